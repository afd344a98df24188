// Kernels of the learned current denoiser: a 3x3 circular-padding
// convolutional encoder-decoder run in bfloat16 with FP32 accumulation on the
// tensor cores (mma.sync m16n8k16, operands staged in shared memory with
// cp.async and fed with ldmatrix), its backward pass and its Adam update.
//
// Tensors are NHWC bfloat16 with the channel count a multiple of 16 (the
// 3-channel current is padded with zeros); gradients are FP32 except where
// they enter a tensor-core product (dz, rounded to bfloat16).
//
//   k_conv   implicit GEMM, persistent: a CTA keeps a tile of output
//            channels' weights in shared memory and runs through 8x16-pixel
//            tiles with a double-buffered halo patch; warp = one pixel row
//            (m16) x the channel tile.  The same
//            kernel computes the input gradient with flipped, transposed
//            weights (dgrad).  Epilogues: bias + ReLU (+ skip) to bfloat16,
//            raw FP32, or the network's residual output in field layout.
//   k_wgrad  weight gradient: per tap a (cout x cin) GEMM over all pixels,
//            split over CTAs (FP32 atomics into the gradient).
//   k_conv_first  the thin first layer (3 -> 32 with the input packing) on
//            the CUDA cores, for passes below 2^18 pixels.
//   elementwise: 2x2 mean pooling / nearest upsampling and
//            their adjoints, ReLU backward with the bias gradient, MSE loss,
//            Adam, weight packing.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>

#include "nn_internal.h"

namespace pic {
namespace nn {

namespace {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ uint32_t saddr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr(sdst)), "l"(gsrc)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void ldsm_x4(uint32_t r[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(saddr(p)));
}
__device__ __forceinline__ void ldsm_x2(uint32_t r[2], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];"
                 : "=r"(r[0]), "=r"(r[1])
                 : "r"(saddr(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t r[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(saddr(p)));
}

// D += A (16x16, row) * B (16x8, col), bf16 in, fp32 accumulate
__device__ __forceinline__ void mma_bf16(float d[4], const uint32_t a[4], uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// ------------------------------------------------------------------ conv
// Launched as programmatic dependents (PDL): a CTA stages its weights, which
// no earlier kernel of the forward pass writes, before waiting for the
// previous kernel, and lets the next kernel start staging once its own
// products are issued.
// UP: the input is the half-resolution tensor read through nearest 2x
// upsampling; the patch then holds the 6 x 10 source pixels of the tile's
// 10 x 18 halo (tiles start on even pixels) and each lane addresses its own
// source pixel, a quarter of the shared memory and of the loads.
constexpr int CPH = PH / 2 + 1, CPW = PW / 2 + 1;  // 6 x 10
template <int CIN, int CT, bool UP = false>
struct ConvSmem {
    static constexpr int CS = CIN + 8;  // row stride in elements (16 B of padding: no bank conflicts)
    static constexpr int PATCH = (UP ? CPH * CPW : PH * PW) * CS;
    static constexpr int WTS = 9 * CT * CS;
    // the CTA's weights, then two patches
    static constexpr size_t bytes = (size_t)(WTS + 2 * PATCH) * 2;
};

// Persistent: CTA (blockIdx.x, blockIdx.z) keeps the weights of output
// channels [z CT, z CT + CT) in shared memory and runs through the tiles
// blockIdx.x, blockIdx.x + gridDim.x, ... of all images; the next tile's
// patch is copied in while the current one is computed.
template <int CIN, int CT, bool UP = false>
__global__ void __launch_bounds__(CONV_THREADS) k_conv(const ConvParams p) {
    using L = ConvSmem<CIN, CT, UP>;
    extern __shared__ __align__(16) unsigned char smem[];
    bf16* sW = reinterpret_cast<bf16*>(smem);
    bf16* sP0 = sW + L::WTS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tilesx = p.W / TW, tiles_img = tilesx * (p.H / TH);
    const int ntiles = p.B * tiles_img;
    const int co0 = blockIdx.z * CT;
    constexpr int CH = CIN / 8;  // 16-byte chunks per pixel
    // input pixel (y, x); with p.up the input is the half-resolution tensor
    // read at (y/2, x/2): nearest 2x upsampling fused into the load
    const int sh = p.up ? 1 : 0;
    const int Hi = p.H >> sh, Wi = p.W >> sh;

    auto load_patch = [&](int tile, bf16* sP) {
        const int b = tile / tiles_img, tl = tile - b * tiles_img;
        const int ty0 = (tl / tilesx) * TH, tx0 = (tl % tilesx) * TW;
        if constexpr (UP) {
            // source pixels (ty0/2 - 1 + cy, tx0/2 - 1 + cx), periodic
            for (int i = tid; i < CPH * CPW * CH; i += CONV_THREADS) {
                const int pix = i / CH, c = i - pix * CH;
                const int cy = pix / CPW, cx = pix - cy * CPW;
                const int y = wrap((ty0 >> 1) - 1 + cy, Hi), x = wrap((tx0 >> 1) - 1 + cx, Wi);
                cp_async16(sP + pix * L::CS + c * 8,
                           p.x + (((size_t)b * Hi + y) * Wi + x) * CIN + c * 8);
            }
            return;
        }
        for (int i = tid; i < PH * PW * CH; i += CONV_THREADS) {
            const int pix = i / CH, c = i - pix * CH;
            const int r = pix / PW, q = pix - r * PW;
            const int y = wrap(ty0 - 1 + r, p.H) >> sh, x = wrap(tx0 - 1 + q, p.W) >> sh;
            cp_async16(sP + pix * L::CS + c * 8,
                       p.x + (((size_t)b * Hi + y) * Wi + x) * CIN + c * 8);
        }
    };

    for (int i = tid; i < 9 * CT * CH; i += CONV_THREADS) {
        const int row = i / CH, c = i - row * CH;
        const int tap = row / CT, n = row - tap * CT;
        cp_async16(sW + row * L::CS + c * 8,
                   p.w + ((size_t)tap * p.cout_pad + co0 + n) * CIN + c * 8);
    }
    pdl_wait();  // the input is the previous kernel's output
    if ((int)blockIdx.x < ntiles) load_patch(blockIdx.x, sP0);
    cp_async_commit();

    constexpr int NT = CT / 8;
    const int r = warp;  // the warp's output pixel row inside the tile
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        bf16* sP = sP0 + (it & 1) * L::PATCH;
        cp_async_wait<0>();
        __syncthreads();  // this tile's patch is in; every warp is done with the other buffer
        const int nxt = tile + gridDim.x;
        if (nxt < ntiles) load_patch(nxt, sP0 + ((it + 1) & 1) * L::PATCH);
        cp_async_commit();

        float acc[NT][4];
#pragma unroll
        for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll 1
        for (int tap = 0; tap < 9; ++tap) {
            const int ky = tap / 3, kx = tap - 3 * (tap / 3);
            // halo pixel (r + ky, px + kx); with UP its source pixel ((f + 1) >> 1)
            const int px = lane & 15;
            const int pix = UP ? ((r + ky + 1) >> 1) * CPW + ((px + kx + 1) >> 1)
                               : (r + ky) * PW + kx + px;
            const bf16* pa = sP + pix * L::CS + (lane >> 4) * 8;
            const bf16* pw = sW + tap * CT * L::CS;
#pragma unroll
            for (int kc = 0; kc < CIN / 16; ++kc) {
                uint32_t a[4];
                ldsm_x4(a, pa + kc * 16);
                if constexpr (NT == 1) {
                    uint32_t bb[2];
                    ldsm_x2(bb, pw + (lane & 7) * L::CS + kc * 16 + ((lane >> 3) & 1) * 8);
                    mma_bf16(acc[0], a, bb[0], bb[1]);
                } else {
#pragma unroll
                    for (int nt = 0; nt < NT; nt += 2) {
                        const int j = lane >> 3;
                        uint32_t bb[4];
                        ldsm_x4(bb, pw + (nt * 8 + (j >> 1) * 8 + (lane & 7)) * L::CS + kc * 16 +
                                        (j & 1) * 8);
                        mma_bf16(acc[nt], a, bb[0], bb[1]);
                        mma_bf16(acc[nt + 1], a, bb[2], bb[3]);
                    }
                }
            }
        }
        if (tile + gridDim.x >= ntiles) pdl_trigger();

        // epilogue: rows g, g+8 of the warp's 16 pixels; columns 2(lane%4), +1 of each n-tile
        const int b = tile / tiles_img, tl = tile - b * tiles_img;
        const int ty0 = (tl / tilesx) * TH, tx0 = (tl % tilesx) * TW;
        const int g = lane >> 2, cq = (lane & 3) * 2;
        const int y = ty0 + r;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int x = tx0 + g + 8 * h;
            const size_t pix = ((size_t)b * p.H + y) * p.W + x;
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const int co = co0 + nt * 8 + cq;
                float v0 = acc[nt][2 * h], v1 = acc[nt][2 * h + 1];
                if (p.epi == EPI_GRAD) {
                    *reinterpret_cast<float2*>(p.g_out + pix * p.cout_pad + co) = make_float2(v0, v1);
                    continue;
                }
                if (p.bias) {
                    if (co < p.cout) v0 += p.bias[co];
                    if (co + 1 < p.cout) v1 += p.bias[co + 1];
                }
                if (p.epi == EPI_FINAL) {
                    // residual output in field layout: out = res * rs + z * os
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int c = co + e;
                        if (c >= p.cout) continue;
                        const size_t o = (size_t)b * p.bstride + (size_t)c * p.cstride + p.offset +
                                         (size_t)y * p.pitch + x;
                        p.fout[o] = p.res[o] * p.rs + (e ? v1 : v0) * p.os;
                    }
                    continue;
                }
                if (p.relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                const __nv_bfloat162 a2 = __floats2bfloat162_rn(v0, v1);
                if (p.a_out) *reinterpret_cast<__nv_bfloat162*>(p.a_out + pix * p.cout_pad + co) = a2;
                if (p.skip) {
                    const __nv_bfloat162 s2 =
                        *reinterpret_cast<const __nv_bfloat162*>(p.skip + pix * p.cout_pad + co);
                    const float2 af = __bfloat1622float2(a2), sf = __bfloat1622float2(s2);
                    *reinterpret_cast<__nv_bfloat162*>(p.y_out + pix * p.cout_pad + co) =
                        __floats2bfloat162_rn(af.x + sf.x, af.y + sf.y);
                }
            }
        }
    }
    cp_async_wait<0>();
}

// ----------------------------------------------------------------- wgrad
// dW[tap][ci][co] += sum over pixels p of x[p + tap offset][ci] * dz[p][co].
// Per tap a GEMM with M = co, N = ci, K = pixels: CTA (s, tap) takes the
// chunks of WG_PIX consecutive pixels (flattened b, y, x order) s, s +
// gridDim.x, ... through a WG_STAGES-deep cp.async pipeline.  The warps split
// the (CO/16) x (CI/16) output blocks and, when there are fewer blocks than
// warps, the 16-pixel k-steps of a chunk as well.  With p.up the input is the
// half-resolution tensor read at (y/2, x/2) (fused nearest upsampling).
template <int CI, int CO>
struct WgradSmem {
    static constexpr int XS = CI + 8, DS = CO + 8;
    static constexpr int STAGE = WG_PIX * (XS + DS);
    static constexpr size_t bytes = (size_t)WG_STAGES * STAGE * 2;
};

template <int CI, int CO>
__global__ void __launch_bounds__(WG_THREADS) k_wgrad(const WgradParams p) {
    using L = WgradSmem<CI, CO>;
    extern __shared__ __align__(16) unsigned char smem[];
    bf16* sbase = reinterpret_cast<bf16*>(smem);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tap = blockIdx.y, ky = tap / 3, kx = tap - 3 * (tap / 3);
    const long long HW = (long long)p.H * p.W;
    const long long nchunks = (long long)p.B * HW / WG_PIX;
    const int sh = p.up ? 1 : 0;
    const int Hi = p.H >> sh, Wi = p.W >> sh;
    constexpr int MB = CO / 16, NB = CI / 16, NBLK = MB * NB;
    constexpr bool SPLITK = NBLK < WG_WARPS;
    constexpr int KS = SPLITK ? WG_WARPS / NBLK : 1;                  // k-step phases
    constexpr int PER = SPLITK ? 1 : (NBLK + WG_WARPS - 1) / WG_WARPS;  // blocks per warp
    const int blk0 = SPLITK ? warp % NBLK : warp;
    const int kph = SPLITK ? warp / NBLK : 0;
    float acc[PER][2][4];
#pragma unroll
    for (int k = 0; k < PER; ++k)
#pragma unroll
        for (int h = 0; h < 2; ++h) acc[k][h][0] = acc[k][h][1] = acc[k][h][2] = acc[k][h][3] = 0.f;

    auto load = [&](long long c, int stage) {
        bf16* sX = sbase + stage * L::STAGE;
        bf16* sD = sX + WG_PIX * L::XS;
        const long long pix0 = c * WG_PIX;
        // the chunk's first pixel (b0, y0, x0), once; the chunk spans < 64 / 16 + 1 rows
        const int b0 = (int)(pix0 / HW);
        const int rem0 = (int)(pix0 - (long long)b0 * HW);
        const int y0 = rem0 / p.W, x0 = rem0 - y0 * p.W;
        constexpr int CHX = CI / 8, CHD = CO / 8;
        for (int i = tid; i < WG_PIX * CHX; i += WG_THREADS) {
            const int px = i / CHX, cc = i - px * CHX;
            int x = x0 + px, y = y0, b = b0;
            while (x >= p.W) {  // at most WG_PIX / 16 times (W >= 16)
                x -= p.W;
                if (++y == p.H) {
                    y = 0;
                    ++b;
                }
            }
            const int ys = wrap(y + ky - 1, p.H) >> sh, xs = wrap(x + kx - 1, p.W) >> sh;
            cp_async16(sX + px * L::XS + cc * 8, p.x + (((size_t)b * Hi + ys) * Wi + xs) * CI + cc * 8);
        }
        for (int i = tid; i < WG_PIX * CHD; i += WG_THREADS) {
            const int px = i / CHD, cc = i - px * CHD;
            cp_async16(sD + px * L::DS + cc * 8, p.dz + (size_t)(pix0 + px) * CO + cc * 8);
        }
    };

    const long long c0 = blockIdx.x;
    const long long ns = gridDim.x;
    // prefetch WG_STAGES - 1 chunks
#pragma unroll
    for (int k = 0; k < WG_STAGES - 1; ++k) {
        if (c0 + k * ns < nchunks) load(c0 + k * ns, k);
        cp_async_commit();
    }
    int stage = 0;
    for (long long c = c0; c < nchunks; c += ns) {
        const long long cn = c + (WG_STAGES - 1) * ns;
        if (cn < nchunks) load(cn, (stage + WG_STAGES - 1) % WG_STAGES);
        cp_async_commit();
        cp_async_wait<WG_STAGES - 1>();  // the chunk of this iteration has landed
        __syncthreads();
        const bf16* sX = sbase + stage * L::STAGE;
        const bf16* sD = sX + WG_PIX * L::XS;
        const int j = lane >> 3;
#pragma unroll
        for (int ks = kph; ks < WG_PIX / 16; ks += KS) {
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                const int blk = blk0 + k * WG_WARPS;
                if (blk >= NBLK) break;
                const int mb = blk / NB, nb = blk - mb * NB;
                uint32_t a[4], bb[4];
                // A (co x px) from dz stored [px][co]: transposing load
                ldsm_x4_t(a, sD + (ks * 16 + (j >> 1) * 8 + (lane & 7)) * L::DS + mb * 16 + (j & 1) * 8);
                // B (px x ci) from x stored [px][ci]: transposing load, two n-tiles
                ldsm_x4_t(bb, sX + (ks * 16 + (j & 1) * 8 + (lane & 7)) * L::XS + nb * 16 + (j >> 1) * 8);
                mma_bf16(acc[k][0], a, bb[0], bb[1]);
                mma_bf16(acc[k][1], a, bb[2], bb[3]);
            }
        }
        __syncthreads();  // the stage is refilled by a later iteration
        stage = (stage + 1) % WG_STAGES;
    }
    cp_async_wait<0>();
    // accumulate into dW[tap][ci][co] (real channel counts)
    const int g = lane >> 2, cq = (lane & 3) * 2;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int blk = blk0 + k * WG_WARPS;
        if (blk >= NBLK) break;
        const int mb = blk / NB, nb = blk - mb * NB;
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int co = mb * 16 + g + (e >= 2 ? 8 : 0);
                const int ci = nb * 16 + h * 8 + cq + (e & 1);
                if (co < p.cout && ci < p.cin)
                    atomicAdd(p.dw + ((size_t)tap * p.cin + ci) * p.cout + co, acc[k][h][e]);
            }
    }
}

// ----------------------------------------------------------- elementwise

// The network's thin first layer on the CUDA cores.  c1 (3 -> 32 channels)
// has 27 inputs per output: as an implicit GEMM on the tensor cores most of
// each tile is padding, and at small grids its time is launch and pipeline
// latency.  It keeps the arithmetic of the tensor-core path: bfloat16 inputs
// and weights, FP32 products and sums, bias, then the epilogue.
constexpr int THIN_T = 16;  // 16 x 16 output pixels per CTA, one per thread

__device__ __forceinline__ int wrap_idx(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// c1 fused with the input packing: the current (field layout) is scaled and
// rounded to bfloat16 (the network input, also stored NHWC with 16 channels
// for the first layer's weight gradient), then the 3x3 circular convolution
// with bias and ReLU gives the 32-channel bfloat16 activation.
__global__ void __launch_bounds__(256) k_conv_first(const float* J, long long bstride,
                                                    long long cstride, int pitch, int offset,
                                                    int H, int W, float inv_scale, const bf16* w,
                                                    int cout_pad, const float* bias, bf16* xin,
                                                    bf16* a_out) {
    constexpr int C1 = 32, CI = 3, CINP = 16, E = THIN_T + 2;
    __shared__ float sX[CI][E][E];
    __shared__ __align__(16) float sW[9 * CI][C1];  // [tap * 3 + ci][co]
    const int tid = threadIdx.x, b = blockIdx.z;
    const int x0 = blockIdx.x * THIN_T, y0 = blockIdx.y * THIN_T;
    pdl_wait();
    for (int i = tid; i < 9 * CI * C1; i += blockDim.x) {
        const int co = i % C1, k = i / C1, tap = k / CI, ci = k - tap * CI;
        sW[k][co] = __bfloat162float(w[((size_t)tap * cout_pad + co) * CINP + ci]);
    }
    for (int i = tid; i < CI * E * E; i += blockDim.x) {
        const int c = i / (E * E), r = (i / E) % E, q = i % E;
        const int yy = wrap_idx(y0 + r - 1, H), xx = wrap_idx(x0 + q - 1, W);
        const float v = J[b * bstride + c * cstride + offset + (long long)yy * pitch + xx] * inv_scale;
        sX[c][r][q] = __bfloat162float(__float2bfloat16_rn(v));
    }
    __syncthreads();
    pdl_trigger();
    const int ty = tid / THIN_T, tx = tid % THIN_T;
    const size_t pix = ((size_t)b * H + y0 + ty) * W + x0 + tx;
    {
        __align__(16) bf16 v[CINP];
#pragma unroll
        for (int c = 0; c < CINP; ++c) v[c] = __float2bfloat16_rn(c < CI ? sX[c][ty + 1][tx + 1] : 0.f);
        uint4* o = reinterpret_cast<uint4*>(xin + pix * CINP);
        o[0] = reinterpret_cast<const uint4*>(v)[0];
        o[1] = reinterpret_cast<const uint4*>(v)[1];
    }
    float acc[C1];
#pragma unroll
    for (int co = 0; co < C1; ++co) acc[co] = 0.f;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
        const int ky = tap / 3, kx = tap - 3 * (tap / 3);
#pragma unroll
        for (int ci = 0; ci < CI; ++ci) {
            const float xv = sX[ci][ty + ky][tx + kx];
            const float4* wr = reinterpret_cast<const float4*>(sW[tap * CI + ci]);
#pragma unroll
            for (int q = 0; q < C1 / 4; ++q) {
                const float4 wv = wr[q];
                acc[4 * q] += xv * wv.x;
                acc[4 * q + 1] += xv * wv.y;
                acc[4 * q + 2] += xv * wv.z;
                acc[4 * q + 3] += xv * wv.w;
            }
        }
    }
    __align__(16) bf16 o[C1];
#pragma unroll
    for (int co = 0; co < C1; ++co) o[co] = __float2bfloat16_rn(fmaxf(acc[co] + bias[co], 0.f));
    uint4* dst = reinterpret_cast<uint4*>(a_out + pix * C1);
#pragma unroll
    for (int q = 0; q < C1 / 8; ++q) dst[q] = reinterpret_cast<const uint4*>(o)[q];
}

// The network input on large lattices, where c1 runs as an implicit GEMM on
// the tensor cores: the current (field layout) scaled and rounded to
// bfloat16, NHWC with 16 channels (3 used).
__global__ void k_pack_input(const float* J, long long bstride, long long cstride, int pitch,
                             int offset, int B, int H, int W, float inv_scale, bf16* out) {
    pdl_wait();
    pdl_trigger();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)B * H * W) return;
    const int x = (int)(i % W);
    const long long t = i / W;
    const int y = (int)(t % H), b = (int)(t / H);
    const float* s = J + b * bstride + offset + (long long)y * pitch + x;
    __align__(16) bf16 v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16_rn(c < 3 ? s[c * cstride] * inv_scale : 0.f);
    uint4* o = reinterpret_cast<uint4*>(out + i * 16);
    o[0] = reinterpret_cast<const uint4*>(v)[0];
    o[1] = reinterpret_cast<const uint4*>(v)[1];
}

// 2x2 mean pooling, bfloat16 -> bfloat16 (FP32 sum of the four)
__global__ void k_pool_fwd(const bf16* in, int B, int H, int W, int C, bf16* out) {
    pdl_wait();
    pdl_trigger();
    const int G = C / 8;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int Ho = H / 2, Wo = W / 2;
    if (i >= (long long)B * Ho * Wo * G) return;
    const int gi = (int)(i % G);
    const long long pix = i / G;
    const int x = (int)(pix % Wo);
    const long long t = pix / Wo;
    const int y = (int)(t % Ho), b = (int)(t / Ho);
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
            const uint4 u = *reinterpret_cast<const uint4*>(
                in + (((size_t)b * H + 2 * y + dy) * W + 2 * x + dx) * C + gi * 8);
            const bf16* v = reinterpret_cast<const bf16*>(&u);
#pragma unroll
            for (int k = 0; k < 8; ++k) s[k] += __bfloat162float(v[k]);
        }
    __align__(16) bf16 o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) o[k] = __float2bfloat16_rn(0.25f * s[k]);
    *reinterpret_cast<uint4*>(out + pix * C + gi * 8) = *reinterpret_cast<const uint4*>(o);
}

// nearest 2x upsampling, bfloat16 (out has 2H x 2W)
__global__ void k_up_fwd(const bf16* in, int B, int H, int W, int C, bf16* out) {
    const int G = C / 8;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int Ho = 2 * H, Wo = 2 * W;
    if (i >= (long long)B * Ho * Wo * G) return;
    const int gi = (int)(i % G);
    const long long pix = i / G;
    const int x = (int)(pix % Wo);
    const long long t = pix / Wo;
    const int y = (int)(t % Ho), b = (int)(t / Ho);
    *reinterpret_cast<uint4*>(out + pix * C + gi * 8) = *reinterpret_cast<const uint4*>(
        in + (((size_t)b * H + y / 2) * W + x / 2) * C + gi * 8);
}

// adjoint of pooling: out (H x W) = in (H/2 x W/2) / 4, FP32

// the gradient arriving at the ReLU of the pixel pix (NHWC index on the
// layer's grid, B x H x W) for channels c .. c + 7: read directly (RB_DIRECT),
// through the adjoint of the 2x2 mean pooling (RB_POOL: a quarter of the
// coarse pixel's value) or of the nearest 2x upsampling (RB_UP: the sum of
// the four fine pixels), in the FP32 order the separate adjoint kernels had
enum { RB_DIRECT = 0, RB_POOL = 1, RB_UP = 2 };
__device__ __forceinline__ void rb_source(int mode, const float* src, long long pix, int H, int W,
                                          int C, int c, float v[8]) {
    if (mode == RB_DIRECT) {
        const float4 d0 = *reinterpret_cast<const float4*>(src + pix * C + c);
        const float4 d1 = *reinterpret_cast<const float4*>(src + pix * C + c + 4);
        v[0] = d0.x; v[1] = d0.y; v[2] = d0.z; v[3] = d0.w;
        v[4] = d1.x; v[5] = d1.y; v[6] = d1.z; v[7] = d1.w;
        return;
    }
    const int x = (int)(pix % W);
    const long long t = pix / W;
    const int y = (int)(t % H), b = (int)(t / H);
    if (mode == RB_POOL) {
        const float* q = src + (((size_t)b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c;
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = q[k] * 0.25f;
        return;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = 0.f;
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
            const float* q = src + (((size_t)b * 2 * H + 2 * y + dy) * 2 * W + 2 * x + dx) * C + c;
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] += q[k];
        }
}

// dz = bf16((dy + extra) * (a > 0)); db[c] += sum over pixels of the FP32 product
__global__ void __launch_bounds__(256) k_relu_back(int mode, const float* src, int H, int W,
                                                   const float* extra, const bf16* a,
                                                   long long npix, int C, bf16* dz, float* db) {
    __shared__ float sdb[128];
    for (int c = threadIdx.x; c < C; c += blockDim.x) sdb[c] = 0.f;
    __syncthreads();
    const int G = C / 8;
    float part[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int myg = -1;
    const long long total = npix * G;
    // the grid stride is a multiple of G, so a thread keeps its channel group
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const int gi = (int)(i % G);
        myg = gi;
        const long long pix = i / G;
        float v[8];
        rb_source(mode, src, pix, H, W, C, gi * 8, v);
        if (extra) {
            const float4 e0 = *reinterpret_cast<const float4*>(extra + pix * C + gi * 8);
            const float4 e1 = *reinterpret_cast<const float4*>(extra + pix * C + gi * 8 + 4);
            v[0] += e0.x; v[1] += e0.y; v[2] += e0.z; v[3] += e0.w;
            v[4] += e1.x; v[5] += e1.y; v[6] += e1.z; v[7] += e1.w;
        }
        if (a) {
            const uint4 u = *reinterpret_cast<const uint4*>(a + pix * C + gi * 8);
            const bf16* av = reinterpret_cast<const bf16*>(&u);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (!(__bfloat162float(av[k]) > 0.f)) v[k] = 0.f;
        }
        __align__(16) bf16 o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            part[k] += v[k];
            o[k] = __float2bfloat16_rn(v[k]);
        }
        *reinterpret_cast<uint4*>(dz + pix * C + gi * 8) = *reinterpret_cast<const uint4*>(o);
    }
    if (myg >= 0)
#pragma unroll
        for (int k = 0; k < 8; ++k) atomicAdd(&sdb[myg * 8 + k], part[k]);
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) atomicAdd(db + c, sdb[c]);
}

// MSE of the normalised output against the normalised target; dz11 (16
// channels, bfloat16) = bf16(2 (out - t) / N); db11 += the FP32 gradient.
__global__ void __launch_bounds__(256) k_mse(const float* out, const float* target,
                                             long long bstride, long long cstride, int pitch,
                                             int offset, int B, int H, int W, float inv_scale,
                                             double inv_n, bf16* dz, float* db, double* loss) {
    __shared__ double sred[8];
    __shared__ float sdb[3];
    if (threadIdx.x < 3) sdb[threadIdx.x] = 0.f;
    __syncthreads();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    float gsum[3] = {0.f, 0.f, 0.f};
    if (i < (long long)B * H * W) {
        const int x = (int)(i % W);
        const long long t = i / W;
        const int y = (int)(t % H), b = (int)(t / H);
        const long long o = b * bstride + offset + (long long)y * pitch + x;
        // out is the normalised network output in a dense [B][3][H][W] buffer
        const long long od = ((long long)b * 3) * H * W + (long long)y * W + x;
        __align__(16) bf16 v[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16_rn(0.f);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float d = out[od + (long long)c * H * W] - target[o + c * cstride] * inv_scale;
            l += (double)d * d;
            const float gr = (float)(2.0 * inv_n) * d;
            gsum[c] = gr;
            v[c] = __float2bfloat16_rn(gr);
        }
        uint4* q = reinterpret_cast<uint4*>(dz + i * 16);
        q[0] = reinterpret_cast<const uint4*>(v)[0];
        q[1] = reinterpret_cast<const uint4*>(v)[1];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float s = gsum[c];
#pragma unroll
        for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
        if ((threadIdx.x & 31) == 0) atomicAdd(&sdb[c], s);
    }
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) l += __shfl_xor_sync(0xffffffffu, l, k);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sred[w];
        atomicAdd(loss, s * inv_n);
    }
    if (threadIdx.x < 3) atomicAdd(db + threadIdx.x, sdb[threadIdx.x]);
}

// Adam (Kingma & Ba, Algorithm 1) on the FP32 master parameters; c1, c2 are
// the bias corrections 1/(1 - beta^t).
// Low-wavenumber restoration, out <- out + L^n (a - b), as two separable
// passes: n passes of the periodic binomial stencil (1/4, 1/2, 1/4) compose to
// the (2n+1)-tap kernel C(2n, k) / 4^n along each axis, which multiplies the
// Fourier mode (mx, my) of an H x W periodic lattice by
// (cos^2(pi mx / W) cos^2(pi my / H))^n.  Rows first (k_lowk_x: the row
// segment and its halo staged in shared memory, coalesced), then columns
// (k_lowk_y: a 64-row x 32-column tile and its halo rows).
// i mod n in [0, n) for any i (the halo may wrap several times on small lattices)
__device__ __forceinline__ int wrap_any(int i, int n) {
    if (i >= 0 && i < n) return i;  // nearly every index: no division
    i %= n;
    return i < 0 ? i + n : i;
}

constexpr int LK_ROW = 256;                    // outputs per row of the row pass
// rows per CTA of the row pass and of the copy: 8 on large lattices (fewer,
// longer CTAs), 1 on small ones (more CTAs in flight)
__host__ __device__ inline int lk_rows(int B, int H, int W) {
    return 3LL * B * H * W >= (1LL << 23) ? 8 : 1;
}
constexpr int LK_TY = 64, LK_TX = 32, LK_YT = 8;  // column pass: tile rows, columns, thread rows

// t = rows of (a - b) (b.p null: a) filtered along x; t dense [B][3][H][W].
// CTA = LK_ROW columns of lk_rows rows.
__global__ void k_lowk_x(FieldView a, FieldView b, float* t, LowkTaps w, int B, int H, int W) {
    extern __shared__ float sRow[];  // LK_ROW + 2n values
    const int n = w.n;
    const int x0 = blockIdx.x * LK_ROW;
    const int c = blockIdx.z % 3, smp = blockIdx.z / 3;
    const int x = x0 + threadIdx.x;
    const int rows = lk_rows(B, H, W);
    for (int y = blockIdx.y * rows; y < min(H, (int)(blockIdx.y + 1) * rows); ++y) {
        const float* pa = a.p + smp * a.bstride + c * a.cstride + a.offset + (long long)y * a.pitch;
        const float* pb =
            b.p ? b.p + smp * b.bstride + c * b.cstride + b.offset + (long long)y * b.pitch : nullptr;
        __syncthreads();  // the previous row's reads of sRow are done
        for (int i = threadIdx.x; i < LK_ROW + 2 * n; i += blockDim.x) {
            const int xs = wrap_any(x0 + i - n, W);
            sRow[i] = pb ? pa[xs] - pb[xs] : pa[xs];
        }
        __syncthreads();
        if (x < W) {
            float v = 0.f;
            for (int k = 0; k <= 2 * n; ++k) v = fmaf(w.w[k], sRow[threadIdx.x + k], v);
            t[((long long)blockIdx.z * H + y) * W + x] = v;
        }
    }
}

// out += columns of t filtered along y
__global__ void k_lowk_y(const float* t, FieldView o, LowkTaps w, int B, int H, int W) {
    extern __shared__ float sCol[];  // (LK_TY + 2n) rows x (LK_TX + 1)
    const int n = w.n;
    const int x0 = blockIdx.x * LK_TX, y0 = blockIdx.y * LK_TY;
    const int c = blockIdx.z % 3, smp = blockIdx.z / 3;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x = x0 + tx;
    const float* pt = t + (long long)blockIdx.z * H * W;
    for (int r = ty; r < LK_TY + 2 * n; r += LK_YT)
        sCol[r * (LK_TX + 1) + tx] = x < W ? pt[(long long)wrap_any(y0 + r - n, H) * W + x] : 0.f;
    __syncthreads();
    if (x >= W) return;
    float* po = o.p + smp * o.bstride + c * o.cstride + o.offset + x;
    for (int r = ty; r < LK_TY && y0 + r < H; r += LK_YT) {
        float v = 0.f;
        for (int k = 0; k <= 2 * n; ++k) v = fmaf(w.w[k], sCol[(r + k) * (LK_TX + 1) + tx], v);
        po[(long long)(y0 + r) * o.pitch] += v;
    }
}

// o = a, element by element (layouts may differ); CTA = 256 columns of
// lk_rows rows of one component of one sample (blockIdx.z)
__global__ void k_field_copy(FieldView a, FieldView o, int B, int H, int W) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= W) return;
    const int c = blockIdx.z % 3, smp = blockIdx.z / 3;
    const float* pa = a.p + smp * a.bstride + c * a.cstride + a.offset + x;
    float* po = o.p + smp * o.bstride + c * o.cstride + o.offset + x;
    const int rows = lk_rows(B, H, W);
    for (int y = blockIdx.y * rows; y < min(H, (int)(blockIdx.y + 1) * rows); ++y)
        po[(long long)y * o.pitch] = pa[(long long)y * a.pitch];
}

// The same copy with per-sample base pointers: sample b of a starts at
// atab[b] (when atab is set, else a.p + b a.bstride) and sample b of o at
// otab[b] (else o.p + b o.bstride); o2 (when o2.p is set) receives a second
// copy.  Gathers the currents of separate simulations into one dense batch of
// samples and writes them back.
__global__ void k_field_copy_tab(FieldView a, const float* const* atab, FieldView o,
                                 float* const* otab, FieldView o2, int B, int H, int W) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= W) return;
    const int c = blockIdx.z % 3, smp = blockIdx.z / 3;
    const float* pa = (atab ? atab[smp] : a.p + smp * a.bstride) + c * a.cstride + a.offset + x;
    float* po = (otab ? otab[smp] : o.p + smp * o.bstride) + c * o.cstride + o.offset + x;
    float* po2 = o2.p ? o2.p + smp * o2.bstride + c * o2.cstride + o2.offset + x : nullptr;
    const int rows = lk_rows(B, H, W);
    for (int y = blockIdx.y * rows; y < min(H, (int)(blockIdx.y + 1) * rows); ++y) {
        const float v = pa[(long long)y * a.pitch];
        po[(long long)y * o.pitch] = v;
        if (po2) po2[(long long)y * o2.pitch] = v;
    }
}

__global__ void k_adam(float* p, const float* g, float* m, float* v, long long n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// master FP32 weights [tap][ci][co] -> bfloat16 forward [tap][co_pad][ci_pad]
// and input-gradient [tap'][ci_padn][co_pad16] layouts (tap' = 8 - tap)
__global__ void k_pack_weights(const PackTable t, const float* master, bf16* wf, bf16* wd,
                               bf16* wp) {
    const int l = blockIdx.y;
    if (l >= t.n) return;
    const LayerDesc& d = t.layer[l];
    const long long nf = wf ? 9LL * d.cout_pad * d.cin_pad : 0;
    const long long nd = wd ? 9LL * d.dg_cout_pad * d.dg_cin_pad : 0;
    const long long np = (wp && d.wp_off >= 0) ? 16LL * d.cout_pad * d.cin_pad : 0;
    const float* w = master + d.woff;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nf + nd + np;
         i += (long long)gridDim.x * blockDim.x) {
        if (i >= nf + nd) {
            // combined tap t = parity (a, b) x (u, v) of an upsampling layer: the
            // sum of the 3x3 taps (dy, dx) whose upsampled row and column land
            // on x pixel (i + u, j + v) for an output pixel of parity (a, b)
            const long long k = i - nf - nd;
            const int ci = (int)(k % d.cin_pad);
            const long long r = k / d.cin_pad;
            const int co = (int)(r % d.cout_pad), tp = (int)(r / d.cout_pad);
            const int a = tp >> 3, b = (tp >> 2) & 1, uu = (tp >> 1) & 1, vv = tp & 1;
            // offsets dy in [ylo, yhi] (a = 0: {-1}, {0, 1}; a = 1: {-1, 0}, {1})
            const int ylo = uu == 0 ? -1 : (a == 0 ? 0 : 1), yhi = uu == 0 ? (a == 0 ? -1 : 0) : 1;
            const int xlo = vv == 0 ? -1 : (b == 0 ? 0 : 1), xhi = vv == 0 ? (b == 0 ? -1 : 0) : 1;
            float v = 0.f;
            if (ci < d.cin && co < d.cout)
                for (int dy = ylo; dy <= yhi; ++dy)
                    for (int dx = xlo; dx <= xhi; ++dx)
                        v += w[((long long)((dy + 1) * 3 + dx + 1) * d.cin + ci) * d.cout + co];
            wp[d.wp_off + k] = __float2bfloat16_rn(v);
        } else if (i < nf) {
            const int ci = (int)(i % d.cin_pad);
            const long long r = i / d.cin_pad;
            const int co = (int)(r % d.cout_pad), tap = (int)(r / d.cout_pad);
            const float v = (ci < d.cin && co < d.cout) ? w[((long long)tap * d.cin + ci) * d.cout + co] : 0.f;
            wf[d.wf_off + i] = __float2bfloat16_rn(v);
        } else if (d.dg_cout_pad > 0) {
            const long long k = i - nf;
            const int co = (int)(k % d.dg_cin_pad);   // the layer's output channel (k of the dgrad GEMM)
            const long long r = k / d.dg_cin_pad;
            const int ci = (int)(r % d.dg_cout_pad), tp = (int)(r / d.dg_cout_pad);
            const int tap = 8 - tp;
            const float v = (ci < d.cin && co < d.cout) ? w[((long long)tap * d.cin + ci) * d.cout + co] : 0.f;
            wd[d.wd_off + k] = __float2bfloat16_rn(v);
        }
    }
}

template <int CIN, int CT, bool UP = false>
cudaError_t conv_attr() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_conv<CIN, CT, UP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)ConvSmem<CIN, CT, UP>::bytes);
    done = e == cudaSuccess;
    return e;
}

template <int CI, int CO>
cudaError_t wgrad_attr() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_wgrad<CI, CO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)WgradSmem<CI, CO>::bytes);
    done = e == cudaSuccess;
    return e;
}

template <int CIN, int CT, bool UP = false>
cudaError_t conv_T(const ConvParams& p, cudaStream_t s) {
    cudaError_t e = conv_attr<CIN, CT, UP>();
    if (e != cudaSuccess) return e;
    static int per_sm = 0, sms = 0;
    if (!per_sm) {
        int dev = 0, smem = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return e;
        if ((e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) !=
            cudaSuccess)
            return e;
        per_sm = smem / (int)(ConvSmem<CIN, CT, UP>::bytes + 1024);
        if (per_sm < 1) per_sm = 1;
        if (per_sm * CONV_THREADS > 2048) per_sm = 2048 / CONV_THREADS;
    }
    const int ntiles = p.B * (p.W / TW) * (p.H / TH), zt = p.cout_pad / CT;
    // resident CTAs shared by the output-channel tiles
    int gx = (sms * per_sm + zt - 1) / zt;
    if (gx > ntiles) gx = ntiles;
    if (gx < 1) gx = 1;
    const dim3 grid(gx, 1, zt);
    return launch_pdl(k_conv<CIN, CT, UP>, grid, dim3(CONV_THREADS), ConvSmem<CIN, CT, UP>::bytes,
                      s, p);
}

template <int CI, int CO>
cudaError_t wgrad_T(const WgradParams& p, int nsplit, cudaStream_t s) {
    cudaError_t e = wgrad_attr<CI, CO>();
    if (e != cudaSuccess) return e;
    k_wgrad<CI, CO><<<dim3(nsplit, 9), WG_THREADS, WgradSmem<CI, CO>::bytes, s>>>(p);
    return cudaGetLastError();
}

int blocks(long long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

#define PIC_CONV_SHAPES(X) \
    X(16, 32) X(16, 64) X(16, 8) X(32, 32) X(32, 64) X(32, 8) X(64, 32) X(64, 64) X(128, 32)
#define PIC_WGRAD_SHAPES(X) \
    X(16, 32) X(32, 32) X(32, 64) X(64, 64) X(64, 128) X(128, 128) X(128, 64) X(64, 32) X(32, 16)

cudaError_t init_kernels() {
    cudaError_t e = init_tc_kernels();
    if (e == cudaSuccess) e = conv_attr<128, 32, true>();
    if (e == cudaSuccess) e = conv_attr<64, 32, true>();
#define PIC_C_ATTR(A, B) if (e == cudaSuccess) e = conv_attr<A, B>();
#define PIC_W_ATTR(A, B) if (e == cudaSuccess) e = wgrad_attr<A, B>();
    PIC_CONV_SHAPES(PIC_C_ATTR)
    PIC_WGRAD_SHAPES(PIC_W_ATTR)
#undef PIC_C_ATTR
#undef PIC_W_ATTR
    return e;
}

// CIN in {16, 32, 64, 128}; CT in {8, 32, 64} (cout_pad a multiple of CT).
// CIN = 128 always runs with CT = 32: 64 channels' weights and two patches
// would not fit in shared memory.
cudaError_t launch_conv(const ConvParams& p, int cin, int ct, cudaStream_t s) {
    if (p.H % TH || p.W % TW || p.cout_pad % ct) return cudaErrorInvalidValue;
    if (conv_out_tc_supported(p, cin)) return launch_conv_out_tc(p, s);
    if (conv_up_tc_supported(p, cin)) return launch_conv_up_tc(p, cin, s);
    if (conv_tc_supported(p, cin)) return launch_conv_tc(p, cin, s);
    if (cin == 128 && ct == 64) ct = 32;
    // the decoder's upsampling layers (c7: 128 -> 64, c9: 64 -> 32) read
    // their source pixels directly
    if (p.up && cin == 128 && ct == 32) return conv_T<128, 32, true>(p, s);
    if (p.up && cin == 64 && ct == 32) return conv_T<64, 32, true>(p, s);
#define PIC_CONV_CASE(CI, C) \
    if (cin == CI && ct == C) return conv_T<CI, C>(p, s);
    PIC_CONV_SHAPES(PIC_CONV_CASE)
#undef PIC_CONV_CASE
    return cudaErrorInvalidValue;
}

// CI = x channels, CO = dz channels (both padded to 16)
cudaError_t launch_wgrad(const WgradParams& p, int ci, int co, cudaStream_t s) {
    const long long npix = (long long)p.B * p.H * p.W;
    if (npix % WG_PIX || p.W < 16 || (p.up && (p.H % 2 || p.W % 2))) return cudaErrorInvalidValue;
    if (wgrad_tc_supported(p, ci, co)) return launch_wgrad_tc(p, ci, co, s);
    const long long nchunks = npix / WG_PIX;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // about four CTAs per SM over the nine taps
    int nsplit = (int)std::min<long long>(nchunks, std::max(1, 4 * sms / 9));
#define PIC_WG_CASE(A, B) \
    if (ci == A && co == B) return wgrad_T<A, B>(p, nsplit, s);
    PIC_WGRAD_SHAPES(PIC_WG_CASE)
#undef PIC_WG_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_conv_first(const float* J, long long bstride, long long cstride, int pitch,
                              int offset, int B, int H, int W, float inv_scale,
                              const __nv_bfloat16* w, int cout_pad, const float* bias,
                              __nv_bfloat16* xin, __nv_bfloat16* a_out, cudaStream_t s) {
    if (B <= 0) return cudaSuccess;
    if (H % THIN_T || W % THIN_T) return cudaErrorInvalidValue;
    return launch_pdl(k_conv_first, dim3(W / THIN_T, H / THIN_T, B), dim3(256), 0, s, J, bstride,
                      cstride, pitch, offset, H, W, inv_scale, w, cout_pad, bias, xin, a_out);
}

cudaError_t launch_pack_input(const float* J, long long bstride, long long cstride, int pitch,
                              int offset, int B, int H, int W, float inv_scale, __nv_bfloat16* out,
                              cudaStream_t s) {
    const long long n = (long long)B * H * W;
    if (n == 0) return cudaSuccess;
    return launch_pdl(k_pack_input, dim3(blocks(n, 256)), dim3(256), 0, s, J, bstride, cstride,
                      pitch, offset, B, H, W, inv_scale, out);
}

cudaError_t launch_pool_fwd(const __nv_bfloat16* in, int B, int H, int W, int C,
                            __nv_bfloat16* out, cudaStream_t s) {
    const long long n = (long long)B * (H / 2) * (W / 2) * (C / 8);
    return launch_pdl(k_pool_fwd, dim3(blocks(n, 256)), dim3(256), 0, s, in, B, H, W, C, out);
}

cudaError_t launch_up_fwd(const __nv_bfloat16* in, int B, int H, int W, int C, __nv_bfloat16* out,
                          cudaStream_t s) {
    const long long n = (long long)B * (2 * H) * (2 * W) * (C / 8);
    k_up_fwd<<<blocks(n, 256), 256, 0, s>>>(in, B, H, W, C, out);
    return cudaGetLastError();
}

namespace {
cudaError_t relu_back_launch(int mode, const float* src, int B, int H, int W, const float* extra,
                             const __nv_bfloat16* a, int C, __nv_bfloat16* dz, float* db,
                             cudaStream_t s) {
    const long long npix = (long long)B * H * W;
    const int G = C / 8;
    // threads a multiple of G: each thread keeps one channel group
    const long long work = npix * G;
    long long nb = std::min<long long>((work + 255) / 256, 4 * 152);
    if (nb < 1) nb = 1;
    k_relu_back<<<(int)nb, 256, 0, s>>>(mode, src, H, W, extra, a, npix, C, dz, db);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_relu_back(const float* dy, const float* extra, const __nv_bfloat16* a,
                             long long npix, int C, __nv_bfloat16* dz, float* db, cudaStream_t s) {
    if (npix > 0x7fffffffLL) return cudaErrorInvalidValue;
    return relu_back_launch(RB_DIRECT, dy, 1, 1, (int)npix, extra, a, C, dz, db, s);
}

cudaError_t launch_pool_relu_back(const float* dp, int B, int H, int W, int C, const float* extra,
                                  const __nv_bfloat16* a, __nv_bfloat16* dz, float* db,
                                  cudaStream_t s) {
    return relu_back_launch(RB_POOL, dp, B, H, W, extra, a, C, dz, db, s);
}

cudaError_t launch_up_relu_back(const float* du, int B, int H, int W, int C,
                                const __nv_bfloat16* a, __nv_bfloat16* dz, float* db,
                                cudaStream_t s) {
    return relu_back_launch(RB_UP, du, B, H, W, nullptr, a, C, dz, db, s);
}

cudaError_t launch_mse(const float* out, const float* target, long long bstride, long long cstride,
                       int pitch, int offset, int B, int H, int W, float inv_scale,
                       __nv_bfloat16* dz, float* db, double* loss, cudaStream_t s) {
    const long long n = (long long)B * H * W;
    const double inv_n = 1.0 / (3.0 * (double)n);
    k_mse<<<blocks(n, 256), 256, 0, s>>>(out, target, bstride, cstride, pitch, offset, B, H, W,
                                         inv_scale, inv_n, dz, db, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, long long n, float lr,
                        float b1, float b2, float eps, float c1, float c2, cudaStream_t s) {
    k_adam<<<blocks(n, 256), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

LowkTaps lowk_taps(int n) {
    LowkTaps w;
    memset(&w, 0, sizeof w);
    w.n = n;
    // C(2n, k) / 4^n by Pascal's rule in FP64 (exact up to n = 26), then FP32
    double row[2 * LOWK_MAX + 1] = {1.0};
    for (int m = 1; m <= 2 * n; ++m) {
        for (int k = m; k >= 1; --k) row[k] = 0.5 * (row[k] + row[k - 1]);
        row[0] *= 0.5;
    }
    for (int k = 0; k <= 2 * n; ++k) w.w[k] = (float)row[k];
    return w;
}

cudaError_t launch_lowk(const FieldView& a, const FieldView& b, float* t, const FieldView& o,
                        int n, int B, int H, int W, cudaStream_t s) {
    if (n <= 0 || (long long)B * H * W == 0) return cudaSuccess;
    if (n > LOWK_MAX) return cudaErrorInvalidValue;
    const LowkTaps w = lowk_taps(n);
    const int rows = lk_rows(B, H, W);
    const dim3 gx((W + LK_ROW - 1) / LK_ROW, (H + rows - 1) / rows, 3 * B);
    k_lowk_x<<<gx, LK_ROW, (LK_ROW + 2 * n) * sizeof(float), s>>>(a, b, t, w, B, H, W);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const dim3 gy((W + LK_TX - 1) / LK_TX, (H + LK_TY - 1) / LK_TY, 3 * B);
    k_lowk_y<<<gy, dim3(LK_TX, LK_YT), (LK_TY + 2 * n) * (LK_TX + 1) * sizeof(float), s>>>(
        t, o, w, B, H, W);
    return cudaGetLastError();
}

cudaError_t launch_field_copy_tab(const FieldView& a, const float* const* atab, const FieldView& o,
                                  float* const* otab, const FieldView& o2, int B, int H, int W,
                                  cudaStream_t s) {
    const long long n = (long long)B * 3 * H * W;
    if (n == 0) return cudaSuccess;
    const int rows = lk_rows(B, H, W);
    k_field_copy_tab<<<dim3((W + 255) / 256, (H + rows - 1) / rows, 3 * B), 256, 0, s>>>(
        a, atab, o, otab, o2, B, H, W);
    return cudaGetLastError();
}

cudaError_t launch_field_copy(const FieldView& a, const FieldView& o, int B, int H, int W,
                              cudaStream_t s) {
    const long long n = (long long)B * 3 * H * W;
    if (n == 0) return cudaSuccess;
    const int rows = lk_rows(B, H, W);
    k_field_copy<<<dim3((W + 255) / 256, (H + rows - 1) / rows, 3 * B), 256, 0, s>>>(a, o, B, H, W);
    return cudaGetLastError();
}

cudaError_t launch_pack_weights(const PackTable& t, const float* master, __nv_bfloat16* wf,
                                __nv_bfloat16* wd, cudaStream_t s, __nv_bfloat16* wp) {
    k_pack_weights<<<dim3(64, t.n), 256, 0, s>>>(t, master, wf, wd, wp);
    return cudaGetLastError();
}

}  // namespace nn
}  // namespace pic
