// 3x3 circular convolution on the 5th-generation tensor cores (tcgen05):
// the implicit GEMM D[pixels x cout] = sum over taps and input channels of
// X[shifted pixel][cin] * W[tap][cout][cin], bfloat16 operands in shared
// memory, FP32 accumulator in tensor memory (TMEM).
//
// Work unit = one segment of M = 128 consecutive output pixels of one image
// row x all NT output channels; persistent CTAs run through the segments.
// Shared memory holds two 3 x (M + 2) input patches (a segment's rows
// y-1..y+1 with the circular halo) and the weights of all nine taps, both in the K-major canonical layout without swizzle: 8 x 16 B
// core matrices, an operand's 8-row groups 128 B apart (SBO) and its 8-column
// k-groups one "plane" apart (LBO).  For tap (ky, kx) the A operand is simply
// the patch row ky starting at column kx, so each tap is a plain descriptor
// offset and no im2col copy exists.  One thread issues the 9 x cin/16
// tcgen05.mma (M = 128, N = NT, K = 16) into one TMEM accumulator and commits
// them to an mbarrier; each warp then reads its 32 TMEM lanes (pixels) and
// runs the same epilogues as the mma.sync kernel (bias + ReLU (+ skip) to
// bfloat16, raw FP32, residual output in field layout).
//
// Output channels beyond N = 64 are split over CTAs (blockIdx.y takes channels
// [64 y, 64 y + 64)).  Inputs of 128 channels (the encoder's last level and
// the decoder's first layer) do not fit twice in shared memory: their kernel
// keeps all nine taps of the CTA's weights and two patches of 32 channels, and
// runs each work unit as four passes over the channel quarters into the same
// accumulator, loading the next quarter while the tensor cores multiply the
// current one.
//
// Every wait is bounded; on a timeout the kernel flags it in the status word,
// frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "nn_internal.h"

namespace pic {
namespace nn {

namespace {

using bf16 = __nv_bfloat16;

constexpr int TC_M = 128;             // pixels of one row segment (MMA M)
constexpr int TC_R = 2;               // rows per work unit: one accumulator each
constexpr int TC_THREADS = 256;       // 8 warps: two per 32 TMEM lanes (column halves)
constexpr int TC_PW = TC_M + 2;       // patch row length (halo)
constexpr int TC_PR = TC_R + 2;       // patch rows

__device__ __forceinline__ uint32_t saddr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr(sdst)), "l"(gsrc)
                 : "memory");
}
__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// shared-memory matrix descriptor: K-major, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo & 0x3FFFF) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFF) >> 4) << 32) | ((uint64_t)1 << 46);
}

template <int CIN, int NT>
struct TcSmem {
    static constexpr int KG = CIN / 8;                        // k-groups
    static constexpr int PPLANE = TC_PR * TC_PW * 16;         // bytes of one k-group of a patch
    static constexpr int PATCH = KG * PPLANE;                 // bytes of one patch
    static constexpr int WPLANE = NT * 16;                    // bytes of one k-group of one tap
    static constexpr int WTAP = KG * WPLANE;
    static constexpr size_t off_w = 2 * (size_t)PATCH;        // two patches, then the weights
    static constexpr size_t off_bias = off_w + 9 * WTAP;       // NT floats
    static constexpr size_t off_bar = (off_bias + NT * 4 + 15) & ~(size_t)15;
    static constexpr size_t bytes = off_bar + 32;             // 2 mbarriers + TMEM slot
    static constexpr int NTC = NT < 32 ? 32 : NT;             // TMEM columns of one row's accumulator
    static constexpr int TMEM_COLS = 2 * TC_R * NTC;          // two work units in flight
};

// The channel-pass kernel: two patches of KC channels, then all CIN channels
// of the nine taps' weights.
template <int CIN, int NT, int KC>
struct TcSmemKC {
    static constexpr int KG = CIN / 8;                        // k-groups of the weights
    static constexpr int KGC = KC / 8;                        // k-groups of one patch
    static constexpr int PPLANE = TC_PR * TC_PW * 16;
    static constexpr int PATCH = KGC * PPLANE;
    static constexpr int WPLANE = NT * 16;
    static constexpr int WTAP = KG * WPLANE;
    static constexpr size_t off_w = 2 * (size_t)PATCH;
    static constexpr size_t off_bias = off_w + 9 * (size_t)WTAP;
    static constexpr size_t off_bar = (off_bias + NT * 4 + 15) & ~(size_t)15;
    static constexpr size_t bytes = off_bar + 32;             // 2 mbarriers + TMEM slot
    static constexpr int NTC = NT < 32 ? 32 : NT;
    static constexpr int TMEM_COLS = 2 * TC_R * NTC;
};

// wait for phase `parity` of an mbarrier, about a second at most
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, q;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > 2000000000LL) return false;
        __nanosleep(64);
    }
}

// patch of work unit `seg` (rows y0-1..y0+R, columns x0-1..x0+M, circular)
// into k-group planes of 16 B per pixel; a thread takes whole pixels (their
// CIN channels are contiguous in memory)
// KGP k-groups per patch plane set, starting at input channel c0 (the
// two-pass kernel loads one channel half at a time)
template <int CIN, int KGP, int PPLANE>
__device__ __forceinline__ void load_patch_ch(const ConvParams& p, unsigned char* sP, int seg,
                                              int c0, int tid) {
    const int segs = p.W / TC_M, rows = p.H / TC_R;
    const int x0 = (seg % segs) * TC_M;
    const int y0 = ((seg / segs) % rows) * TC_R;
    const int b = seg / (segs * rows);
    const int sh = p.up ? 1 : 0;
    const int Hi = p.H >> sh, Wi = p.W >> sh;
    for (int pix = tid; pix < TC_PR * TC_PW; pix += TC_THREADS) {
        const int r = pix / TC_PW, q = pix - r * TC_PW;
        const int ys = wrap(y0 - 1 + r, p.H) >> sh, xs = wrap(x0 - 1 + q, p.W) >> sh;
        const bf16* src = p.x + (((size_t)b * Hi + ys) * Wi + xs) * CIN + c0;
        unsigned char* dst = sP + pix * 16;
#pragma unroll
        for (int kg = 0; kg < KGP; ++kg) cp_async16(dst + kg * PPLANE, src + kg * 8);
    }
}

template <int CIN, int NT>
__device__ __forceinline__ void load_patch(const ConvParams& p, unsigned char* sP, int seg, int tid) {
    using L = TcSmem<CIN, NT>;
    const int segs = p.W / TC_M, rows = p.H / TC_R;
    const int x0 = (seg % segs) * TC_M;
    const int y0 = ((seg / segs) % rows) * TC_R;
    const int b = seg / (segs * rows);
    const int sh = p.up ? 1 : 0;
    const int Hi = p.H >> sh, Wi = p.W >> sh;
    for (int pix = tid; pix < TC_PR * TC_PW; pix += TC_THREADS) {
        const int r = pix / TC_PW, q = pix - r * TC_PW;
        const int ys = wrap(y0 - 1 + r, p.H) >> sh, xs = wrap(x0 - 1 + q, p.W) >> sh;
        const bf16* src = p.x + (((size_t)b * Hi + ys) * Wi + xs) * CIN;
        unsigned char* dst = sP + pix * 16;
#pragma unroll
        for (int kg = 0; kg < L::KG; ++kg) cp_async16(dst + kg * L::PPLANE, src + kg * 8);
    }
}

// the epilogues on one accumulator (row rr of unit seg): TMEM lane = pixel
// x0 + lane of the row, column = output channel
template <int NT>
__device__ __forceinline__ void epilogue(const ConvParams& p, const float* sBias, uint32_t acc,
                                         int seg, int rr, int warp, int lane, int co0) {
    // warps w and w + 4 read TMEM lanes 32 (w % 4)..+31: the first and the
    // second half of the 16-column chunks
    const int lg = warp & 3, half = warp >> 2;
    const int segs = p.W / TC_M, rows = p.H / TC_R;
    const int x = (seg % segs) * TC_M + 32 * lg + lane;
    const int y = ((seg / segs) % rows) * TC_R + rr;
    const int b = seg / (segs * rows);
    const size_t pix = ((size_t)b * p.H + y) * p.W + x;
#pragma unroll 1
    for (int c0 = 16 * half; c0 < NT; c0 += 32) {
        uint32_t r[16];
        const uint32_t taddr = acc + ((uint32_t)(32 * lg) << 16) + c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
            "%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
              "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
              "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (co0 + c0 >= p.cout_pad) continue;
        const int cg = co0 + c0;  // output channel of column c0
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
        if (p.epi == EPI_GRAD) {
            float4* o = reinterpret_cast<float4*>(p.g_out + pix * p.cout_pad + cg);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                o[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
            continue;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] += sBias[c0 + j];  // zero past cout and without bias
        if (p.epi == EPI_FINAL) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int c = cg + j;
                if (c >= p.cout) continue;
                const size_t o = (size_t)b * p.bstride + (size_t)c * p.cstride + p.offset +
                                 (size_t)y * p.pitch + x;
                p.fout[o] = p.res[o] * p.rs + v[j] * p.os;
            }
            continue;
        }
        if (p.relu) {
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j], 0.f);
        }
        __align__(16) __nv_bfloat162 a2[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) a2[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
        uint4* ao = reinterpret_cast<uint4*>(p.a_out + pix * p.cout_pad + cg);
        ao[0] = reinterpret_cast<const uint4*>(a2)[0];
        ao[1] = reinterpret_cast<const uint4*>(a2)[1];
        if (p.skip) {
            const uint4* sk = reinterpret_cast<const uint4*>(p.skip + pix * p.cout_pad + cg);
            __align__(16) uint4 sv[2] = {sk[0], sk[1]};
            const __nv_bfloat162* s2 = reinterpret_cast<const __nv_bfloat162*>(sv);
            __align__(16) __nv_bfloat162 y2[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float2 af = __bfloat1622float2(a2[j]), sf = __bfloat1622float2(s2[j]);
                y2[j] = __floats2bfloat162_rn(af.x + sf.x, af.y + sf.y);
            }
            uint4* yo = reinterpret_cast<uint4*>(p.y_out + pix * p.cout_pad + cg);
            yo[0] = reinterpret_cast<const uint4*>(y2)[0];
            yo[1] = reinterpret_cast<const uint4*>(y2)[1];
        }
    }
}

// Persistent: the CTA keeps the nine taps' weights in shared memory and runs
// through segments blockIdx.x, blockIdx.x + gridDim.x, ...  Two patches and
// two TMEM accumulators: while the tensor cores work on segment i, the CTA
// stores segment i-1's results and loads segment i+1's patch.
template <int CIN, int NT>
__global__ void __launch_bounds__(TC_THREADS) k_conv_tc(const ConvParams p) {
    using L = TcSmem<CIN, NT>;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sW = smem + L::off_w;
    float* sBias = reinterpret_cast<float*>(smem + L::off_bias);
    const uint32_t bar0 = saddr(smem + L::off_bar);           // mbarriers of accumulators 0, 1
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L::off_bar + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nseg = p.B * (p.H / TC_R) * (p.W / TC_M);
    if ((int)blockIdx.x >= nseg) return;
    const int co0 = blockIdx.y * NT;  // the CTA's output channels

    // weights of the nine taps: packed [tap][cout_pad][CIN] -> [tap][kg][n][8]
    for (int i = tid; i < 9 * NT * L::KG; i += TC_THREADS) {
        const int kg = i % L::KG;
        const int rn = i / L::KG;
        const int n = rn % NT, tap = rn / NT;
        unsigned char* dst = sW + tap * L::WTAP + kg * L::WPLANE + n * 16;
        if (co0 + n < p.cout_pad)
            cp_async16(dst, p.w + ((size_t)tap * p.cout_pad + co0 + n) * CIN + kg * 8);
        else
            *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
    }
    for (int c = tid; c < NT; c += TC_THREADS)
        sBias[c] = (p.bias && co0 + c < p.cout && p.epi != EPI_GRAD) ? p.bias[co0 + c] : 0.f;
    pdl_wait();  // the input is the previous kernel's output
    pdl_trigger();
    load_patch<CIN, NT>(p, smem, blockIdx.x, tid);
    asm volatile("cp.async.commit_group;" ::: "memory");
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         saddr(tslot)),
                     "r"(L::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    // D f32 (bits 4-5), A and B bf16 (7-9, 10-12), both K-major, N >> 3 at 17, M >> 4 at 24
    constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) |
                               ((uint32_t)(TC_M >> 4) << 24);
    bool ok = true;
    int i = 0, prev = -1;
    for (int seg = blockIdx.x; seg < nseg; seg += gridDim.x, ++i) {
        const int buf = i & 1;
        // this segment's patch (and, the first time, the weights) has landed
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint32_t pa = saddr(smem + buf * L::PATCH), pw = saddr(sW);
#pragma unroll 1
            for (int tap = 0; tap < 9; ++tap) {
                const int ky = tap / 3, kx = tap - 3 * (tap / 3);
#pragma unroll
                for (int kc = 0; kc < CIN / 16; ++kc) {
                    const uint64_t bd =
                        smem_desc(pw + tap * L::WTAP + (2 * kc) * L::WPLANE, L::WPLANE, 128);
                    const uint32_t accum = (tap | kc) != 0;
#pragma unroll
                    for (int rr = 0; rr < TC_R; ++rr) {
                        const uint32_t acc = tmem + (buf * TC_R + rr) * L::NTC;
                        const uint64_t ad = smem_desc(
                            pa + (2 * kc) * L::PPLANE + ((rr + ky) * TC_PW + kx) * 16, L::PPLANE, 128);
                        asm volatile(
                            "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n\t}" ::"r"(acc),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                    }
                }
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    bar0 + 8 * buf));
        }
        // once the previous unit's products are complete, its patch buffer
        // takes the next unit's patch, and its results are stored while the
        // tensor cores run this unit
        if (prev >= 0) {
            const int pb = (i - 1) & 1;
            if (ok && !wait_bar(bar0 + 8 * pb, ((i - 1) >> 1) & 1)) ok = false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
        const int nxt = seg + gridDim.x;
        if (nxt < nseg) load_patch<CIN, NT>(p, smem + (buf ^ 1) * L::PATCH, nxt, tid);
        asm volatile("cp.async.commit_group;" ::: "memory");
        if (prev >= 0 && ok) {
            const int pb = (i - 1) & 1;
            for (int rr = 0; rr < TC_R; ++rr)
                epilogue<NT>(p, sBias, tmem + (pb * TC_R + rr) * L::NTC, prev, rr, warp, lane, co0);
        }
        prev = seg;
    }
    if (prev >= 0) {
        const int pb = (i - 1) & 1;
        if (ok && !wait_bar(bar0 + 8 * pb, ((i - 1) >> 1) & 1)) ok = false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (ok)
            for (int rr = 0; rr < TC_R; ++rr)
                epilogue<NT>(p, sBias, tmem + (pb * TC_R + rr) * L::NTC, prev, rr, warp, lane, co0);
    }
    if (!ok && tid == 0) {
        if (p.status) atomicOr(p.status, 2u);  // a bounded wait ran out
        // the products still in flight, once more, before the accumulators
        // are freed: the last commit on each of the two barriers (unit j
        // commits on barrier j & 1, phase (j >> 1) & 1)
        for (int j = i - 1; j >= 0 && j >= i - 2; --j) wait_bar(bar0 + 8 * (j & 1), (j >> 1) & 1);
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(L::TMEM_COLS));
}

// Passes over the input channels (CIN = NCH KC) per work unit: the CTA keeps
// its nine taps' weights of all CIN channels and two patches of KC channels.
// Chunk g (unit g / NCH, channels (g % NCH) KC ...) goes to patch g & 1 and
// its products to the unit's accumulator (unit & 1), committed on mbarrier
// g & 1 (its (g >> 1)-th commit there).  While the tensor cores multiply
// chunk g, the CTA waits for chunk g - 1's products (freeing the other patch,
// and completing the previous unit after its last chunk), loads chunk g + 1
// there and, at a unit's first chunk, stores the previous unit's results.
template <int CIN, int NT, int KC>
__global__ void __launch_bounds__(TC_THREADS) k_conv_tc_kc(const ConvParams p) {
    using L = TcSmemKC<CIN, NT, KC>;
    constexpr int NCH = CIN / KC;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sW = smem + L::off_w;
    float* sBias = reinterpret_cast<float*>(smem + L::off_bias);
    const uint32_t bar0 = saddr(smem + L::off_bar);  // mbarriers of patches 0, 1
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L::off_bar + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nseg = p.B * (p.H / TC_R) * (p.W / TC_M);
    if ((int)blockIdx.x >= nseg) return;
    const int co0 = blockIdx.y * NT;
    // this CTA's units: blockIdx.x, blockIdx.x + gridDim.x, ...
    const int nunit = (nseg - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    const int nchunk = nunit * NCH;
    auto seg_of = [&](int u) { return (int)blockIdx.x + u * (int)gridDim.x; };

    for (int i = tid; i < 9 * NT * L::KG; i += TC_THREADS) {
        const int kg = i % L::KG;
        const int rn = i / L::KG;
        const int n = rn % NT, tap = rn / NT;
        unsigned char* dst = sW + tap * L::WTAP + kg * L::WPLANE + n * 16;
        if (co0 + n < p.cout_pad)
            cp_async16(dst, p.w + ((size_t)tap * p.cout_pad + co0 + n) * CIN + kg * 8);
        else
            *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
    }
    for (int c = tid; c < NT; c += TC_THREADS)
        sBias[c] = (p.bias && co0 + c < p.cout && p.epi != EPI_GRAD) ? p.bias[co0 + c] : 0.f;
    pdl_wait();  // the input is the previous kernel's output
    pdl_trigger();
    load_patch_ch<CIN, L::KGC, L::PPLANE>(p, smem, seg_of(0), 0, tid);
    asm volatile("cp.async.commit_group;" ::: "memory");
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         saddr(tslot)),
                     "r"(L::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) |
                               ((uint32_t)(TC_M >> 4) << 24);
    bool ok = true;
#pragma unroll 1
    for (int g = 0; g < nchunk; ++g) {
        const int u = g / NCH, c = g - u * NCH, pbuf = g & 1;
        // chunk g's patch (and, the first time, the weights) has landed
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint32_t pa = saddr(smem + pbuf * L::PATCH), pw = saddr(sW);
#pragma unroll 1
            for (int tap = 0; tap < 9; ++tap) {
                const int ky = tap / 3, kx = tap - 3 * (tap / 3);
#pragma unroll
                for (int kc = 0; kc < KC / 16; ++kc) {
                    const uint64_t bd = smem_desc(
                        pw + tap * L::WTAP + (c * L::KGC + 2 * kc) * L::WPLANE, L::WPLANE, 128);
                    const uint32_t accum = (c | tap | kc) != 0;
#pragma unroll
                    for (int rr = 0; rr < TC_R; ++rr) {
                        const uint32_t acc = tmem + ((u & 1) * TC_R + rr) * L::NTC;
                        const uint64_t ad = smem_desc(
                            pa + (2 * kc) * L::PPLANE + ((rr + ky) * TC_PW + kx) * 16, L::PPLANE,
                            128);
                        asm volatile(
                            "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n\t}" ::"r"(acc),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                    }
                }
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    bar0 + 8 * pbuf));
        }
        if (g >= 1) {  // chunk g - 1's products: its patch is free, its unit may be complete
            const int gp = g - 1;
            if (ok && !wait_bar(bar0 + 8 * (gp & 1), (gp >> 1) & 1)) ok = false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
        if (g + 1 < nchunk) {
            const int un = (g + 1) / NCH, cn = (g + 1) - un * NCH;
            load_patch_ch<CIN, L::KGC, L::PPLANE>(p, smem + (pbuf ^ 1) * L::PATCH, seg_of(un),
                                                  cn * KC, tid);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        if (c == 0 && u >= 1 && ok)  // unit u - 1 ended with chunk g - 1
            for (int rr = 0; rr < TC_R; ++rr)
                epilogue<NT>(p, sBias, tmem + (((u - 1) & 1) * TC_R + rr) * L::NTC, seg_of(u - 1),
                             rr, warp, lane, co0);
    }
    // the last chunk's products, then the last unit's results
    if (ok && !wait_bar(bar0 + 8 * ((nchunk - 1) & 1), ((nchunk - 1) >> 1) & 1)) ok = false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok)
        for (int rr = 0; rr < TC_R; ++rr)
            epilogue<NT>(p, sBias, tmem + (((nunit - 1) & 1) * TC_R + rr) * L::NTC,
                         seg_of(nunit - 1), rr, warp, lane, co0);
    if (!ok && tid == 0) {
        if (p.status) atomicOr(p.status, 2u);  // a bounded wait ran out
        // the products still in flight, once more, before the accumulators
        // are freed: the last commit on each of the two barriers
        for (int j = nchunk - 1; j >= 0 && j >= nchunk - 2; --j)
            wait_bar(bar0 + 8 * (j & 1), (j >> 1) & 1);
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(L::TMEM_COLS));
}

// Persistent grid size of a shape: CTAs resident at once (shared memory and
// 512 TMEM columns per SM); also raises the shared-memory limit.  Called once
// per shape before any graph capture (init_tc_kernels).
template <int CIN, int NT, int KC>
int& tc_grid_cap() {
    static int cap = 0;
    return cap;
}

// KC == CIN: the one-pass kernel (two patches); KC < CIN: the two-pass one
template <int CIN, int NT, int KC>
struct TcShape {
    static constexpr bool kOnePass = KC == CIN;
    static constexpr size_t bytes = kOnePass ? TcSmem<CIN, NT>::bytes : TcSmemKC<CIN, NT, KC>::bytes;
    static constexpr int tmem_cols = kOnePass ? TcSmem<CIN, NT>::TMEM_COLS : TcSmemKC<CIN, NT, KC>::TMEM_COLS;
    static void (*kernel())(const ConvParams) {
        if constexpr (kOnePass) return k_conv_tc<CIN, NT>;
        else return k_conv_tc_kc<CIN, NT, KC>;
    }
};

template <int CIN, int NT, int KC>
cudaError_t tc_prepare() {
    using S = TcShape<CIN, NT, KC>;
    static_assert(S::bytes <= 227 * 1024, "tcgen05 convolution shape exceeds shared memory");
    if (tc_grid_cap<CIN, NT, KC>()) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(S::kernel(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)S::bytes);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, smem = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    if ((e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) !=
        cudaSuccess)
        return e;
    // resident CTAs: shared memory (plus the 1 KB the system keeps per CTA),
    // TMEM columns, threads
    int per = smem / (int)(S::bytes + 1024);
    per = per < 1 ? 1 : per;
    if (per * S::tmem_cols > 512) per = 512 / S::tmem_cols;
    if (per * TC_THREADS > 2048) per = 2048 / TC_THREADS;
    tc_grid_cap<CIN, NT, KC>() = sms * per;
    return cudaSuccess;
}

// grid: (persistent CTAs over the work units, output-channel tiles of NT)
template <int CIN, int NT, int KC>
cudaError_t conv_tc_T(const ConvParams& p, cudaStream_t s) {
    using S = TcShape<CIN, NT, KC>;
    cudaError_t e = tc_prepare<CIN, NT, KC>();
    if (e != cudaSuccess) return e;
    const int nseg = p.B * (p.H / TC_R) * (p.W / TC_M);
    const int ntile = (p.cout_pad + NT - 1) / NT;
    int gx = tc_grid_cap<CIN, NT, KC>() / ntile;
    gx = gx < 1 ? 1 : (gx > nseg ? nseg : gx);
    return launch_pdl(S::kernel(), dim3(gx, ntile), dim3(TC_THREADS), S::bytes, s, p);
}

}  // namespace

// the (CIN, N, channels per pass) shapes built for the tensor-core path (one
// pass: two patches and nine taps of weights within 227 KB of shared memory;
// CIN = 128: four passes of 32 channels through two patches); output
// channels beyond N = 64 are split over CTAs
#define PIC_TC_SHAPES(X) \
    X(16, 32, 16) X(32, 32, 32) X(32, 64, 32) X(64, 32, 64) X(64, 64, 64) X(32, 16, 32) X(128, 64, 32)

// the N of a launch: the padded output channels rounded up to 16, 32 or 64
// (more than 64: tiles of 64)
static int tc_nt(int cout_pad) {
    return cout_pad <= 16 ? 16 : (cout_pad <= 32 ? 32 : 64);
}

bool conv_tc_supported(const ConvParams& p, int cin) {
    if (p.force_tc < 0 || p.W % TC_M || p.H % TC_R || p.cout_pad > 128) return false;
    // small problems (a few hundred work units) finish sooner on the mma.sync
    // kernel, whose CTAs do not each stage all nine taps of weights
    if ((long long)p.B * (p.H / TC_R) * (p.W / TC_M) < 600 && p.force_tc <= 0) return false;
    const int nt = tc_nt(p.cout_pad);
    // a 16-wide tile (the 3-channel output layer) is faster on the mma.sync
    // kernel (measured on GB300: 66 against 84 us at 1024^2)
    if (nt == 16 && p.force_tc <= 0) return false;
#define PIC_TC_HAS(A, B, C) if (cin == A && nt == B) return true;
    PIC_TC_SHAPES(PIC_TC_HAS)
#undef PIC_TC_HAS
    return false;
}

cudaError_t launch_conv_tc(const ConvParams& p, int cin, cudaStream_t s) {
    const int nt = tc_nt(p.cout_pad);
#define PIC_TC_CASE(A, B, C) \
    if (cin == A && nt == B) return conv_tc_T<A, B, C>(p, s);
    PIC_TC_SHAPES(PIC_TC_CASE)
#undef PIC_TC_CASE
    return cudaErrorInvalidValue;
}

cudaError_t init_tc_kernels() {
    cudaError_t e = cudaSuccess;
#define PIC_TC_PREP(A, B, C) \
    if (e == cudaSuccess) e = tc_prepare<A, B, C>();
    PIC_TC_SHAPES(PIC_TC_PREP)
#undef PIC_TC_PREP
    return e;
}

}  // namespace nn
}  // namespace pic
