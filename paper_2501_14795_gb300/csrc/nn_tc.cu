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
// Beside it: the two layers that read a 2x upsampled input as four 2x2
// convolutions of the coarse grid (k_conv_up_tc), the 3-channel output layer
// with its nine taps in the GEMM's N (k_conv_out_tc), and the weight
// gradients (k_wgrad_tc, k_wgrad_tcn), each described where it is defined.
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
// (b, y, x): the output pixel of this thread's TMEM lane
template <int NT>
__device__ __forceinline__ void epilogue_at(const ConvParams& p, const float* sBias, uint32_t acc,
                                            int b, int y, int x, int warp, int lane, int co0) {
    // warps w and w + 4 read TMEM lanes 32 (w % 4)..+31: the first and the
    // second half of the 16-column chunks
    const int lg = warp & 3, half = warp >> 2;
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
        if (p.a_out) {
            uint4* ao = reinterpret_cast<uint4*>(p.a_out + pix * p.cout_pad + cg);
            ao[0] = reinterpret_cast<const uint4*>(a2)[0];
            ao[1] = reinterpret_cast<const uint4*>(a2)[1];
        }
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

// row rr of work unit seg (TC_R rows of TC_M pixels): lane = pixel x0 + lane
template <int NT>
__device__ __forceinline__ void epilogue(const ConvParams& p, const float* sBias, uint32_t acc,
                                         int seg, int rr, int warp, int lane, int co0) {
    const int segs = p.W / TC_M, rows = p.H / TC_R;
    const int x = (seg % segs) * TC_M + 32 * (warp & 3) + lane;
    const int y = ((seg / segs) % rows) * TC_R + rr;
    const int b = seg / (segs * rows);
    epilogue_at<NT>(p, sBias, acc, b, y, x, warp, lane, co0);
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
            ok = __all_sync(0xffffffffu, ok);  // the warp's TMEM loads are collective
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
        ok = __all_sync(0xffffffffu, ok);
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
            ok = __all_sync(0xffffffffu, ok);  // the warp's TMEM loads are collective
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
    ok = __all_sync(0xffffffffu, ok);
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

// ------------------------------------------- convolution of a 2x upsampled input
// A 3x3 convolution of the nearest-neighbour 2x upsampling of x is, for each
// parity (a, b) of the output pixel (2i + a, 2j + b), a 2x2 convolution of x
// itself: output row offsets dy -1, 0, 1 land on x rows i + floor((a + dy) / 2),
// so the taps that land on the same x pixel add their weights
// (a = 0: dy = -1 -> i - 1, dy = 0, 1 -> i; a = 1: dy = -1, 0 -> i, dy = 1 ->
// i + 1; the same for columns).  Sixteen combined taps (four parities x 2x2,
// summed in FP32 from the master weights, then rounded to bfloat16 once)
// replace nine taps on a grid four times larger: 4/9 of the products.  A work
// unit is a row segment of 128 x pixels (row i, columns j0 ..); its patch is
// x rows i - 1 .. i + 1, columns j0 - 1 .. j0 + 128, and it has four
// accumulators, one per parity, whose lanes m are the output pixels
// (2i + a, 2 (j0 + m) + b).  Otherwise as k_conv_tc: persistent, weights
// resident, two patches and two sets of accumulators in flight.
constexpr int UP_PR = 3;                 // patch rows
constexpr int UP_PW = TC_M + 2;          // patch columns

template <int CIN, int NT, int KC>
struct UpSmem {
    static constexpr int KG = CIN / 8;      // k-groups of the weights
    static constexpr int KGC = KC / 8;      // k-groups of one patch (one pass over KC channels)
    static constexpr int PPLANE = UP_PR * UP_PW * 16;
    static constexpr int PATCH = KGC * PPLANE;
    static constexpr int WPLANE = NT * 16;
    static constexpr int WTAP = KG * WPLANE;
    static constexpr size_t off_w = 2 * (size_t)PATCH;
    static constexpr size_t off_bias = off_w + 16 * (size_t)WTAP;
    static constexpr size_t off_bar = (off_bias + NT * 4 + 15) & ~(size_t)15;
    static constexpr size_t bytes = off_bar + 32;
    static constexpr int NTC = NT < 32 ? 32 : NT;
    static constexpr int TMEM_COLS = 2 * 4 * NTC;   // two units of four parities
    static_assert(bytes <= 227 * 1024 && TMEM_COLS <= 512, "upsampling tile does not fit");
};

// channels c0 .. c0 + KC - 1 of unit seg's patch
template <int CIN, int NT, int KC>
__device__ __forceinline__ void load_patch_up(const ConvParams& p, unsigned char* sP, int seg,
                                              int c0, int tid) {
    using L = UpSmem<CIN, NT, KC>;
    const int Hi = p.H >> 1, Wi = p.W >> 1;
    const int segs = Wi / TC_M;
    const int j0 = (seg % segs) * TC_M;
    const int i = (seg / segs) % Hi;
    const int b = seg / (segs * Hi);
    for (int pix = tid; pix < UP_PR * UP_PW; pix += TC_THREADS) {
        const int r = pix / UP_PW, q = pix - r * UP_PW;
        const int ys = wrap(i - 1 + r, Hi), xs = wrap(j0 - 1 + q, Wi);
        const bf16* src = p.x + (((size_t)b * Hi + ys) * Wi + xs) * CIN + c0;
        unsigned char* dst = sP + pix * 16;
#pragma unroll
        for (int kg = 0; kg < L::KGC; ++kg) cp_async16(dst + kg * L::PPLANE, src + kg * 8);
    }
}

// the four parities' results of unit seg (accumulators acc0 + parity NTC):
// bf16(relu(z + bias)) and, with a skip, bf16(a + skip).  The skip values
// and the four accumulators' columns are all requested before the first
// store, so their latencies overlap instead of adding up per parity.
template <int NTC, int NT>
__device__ __forceinline__ void epilogue_up(const ConvParams& p, const float* sBias, uint32_t acc0,
                                            int seg, int warp, int lane, int co0) {
    const int Hi = p.H >> 1, Wi = p.W >> 1;
    const int segs = Wi / TC_M;
    const int lg = warp & 3, half = warp >> 2;
    const int j = (seg % segs) * TC_M + 32 * lg + lane;
    const int i = (seg / segs) % Hi;
    const int b = seg / (segs * Hi);
#pragma unroll 1
    for (int c0 = 16 * half; c0 < NT; c0 += 32) {
        if (co0 + c0 >= p.cout_pad) continue;  // uniform over the warp
        const int cg = co0 + c0;
        size_t pix[4];
#pragma unroll
        for (int ph = 0; ph < 4; ++ph)
            pix[ph] = ((size_t)b * p.H + 2 * i + (ph >> 1)) * p.W + 2 * j + (ph & 1);
        uint4 sk[4][2];
        if (p.skip) {
#pragma unroll
            for (int ph = 0; ph < 4; ++ph) {
                const uint4* src = reinterpret_cast<const uint4*>(p.skip + pix[ph] * p.cout_pad + cg);
                sk[ph][0] = src[0];
                sk[ph][1] = src[1];
            }
        }
        uint32_t r[4][16];
#pragma unroll
        for (int ph = 0; ph < 4; ++ph) {
            const uint32_t taddr = acc0 + ph * NTC + ((uint32_t)(32 * lg) << 16) + c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
                "%12,%13,%14,%15}, [%16];"
                : "=r"(r[ph][0]), "=r"(r[ph][1]), "=r"(r[ph][2]), "=r"(r[ph][3]), "=r"(r[ph][4]),
                  "=r"(r[ph][5]), "=r"(r[ph][6]), "=r"(r[ph][7]), "=r"(r[ph][8]), "=r"(r[ph][9]),
                  "=r"(r[ph][10]), "=r"(r[ph][11]), "=r"(r[ph][12]), "=r"(r[ph][13]),
                  "=r"(r[ph][14]), "=r"(r[ph][15])
                : "r"(taddr));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int ph = 0; ph < 4; ++ph) {
            float v[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                v[q] = __uint_as_float(r[ph][q]) + sBias[c0 + q];
                if (p.relu) v[q] = fmaxf(v[q], 0.f);
            }
            __align__(16) __nv_bfloat162 a2[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) a2[q] = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
            if (p.a_out) {
                uint4* ao = reinterpret_cast<uint4*>(p.a_out + pix[ph] * p.cout_pad + cg);
                ao[0] = reinterpret_cast<const uint4*>(a2)[0];
                ao[1] = reinterpret_cast<const uint4*>(a2)[1];
            }
            if (p.skip) {
                const __nv_bfloat162* s2 = reinterpret_cast<const __nv_bfloat162*>(sk[ph]);
                __align__(16) __nv_bfloat162 y2[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float2 af = __bfloat1622float2(a2[q]), sf = __bfloat1622float2(s2[q]);
                    y2[q] = __floats2bfloat162_rn(af.x + sf.x, af.y + sf.y);
                }
                uint4* yo = reinterpret_cast<uint4*>(p.y_out + pix[ph] * p.cout_pad + cg);
                yo[0] = reinterpret_cast<const uint4*>(y2)[0];
                yo[1] = reinterpret_cast<const uint4*>(y2)[1];
            }
        }
    }
}

// p.wp: the sixteen combined taps, packed [parity][u][v][cout_pad][CIN].
// Passes of KC input channels (CIN / KC per unit) through two patches, as in
// k_conv_tc_kc: chunk g (unit g / NCH, channels (g % NCH) KC ...) goes to
// patch g & 1, its products to the unit's four accumulators (unit & 1),
// committed on mbarrier g & 1; while the tensor cores multiply chunk g the
// CTA waits for chunk g - 1, loads chunk g + 1 and, at a unit's first chunk,
// stores the previous unit's results.
template <int CIN, int NT, int KC>
__global__ void __launch_bounds__(TC_THREADS) k_conv_up_tc(const ConvParams p) {
    using L = UpSmem<CIN, NT, KC>;
    constexpr int NCH = CIN / KC;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sW = smem + L::off_w;
    float* sBias = reinterpret_cast<float*>(smem + L::off_bias);
    const uint32_t bar0 = saddr(smem + L::off_bar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L::off_bar + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nseg = p.B * (p.H >> 1) * ((p.W >> 1) / TC_M);
    if ((int)blockIdx.x >= nseg) return;
    const int co0 = blockIdx.y * NT;
    const int nunit = (nseg - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    const int nchunk = nunit * NCH;
    auto seg_of = [&](int u) { return (int)blockIdx.x + u * (int)gridDim.x; };
    for (int idx = tid; idx < 16 * NT * L::KG; idx += TC_THREADS) {
        const int kg = idx % L::KG;
        const int rn = idx / L::KG;
        const int n = rn % NT, tap = rn / NT;
        unsigned char* dst = sW + tap * L::WTAP + kg * L::WPLANE + n * 16;
        if (co0 + n < p.cout_pad)
            cp_async16(dst, p.wp + ((size_t)tap * p.cout_pad + co0 + n) * CIN + kg * 8);
        else
            *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
    }
    for (int c = tid; c < NT; c += TC_THREADS)
        sBias[c] = (p.bias && co0 + c < p.cout) ? p.bias[co0 + c] : 0.f;
    pdl_wait();
    pdl_trigger();
    load_patch_up<CIN, NT, KC>(p, smem, seg_of(0), 0, tid);
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
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint32_t pa = saddr(smem + pbuf * L::PATCH), pw = saddr(sW);
#pragma unroll 1
            for (int ph = 0; ph < 4; ++ph) {
                const int a = ph >> 1, bp = ph & 1;
                const uint32_t acc = tmem + ((u & 1) * 4 + ph) * L::NTC;
#pragma unroll
                for (int t4 = 0; t4 < 4; ++t4) {
                    // patch row 1 + u, column 1 + v (u, v = offsets of the x pixel)
                    const int du = a - 1 + (t4 >> 1), dv = bp - 1 + (t4 & 1);
                    const int tap = ph * 4 + t4;
#pragma unroll
                    for (int kc = 0; kc < KC / 16; ++kc) {
                        const uint64_t bd = smem_desc(
                            pw + tap * L::WTAP + (c * L::KGC + 2 * kc) * L::WPLANE, L::WPLANE, 128);
                        const uint64_t ad = smem_desc(
                            pa + (2 * kc) * L::PPLANE + ((1 + du) * UP_PW + 1 + dv) * 16, L::PPLANE,
                            128);
                        const uint32_t accum = (c | t4 | kc) != 0;
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
            ok = __all_sync(0xffffffffu, ok);  // the warp's TMEM loads are collective
        }
        if (g + 1 < nchunk) {
            const int un = (g + 1) / NCH, cn = (g + 1) - un * NCH;
            load_patch_up<CIN, NT, KC>(p, smem + (pbuf ^ 1) * L::PATCH, seg_of(un), cn * KC, tid);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        if (c == 0 && u >= 1 && ok)  // unit u - 1 ended with chunk g - 1
            epilogue_up<L::NTC, NT>(p, sBias, tmem + ((u - 1) & 1) * 4 * L::NTC, seg_of(u - 1),
                                    warp, lane, co0);
    }
    if (ok && !wait_bar(bar0 + 8 * ((nchunk - 1) & 1), ((nchunk - 1) >> 1) & 1)) ok = false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    ok = __all_sync(0xffffffffu, ok);
    if (ok)
        epilogue_up<L::NTC, NT>(p, sBias, tmem + ((nunit - 1) & 1) * 4 * L::NTC,
                                seg_of(nunit - 1), warp, lane, co0);
    if (!ok && tid == 0) {
        if (p.status) atomicOr(p.status, 2u);
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

template <int CIN, int NT, int KC>
int& up_grid_cap() {
    static int cap = 0;
    return cap;
}

// the attribute and the grid cap (one CTA per SM: the patches and sixteen taps
// take most of the shared memory), once per shape before any graph capture
template <int CIN, int NT, int KC>
cudaError_t up_prepare() {
    using L = UpSmem<CIN, NT, KC>;
    if (up_grid_cap<CIN, NT, KC>()) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_conv_up_tc<CIN, NT, KC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, smem = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    if ((e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) !=
        cudaSuccess)
        return e;
    int per = smem / (int)(L::bytes + 1024);
    per = per < 1 ? 1 : per;
    if (per * L::TMEM_COLS > 512) per = 512 / L::TMEM_COLS;
    up_grid_cap<CIN, NT, KC>() = sms * per;
    return cudaSuccess;
}

template <int CIN, int NT, int KC>
cudaError_t conv_up_tc_T(const ConvParams& p, cudaStream_t s) {
    using L = UpSmem<CIN, NT, KC>;
    cudaError_t e = up_prepare<CIN, NT, KC>();
    if (e != cudaSuccess) return e;
    const int nseg = p.B * (p.H >> 1) * ((p.W >> 1) / TC_M);
    const int ntile = (p.cout_pad + NT - 1) / NT;
    int gx = up_grid_cap<CIN, NT, KC>() / ntile;
    gx = gx < 1 ? 1 : (gx > nseg ? nseg : gx);
    return launch_pdl(k_conv_up_tc<CIN, NT, KC>, dim3(gx, ntile), dim3(TC_THREADS), L::bytes, s,
                      p);
}

// ------------------------------------------------- the output layer (32 -> 3)
// out[y][x][co] = sum over taps (ky, kx) and ci of a[y + ky - 1][x + kx - 1][ci]
// w[ky][kx][ci][co].  With three outputs, the nine-tap GEMM has N = 3 and
// every MMA reads a 128-pixel operand for almost nothing; here the taps go
// into N instead: per input row r, one GEMM gives D_r[pixel][(tap, co)] =
// sum over ci of a[r][pixel][ci] w[tap][ci][co] (27 of 32 columns), and the
// epilogue adds, for output pixel x of row y, D_{y+ky-1}[x + kx - 1][(ky, kx,
// co)] over the nine taps.  A work unit is OT_R output rows by 126 output
// columns: its patch is the OT_R + 2 input rows around them and the 128 input
// pixels x0 - 1 .. x0 + 126 (TMEM lane m = pixel x0 - 1 + m, circular), one
// accumulator of 32 columns per input row.  In the epilogue each lane sums
// its pixel's centre, left-tap and right-tap contributions over ky; the
// output at lane m takes the centre of m, the left-tap sum of m - 1 and the
// right-tap sum of m + 1 (warp shuffles, across warps through shared memory).
constexpr int OT_R = 4;                  // output rows per unit (even; 2 measured slower)
constexpr int OT_DR = OT_R + 2;          // input rows (TMEM accumulators)
constexpr int OT_P = TC_M - 2;           // output columns per unit
constexpr int OT_N = 32;                 // GEMM columns: 9 taps x 3 outputs, padded

struct OutSmem {
    static constexpr int CIN = 32, KG = CIN / 8;
    static constexpr int PPLANE = OT_DR * TC_M * 16;   // one k-group of the patch
    static constexpr int PATCH = KG * PPLANE;
    static constexpr int WPLANE = OT_N * 16;
    static constexpr size_t off_w = 2 * (size_t)PATCH;
    static constexpr size_t off_x = off_w + KG * WPLANE;           // edge exchange
    static constexpr size_t off_bar = off_x + 2 * 2 * 4 * 3 * 4;    // [row slot][side][quarter][co]
    static constexpr size_t bytes = off_bar + 16;
    static constexpr int TMEM_COLS = OT_DR * OT_N <= 128 ? 128 : (OT_DR * OT_N <= 256 ? 256 : 512);
};

__device__ __forceinline__ void load_patch_out(const ConvParams& p, unsigned char* sP, int unit,
                                               int tid) {
    using L = OutSmem;
    const int segs = (p.W + OT_P - 1) / OT_P, bands = p.H / OT_R;
    const int x0 = (unit % segs) * OT_P;
    const int y0 = ((unit / segs) % bands) * OT_R;
    const int b = unit / (segs * bands);
    // consecutive threads take consecutive 16-byte pieces of a pixel's 64 bytes
    for (int i = tid; i < OT_DR * TC_M * L::KG; i += TC_THREADS) {
        const int kg = i % L::KG, pix = i / L::KG;
        const int r = pix / TC_M, m = pix - r * TC_M;
        const int ys = wrap(y0 - 1 + r, p.H);
        int xs = x0 - 1 + m;
        xs = xs < 0 ? xs + p.W : (xs >= p.W ? xs - p.W : xs);
        if (xs >= p.W) xs -= p.W;  // the last unit's lanes past the right edge wrap again
        cp_async16(sP + kg * L::PPLANE + pix * 16,
                   p.x + (((size_t)b * p.H + ys) * p.W + xs) * L::CIN + kg * 8);
    }
}

// p.w: the layer's forward packing [9][cout_pad][32]; EPI_FINAL only
// two CTAs per SM (TMEM 2 x 256 columns): up to 128 registers a thread
__global__ void __launch_bounds__(TC_THREADS, 2) k_conv_out_tc(const ConvParams p) {
    using L = OutSmem;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sW = smem + L::off_w;
    float* sX = reinterpret_cast<float*>(smem + L::off_x);
    const uint32_t bar = saddr(smem + L::off_bar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L::off_bar + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int segs = (p.W + OT_P - 1) / OT_P, bands = p.H / OT_R;
    const int nunit = p.B * bands * segs;
    if ((int)blockIdx.x >= nunit) return;
    // B: row n = tap 3 + co of the GEMM (zero past the real outputs), k-group kg
    for (int i = tid; i < OT_N * L::KG; i += TC_THREADS) {
        const int n = i / L::KG, kg = i - n * L::KG;
        const int tap = n / 3, co = n - 3 * tap;
        unsigned char* dst = sW + kg * L::WPLANE + n * 16;
        if (tap < 9 && co < p.cout)
            cp_async16(dst, p.w + ((size_t)tap * p.cout_pad + co) * L::CIN + kg * 8);
        else
            *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
    }
    float bias[3];
#pragma unroll
    for (int co = 0; co < 3; ++co) bias[co] = (p.bias && co < p.cout) ? p.bias[co] : 0.f;
    pdl_wait();
    pdl_trigger();
    load_patch_out(p, smem, blockIdx.x, tid);
    asm volatile("cp.async.commit_group;" ::: "memory");
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
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
    constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OT_N >> 3) << 17) |
                               ((uint32_t)(TC_M >> 4) << 24);
    const int lq = warp & 3, half = warp >> 2;
    const int m = 32 * lq + lane;  // TMEM lane: input pixel x0 - 1 + m
    bool ok = true;
    int it = 0;
#pragma unroll 1
    for (int unit = blockIdx.x; unit < nunit; unit += gridDim.x, ++it) {
        const int buf = it & 1;
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint32_t pa = saddr(smem + buf * L::PATCH), pw = saddr(sW);
#pragma unroll
            for (int r = 0; r < OT_DR; ++r)
#pragma unroll
                for (int kc = 0; kc < L::CIN / 16; ++kc) {
                    const uint64_t bd = smem_desc(pw + (2 * kc) * L::WPLANE, L::WPLANE, 128);
                    const uint64_t ad =
                        smem_desc(pa + (2 * kc) * L::PPLANE + r * TC_M * 16, L::PPLANE, 128);
                    const uint32_t accum = kc != 0;
                    asm volatile(
                        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n\t}" ::"r"(
                            tmem + r * OT_N),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    bar));
        }
        // the next unit's patch into the other buffer (its products were read
        // before the previous unit's epilogue ended)
        const int nxt = unit + gridDim.x;
        if (nxt < nunit) load_patch_out(p, smem + (buf ^ 1) * L::PATCH, nxt, tid);
        asm volatile("cp.async.commit_group;" ::: "memory");
        const int x0 = (unit % segs) * OT_P;
        const int y0 = ((unit / segs) % bands) * OT_R;
        const int b = unit / (segs * bands);
        const int x = x0 - 1 + m;
        const bool mine = m >= 1 && m <= OT_P && x < p.W;  // this lane's output column
        // the residual of this lane's two output pixels, requested before the wait
        float res[OT_R / 2][3];
#pragma unroll
        for (int round = 0; round < OT_R / 2; ++round)
#pragma unroll
            for (int co = 0; co < 3; ++co) {
                res[round][co] = 0.f;
                if (mine && co < p.cout)
                    res[round][co] = p.res[(size_t)b * p.bstride + (size_t)co * p.cstride + p.offset +
                                           (size_t)(y0 + half + 2 * round) * p.pitch + x];
            }
        if (ok && !wait_bar(bar, it & 1)) ok = false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int okall = __syncthreads_and(ok);
        if (!okall) {
            ok = false;
            break;
        }
        // OT_R / 2 rounds: warps 0-3 the even output rows, warps 4-7 the odd ones
#pragma unroll
        for (int round = 0; round < OT_R / 2; ++round) {
            const int o = half + 2 * round;
            float C[3] = {0.f, 0.f, 0.f}, Lt[3] = {0.f, 0.f, 0.f}, Rt[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) {
                uint32_t v[32];
                const uint32_t taddr = tmem + ((uint32_t)(32 * lq) << 16) + (uint32_t)((o + ky) * OT_N);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
                    "%12,%13,%14,%15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                      "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                      "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                    : "r"(taddr));
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
                    "%12,%13,%14,%15}, [%16];"
                    : "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                      "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
                      "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(taddr + 16));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int co = 0; co < 3; ++co) {
                    Lt[co] += __uint_as_float(v[(3 * ky + 0) * 3 + co]);  // kx = 0: feeds x + 1
                    C[co] += __uint_as_float(v[(3 * ky + 1) * 3 + co]);
                    Rt[co] += __uint_as_float(v[(3 * ky + 2) * 3 + co]);  // kx = 2: feeds x - 1
                }
            }
            // the warp's edge lanes hand their sums to the neighbouring quarters
            float* xs = sX + (half * 2) * 4 * 3;  // [side][quarter][co] of this row slot
            if (lane == 31)
#pragma unroll
                for (int co = 0; co < 3; ++co) xs[(0 * 4 + lq) * 3 + co] = Lt[co];
            if (lane == 0)
#pragma unroll
                for (int co = 0; co < 3; ++co) xs[(1 * 4 + lq) * 3 + co] = Rt[co];
            __syncthreads();
            float out[3];
#pragma unroll
            for (int co = 0; co < 3; ++co) {
                float left = __shfl_up_sync(0xffffffffu, Lt[co], 1);
                float right = __shfl_down_sync(0xffffffffu, Rt[co], 1);
                if (lane == 0) left = lq > 0 ? xs[(0 * 4 + lq - 1) * 3 + co] : 0.f;
                if (lane == 31) right = lq < 3 ? xs[(1 * 4 + lq + 1) * 3 + co] : 0.f;
                out[co] = C[co] + left + right;
            }
            if (mine) {
                const int y = y0 + o;
#pragma unroll
                for (int co = 0; co < 3; ++co) {
                    if (co >= p.cout) continue;
                    const size_t oi = (size_t)b * p.bstride + (size_t)co * p.cstride + p.offset +
                                      (size_t)y * p.pitch + x;
                    p.fout[oi] = res[round][co] * p.rs + (out[co] + bias[co]) * p.os;
                }
            }
            __syncthreads();  // the exchange slots are reused next round
        }
    }
    if (!ok && tid == 0) {
        if (p.status) atomicOr(p.status, 2u);  // a bounded wait ran out
        wait_bar(bar, it & 1);                  // the products in flight, once more
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(L::TMEM_COLS));
}

int& out_grid_cap() {
    static int cap = 0;
    return cap;
}

cudaError_t out_prepare() {
    using L = OutSmem;
    if (out_grid_cap()) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_conv_out_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)L::bytes);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, smem = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    if ((e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) !=
        cudaSuccess)
        return e;
    int per = smem / (int)(L::bytes + 1024);
    per = per < 1 ? 1 : per;
    if (per * L::TMEM_COLS > 512) per = 512 / L::TMEM_COLS;
    if (per * TC_THREADS > 2048) per = 2048 / TC_THREADS;
    out_grid_cap() = sms * per;
    return cudaSuccess;
}

// ------------------------------------------------------------ weight gradient
// dW[ky][kx][ci][co] = sum over output pixels p of x[p + (ky - 1, kx - 1)][ci] dz[p][co]
// (x read through the nearest-neighbour doubling when the layer upsamples).
// For one kx the three ky taps form one GEMM: M = (ky, ci) in TMEM lanes, N =
// co in columns, K = pixels.  A CTA takes tiles of R rows x P columns of
// output pixels (R P = TP): the patch of x around the tile (R + 2 rows, P + 2
// columns, circular) and the tile of dz go to shared memory, and for each kx,
// output row and 16 pixels one MMA runs per 128 lanes of (ky, ci).
//
// The patch is stored [row][8-channel group][pixel], 16 B per pixel and group:
// a core matrix (8 pixels x 8 channels) is 128 contiguous bytes, the next 8
// pixels follow (K stride 128 B) and the next 8 lanes of M, the next channel
// group or after the last group the first group of the next row, sit one row
// segment of (P + 2) 16 B further (M stride): the ky taps are consecutive
// lane groups and the kx shift is a 16-byte offset of the start address.  dz
// is stored [8-channel group][pixel] (K stride 128 B, N stride TP 16 B).
// Both operands are MN-major (channels contiguous, as in memory), copied with
// cp.async in 16-byte pieces, no transpose; NS stages in flight, each tile's
// products committed to its stage's mbarrier.  Lanes past the third ky row
// (when 3 CI is not a multiple of 128) read the rows below the patch and are
// never stored.  At the end each lane adds its (ky, ci) row, CO columns per
// kx, into dW with atomics (all CTAs of a launch add into the same values).
constexpr int WT_THREADS = 256;  // 8 warps; in the epilogue warps w and w + 4 share lane quarter w

template <int CI, int CO, int KXS, int TP>
struct WtSmem {
    static constexpr int NG = CI / 8;                   // channel groups of x
    static constexpr int GO = CO / 8;                   // channel groups of dz
    static constexpr int NCH = (3 * NG + 15) / 16;      // MMAs of 128 lanes per kx and 16 pixels
    static constexpr int CSMAX = 66 * 16;               // row segment of one group, P = 64
    static constexpr int PATCH = (TP / 64 + 2) * NG * CSMAX;  // P = 64 is the largest patch
    static constexpr int DZ = TP * CO * 2;
    static constexpr int STAGE = PATCH + DZ;
    static constexpr int SLACK_ROWS = (16 * NCH - 1) / NG > 2 ? (16 * NCH - 1) / NG - 2 : 0;
    static constexpr int SLACK = SLACK_ROWS * NG * CSMAX;   // rows read below the last patch
    static constexpr int COLS = KXS * NCH * CO;
    static constexpr int TMEM_COLS =
        COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128 : COLS <= 256 ? 256 : 512;
    // stages: three, or two, if two CTAs then fit an SM (their issue and
    // loads overlap); else as many as fit, at most three
    static constexpr int FIX = SLACK + 64 + 1024;   // + the 1 KB the system keeps per CTA
    static constexpr bool TWO = 2 * TMEM_COLS <= 512;
    static constexpr int NSF = (227 * 1024 - SLACK - 64) / STAGE;
    static constexpr int NS = TWO && 2 * (3 * STAGE + FIX) <= 228 * 1024   ? 3
                              : TWO && 2 * (2 * STAGE + FIX) <= 228 * 1024 ? 2
                              : NSF > 3                                    ? 3
                                                                           : NSF;
    static constexpr size_t off_bar = (size_t)NS * STAGE + SLACK;
    static constexpr size_t bytes = off_bar + 8 * NS + 16;  // mbarriers + TMEM slot
    static_assert(NS >= 2 && COLS <= 512 && (NG & (NG - 1)) == 0 && (GO & (GO - 1)) == 0,
                  "weight-gradient tile does not fit");
};

// tile t (batch b, tile row ty, tile column tx) of output pixels: the patch of
// x and the tile of dz into a stage
template <int CI, int CO, int KXS, int TP>
__device__ __forceinline__ void wt_load(const WgradParams& p, unsigned char* st, long long t,
                                        int pl, int tid) {
    using L = WtSmem<CI, CO, KXS, TP>;
    const int P = 1 << pl, R = TP >> pl;
    const int tilesx = p.W >> pl, tpb = tilesx * (p.H / R);
    const int b = (int)(t / tpb);
    const int rem = (int)(t - (long long)b * tpb);
    const int ty = rem / tilesx, tx = rem - ty * tilesx;
    const int y0 = ty * R, x0 = tx * P;
    const int sh = p.up ? 1 : 0;
    const int Hi = p.H >> sh, Wi = p.W >> sh;
    const int CS = (P + 2) * 16;
    const bf16* xb = p.x + (size_t)b * Hi * Wi * CI;
    // patch rows y0 - 1 .. y0 + R, columns x0 - 1 .. x0 + P; consecutive
    // threads take consecutive 16-byte pieces of a pixel's channels
    const int rowpieces = (P + 2) * L::NG;
    for (int pr = 0; pr < R + 2; ++pr) {
        const bf16* xr = xb + (size_t)(wrap(y0 - 1 + pr, p.H) >> sh) * Wi * CI;
        unsigned char* dr = st + pr * L::NG * CS;
        for (int j = tid; j < rowpieces; j += WT_THREADS) {
            const int pc = j / L::NG, g = j - pc * L::NG;
            cp_async16(dr + g * CS + pc * 16, xr + (size_t)(wrap(x0 - 1 + pc, p.W) >> sh) * CI + g * 8);
        }
    }
    // dz: tile pixel k = r P + c of group g at g TP 16 + k 16
    unsigned char* sd = st + L::PATCH;
    const bf16* dzb = p.dz + (((size_t)b * p.H + y0) * p.W + x0) * CO;
    for (int j = tid; j < TP * L::GO; j += WT_THREADS) {
        const int k = j / L::GO, g = j - k * L::GO;
        const int r = k >> pl, c = k & (P - 1);
        cp_async16(sd + g * (TP * 16) + k * 16, dzb + ((size_t)r * p.W + c) * CO + g * 8);
    }
}

// grid (3 / KXS: the kx taps of a CTA, splits of the tiles); pl = log2 P
template <int CI, int CO, int KXS, int TP>
__global__ void __launch_bounds__(WT_THREADS) k_wgrad_tc(const WgradParams p, const int pl) {
    using L = WtSmem<CI, CO, KXS, TP>;
    constexpr int NS = L::NS;
    extern __shared__ __align__(1024) unsigned char smem[];
    const uint32_t bar0 = saddr(smem + L::off_bar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L::off_bar + 8 * NS);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int P = 1 << pl, R = TP >> pl;
    const long long ntiles = (long long)p.B * (p.W >> pl) * (p.H / R);
    const int kx0 = blockIdx.x * KXS;
    const long long t0 = blockIdx.y, ts = gridDim.y;
    if (t0 >= ntiles) return;
    const int nmine = (int)((ntiles - t0 + ts - 1) / ts);  // this CTA's tiles
    pdl_wait();
    pdl_trigger();
    if (tid == 0) {
        for (int k = 0; k < NS; ++k)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8 * k));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         saddr(tslot)),
                     "r"(L::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
#pragma unroll
    for (int k = 0; k < NS - 1; ++k) {
        if (k < nmine) wt_load<CI, CO, KXS, TP>(p, smem + k * L::STAGE, t0 + k * ts, pl, tid);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    // D f32, A and B bf16, both MN-major (bits 15, 16), N = CO, M = 128
    constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                               ((uint32_t)(CO >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    const uint32_t CS = (uint32_t)(P + 2) * 16;
    bool ok = true;
    for (int i = 0; i < nmine; ++i) {
        const int stg = i % NS;
        asm volatile("cp.async.wait_group %0;" ::"n"(NS - 2) : "memory");  // tile i landed
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            // descriptors of the stage's patch and dz tile; an offset of n 16-byte
            // units is added to the start-address field (addresses stay below 256 KB)
            const uint32_t pa = saddr(smem + stg * L::STAGE), pb = pa + L::PATCH;
            const uint64_t a0 = smem_desc(pa, 128, CS) + (uint64_t)kx0;
            const uint64_t b0 = smem_desc(pb, 128, TP * 16);
            for (int r = 0; r < R; ++r)
                for (int c = 0; c < P; c += 16) {
                    const uint64_t bd = b0 + (uint64_t)(r * P + c);
                    const uint64_t ar = a0 + (uint64_t)(r * L::NG * (P + 2) + c);
                    const uint32_t accum = (i | r | c) != 0;
#pragma unroll
                    for (int kxl = 0; kxl < KXS; ++kxl)
#pragma unroll
                        for (int h = 0; h < L::NCH; ++h) {
                            const uint64_t ad = ar + (uint64_t)(kxl + h * 16 * (P + 2));
                            asm volatile(
                                "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n\t}" ::"r"(
                                    tmem + (uint32_t)((kxl * L::NCH + h) * CO)),
                                "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                        }
                }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    bar0 + 8 * stg));
        }
        // tile i + NS - 1 into the stage tile i - 1 used, once its products are done
        const int nx = i + NS - 1;
        if (nx < nmine) {
            if (i >= 1) {
                const int j = i - 1;
                if (ok && !wait_bar(bar0 + 8 * (j % NS), (j / NS) & 1)) ok = false;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            }
            wt_load<CI, CO, KXS, TP>(p, smem + (nx % NS) * L::STAGE, t0 + nx * ts, pl, tid);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    // every tile's products: the last commit on each stage not yet waited for
    for (int j = nmine - 1; j >= 0 && j >= nmine - NS; --j)
        if (ok && !wait_bar(bar0 + 8 * (j % NS), (j / NS) & 1)) ok = false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    ok = __syncthreads_and(ok);
    if (ok) {
        const int lq = warp & 3;        // TMEM lane quarter of this warp
        const int m = 32 * lq + lane;   // this thread's lane (row of M)
        const bool vec = (p.cout & 3) == 0 && ((uintptr_t)p.dw & 15) == 0;
#pragma unroll 1
        for (int h = 0; h < L::NCH; ++h) {
            const int G = 16 * h + (m >> 3);             // lane group: (ky, channel group)
            const int ky = G / L::NG, ci = (G - ky * L::NG) * 8 + (m & 7);
            const bool valid = ky < 3 && ci < p.cin;
#pragma unroll 1
            for (int kxl = 0; kxl < KXS; ++kxl)
#pragma unroll 1
                for (int cc = 16 * (warp >> 2); cc < CO; cc += 32) {
                    uint32_t v[16];
                    const uint32_t taddr = tmem + ((uint32_t)(32 * lq) << 16) +
                                           (uint32_t)((kxl * L::NCH + h) * CO + cc);
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,"
                        "%10,%11,%12,%13,%14,%15}, [%16];"
                        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                          "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                          "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                        : "r"(taddr));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (!valid) continue;
                    float* dst = p.dw + ((size_t)(3 * ky + kx0 + kxl) * p.cin + ci) * p.cout + cc;
                    if (vec) {
#pragma unroll
                        for (int q = 0; q < 16; q += 4)
                            if (cc + q < p.cout)
                                atomicAdd(reinterpret_cast<float4*>(dst + q),
                                          make_float4(__uint_as_float(v[q]), __uint_as_float(v[q + 1]),
                                                      __uint_as_float(v[q + 2]),
                                                      __uint_as_float(v[q + 3])));
                    } else {
#pragma unroll
                        for (int q = 0; q < 16; ++q)
                            if (cc + q < p.cout) atomicAdd(dst + q, __uint_as_float(v[q]));
                    }
                }
        }
    } else if (tid == 0) {
        if (p.status) atomicOr(p.status, 2u);  // a bounded wait ran out
        // the products still in flight, once more, before the accumulator is freed
        for (int j = nmine - 1; j >= 0 && j >= nmine - NS; --j)
            wait_bar(bar0 + 8 * (j % NS), (j / NS) & 1);
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(L::TMEM_COLS));
}

template <int CI, int CO, int KXS, int TP>
cudaError_t wgrad_tc_T(const WgradParams& p, int pl, cudaStream_t s) {
    using L = WtSmem<CI, CO, KXS, TP>;
    static int per_sm = 0;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (per_sm == 0) {
        int smem = 0;
        e = cudaFuncSetAttribute(k_wgrad_tc<CI, CO, KXS, TP>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (e != cudaSuccess) return e;
        // resident CTAs: shared memory (plus the 1 KB the system keeps per CTA),
        // TMEM columns, threads
        int per = smem / (int)(L::bytes + 1024);
        if (per * L::TMEM_COLS > 512) per = 512 / L::TMEM_COLS;
        if (per * WT_THREADS > 2048) per = 2048 / WT_THREADS;
        per_sm = per < 1 ? 1 : per;
    }
    const int gx = 3 / KXS;
    const long long ntiles = (long long)p.B * (p.W >> pl) * (p.H / (TP >> pl));
    long long split = (long long)sms * per_sm / gx;  // one wave
    split = split < 1 ? 1 : (split > ntiles ? ntiles : split);
    return launch_pdl(k_wgrad_tc<CI, CO, KXS, TP>, dim3(gx, (unsigned)split), dim3(WT_THREADS),
                      L::bytes, s, p, pl);
}

// ------------------------------------------- weight gradient, kx taps in N
// The same sums with the three kx taps side by side in N.  With q the patch
// column (the patch spans columns x0 - 1 .. x0 + P of the tile's rows,
// padded with zeros to QW = P + 16 columns) and dzk[kx] the dz tile shifted
// right by kx pixels (dz[r][q - kx], zero outside the tile):
//   D[(ky, ci)][(kx, co)] += sum over q of patch[r + ky][q][ci] dzk[kx][r][q][co]
// so one MMA of N = 3 CO covers the three kx taps of 16 patch columns, where
// the first kernel issues one MMA of N = CO per tap: the 128-lane A operand
// is read from shared memory a third as often.  The padding makes K = P + 16
// per row instead of P.  dzk is stored [kx][8-channel group][row][column]
// (N stride R QW 16 B), the patch as in the first kernel with rows of QW
// pixels.  Tiles are 64 columns wide; a CTA takes the lane chunks CHS of
// (ky, ci) whose accumulators (CHS 3 CO columns) fit TMEM: all of them, or
// for 128 input channels one ky per CTA (then it loads only that tap's R
// patch rows).
constexpr int WN_P = 64;
constexpr int WN_QW = WN_P + 16;

template <int CI, int CO, int TP, int CHS>
struct WnSmem {
    static constexpr int NG = CI / 8, GO = CO / 8, R = TP / WN_P;
    static constexpr int NCH = (3 * NG + 15) / 16;
    static constexpr int N = 3 * CO;
    static constexpr int CS = WN_QW * 16;   // one row of one channel group
    static constexpr int RS = NG * CS;      // one patch row
    // patch rows a CTA loads: every ky, or (CHS = 1, 16 groups a ky) its own
    static constexpr int NR = CHS == NCH ? R + 2 : R;
    static constexpr int PATCH = NR * RS;
    // lanes past the third ky read this many rows below the patch (into the dzk
    // tile that follows it in the stage)
    static constexpr int SLACK_ROWS =
        CHS == NCH && (16 * NCH - 1) / NG > 2 ? (16 * NCH - 1) / NG - 2 : 0;
    static constexpr int PL = R * WN_QW * 16;   // one (kx, group) plane of dzk
    static constexpr int DZK = 3 * GO * PL;
    static constexpr int STAGE = PATCH + DZK;
    static constexpr int COLS = CHS * N;
    static constexpr int TMEM_COLS =
        COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128 : COLS <= 256 ? 256 : 512;
    static constexpr int FIX = 64 + 1024;
    static constexpr bool TWO = 2 * TMEM_COLS <= 512;
    static constexpr int NSF = (227 * 1024 - 64) / STAGE;
    static constexpr int NS = TWO && 2 * (3 * STAGE + FIX) <= 228 * 1024   ? 3
                              : TWO && 2 * (2 * STAGE + FIX) <= 228 * 1024 ? 2
                              : NSF > 3                                    ? 3
                                                                           : NSF;
    static constexpr size_t off_bar = (size_t)NS * STAGE;
    static constexpr size_t bytes = off_bar + 8 * NS + 16;  // mbarriers + TMEM slot
    static_assert(NS >= 2 && COLS <= 512 && N <= 256 && SLACK_ROWS * RS <= DZK &&
                      (CHS == NCH || (CHS == 1 && NG == 16)),
                  "weight-gradient tile (kx in N) does not fit");
};

// the zero columns of every stage: patch columns P + 2 .. QW - 1, and the
// columns of each dzk copy outside kx .. kx + P - 1 (the loads never write them)
template <int CI, int CO, int TP, int CHS>
__device__ __forceinline__ void wn_zero(unsigned char* smem, int tid) {
    using L = WnSmem<CI, CO, TP, CHS>;
    constexpr int PZ = WN_QW - (WN_P + 2);                 // 14 patch columns a row
    constexpr int NPZ = L::NR * L::NG * PZ;
    constexpr int DZ_Z = 16;                                // 16 dzk columns a row and copy
    constexpr int NDZ = 3 * L::GO * L::R * DZ_Z;
    const uint4 z = make_uint4(0, 0, 0, 0);
    for (int st = 0; st < L::NS; ++st) {
        unsigned char* base = smem + st * L::STAGE;
        for (int i = tid; i < NPZ; i += WT_THREADS) {
            const int row = i / (L::NG * PZ), rem = i - row * (L::NG * PZ);
            const int g = rem / PZ, q = WN_P + 2 + (rem - g * PZ);
            *reinterpret_cast<uint4*>(base + row * L::RS + g * L::CS + q * 16) = z;
        }
        for (int i = tid; i < NDZ; i += WT_THREADS) {
            const int plane = i / (L::R * DZ_Z), rem = i - plane * (L::R * DZ_Z);
            const int r = rem / DZ_Z, j = rem - r * DZ_Z;
            const int kx = plane / L::GO;
            // columns 0 .. kx - 1 and kx + P .. QW - 1: 16 of them
            const int q = j < kx ? j : WN_P + j;
            *reinterpret_cast<uint4*>(base + L::PATCH + plane * L::PL + (r * WN_QW + q) * 16) = z;
        }
    }
}

template <int CI, int CO, int TP, int CHS>
__device__ __forceinline__ void wn_load(const WgradParams& p, unsigned char* st, long long t, int lo,
                                        int tid) {
    using L = WnSmem<CI, CO, TP, CHS>;
    constexpr int R = L::R;
    const int tilesx = p.W / WN_P, tpb = tilesx * (p.H / R);
    const int b = (int)(t / tpb);
    const int rem = (int)(t - (long long)b * tpb);
    const int ty = rem / tilesx, tx = rem - ty * tilesx;
    const int y0 = ty * R, x0 = tx * WN_P;
    const int sh = p.up ? 1 : 0;
    const int Hi = p.H >> sh, Wi = p.W >> sh;
    const bf16* xb = p.x + (size_t)b * Hi * Wi * CI;
    // patch rows y0 - 1 + lo + j, columns x0 - 1 .. x0 + P
    constexpr int ROWP = (WN_P + 2) * L::NG;
    for (int j = 0; j < L::NR; ++j) {
        const bf16* xr = xb + (size_t)(wrap(y0 - 1 + lo + j, p.H) >> sh) * Wi * CI;
        unsigned char* dr = st + j * L::RS;
        for (int i = tid; i < ROWP; i += WT_THREADS) {
            const int q = i / L::NG, g = i - q * L::NG;
            cp_async16(dr + g * L::CS + q * 16, xr + (size_t)(wrap(x0 - 1 + q, p.W) >> sh) * CI + g * 8);
        }
    }
    // dzk: tile pixel (r, c) of group g into column c + kx of each copy; the
    // second and third copies of a piece come from L1
    unsigned char* sd = st + L::PATCH;
    const bf16* dzb = p.dz + (((size_t)b * p.H + y0) * p.W + x0) * CO;
    for (int i = tid; i < TP * L::GO; i += WT_THREADS) {
        const int k = i / L::GO, g = i - k * L::GO;
        const int r = k / WN_P, c = k - r * WN_P;
        const bf16* src = dzb + ((size_t)r * p.W + c) * CO + g * 8;
#pragma unroll
        for (int kx = 0; kx < 3; ++kx)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(saddr(
                             sd + (kx * L::GO + g) * L::PL + (r * WN_QW + c + kx) * 16)),
                         "l"(src)
                         : "memory");
    }
}

// grid (NCH / CHS lane chunks, splits of the tiles)
template <int CI, int CO, int TP, int CHS>
__global__ void __launch_bounds__(WT_THREADS) k_wgrad_tcn(const WgradParams p) {
    using L = WnSmem<CI, CO, TP, CHS>;
    constexpr int NS = L::NS, R = L::R;
    extern __shared__ __align__(1024) unsigned char smem[];
    const uint32_t bar0 = saddr(smem + L::off_bar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L::off_bar + 8 * NS);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long ntiles = (long long)p.B * (p.W / WN_P) * (p.H / R);
    const int h0 = blockIdx.x * CHS;            // first lane chunk of this CTA
    const int lo = (16 * h0) / L::NG;           // first patch row (relative to y0 - 1)
    const long long t0 = blockIdx.y, ts = gridDim.y;
    if (t0 >= ntiles) return;
    const int nmine = (int)((ntiles - t0 + ts - 1) / ts);
    pdl_wait();
    pdl_trigger();
    if (tid == 0) {
        for (int k = 0; k < NS; ++k)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8 * k));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         saddr(tslot)),
                     "r"(L::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    wn_zero<CI, CO, TP, CHS>(smem, tid);
#pragma unroll
    for (int k = 0; k < NS - 1; ++k) {
        if (k < nmine) wn_load<CI, CO, TP, CHS>(p, smem + k * L::STAGE, t0 + k * ts, lo, tid);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    // D f32, A and B bf16, both MN-major, N = 3 CO, M = 128
    constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                               ((uint32_t)(L::N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    bool ok = true;
    for (int i = 0; i < nmine; ++i) {
        const int stg = i % NS;
        asm volatile("cp.async.wait_group %0;" ::"n"(NS - 2) : "memory");  // tile i landed
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            // start-address offsets in 16-byte units (addresses stay below 256 KB)
            const uint32_t pa = saddr(smem + stg * L::STAGE), pb = pa + L::PATCH;
            const uint64_t a0 = smem_desc(pa, 128, L::CS);
            const uint64_t b0 = smem_desc(pb, 128, L::PL);
#pragma unroll 1
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int sk = 0; sk < WN_QW / 16; ++sk) {
                    const uint64_t bd = b0 + (uint64_t)(r * WN_QW + 16 * sk);
                    const uint32_t accum = (i | r | sk) != 0;
#pragma unroll
                    for (int hl = 0; hl < CHS; ++hl) {
                        const uint64_t ad =
                            a0 + (uint64_t)(((r - lo) * L::NG + 16 * (h0 + hl)) * WN_QW + 16 * sk);
                        asm volatile(
                            "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n\t}" ::"r"(
                                tmem + (uint32_t)(hl * L::N)),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                    }
                }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    bar0 + 8 * stg));
        }
        const int nx = i + NS - 1;
        if (nx < nmine) {
            if (i >= 1) {
                const int j = i - 1;
                if (ok && !wait_bar(bar0 + 8 * (j % NS), (j / NS) & 1)) ok = false;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            }
            wn_load<CI, CO, TP, CHS>(p, smem + (nx % NS) * L::STAGE, t0 + nx * ts, lo, tid);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int j = nmine - 1; j >= 0 && j >= nmine - NS; --j)
        if (ok && !wait_bar(bar0 + 8 * (j % NS), (j / NS) & 1)) ok = false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    ok = __syncthreads_and(ok);
    if (ok) {
        const int lq = warp & 3;
        const int m = 32 * lq + lane;
        const bool vec = (p.cout & 3) == 0 && ((uintptr_t)p.dw & 15) == 0;
#pragma unroll 1
        for (int hl = 0; hl < CHS; ++hl) {
            const int G = 16 * (h0 + hl) + (m >> 3);
            const int ky = G / L::NG, ci = (G - ky * L::NG) * 8 + (m & 7);
            const bool valid = ky < 3 && ci < p.cin;
#pragma unroll 1
            for (int cc = 16 * (warp >> 2); cc < L::N; cc += 32) {
                uint32_t v[16];
                const uint32_t taddr =
                    tmem + ((uint32_t)(32 * lq) << 16) + (uint32_t)(hl * L::N + cc);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,"
                    "%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                      "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                      "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (!valid) continue;
                const int kx = cc / CO, co = cc - kx * CO;  // a 16-column chunk lies in one kx
                float* dst = p.dw + ((size_t)(3 * ky + kx) * p.cin + ci) * p.cout + co;
                if (vec) {
#pragma unroll
                    for (int q = 0; q < 16; q += 4)
                        if (co + q < p.cout)
                            atomicAdd(reinterpret_cast<float4*>(dst + q),
                                      make_float4(__uint_as_float(v[q]), __uint_as_float(v[q + 1]),
                                                  __uint_as_float(v[q + 2]),
                                                  __uint_as_float(v[q + 3])));
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if (co + q < p.cout) atomicAdd(dst + q, __uint_as_float(v[q]));
                }
            }
        }
    } else if (tid == 0) {
        if (p.status) atomicOr(p.status, 2u);
        for (int j = nmine - 1; j >= 0 && j >= nmine - NS; --j)
            wait_bar(bar0 + 8 * (j % NS), (j / NS) & 1);
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(L::TMEM_COLS));
}

template <int CI, int CO, int TP, int CHS>
cudaError_t wgrad_tcn_T(const WgradParams& p, cudaStream_t s) {
    using L = WnSmem<CI, CO, TP, CHS>;
    static int per_sm = 0;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (per_sm == 0) {
        int smem = 0;
        e = cudaFuncSetAttribute(k_wgrad_tcn<CI, CO, TP, CHS>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (e != cudaSuccess) return e;
        int per = smem / (int)(L::bytes + 1024);
        if (per * L::TMEM_COLS > 512) per = 512 / L::TMEM_COLS;
        if (per * WT_THREADS > 2048) per = 2048 / WT_THREADS;
        per_sm = per < 1 ? 1 : per;
    }
    const int gx = L::NCH / CHS;
    const long long ntiles = (long long)p.B * (p.W / WN_P) * (p.H / L::R);
    long long split = (long long)sms * per_sm / gx;  // one wave
    split = split < 1 ? 1 : (split > ntiles ? ntiles : split);
    return launch_pdl(k_wgrad_tcn<CI, CO, TP, CHS>, dim3(gx, (unsigned)split), dim3(WT_THREADS),
                      L::bytes, s, p);
}

}  // namespace

// (CI, CO, kx taps per CTA, pixels per tile): three kx per CTA while their
// accumulators fit the 512 TMEM columns, smaller tiles where a stage of 256
// pixels would not leave two stages in shared memory
#define PIC_WT_SHAPES(X)                                                                \
    X(16, 32, 3, 256) X(32, 32, 3, 256) X(32, 64, 3, 256) X(32, 16, 3, 256)             \
    X(64, 64, 3, 256) X(64, 32, 3, 256) X(64, 128, 1, 128) X(128, 128, 1, 128)          \
    X(128, 64, 1, 128)

namespace {
// log2 of the tile width: 64, 32 or 16 columns, the widest that divides W
// (-1: none, or the tile rows do not divide H)
int wt_log2p(const WgradParams& p, int tp) {
    const int pl = p.W % 64 == 0 ? 6 : (p.W % 32 == 0 ? 5 : (p.W % 16 == 0 ? 4 : -1));
    if (pl < 0 || p.H % (tp >> pl)) return -1;
    return pl;
}
}  // namespace

// (CI, CO, pixels per tile, lane chunks per CTA) of the kx-in-N kernel
// (measured per layer at 256^2 x 16: faster than the first kernel for these
// four; for 32 -> 32 (where the first kernel keeps two CTAs per SM), 64 -> 64
// and 32 -> 64 (where the three dz copies and the halo rows of 128-pixel
// tiles double the copies per pixel) the first kernel is faster)
#define PIC_WN_SHAPES(X) X(16, 32, 256, 1) X(32, 16, 256, 1) X(64, 32, 128, 2) X(128, 64, 128, 1)

namespace {
// the kx-in-N kernel: tiles of 64 columns and TP / 64 rows
bool wn_fits(const WgradParams& p, int tp) { return p.W % WN_P == 0 && p.H % (tp / WN_P) == 0; }
}  // namespace

bool wgrad_tc_supported(const WgradParams& p, int ci, int co) {
    if (p.force_tc < 0) return false;
#define PIC_WT_HAS(A, B, K, T) \
    if (ci == A && co == B) return wt_log2p(p, T) >= 0;
    PIC_WT_SHAPES(PIC_WT_HAS)
#undef PIC_WT_HAS
    return false;
}

cudaError_t launch_wgrad_tc(const WgradParams& p, int ci, int co, cudaStream_t s) {
#define PIC_WN_CASE(A, B, T, C) \
    if (ci == A && co == B && wn_fits(p, T)) return wgrad_tcn_T<A, B, T, C>(p, s);
    PIC_WN_SHAPES(PIC_WN_CASE)
#undef PIC_WN_CASE
#define PIC_WT_CASE(A, B, K, T) \
    if (ci == A && co == B) {                                                       \
        const int pl = wt_log2p(p, T);                                              \
        return pl < 0 ? cudaErrorInvalidValue : wgrad_tc_T<A, B, K, T>(p, pl, s);   \
    }
    PIC_WT_SHAPES(PIC_WT_CASE)
#undef PIC_WT_CASE
    return cudaErrorInvalidValue;
}

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
    // small problems finish sooner on the mma.sync kernel, whose CTAs do not
    // each stage all nine taps of weights (measured in the denoised step with
    // programmatic dependent launch: from 200 work units on the tcgen05 kernel
    // is faster, 512^2 0.306 -> 0.278 ms; 256 units of 32 channels at 256^2
    // are within 1 % either way)
    if ((long long)p.B * (p.H / TC_R) * (p.W / TC_M) < 200 && p.force_tc <= 0) return false;
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

// (CIN, N, channels per pass) shapes of the upsampling convolution: c9 (64 ->
// 32) in one pass; c7 (128 -> 64) as two tiles of 32 output channels (the
// sixteen taps of 64 output channels and 128 inputs would not fit) and four
// passes of 32 input channels
#define PIC_UP_SHAPES(X) X(64, 32, 64) X(128, 32, 32)

static int up_nt(int cin, int cout_pad) { return cin == 128 ? 32 : tc_nt(cout_pad); }

bool conv_up_tc_supported(const ConvParams& p, int cin) {
    if (!p.up || !p.wp || p.force_tc < 0 || p.epi != EPI_ACT) return false;
    if (p.H % 2 || (p.W >> 1) % TC_M || p.cout_pad > 128) return false;
    // no size rule: with 4/9 of the products it beats the mma.sync kernel from
    // the smallest grids it takes on (measured at 256^2 and 512^2 in the step)
    const int nt = up_nt(cin, p.cout_pad);
#define PIC_UP_HAS(A, B, C) if (cin == A && nt == B) return true;
    PIC_UP_SHAPES(PIC_UP_HAS)
#undef PIC_UP_HAS
    return false;
}

cudaError_t launch_conv_up_tc(const ConvParams& p, int cin, cudaStream_t s) {
    const int nt = up_nt(cin, p.cout_pad);
#define PIC_UP_CASE(A, B, C) \
    if (cin == A && nt == B) return conv_up_tc_T<A, B, C>(p, s);
    PIC_UP_SHAPES(PIC_UP_CASE)
#undef PIC_UP_CASE
    return cudaErrorInvalidValue;
}

bool conv_out_tc_supported(const ConvParams& p, int cin) {
    return p.force_tc >= 0 && p.epi == EPI_FINAL && !p.up && cin == 32 && p.cout <= 3 &&
           p.cout_pad >= 3 && p.H % OT_R == 0 && p.W >= TC_M;
}

cudaError_t launch_conv_out_tc(const ConvParams& p, cudaStream_t s) {
    cudaError_t e = out_prepare();
    if (e != cudaSuccess) return e;
    const int nunit = p.B * (p.H / OT_R) * ((p.W + OT_P - 1) / OT_P);
    int gx = out_grid_cap();
    gx = gx < 1 ? 1 : (gx > nunit ? nunit : gx);
    return launch_pdl(k_conv_out_tc, dim3(gx), dim3(TC_THREADS), OutSmem::bytes, s, p);
}

cudaError_t init_tc_kernels() {
    cudaError_t e = out_prepare();
#define PIC_TC_PREP(A, B, C) \
    if (e == cudaSuccess) e = tc_prepare<A, B, C>();
    PIC_TC_SHAPES(PIC_TC_PREP)
#undef PIC_TC_PREP
#define PIC_UP_PREP(A, B, C) \
    if (e == cudaSuccess) e = up_prepare<A, B, C>();
    PIC_UP_SHAPES(PIC_UP_PREP)
#undef PIC_UP_PREP
    return e;
}

}  // namespace nn
}  // namespace pic
