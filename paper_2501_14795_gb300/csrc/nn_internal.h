// Internal declarations of the denoiser kernels (nn_kernels.cu) shared with
// their host runtime (denoiser.cu).  Not part of the public ABI.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstdlib>
#include <utility>

namespace pic {
namespace nn {

// convolution tile: 8 x 16 output pixels per CTA, one pixel row per warp
constexpr int TH = 8, TW = 16;
constexpr int PH = TH + 2, PW = TW + 2;
constexpr int CONV_THREADS = 256;
// weight gradient: chunks of WG_PIX consecutive pixels (flattened b, y, x)
// through a WG_STAGES-deep pipeline
constexpr int WG_PIX = 64, WG_STAGES = 3;
constexpr int WG_THREADS = 256, WG_WARPS = 8;

enum { EPI_ACT = 0, EPI_FINAL = 1, EPI_GRAD = 2 };

struct ConvParams {
    const __nv_bfloat16* x;  // input NHWC, channels = the kernel's CIN
    int B, H, W;             // output (and, without up, input) size
    int up;                  // x is H/2 x W/2, read at (y/2, x/2): fused 2x upsampling
    const __nv_bfloat16* w;  // packed [9][cout_pad][CIN]
    const __nv_bfloat16* wp; // with up: the sixteen combined taps of the four output
                             // parities, packed [16][cout_pad][CIN] (null: not packed)
    const float* bias;       // [cout] or null
    int cout, cout_pad;
    int epi, relu;
    // EPI_ACT: a_out = bf16(relu(z + bias)); with skip: y_out = bf16(a + skip)
    // (a_out may then be null: the activation is kept only for a backward pass)
    __nv_bfloat16* a_out;
    const __nv_bfloat16* skip;
    __nv_bfloat16* y_out;
    // EPI_GRAD: g_out = z (FP32 NHWC, cout_pad channels)
    float* g_out;
    // EPI_FINAL: fout[o] = res[o] * rs + (z + bias) * os for c < cout, with
    // o = b*bstride + c*cstride + offset + y*pitch + x (field layout)
    const float* res;
    float* fout;
    long long bstride, cstride;
    int pitch, offset;
    float rs, os;
    unsigned* status;        // tensor-core path: bit 2 set when a bounded wait ran out (may be null)
    int force_tc;            // take the tensor-core path whenever the shape allows (tests)
};

// A three-component current in field layout: element (b, c, y, x) at
// p[b*bstride + c*cstride + offset + y*pitch + x].
struct FieldView {
    float* p;
    long long bstride, cstride;
    int pitch, offset;
};

// taps of the (2n+1)-point kernel C(2n, k) / 4^n (n passes of the binomial stencil)
constexpr int LOWK_MAX = 64;
struct LowkTaps {
    int n;
    float w[2 * LOWK_MAX + 1];
};

struct WgradParams {
    const __nv_bfloat16* x;   // layer input NHWC (CI channels)
    const __nv_bfloat16* dz;  // output gradient NHWC (CO channels)
    int B, H, W;              // output size
    int up;                   // x is H/2 x W/2, read at (y/2, x/2)
    int cin, cout;            // real channel counts
    float* dw;                // += into [9][cin][cout]
    int force_tc;             // 1: the tcgen05 kernel whenever the shape allows, -1: never
    unsigned* status;         // tcgen05 kernel: bit 2 set when a bounded wait ran out (may be null)
};

struct LayerDesc {
    int cin, cout;            // real channel counts
    int cin_pad, cout_pad;    // forward GEMM: k = cin_pad (x16), n = cout_pad (x CT)
    int dg_cin_pad, dg_cout_pad;  // input-gradient GEMM: k = cout padded to 16, n = cin (0: none)
    long long woff;           // weights in the master vector ([9][cin][cout], then bias)
    long long wf_off, wd_off; // packed bfloat16 arrays
    long long wp_off;         // combined taps of an upsampling layer ([16][cout_pad][cin_pad];
                              // -1: none)
};

constexpr int MAX_LAYERS = 16;
struct PackTable {
    int n;
    LayerDesc layer[MAX_LAYERS];
};

// raise every kernel shape's shared-memory limit (before any graph capture)
cudaError_t init_kernels();
// mma.sync implicit GEMM (any shape of the network), or the tcgen05 kernel
// (nn_tc.cu) when the row length is a multiple of 128 and the shape is built
// Programmatic dependent launch: the kernel may start before the previous
// kernel in the stream has finished; it must call pdl_wait() before touching
// global memory other than the packed weights and biases (pdl_trigger(),
// called after the wait, lets the next kernel start, so a kernel two launches
// later never overlaps one that is still reading).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;"); }

// Programmatic dependent launch is on unless PIC_NN_PDL=0 in the environment:
// measured on GB300 in the step graph of a denoised 4-ppc run it saves the
// layers' launch gaps (256^2: 0.1375 -> 0.1315 ms per step, 1024^2: 0.799 ->
// 0.773 ms).  (With the earlier, longer-tailed kernels it cost ~10 us at 256^2.)
inline bool pdl_enabled() {
    static const int on = [] {
        const char* v = getenv("PIC_NN_PDL");
        return (v && v[0] == '0') ? 0 : 1;
    }();
    return on != 0;
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

cudaError_t launch_conv(const ConvParams& p, int cin, int ct, cudaStream_t s);
bool conv_tc_supported(const ConvParams& p, int cin);
cudaError_t launch_conv_tc(const ConvParams& p, int cin, cudaStream_t s);
// the output layer (32 -> 3, EPI_FINAL) with its nine taps in the GEMM's N (tcgen05)
bool conv_out_tc_supported(const ConvParams& p, int cin);
cudaError_t launch_conv_out_tc(const ConvParams& p, cudaStream_t s);
// a 3x3 convolution of a 2x upsampled input as four 2x2 convolutions (tcgen05)
bool conv_up_tc_supported(const ConvParams& p, int cin);
cudaError_t launch_conv_up_tc(const ConvParams& p, int cin, cudaStream_t s);
cudaError_t init_tc_kernels();
// weight gradient on the tensor cores (ci, co: padded channel counts)
bool wgrad_tc_supported(const WgradParams& p, int ci, int co);
cudaError_t launch_wgrad_tc(const WgradParams& p, int ci, int co, cudaStream_t s);
cudaError_t launch_wgrad(const WgradParams& p, int ci, int co, cudaStream_t s);
// the first layer (3 -> 32, ReLU) fused with the input packing, and the
// output layer (32 -> 3) with the residual epilogue, on the CUDA cores; H and
// W multiples of 16
cudaError_t launch_conv_first(const float* J, long long bstride, long long cstride, int pitch,
                              int offset, int B, int H, int W, float inv_scale,
                              const __nv_bfloat16* w, int cout_pad, const float* bias,
                              __nv_bfloat16* xin, __nv_bfloat16* a_out, cudaStream_t s);
cudaError_t launch_pack_input(const float* J, long long bstride, long long cstride, int pitch,
                              int offset, int B, int H, int W, float inv_scale, __nv_bfloat16* out,
                              cudaStream_t s);
cudaError_t launch_pool_fwd(const __nv_bfloat16* in, int B, int H, int W, int C,
                            __nv_bfloat16* out, cudaStream_t s);
cudaError_t launch_up_fwd(const __nv_bfloat16* in, int B, int H, int W, int C, __nv_bfloat16* out,
                          cudaStream_t s);
// ReLU backward: dz = bf16((dy + extra) * (a > 0)), db += the FP32 sum over
// pixels; dy read directly (npix pixels), through the adjoint of the 2x2 mean
// pooling (dp on the H/2 x W/2 grid; dz on B x H x W) or of the nearest 2x
// upsampling (du on the 2H x 2W grid; dz on B x H x W)
cudaError_t launch_relu_back(const float* dy, const float* extra, const __nv_bfloat16* a,
                             long long npix, int C, __nv_bfloat16* dz, float* db, cudaStream_t s);
cudaError_t launch_pool_relu_back(const float* dp, int B, int H, int W, int C, const float* extra,
                                  const __nv_bfloat16* a, __nv_bfloat16* dz, float* db,
                                  cudaStream_t s);
cudaError_t launch_up_relu_back(const float* du, int B, int H, int W, int C,
                                const __nv_bfloat16* a, __nv_bfloat16* dz, float* db,
                                cudaStream_t s);
cudaError_t launch_mse(const float* out, const float* target, long long bstride, long long cstride,
                       int pitch, int offset, int B, int H, int W, float inv_scale,
                       __nv_bfloat16* dz, float* db, double* loss, cudaStream_t s);
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, long long n, float lr,
                        float b1, float b2, float eps, float c1, float c2, cudaStream_t s);
// o += L^n (a - b) (b.p null: L^n a), L one pass of the periodic binomial
// smoothing; t is dense scratch of 3 B H W floats; 0 <= n <= LOWK_MAX
cudaError_t launch_lowk(const FieldView& a, const FieldView& b, float* t, const FieldView& o,
                        int n, int B, int H, int W, cudaStream_t s);
// o = a (three-component currents of B samples, any layouts)
cudaError_t launch_field_copy(const FieldView& a, const FieldView& o, int B, int H, int W,
                              cudaStream_t s);
// o = a (and o2 = a when o2.p is set) with per-sample base pointers from the
// device tables atab / otab where they are non-null
cudaError_t launch_field_copy_tab(const FieldView& a, const float* const* atab, const FieldView& o,
                                  float* const* otab, const FieldView& o2, int B, int H, int W,
                                  cudaStream_t s);
// bfloat16 packings of the master weights: wf (forward), wd (input
// gradient), and wp (the combined taps of the layers with wp_off >= 0); a
// null array is skipped
cudaError_t launch_pack_weights(const PackTable& t, const float* master, __nv_bfloat16* wf,
                                __nv_bfloat16* wd, cudaStream_t s, __nv_bfloat16* wp = nullptr);

}  // namespace nn
}  // namespace pic
