// Host runtime of the learned current denoiser behind the C ABI of
// include/pic.h: parameters (FP32 master copy, Adam moments, bfloat16 packed
// copies), activation and gradient buffers for up to batch_max samples, the
// forward pass, the backward pass, the Adam step, the kernel-level probes and
// the hook that runs the network in a simulation's current-filter slot.
//
// Network (3 levels, 32/64/128 channels, 3x3 circular convolutions, ReLU,
// 2x2 mean pooling, nearest upsampling, additive skips, residual output):
//   c1 3->32, c2 32->32 [s1] | pool | c3 32->64, c4 64->64 [s2] | pool |
//   c5 64->128, c6 128->128 | up | c7 128->64 (+s2), c8 64->64 | up |
//   c9 64->32 (+s1), c10 32->32, c11 32->3;  out = x + c11.
// Optional low-wavenumber restoration after the network (n > 0 passes):
//   out <- out + L^n (x - out), L one pass of the periodic binomial smoothing,
// which gives back the long-wavelength part of what the network removed (a
// mean-squared-error denoiser shrinks a weak coherent mode with the noise).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "host_internal.h"
#include "nn_internal.h"

using namespace pic;
using namespace pic::nn;
using namespace pic::host;
using bf16 = __nv_bfloat16;

namespace {

struct LayerSpec {
    int cin, cout, level;
    bool relu;
    int skip;  // layer index whose output is added, or -1
};
constexpr int NL = 11;
constexpr LayerSpec kLayers[NL] = {
    {3, 32, 0, true, -1},   {32, 32, 0, true, -1},  {32, 64, 1, true, -1},
    {64, 64, 1, true, -1},  {64, 128, 2, true, -1}, {128, 128, 2, true, -1},
    {128, 64, 1, true, 3},  {64, 64, 1, true, -1},  {64, 32, 0, true, 1},
    {32, 32, 0, true, -1},  {32, 3, 0, false, -1},
};

int pad16(int c) { return (c + 15) / 16 * 16; }
// c7 and c9 read the coarser level through the 2x upsampling
bool up_input(int l) { return l == 6 || l == 8; }
// below this many pixels per forward pass the thin first layer runs on the CUDA cores
constexpr long long kThinPixels = 1LL << 18;
// output-channel tile of the convolution kernel for a given channel count
int ctile(int cout) { return cout <= 8 ? 8 : (cout >= 64 ? 64 : 32); }
int padct(int cout) { const int t = ctile(cout); return (cout + t - 1) / t * t; }

}  // namespace

struct pic_denoiser {
    int H = 0, W = 0, Bmax = 0;
    double scale = 1.0;
    cudaStream_t stream = nullptr;
    PackTable tab;
    long long np = 0;
    long long boff[NL];
    float *master = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    long long adam_t = 0;
    bf16 *wf = nullptr, *wd = nullptr, *wp = nullptr;
    // activations (Bmax samples)
    bf16* xin = nullptr;
    bf16* a[NL] = {};
    bf16 *y7 = nullptr, *y9 = nullptr, *p1 = nullptr, *p2 = nullptr;
    float* out = nullptr;  // normalised output, dense [B][3][H][W]
    // gradients
    bf16* dz = nullptr;
    float *G0 = nullptr, *G1 = nullptr, *S1 = nullptr, *S2 = nullptr;
    double* dloss = nullptr;
    unsigned* status = nullptr;      // device word: bit 2 = a bounded wait in a kernel ran out
    unsigned* cur_status = nullptr;  // where the next launches report (own word or a simulation's)
    int force_tc = 0;                // PIC_DENOISER_TC: always (1) / never (-1) the tcgen05 path
    int restore = 0;                 // passes of the low-wavenumber restoration (0: off)
    // host-buffer staging
    float *stage_in = nullptr, *stage_t = nullptr;
    std::vector<void*> allocs;
    std::string err;
};

namespace {

pic_status dfail(pic_denoiser* d, pic_status code, const char* fmt, ...) {
    if (d) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        d->err = buf;
    }
    return code;
}

#define DCK(call)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return dfail(d, e_ == cudaErrorMemoryAllocation ? PIC_ENOMEM : PIC_ECUDA,       \
                         "%s failed: %s", #call, cudaGetErrorString(e_));                   \
    } while (0)

template <class T>
cudaError_t nalloc(pic_denoiser* d, T** p, size_t count) {
    *p = nullptr;
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
    if (e == cudaSuccess) d->allocs.push_back((void*)*p);
    return e;
}

void build_table(pic_denoiser* d) {
    PackTable& t = d->tab;
    memset(&t, 0, sizeof t);
    t.n = NL;
    long long off = 0, wf = 0, wd = 0, wp = 0;
    for (int l = 0; l < NL; ++l) {
        LayerDesc& L = t.layer[l];
        L.cin = kLayers[l].cin;
        L.cout = kLayers[l].cout;
        L.cin_pad = pad16(L.cin);
        L.cout_pad = padct(L.cout);
        L.woff = off;
        off += 9LL * L.cin * L.cout;
        d->boff[l] = off;
        off += L.cout;
        L.wf_off = wf;
        wf += 9LL * L.cout_pad * L.cin_pad;
        L.wp_off = -1;
        if (up_input(l)) {
            L.wp_off = wp;
            wp += 16LL * L.cout_pad * L.cin_pad;
        }
        if (l > 0) {  // no input gradient for the first layer
            L.dg_cin_pad = pad16(L.cout);
            L.dg_cout_pad = padct(L.cin);
            L.wd_off = wd;
            wd += 9LL * L.dg_cout_pad * L.dg_cin_pad;
        }
    }
    d->np = off;
}

long long packed_fwd(const pic_denoiser* d) {
    const LayerDesc& L = d->tab.layer[NL - 1];
    return L.wf_off + 9LL * L.cout_pad * L.cin_pad;
}
long long packed_up(const pic_denoiser* d) {
    long long n = 0;
    for (int l = 0; l < NL; ++l) {
        const LayerDesc& L = d->tab.layer[l];
        if (L.wp_off >= 0) n = L.wp_off + 16LL * L.cout_pad * L.cin_pad;
    }
    return n;
}
long long packed_dg(const pic_denoiser* d) {
    const LayerDesc& L = d->tab.layer[NL - 1];
    return L.wd_off + 9LL * L.dg_cout_pad * L.dg_cin_pad;
}

int dims(const pic_denoiser* d, int level, int* H, int* W) {
    *H = d->H >> level;
    *W = d->W >> level;
    return 0;
}

// Output-channel tile for a launch: 64 when the grid is large enough to fill
// the GPU twice over, else 32 (more, smaller CTAs for small layers).
int ctile_for(int cout, long long tiles) {
    const int t = ctile(cout);
    if (t == 64 && tiles * ((cout + 63) / 64) < 2 * 152) return 32;
    return t;
}

cudaError_t conv(pic_denoiser* d, int l, int B, const bf16* x, int epi, bf16* a_out,
                 const bf16* skip, bf16* y_out, float* g_out, cudaStream_t s,
                 const float* res = nullptr, float* fout = nullptr, long long bstride = 0,
                 long long cstride = 0, int pitch = 0, int offset = 0, float rs = 0.f,
                 float os = 0.f, int up = 0) {
    const LayerDesc& L = d->tab.layer[l];
    ConvParams p;
    memset(&p, 0, sizeof p);
    int H, W;
    dims(d, kLayers[l].level, &H, &W);
    p.x = x;
    p.B = B;
    p.H = H;
    p.W = W;
    p.up = up;
    p.epi = epi;
    p.status = d->cur_status;
    p.force_tc = d->force_tc;
    const long long tiles = (long long)B * (H / TH) * (W / TW);
    if (epi == EPI_GRAD) {
        p.w = d->wd + L.wd_off;
        p.cout = L.cin;
        p.cout_pad = L.dg_cout_pad;
        p.g_out = g_out;
        return launch_conv(p, L.dg_cin_pad, ctile_for(L.cin, tiles), s);
    }
    p.w = d->wf + L.wf_off;
    p.wp = (up && L.wp_off >= 0) ? d->wp + L.wp_off : nullptr;
    p.bias = d->master + d->boff[l];
    p.cout = L.cout;
    p.cout_pad = L.cout_pad;
    p.relu = kLayers[l].relu;
    p.a_out = a_out;
    p.skip = skip;
    p.y_out = y_out;
    p.res = res;
    p.fout = fout;
    p.bstride = bstride;
    p.cstride = cstride;
    p.pitch = pitch;
    p.offset = offset;
    p.rs = rs;
    p.os = os;
    return launch_conv(p, L.cin_pad, ctile_for(L.cout, tiles), s);
}

// Forward pass of B samples given in field layout (J, with the layout
// parameters); the output goes to `fout` in the same layout as out = J * rs +
// z11 * os.  Returns kernels launched or -1.
int forward(pic_denoiser* d, int B, const float* J, long long bstride, long long cstride,
            int pitch, int offset, float* fout, float rs, float os, cudaStream_t s,
            bool keep = false) {
    cudaError_t e;
    int n = 0;
    const int H0 = d->H, W0 = d->W, H1 = H0 / 2, W1 = W0 / 2;
#define FW(call)                                                                    \
    do {                                                                            \
        if ((e = (call)) != cudaSuccess) {                                          \
            d->err = std::string("denoiser launch failed: ") + cudaGetErrorString(e); \
            return -1;                                                              \
        }                                                                           \
        ++n;                                                                        \
    } while (0)
    // The thin first layer c1 (3 -> 32): on small lattices a CUDA-core kernel
    // fused with the input packing (one launch, no padded tensor-core tile);
    // on large ones, where its multiply-adds take longer than the tensor
    // cores' padded products plus one more pass over memory, the packing
    // kernel and the implicit GEMM (measured on GB300 at 2048^2: 296 against
    // 180 us).  (PIC_DENOISER_TC=always takes the tensor cores at every size.)
    const bool thin = (long long)B * H0 * W0 < kThinPixels && d->force_tc <= 0;
    if (thin) {
        const LayerDesc& L = d->tab.layer[0];
        FW(launch_conv_first(J, bstride, cstride, pitch, offset, B, H0, W0,
                             (float)(1.0 / d->scale), d->wf + L.wf_off, L.cout_pad,
                             d->master + d->boff[0], d->xin, d->a[0], s));
    } else {
        FW(launch_pack_input(J, bstride, cstride, pitch, offset, B, H0, W0, (float)(1.0 / d->scale),
                             d->xin, s));
        FW(conv(d, 0, B, d->xin, EPI_ACT, d->a[0], nullptr, nullptr, nullptr, s));
    }
    FW(conv(d, 1, B, d->a[0], EPI_ACT, d->a[1], nullptr, nullptr, nullptr, s));
    FW(launch_pool_fwd(d->a[1], B, H0, W0, 32, d->p1, s));
    FW(conv(d, 2, B, d->p1, EPI_ACT, d->a[2], nullptr, nullptr, nullptr, s));
    FW(conv(d, 3, B, d->a[2], EPI_ACT, d->a[3], nullptr, nullptr, nullptr, s));
    FW(launch_pool_fwd(d->a[3], B, H1, W1, 64, d->p2, s));
    FW(conv(d, 4, B, d->p2, EPI_ACT, d->a[4], nullptr, nullptr, nullptr, s));
    FW(conv(d, 5, B, d->a[4], EPI_ACT, d->a[5], nullptr, nullptr, nullptr, s));
    // c7 and c9 read the coarser level through the fused 2x upsampling; their
    // activations before the skip sum are kept only for a backward pass (keep)
    FW(conv(d, 6, B, d->a[5], EPI_ACT, keep ? d->a[6] : nullptr, d->a[3], d->y7, nullptr, s,
            nullptr, nullptr, 0, 0, 0, 0, 0.f, 0.f, 1));
    FW(conv(d, 7, B, d->y7, EPI_ACT, d->a[7], nullptr, nullptr, nullptr, s));
    FW(conv(d, 8, B, d->a[7], EPI_ACT, keep ? d->a[8] : nullptr, d->a[1], d->y9, nullptr, s,
            nullptr, nullptr, 0, 0, 0, 0, 0.f, 0.f, 1));
    FW(conv(d, 9, B, d->y9, EPI_ACT, d->a[9], nullptr, nullptr, nullptr, s));
    // c11 on the tensor cores at every size (its nine taps in the GEMM's N; below
    // 128-pixel rows the mma.sync kernel)
    FW(conv(d, 10, B, d->a[9], EPI_FINAL, nullptr, nullptr, nullptr, nullptr, s, J, fout, bstride,
            cstride, pitch, offset, rs, os));
    return n;
}

// Backward pass after forward(... fout = d->out, rs = 1/scale, os = 1) with
// the target in dense field layout; gradients into d->grad, loss into d->dloss.
int backward(pic_denoiser* d, int B, const float* target, cudaStream_t s) {
    cudaError_t e;
    int n = 0;
    const int H0 = d->H, W0 = d->W, H1 = H0 / 2, W1 = W0 / 2, H2 = H0 / 4, W2 = W0 / 4;
    const long long P0 = (long long)B * H0 * W0, P1 = P0 / 4, P2 = P0 / 16;
    const long long HW = (long long)H0 * W0;
    auto wg = [&](int l, const bf16* x, int up = 0) -> cudaError_t {
        const LayerDesc& L = d->tab.layer[l];
        int H, W;
        dims(d, kLayers[l].level, &H, &W);
        WgradParams p;
        p.x = x;
        p.dz = d->dz;
        p.B = B;
        p.H = H;
        p.W = W;
        p.up = up;
        p.cin = L.cin;
        p.cout = L.cout;
        p.dw = d->grad + L.woff;
        p.force_tc = d->force_tc;
        p.status = d->cur_status;
        return launch_wgrad(p, L.cin_pad, pad16(L.cout), s);
    };
    auto db = [&](int l) { return d->grad + d->boff[l]; };
    FW(cudaMemsetAsync(d->grad, 0, sizeof(float) * d->np, s));
    FW(cudaMemsetAsync(d->dloss, 0, sizeof(double), s));
    // c11: loss gradient
    FW(launch_mse(d->out, target, 3 * HW, HW, W0, 0, B, H0, W0, (float)(1.0 / d->scale), d->dz,
                  db(10), d->dloss, s));
    FW(wg(10, d->a[9]));
    FW(conv(d, 10, B, d->dz, EPI_GRAD, nullptr, nullptr, nullptr, d->G1, s));       // dy10
    // c10
    FW(launch_relu_back(d->G1, nullptr, d->a[9], P0, 32, d->dz, db(9), s));
    FW(wg(9, d->y9));
    FW(conv(d, 9, B, d->dz, EPI_GRAD, nullptr, nullptr, nullptr, d->S1, s));        // dy9 (= ds1)
    // c9 (+s1)
    FW(launch_relu_back(d->S1, nullptr, d->a[8], P0, 32, d->dz, db(8), s));
    FW(wg(8, d->a[7], 1));
    FW(conv(d, 8, B, d->dz, EPI_GRAD, nullptr, nullptr, nullptr, d->G0, s));        // du2
    // c8: dy8 = the upsampling adjoint of du2, through the ReLU
    FW(launch_up_relu_back(d->G0, B, H1, W1, 64, d->a[7], d->dz, db(7), s));
    FW(wg(7, d->y7));
    FW(conv(d, 7, B, d->dz, EPI_GRAD, nullptr, nullptr, nullptr, d->S2, s));        // dy7 (= ds2)
    // c7 (+s2)
    FW(launch_relu_back(d->S2, nullptr, d->a[6], P1, 64, d->dz, db(6), s));
    FW(wg(6, d->a[5], 1));
    FW(conv(d, 6, B, d->dz, EPI_GRAD, nullptr, nullptr, nullptr, d->G0, s));        // du1
    // c6: dy6 = the upsampling adjoint of du1, through the ReLU
    FW(launch_up_relu_back(d->G0, B, H2, W2, 128, d->a[5], d->dz, db(5), s));
    FW(wg(5, d->a[4]));
    FW(conv(d, 5, B, d->dz, EPI_GRAD, nullptr, nullptr, nullptr, d->G0, s));        // dy5
    // c5
    FW(launch_relu_back(d->G0, nullptr, d->a[4], P2, 128, d->dz, db(4), s));
    FW(wg(4, d->p2));
    FW(conv(d, 4, B, d->dz, EPI_GRAD, nullptr, nullptr, nullptr, d->G1, s));        // dp2
    // c4: dy4 = the pooling adjoint of dp2 + ds2, through the ReLU
    FW(launch_pool_relu_back(d->G1, B, H1, W1, 64, d->S2, d->a[3], d->dz, db(3), s));
    FW(wg(3, d->a[2]));
    FW(conv(d, 3, B, d->dz, EPI_GRAD, nullptr, nullptr, nullptr, d->G1, s));        // dy3
    // c3
    FW(launch_relu_back(d->G1, nullptr, d->a[2], P1, 64, d->dz, db(2), s));
    FW(wg(2, d->p1));
    FW(conv(d, 2, B, d->dz, EPI_GRAD, nullptr, nullptr, nullptr, d->G0, s));        // dp1
    // c2: dy2 = the pooling adjoint of dp1 + ds1, through the ReLU
    FW(launch_pool_relu_back(d->G0, B, H0, W0, 32, d->S1, d->a[1], d->dz, db(1), s));
    FW(wg(1, d->a[0]));
    FW(conv(d, 1, B, d->dz, EPI_GRAD, nullptr, nullptr, nullptr, d->G0, s));        // dy1
    // c1
    FW(launch_relu_back(d->G0, nullptr, d->a[0], P0, 32, d->dz, db(0), s));
    FW(wg(0, d->xin));
#undef FW
    return n;
}

// Low-wavenumber restoration out <- out + L^n (raw - out) over B samples
// (t: dense scratch of 3 B H W floats).  Returns kernels launched, or -1 with
// the reason in *err.
int low_k_chain(int n, int B, int H, int W, const FieldView& raw, const FieldView& out, float* t,
                cudaStream_t s, std::string* err) {
    if (n <= 0) return 0;
    const cudaError_t e = launch_lowk(raw, out, t, out, n, B, H, W, s);
    if (e != cudaSuccess) {
        *err = std::string("low-wavenumber restoration launch failed: ") + cudaGetErrorString(e);
        return -1;
    }
    return 2;
}

pic_status pack(pic_denoiser* d) {
    DCK(launch_pack_weights(d->tab, d->master, d->wf, d->wd, d->stream, d->wp));
    return PIC_OK;
}

const float* stage(pic_denoiser* d, const float* src, float* buf, size_t count, int on_device,
                   pic_status* st) {
    *st = PIC_OK;
    if (on_device) return src;
    cudaError_t e = cudaMemcpyAsync(buf, src, count * 4, cudaMemcpyHostToDevice, d->stream);
    if (e != cudaSuccess) {
        *st = dfail(d, PIC_ECUDA, "host-to-device copy failed: %s", cudaGetErrorString(e));
        return nullptr;
    }
    return buf;
}

// the device status word after a synchronisation: a bounded wait that ran out
pic_status check_status(pic_denoiser* d) {
    unsigned h = 0;
    DCK(cudaMemcpy(&h, d->status, sizeof h, cudaMemcpyDeviceToHost));
    if (h) {
        DCK(cudaMemset(d->status, 0, sizeof(unsigned)));
        return dfail(d, PIC_ETIMEOUT, "a bounded wait in a tensor-core kernel ran out");
    }
    return PIC_OK;
}

pic_status run_grad(pic_denoiser* d, const float* J_in, const float* J_t, int batch, int on_device,
                    double* loss) {
    if (batch < 1 || batch > d->Bmax) return dfail(d, PIC_EINVAL, "batch %d not in 1..%d", batch, d->Bmax);
    if (!J_in || !J_t) return dfail(d, PIC_EINVAL, "null input");
    const size_t cnt = (size_t)batch * 3 * d->H * d->W;
    pic_status st;
    const float* in = stage(d, J_in, d->stage_in, cnt, on_device, &st);
    if (st != PIC_OK) return st;
    const float* tg = stage(d, J_t, d->stage_t, cnt, on_device, &st);
    if (st != PIC_OK) return st;
    const long long HW = (long long)d->H * d->W;
    if (forward(d, batch, in, 3 * HW, HW, d->W, 0, d->out, (float)(1.0 / d->scale), 1.f,
                d->stream, true) < 0)
        return PIC_ECUDA;
    if (backward(d, batch, tg, d->stream) < 0) return PIC_ECUDA;
    if (loss) {
        DCK(cudaMemcpyAsync(loss, d->dloss, sizeof(double), cudaMemcpyDeviceToHost, d->stream));
    }
    DCK(cudaStreamSynchronize(d->stream));
    return check_status(d);
}

// the current-filter hook: the network applied to J[b] in place
int filter_hook(void* ctx, pic_sim* sim, cudaStream_t s, int b) {
    pic_denoiser* d = static_cast<pic_denoiser*>(ctx);
    const Geom& g = sim->g;
    const FieldView J{sim->J[b], 3 * g.cstride, g.cstride, g.P, GY * g.P + GX};
    // scratch of the restoration (the gradient buffers, idle outside training):
    // the raw current and the row-filtered difference, 3 H W floats each
    const long long n3 = 3LL * d->H * d->W;
    const FieldView raw{d->G0, n3, (long long)d->H * d->W, d->W, 0};
    int k0 = 0;
    if (d->restore > 0) {
        const cudaError_t e = launch_field_copy(J, raw, 1, d->H, d->W, s);
        if (e != cudaSuccess) {
            sim->err = std::string("denoiser copy launch failed: ") + cudaGetErrorString(e);
            return -1;
        }
        k0 = 1;
    }
    d->cur_status = &sim->st->status;  // timeouts show in the simulation's status (ST_TIMEOUT)
    const int k = forward(d, 1, sim->J[b], 3 * g.cstride, g.cstride, g.P, GY * g.P + GX, sim->J[b],
                          1.f, (float)d->scale, s);
    d->cur_status = d->status;
    if (k < 0) {
        sim->err = d->err;
        return k;
    }
    const int kr = low_k_chain(d->restore, 1, d->H, d->W, raw, J, d->G0 + n3, s, &sim->err);
    return kr < 0 ? -1 : k0 + k + kr;
}

}  // namespace

namespace pic {
namespace host {

bool denoiser_fits(const pic_denoiser* d, const Geom& g) { return d && d->W == g.nx && d->H == g.ny; }

// The current-filter slot of B simulations of one grid at once: their
// currents (device table jtab, field layout of g) are gathered into a dense
// batch of samples, run through the network in groups of at most batch_max,
// restored, and written back in place.  Kernel timeouts are reported to
// `status`.  Returns the kernels launched, or -1 with the message in *err.
int denoiser_batch_filter(pic_denoiser* d, float* const* jtab, int B, const Geom& g,
                          unsigned* status, cudaStream_t s, std::string* err) {
    const int H = d->H, W = d->W;
    const long long HW = (long long)H * W;
    const FieldView jl{nullptr, 0, g.cstride, g.P, GY * g.P + GX};
    const FieldView X{d->G1, 3 * HW, HW, W, 0};    // the batch, denoised in place
    const FieldView raw{d->G0, 3 * HW, HW, W, 0};  // the restoration's copy of the input
    const FieldView none{nullptr, 0, 0, 0, 0};
    int n = 0;
    for (int g0 = 0; g0 < B; g0 += d->Bmax) {
        const int nb = std::min(d->Bmax, B - g0);
        cudaError_t e = launch_field_copy_tab(jl, jtab + g0, X, nullptr, d->restore > 0 ? raw : none,
                                              nb, H, W, s);
        if (e != cudaSuccess) {
            *err = std::string("denoiser gather launch failed: ") + cudaGetErrorString(e);
            return -1;
        }
        d->cur_status = status;
        const int k = forward(d, nb, d->G1, 3 * HW, HW, W, 0, d->G1, 1.f, (float)d->scale, s);
        d->cur_status = d->status;
        if (k < 0) {
            *err = d->err;
            return -1;
        }
        const int kr = low_k_chain(d->restore, nb, H, W, raw, X, d->G0 + 3LL * nb * HW, s, err);
        if (kr < 0) return -1;
        e = launch_field_copy_tab(X, nullptr, jl, jtab + g0, none, nb, H, W, s);
        if (e != cudaSuccess) {
            *err = std::string("denoiser scatter launch failed: ") + cudaGetErrorString(e);
            return -1;
        }
        n += 2 + k + kr;
    }
    return n;
}

}  // namespace host
}  // namespace pic

namespace {

// Pack random-access probe weights ([9][cin][cout] FP32, device) for one layer shape.
struct Probe {
    bf16 *wf = nullptr, *wd = nullptr;
    unsigned* st = nullptr;
    // synchronise; a bounded wait that ran out gives PIC_ETIMEOUT
    pic_status finish(cudaStream_t s) {
        if (cudaStreamSynchronize(s) != cudaSuccess) return PIC_ECUDA;
        unsigned h = 0;
        if (cudaMemcpy(&h, st, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) return PIC_ECUDA;
        return h ? PIC_ETIMEOUT : PIC_OK;
    }
    ~Probe() {
        cudaFree(wf);
        cudaFree(wd);
        cudaFree(st);
    }
};

}  // namespace

extern "C" {

int64_t pic_denoiser_num_params(void) {
    pic_denoiser d;
    build_table(&d);
    return d.np;
}

pic_status pic_denoiser_create(int nx, int ny, int batch_max, double scale, void* cuda_stream,
                               pic_denoiser** out) {
    if (!out) return PIC_EINVAL;
    *out = nullptr;
    if (nx < 64 || ny < 32 || nx % 64 || ny % 32 || ny > 65535 || batch_max < 1 || batch_max > 4096 ||
        !(scale > 0) || !std::isfinite(scale))
        return PIC_EINVAL;
    const long long P0 = (long long)batch_max * nx * ny;
    if (P0 > (1LL << 28)) return PIC_EINVAL;
    pic_denoiser* d = new pic_denoiser();
    d->H = ny;
    d->W = nx;
    d->Bmax = batch_max;
    d->scale = scale;
    d->stream = (cudaStream_t)cuda_stream;
    if (const char* v = getenv("PIC_DENOISER_TC"))
        d->force_tc = strcmp(v, "always") == 0 ? 1 : (strcmp(v, "never") == 0 ? -1 : 0);
    build_table(d);
    const long long P1 = P0 / 4, P2 = P0 / 16;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p, size_t n) {
        if (e == cudaSuccess) e = nalloc(d, p, n);
    };
    A(&d->master, d->np);
    A(&d->grad, d->np);
    A(&d->m, d->np);
    A(&d->v, d->np);
    A(&d->wf, packed_fwd(d));
    A(&d->wd, packed_dg(d));
    A(&d->wp, packed_up(d));
    A(&d->xin, P0 * 16);
    const long long lvl[3] = {P0, P1, P2};
    for (int l = 0; l < NL - 1; ++l) A(&d->a[l], lvl[kLayers[l].level] * kLayers[l].cout);
    A(&d->y7, P1 * 64);
    A(&d->y9, P0 * 32);
    A(&d->p1, P1 * 32);
    A(&d->p2, P2 * 64);
    A(&d->out, P0 * 3);
    A(&d->dz, P0 * 32);
    A(&d->G0, P0 * 64);
    A(&d->G1, P0 * 32);
    A(&d->S1, P0 * 32);
    A(&d->S2, P1 * 64);
    A(&d->dloss, 1);
    A(&d->status, 1);
    A(&d->stage_in, P0 * 3);
    A(&d->stage_t, P0 * 3);
    // shared-memory limits of every kernel shape, set before any graph capture
    if (e == cudaSuccess) e = init_kernels();
    if (e == cudaSuccess) e = cudaMemsetAsync(d->status, 0, sizeof(unsigned), d->stream);
    d->cur_status = d->status;
    if (e == cudaSuccess) e = cudaMemsetAsync(d->master, 0, sizeof(float) * d->np, d->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d->m, 0, sizeof(float) * d->np, d->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d->v, 0, sizeof(float) * d->np, d->stream);
    if (e == cudaSuccess)
        e = launch_pack_weights(d->tab, d->master, d->wf, d->wd, d->stream, d->wp);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    if (e != cudaSuccess) {
        pic_denoiser_destroy(d);
        return e == cudaErrorMemoryAllocation ? PIC_ENOMEM : PIC_ECUDA;
    }
    *out = d;
    return PIC_OK;
}

pic_status pic_denoiser_set_params(pic_denoiser* d, const float* params, int on_device) {
    if (!d || !params) return PIC_EINVAL;
    d->err.clear();
    DCK(cudaMemcpyAsync(d->master, params, sizeof(float) * d->np,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, d->stream));
    DCK(cudaMemsetAsync(d->m, 0, sizeof(float) * d->np, d->stream));
    DCK(cudaMemsetAsync(d->v, 0, sizeof(float) * d->np, d->stream));
    d->adam_t = 0;
    pic_status r = pack(d);
    if (r != PIC_OK) return r;
    DCK(cudaStreamSynchronize(d->stream));
    return PIC_OK;
}

pic_status pic_denoiser_get_params(pic_denoiser* d, float* params, int on_device) {
    if (!d || !params) return PIC_EINVAL;
    d->err.clear();
    DCK(cudaMemcpyAsync(params, d->master, sizeof(float) * d->np,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, d->stream));
    DCK(cudaStreamSynchronize(d->stream));
    return PIC_OK;
}

pic_status pic_denoiser_forward(pic_denoiser* d, const float* J_in, float* J_out, int batch,
                                int on_device) {
    if (!d) return PIC_EINVAL;
    d->err.clear();
    if (batch < 1 || batch > d->Bmax) return dfail(d, PIC_EINVAL, "batch %d not in 1..%d", batch, d->Bmax);
    if (!J_in || !J_out) return dfail(d, PIC_EINVAL, "null buffer");
    const size_t cnt = (size_t)batch * 3 * d->H * d->W;
    pic_status st;
    const float* in = stage(d, J_in, d->stage_in, cnt, on_device, &st);
    if (st != PIC_OK) return st;
    float* o = on_device ? J_out : d->stage_t;
    const long long HW = (long long)d->H * d->W;
    FieldView vin{const_cast<float*>(in), 3 * HW, HW, d->W, 0};
    const FieldView vout{o, 3 * HW, HW, d->W, 0};
    if (d->restore > 0 && in == o) {
        // in place: keep the raw current for the restoration
        const FieldView keep{d->G0 + cnt, 3 * HW, HW, d->W, 0};
        DCK(launch_field_copy(vin, keep, batch, d->H, d->W, d->stream));
        vin = keep;
    }
    if (forward(d, batch, in, 3 * HW, HW, d->W, 0, o, 1.f, (float)d->scale, d->stream) < 0)
        return PIC_ECUDA;
    if (low_k_chain(d->restore, batch, d->H, d->W, vin, vout, d->G0, d->stream, &d->err) < 0)
        return PIC_ECUDA;
    if (!on_device)
        DCK(cudaMemcpyAsync(J_out, o, cnt * 4, cudaMemcpyDeviceToHost, d->stream));
    DCK(cudaStreamSynchronize(d->stream));
    return check_status(d);
}

pic_status pic_denoiser_grad(pic_denoiser* d, const float* J_in, const float* J_target, int batch,
                             double* loss, float* grads, int on_device) {
    if (!d) return PIC_EINVAL;
    d->err.clear();
    pic_status r = run_grad(d, J_in, J_target, batch, on_device, loss);
    if (r != PIC_OK) return r;
    if (grads) {
        DCK(cudaMemcpyAsync(grads, d->grad, sizeof(float) * d->np,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            d->stream));
        DCK(cudaStreamSynchronize(d->stream));
    }
    return PIC_OK;
}

pic_status pic_denoiser_train_step(pic_denoiser* d, const float* J_in, const float* J_target,
                                   int batch, float lr, double* loss, int on_device) {
    if (!d) return PIC_EINVAL;
    d->err.clear();
    if (!(lr > 0) || !std::isfinite(lr)) return dfail(d, PIC_EINVAL, "bad learning rate");
    pic_status r = run_grad(d, J_in, J_target, batch, on_device, loss);
    if (r != PIC_OK) return r;
    d->adam_t += 1;
    const double b1 = 0.9, b2 = 0.999;
    const double c1 = 1.0 / (1.0 - std::pow(b1, (double)d->adam_t));
    const double c2 = 1.0 / (1.0 - std::pow(b2, (double)d->adam_t));
    DCK(launch_adam(d->master, d->grad, d->m, d->v, d->np, lr, (float)b1, (float)b2, 1e-8f,
                    (float)c1, (float)c2, d->stream));
    r = pack(d);
    if (r != PIC_OK) return r;
    DCK(cudaStreamSynchronize(d->stream));
    return PIC_OK;
}

pic_status pic_set_denoiser(pic_sim* sim, pic_denoiser* d) {
    if (!sim) return PIC_EINVAL;
    sim->err.clear();
    if (d && (d->H != sim->cfg.ny || d->W != sim->cfg.nx))
        return fail(sim, PIC_EINVAL, "denoiser grid %dx%d differs from the simulation's %dx%d",
                    d->W, d->H, sim->cfg.nx, sim->cfg.ny);
    if (d && sim->window)
        return fail(sim, PIC_EINVAL, "the denoiser pads periodically: not with the moving window");
    PIC_CK(sim, cudaStreamSynchronize(sim->stream));
    sim->jfilter = d ? filter_hook : nullptr;
    sim->jfilter_ctx = d;
    sim->binomial_passes = 0;
    invalidate_graphs(sim);
    return PIC_OK;
}

pic_status pic_denoiser_set_low_k_restore(pic_denoiser* d, int passes) {
    if (!d) return PIC_EINVAL;
    d->err.clear();
    if (passes < 0 || passes > PIC_LOW_K_MAX_PASSES)
        return dfail(d, PIC_EINVAL, "passes %d not in 0..%d", passes, PIC_LOW_K_MAX_PASSES);
    d->restore = passes;
    return PIC_OK;
}

const char* pic_denoiser_last_error(const pic_denoiser* d) {
    return d ? d->err.c_str() : "null handle";
}

void pic_denoiser_destroy(pic_denoiser* d) {
    if (!d) return;
    if (d->stream) cudaStreamSynchronize(d->stream);
    for (void* p : d->allocs) cudaFree(p);
    delete d;
}

// ---- kernel-level probes (device pointers) ----------------------------------

pic_status pic_nn_conv3x3(const void* x, int B, int H, int W, int cin, int cout, const float* w,
                          const float* bias, int relu, const void* skip, void* a_out, void* y_out,
                          void* cuda_stream) {
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (!x || !w || !a_out || B < 1 || H % TH || W % TW || cin < 1 || cin > 128 ||
        !(cout == 32 || cout == 64 || cout == 128) || (skip && !y_out))
        return PIC_EINVAL;
    const int cin_pad = pad16(cin), ct = ctile(cout), cout_pad = padct(cout);
    PackTable t;
    memset(&t, 0, sizeof t);
    t.n = 1;
    LayerDesc& L = t.layer[0];
    L.cin = cin;
    L.cout = cout;
    L.cin_pad = cin_pad;
    L.cout_pad = cout_pad;
    Probe pr;
    if (cudaMalloc((void**)&pr.wf, 2 * 9LL * cout_pad * cin_pad) != cudaSuccess) return PIC_ENOMEM;
    if (launch_pack_weights(t, w, pr.wf, nullptr, s) != cudaSuccess) return PIC_ECUDA;
    if (cudaMalloc((void**)&pr.st, sizeof(unsigned)) != cudaSuccess) return PIC_ENOMEM;
    if (cudaMemsetAsync(pr.st, 0, sizeof(unsigned), s) != cudaSuccess) return PIC_ECUDA;
    ConvParams p;
    memset(&p, 0, sizeof p);
    p.status = pr.st;
    p.force_tc = 1;  // a probe exercises the tensor-core kernel whenever the shape allows
    p.x = (const bf16*)x;
    p.B = B;
    p.H = H;
    p.W = W;
    p.w = pr.wf;
    p.bias = bias;
    p.cout = cout;
    p.cout_pad = cout_pad;
    p.epi = EPI_ACT;
    p.relu = relu;
    p.a_out = (bf16*)a_out;
    p.skip = (const bf16*)skip;
    p.y_out = (bf16*)y_out;
    if (launch_conv(p, cin_pad, ct, s) != cudaSuccess) return PIC_ECUDA;
    return pr.finish(s);
}

pic_status pic_nn_conv3x3_dgrad(const void* dz, int B, int H, int W, int cin, int cout,
                                const float* w, float* dx, void* cuda_stream) {
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (!dz || !w || !dx || B < 1 || H % TH || W % TW || !(cin == 32 || cin == 64 || cin == 128) ||
        cout < 1 || cout > 128)
        return PIC_EINVAL;
    PackTable t;
    memset(&t, 0, sizeof t);
    t.n = 1;
    LayerDesc& L = t.layer[0];
    L.cin = cin;
    L.cout = cout;
    L.cin_pad = pad16(cin);
    L.cout_pad = 0;  // no forward packing
    L.dg_cin_pad = pad16(cout);
    L.dg_cout_pad = padct(cin);
    Probe pr;
    if (cudaMalloc((void**)&pr.wd, 2 * 9LL * L.dg_cout_pad * L.dg_cin_pad) != cudaSuccess)
        return PIC_ENOMEM;
    if (launch_pack_weights(t, w, nullptr, pr.wd, s) != cudaSuccess) return PIC_ECUDA;
    if (cudaMalloc((void**)&pr.st, sizeof(unsigned)) != cudaSuccess) return PIC_ENOMEM;
    if (cudaMemsetAsync(pr.st, 0, sizeof(unsigned), s) != cudaSuccess) return PIC_ECUDA;
    ConvParams p;
    memset(&p, 0, sizeof p);
    p.status = pr.st;
    p.force_tc = 1;
    p.x = (const bf16*)dz;
    p.B = B;
    p.H = H;
    p.W = W;
    p.w = pr.wd;
    p.cout = cin;
    p.cout_pad = L.dg_cout_pad;
    p.epi = EPI_GRAD;
    p.g_out = dx;
    if (launch_conv(p, L.dg_cin_pad, ctile(cin), s) != cudaSuccess) return PIC_ECUDA;
    return pr.finish(s);
}

pic_status pic_nn_low_k_restore(const float* raw, float* out, int B, int H, int W, int passes,
                                void* cuda_stream) {
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (!raw || !out || B < 1 || B > 4096 || H < 1 || H > 65535 || W < 1 || passes < 0 ||
        passes > PIC_LOW_K_MAX_PASSES || (long long)B * H * W > (1LL << 28))
        return PIC_EINVAL;
    const long long n = 3LL * B * H * W, HW = (long long)H * W;
    float* scratch = nullptr;
    if (passes > 0 && cudaMalloc((void**)&scratch, n * sizeof(float)) != cudaSuccess)
        return PIC_ENOMEM;
    const FieldView vr{const_cast<float*>(raw), 3 * HW, HW, W, 0}, vo{out, 3 * HW, HW, W, 0};
    std::string err;
    const int k = low_k_chain(passes, B, H, W, vr, vo, scratch, s, &err);
    const bool ok = k >= 0 && cudaStreamSynchronize(s) == cudaSuccess;
    cudaFree(scratch);
    return ok ? PIC_OK : PIC_ECUDA;
}

pic_status pic_nn_conv3x3_wgrad(const void* x, const void* dz, int B, int H, int W, int cin,
                                int cout, float* dw, void* cuda_stream) {
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (!x || !dz || !dw || B < 1 || H < 1 || W < 16 || ((long long)B * H * W) % WG_PIX ||
        cin < 1 || cin > 128 || cout < 1 || cout > 128)
        return PIC_EINVAL;
    WgradParams p;
    p.x = (const bf16*)x;
    p.dz = (const bf16*)dz;
    p.B = B;
    p.H = H;
    p.W = W;
    p.up = 0;
    p.cin = cin;
    p.cout = cout;
    p.dw = dw;
    p.force_tc = 1;  // a probe exercises the tensor-core kernel whenever the shape allows
    p.status = nullptr;
    if (cudaMemsetAsync(dw, 0, sizeof(float) * 9 * cin * cout, s) != cudaSuccess) return PIC_ECUDA;
    if (launch_wgrad(p, pad16(cin), pad16(cout), s) != cudaSuccess) return PIC_EINVAL;
    return cudaStreamSynchronize(s) == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

}  // extern "C"
