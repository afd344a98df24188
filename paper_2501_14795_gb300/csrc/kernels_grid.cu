// Grid kernels: the fused Yee advance (§3.1 three-step scheme, §4.4 tiled
// field advance), guard-cell copies, field energies, charge density and the
// FP64 charge-conservation residuals, and the initial particle load/sort.
#include <algorithm>

#include "device_util.cuh"
#include "pic_internal.h"

namespace pic {

namespace {

__device__ __forceinline__ long long gidx(const Geom& g, int i, int j) {
    return (long long)(j + GY) * g.P + (i + GX);
}

// ---------------------------------------------------------------- Yee
// One CTA per field tile of YX x YY cells.  Shared memory holds E on cells
// [-1, YX+2) x [-1, YY+2), B on [-1, YX+1) x [-1, YY+1), J on [0, YX+1) x
// [0, YY+1).  In place: B <- B - dt/2 curl E on the B region, then
// E <- E + dt (curl B - J) on [0, YX+1)^2, then B <- B - dt/2 curl E on the
// tile (Eqs. 19-20 on the staggered grid of Fig. 3.1).  The tile of E|B at
// n+1 is written with its periodic images (update_gc_copy), the field
// energies of level n+1 are summed in FP64, and the shared ring of the next
// step's J buffer (cells a neighbouring particle tile's halo reaches) is
// zeroed.  With the moving window (open box along x) the fields outside
// 0 <= i < nx stay zero through the three sub-steps, the x guards are written
// as zeros, and on a step that shifts the window every value is written one
// column to the left (the last column becoming zero): the shift of E and B at
// the end of Listing 3.1 costs no extra pass.
constexpr int YX = 32, YY = 16, YTHREADS = 256;
constexpr int EW = YX + 3, EH = YY + 3;
constexpr int BW = YX + 2, BH = YY + 2;
constexpr int JWY = YX + 1, JHY = YY + 1;

// Shared-memory layouts of the Yee halos: local (q, r) is cell (i0-1+q,
// j0-1+r) for E and B and (i0+q, j0+r) for J.
struct YeePlain {  // the plain-load kernel's arrays [3][EH][EW], [3][BH][BW], [3][JHY][JWY]
    static __device__ __forceinline__ int e(int c, int r, int q) { return (c * EH + r) * EW + q; }
    static __device__ __forceinline__ int b(int c, int r, int q) { return (c * BH + r) * BW + q; }
    static __device__ __forceinline__ int j(int c, int r, int q) { return (c * JHY + r) * JWY + q; }
};
// TMA boxes: E and B as [3][19][40] from cell (i0-4, j0-1) (the box's x origin
// on a 16-byte boundary), J as [3][17][36] from cell (i0, j0)
constexpr int TEW = 40, TEH = 19, TJW = 36, TJH = 17;
struct YeeTma {
    static __device__ __forceinline__ int e(int c, int r, int q) { return (c * TEH + r) * TEW + q + 3; }
    static __device__ __forceinline__ int b(int c, int r, int q) { return (c * TEH + r) * TEW + q + 3; }
    static __device__ __forceinline__ int j(int c, int r, int q) { return (c * TJH + r) * TJW + q; }
};

// The three sub-steps and the write-out of tile (i0, j0) from its halos in
// shared memory (updated in place); the tile's field energies are added to
// we, wb.  Every thread of the CTA calls it.
template <class LAY>
__device__ __forceinline__ void yee_body(const YeeParams& prm, int i0, int j0, float* sE,
                                         float* sB, const float* sJ, float& we, float& wb) {
    const Geom& g = prm.g;
    const int tid = threadIdx.x;
    const long long cs = g.cstride;
    const float hx = g.hdt_dx, hy = g.hdt_dy;
    const bool open = g.open_x != 0;
    // B half step on [-1, YX+1) x [-1, YY+1): local (q, r) <-> cell (i0-1+q, j0-1+r)
    for (int k = tid; k < BW * BH; k += YTHREADS) {
        const int r = k / BW, q = k - r * BW;
        if (open && (i0 - 1 + q < 0 || i0 - 1 + q >= g.nx)) {  // outside the open box
            sB[LAY::b(0, r, q)] = sB[LAY::b(1, r, q)] = sB[LAY::b(2, r, q)] = 0.f;
            continue;
        }
        sB[LAY::b(0, r, q)] -= hy * (sE[LAY::e(2, r + 1, q)] - sE[LAY::e(2, r, q)]);
        sB[LAY::b(1, r, q)] += hx * (sE[LAY::e(2, r, q + 1)] - sE[LAY::e(2, r, q)]);
        sB[LAY::b(2, r, q)] -= hx * (sE[LAY::e(1, r, q + 1)] - sE[LAY::e(1, r, q)]) - hy * (sE[LAY::e(0, r + 1, q)] - sE[LAY::e(0, r, q)]);
    }
    __syncthreads();
    // E full step on cells [0, YX+1) x [0, YY+1): E at (q+1, r+1), B at (q+1, r+1)
    const float dtx = g.dt_dx, dty = g.dt_dy, dt = g.dt;
    for (int k = tid; k < JWY * JHY; k += YTHREADS) {
        const int r = k / JWY, q = k - r * JWY;
        const int e = q + 1, f = r + 1;
        if (open && i0 + q >= g.nx) {
            sE[LAY::e(0, f, e)] = sE[LAY::e(1, f, e)] = sE[LAY::e(2, f, e)] = 0.f;
            continue;
        }
        sE[LAY::e(0, f, e)] += dty * (sB[LAY::b(2, f, e)] - sB[LAY::b(2, f - 1, e)]) - dt * sJ[LAY::j(0, r, q)];
        sE[LAY::e(1, f, e)] += -dtx * (sB[LAY::b(2, f, e)] - sB[LAY::b(2, f, e - 1)]) - dt * sJ[LAY::j(1, r, q)];
        sE[LAY::e(2, f, e)] += dtx * (sB[LAY::b(1, f, e)] - sB[LAY::b(1, f, e - 1)]) -
                       dty * (sB[LAY::b(0, f, e)] - sB[LAY::b(0, f - 1, e)]) - dt * sJ[LAY::j(2, r, q)];
    }
    __syncthreads();
    // B second half step on the tile, write out with images, energies, J ring
    float* Eout = prm.Fout;
    float* Bout = prm.Fout + 3 * cs;
    const int T = g.T;
    const int wshift = open ? *((volatile int*)&prm.st->win_shift) : 0;
    for (int k = tid; k < YX * YY; k += YTHREADS) {
        const int r = k / YX, q = k - r * YX;
        const int i = i0 + q, j = j0 + r;
        if (i >= g.nx || j >= g.ny) continue;
        const int e = q + 1, f = r + 1;
        float bx = sB[LAY::b(0, f, e)] - hy * (sE[LAY::e(2, f + 1, e)] - sE[LAY::e(2, f, e)]);
        float by = sB[LAY::b(1, f, e)] + hx * (sE[LAY::e(2, f, e + 1)] - sE[LAY::e(2, f, e)]);
        float bz = sB[LAY::b(2, f, e)] - (hx * (sE[LAY::e(1, f, e + 1)] - sE[LAY::e(1, f, e)]) -
                                  hy * (sE[LAY::e(0, f + 1, e)] - sE[LAY::e(0, f, e)]));
        const float ex = sE[LAY::e(0, f, e)], ey = sE[LAY::e(1, f, e)], ez = sE[LAY::e(2, f, e)];
        we += ex * ex + ey * ey + ez * ez;
        wb += bx * bx + by * by + bz * bz;
        // images: i' in {i, i+nx if i<2, i-nx if i==nx-1}, same for j
        int jj[2], nj = 1;
        jj[0] = j;
        if (j < 2) jj[nj++] = j + g.ny;
        else if (j == g.ny - 1) jj[nj++] = -1;
        if (!open) {
            int ii[2], ni = 1;
            ii[0] = i;
            if (i < 2) ii[ni++] = i + g.nx;
            else if (i == g.nx - 1) ii[ni++] = -1;
            for (int a = 0; a < ni; ++a)
                for (int b = 0; b < nj; ++b) {
                    const long long o = gidx(g, ii[a], jj[b]);
                    Eout[o] = ex;
                    Eout[cs + o] = ey;
                    Eout[2 * cs + o] = ez;
                    Bout[o] = bx;
                    Bout[cs + o] = by;
                    Bout[2 * cs + o] = bz;
                }
        } else {
            // open box: the value goes to column d = i - shift; the guard
            // columns (and, on a shift, the new last column) get zeros
            const int d = i - wshift;
            for (int b = 0; b < nj; ++b) {
                if (d >= 0) {
                    const long long o = gidx(g, d, jj[b]);
                    Eout[o] = ex;
                    Eout[cs + o] = ey;
                    Eout[2 * cs + o] = ez;
                    Bout[o] = bx;
                    Bout[cs + o] = by;
                    Bout[2 * cs + o] = bz;
                }
                const int z0 = d == 0 ? -1 : (i == g.nx - 1 ? d + 1 : 1);
                const int z1 = i == g.nx - 1 ? g.nx + 1 : (d == 0 ? -1 : 0);
                for (int zc = z0; zc <= z1; ++zc) {
                    const long long o = gidx(g, zc, jj[b]);
#pragma unroll
                    for (int c = 0; c < 3; ++c) Eout[c * cs + o] = Bout[c * cs + o] = 0.f;
                }
            }
        }
        const int mi = i % T, mj = j % T;
        const bool ring = prm.zero_all || mi < 2 || mi == T - 1 || mj < 2 || mj == T - 1;
        if (ring) {
            const long long o = gidx(g, i, j);
            prm.Jnext[o] = 0.f;
            prm.Jnext[cs + o] = 0.f;
            prm.Jnext[2 * cs + o] = 0.f;
        }
    }
}

__device__ __forceinline__ void yee_tile(const YeeParams& prm, int bx, int by) {
    __shared__ float sE[3 * EH * EW];
    __shared__ float sB[3 * BH * BW];
    __shared__ float sJ[3 * JHY * JWY];
    __shared__ double sRed[32];
    const Geom& g = prm.g;
    const int i0 = bx * YX, j0 = by * YY;
    const int tid = threadIdx.x;
    const long long cs = g.cstride;
    const float* Ein = prm.Fin;
    const float* Bin = prm.Fin + 3 * cs;

    for (int k = tid; k < EW * EH; k += YTHREADS) {
        const int r = k / EW, q = k - r * EW;
        const int i = i0 - 1 + q, j = j0 - 1 + r;
        const bool in = i <= g.nx + 1 && j <= g.ny + 1;
        const long long o = gidx(g, i, j);
#pragma unroll
        for (int c = 0; c < 3; ++c) sE[YeePlain::e(c, r, q)] = in ? Ein[c * cs + o] : 0.f;
    }
    for (int k = tid; k < BW * BH; k += YTHREADS) {
        const int r = k / BW, q = k - r * BW;
        const int i = i0 - 1 + q, j = j0 - 1 + r;
        const bool in = i <= g.nx + 1 && j <= g.ny + 1;
        const long long o = gidx(g, i, j);
#pragma unroll
        for (int c = 0; c < 3; ++c) sB[YeePlain::b(c, r, q)] = in ? Bin[c * cs + o] : 0.f;
    }
    for (int k = tid; k < JWY * JHY; k += YTHREADS) {
        const int r = k / JWY, q = k - r * JWY;
        int i = i0 + q, j = j0 + r;
        i = i >= g.nx ? i - g.nx : i;
        j = j >= g.ny ? j - g.ny : j;
        const bool in = i < g.nx && j < g.ny;
        const long long o = gidx(g, i, j);
#pragma unroll
        for (int c = 0; c < 3; ++c) sJ[YeePlain::j(c, r, q)] = in ? prm.J[c * cs + o] : 0.f;
    }
    __syncthreads();
    float we = 0.f, wb = 0.f;
    yee_body<YeePlain>(prm, i0, j0, sE, sB, sJ, we, wb);
    const double dxdy = g.dx * g.dy;
    const long long n = *((volatile long long*)&prm.st->step);
    const double se = dev::block_sum((double)we, sRed);
    if (tid == 0) atomicAdd(&prm.hist_e[n & (HIST - 1)], 0.5 * se * dxdy);
    const double sb = dev::block_sum((double)wb, sRed);
    if (tid == 0) atomicAdd(&prm.hist_b[n & (HIST - 1)], 0.5 * sb * dxdy);
}

// One simulation, persistent: CTA k takes Yee tiles k, k + gridDim.x, ...;
// each tile's E|B and J halos come in by three TMA boxes into one of two
// stages while the other stage is being computed.  J's guard cells hold no
// images, so the J values of cells nx and ny (which the E step needs at the
// tile edges) are patched in from cells 0 after the copy.
// bytes each stage receives, and its layout with every box on a 128-byte boundary
constexpr unsigned TBOX_E = 3 * TEH * TEW * 4, TBOX_J = 3 * TJH * TJW * 4;  // 9120, 7344
constexpr unsigned TTX_BYTES = 2 * TBOX_E + TBOX_J;
constexpr int TOFF_B = ((TBOX_E + 127) / 128) * 128 / 4;        // floats
constexpr int TOFF_J = 2 * TOFF_B;
constexpr int TSTAGE_FLOATS = TOFF_J + ((TBOX_J + 127) / 128) * 128 / 4;
constexpr unsigned TSTAGE_BYTES = TSTAGE_FLOATS * 4;
constexpr size_t YEE_TMA_SMEM = 2 * (size_t)TSTAGE_BYTES + 64 + 32 * sizeof(double);
static_assert(TSTAGE_BYTES % 128 == 0, "stages on 128-byte boundaries");

__global__ void __launch_bounds__(YTHREADS) k_yee_tma(const __grid_constant__ CUtensorMap mapF,
                                                     const __grid_constant__ CUtensorMap mapJ,
                                                     const YeeParams prm) {
    extern __shared__ __align__(128) unsigned char smem[];
    float* stage0 = reinterpret_cast<float*>(smem);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * (size_t)TSTAGE_BYTES);
    double* sRed = reinterpret_cast<double*>(smem + 2 * (size_t)TSTAGE_BYTES + 64);
    const Geom& g = prm.g;
    const int tid = threadIdx.x;
    const long long cs = g.cstride;
    const int nbx = (g.nx + YX - 1) / YX, nt = nbx * ((g.ny + YY - 1) / YY);
    if (tid == 0) {
        dev::mbar_init(bar, 1);
        dev::mbar_init(bar + 1, 1);
        dev::fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int t, int st) {
        float* dst = stage0 + st * TSTAGE_FLOATS;
        const int i0 = (t % nbx) * YX, j0 = (t / nbx) * YY;
        dev::mbar_arrive_expect_tx(bar + st, TTX_BYTES);
        // column i0 of the array is cell i0 - GX = i0 - 4; row j0 is cell j0 - 1
        dev::tma_load_3d(dst, &mapF, i0, j0, 0, bar + st);                    // E
        dev::tma_load_3d(dst + TOFF_B, &mapF, i0, j0, 3, bar + st);           // B
        dev::tma_load_3d(dst + TOFF_J, &mapJ, i0 + GX, j0 + GY, 0, bar + st); // J
    };
    if (tid == 0) {
        if ((int)blockIdx.x < nt) issue(blockIdx.x, 0);
        if ((int)(blockIdx.x + gridDim.x) < nt) issue(blockIdx.x + gridDim.x, 1);
    }
    float we = 0.f, wb = 0.f;
    bool ok = true;
    int it = 0, t_stop = -1;
    for (int t = blockIdx.x; t < nt; t += gridDim.x, ++it) {
        const int st = it & 1;
        float* sE = stage0 + st * TSTAGE_FLOATS;
        float* sB = sE + TOFF_B;
        float* sJ = sE + TOFF_J;
        const int i0 = (t % nbx) * YX, j0 = (t / nbx) * YY;
        if (!dev::mbar_wait_bounded(bar + st, (it >> 1) & 1u)) ok = false;
        if (__syncthreads_or(!ok)) {
            t_stop = t;
            break;
        }
        // J at cells nx (periodic box) and ny: the images of cells 0
        if (!g.open_x && i0 <= g.nx && g.nx <= i0 + YX)
            for (int k = tid; k < 3 * JHY; k += YTHREADS) {
                const int c = k / JHY, r = k - c * JHY;
                int j = j0 + r;
                j = j >= g.ny ? j - g.ny : j;
                sJ[YeeTma::j(c, r, g.nx - i0)] = prm.J[c * cs + gidx(g, 0, j)];
            }
        if (j0 <= g.ny && g.ny <= j0 + YY)
            for (int k = tid; k < 3 * JWY; k += YTHREADS) {
                const int c = k / JWY, q = k - c * JWY;
                int i = i0 + q;
                if (i >= g.nx && (g.open_x || i > g.nx)) continue;  // only cells < nx, and nx when periodic
                i = i >= g.nx ? i - g.nx : i;
                sJ[YeeTma::j(c, g.ny - j0, q)] = prm.J[c * cs + gidx(g, i, 0)];
            }
        __syncthreads();
        yee_body<YeeTma>(prm, i0, j0, sE, sB, sJ, we, wb);
        __syncthreads();  // every thread is done with this stage
        const int nxt = t + 2 * gridDim.x;
        if (tid == 0 && nxt < nt) {
            dev::fence_proxy_async_smem();  // the generic writes above before the async overwrite
            issue(nxt, st);
        }
    }
    if (t_stop >= 0) {
        if (tid == 0) {
            // the copies still in flight, once more, before leaving: this
            // tile's stage and, if it was issued, the next tile's
            dev::mbar_wait_bounded(bar + (it & 1), (it >> 1) & 1u);
            if (t_stop + (int)gridDim.x < nt)
                dev::mbar_wait_bounded(bar + ((it + 1) & 1), ((it + 1) >> 1) & 1u);
            dev::set_status(prm.st, ST_TIMEOUT);
        }
        return;
    }
    const double dxdy = g.dx * g.dy;
    const long long n = *((volatile long long*)&prm.st->step);
    const double se = dev::block_sum((double)we, sRed);
    if (tid == 0) atomicAdd(&prm.hist_e[n & (HIST - 1)], 0.5 * se * dxdy);
    const double sb = dev::block_sum((double)wb, sRed);
    if (tid == 0) atomicAdd(&prm.hist_b[n & (HIST - 1)], 0.5 * sb * dxdy);
}

// 6 CTAs of 256 threads per SM (42 registers): the kernel waits on memory,
// more warps in flight hide more of it.
__global__ void __launch_bounds__(YTHREADS, 6) k_yee(const YeeParams prm) {
    yee_tile(prm, blockIdx.x, blockIdx.y);
}

// batched: one CTA per field tile of the flattened tile list of all members
__global__ void __launch_bounds__(YTHREADS) k_yee_batch(const YeeBatch b) {
    const int gt = blockIdx.x;
    int lo = 0, hi = b.nmembers - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.ytile_start[mid] <= gt) lo = mid;
        else hi = mid - 1;
    }
    const YeeParams& P = b.members[lo];
    const int t = gt - b.ytile_start[lo];
    const int nbx = (P.g.nx + YX - 1) / YX;
    yee_tile(P, t % nbx, t / nbx);
}

// ------------------------------------------------------ binomial filter
// The current filter of Listing 3.1: (1/4, 1/2, 1/4) along x, then along y,
// on each component's periodic lattice.  x pass: J (grid layout) -> dense
// scratch [3][ny][nx]; y pass: scratch -> J (interior; the guard images of J
// are never read).
__global__ void k_binom_x(const Geom g, const float* J, float* tmp) {
    const long long n = 3LL * g.nx * g.ny;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = (int)(k % g.nx);
    const long long r = k / g.nx;
    const int j = (int)(r % g.ny), c = (int)(r / g.ny);
    const float* row = J + c * g.cstride + (long long)(j + GY) * g.P + GX;
    const float l = row[i == 0 ? g.nx - 1 : i - 1], m = row[i], rr = row[i == g.nx - 1 ? 0 : i + 1];
    tmp[k] = 0.25f * l + 0.5f * m + 0.25f * rr;
}

__global__ void k_binom_y(const Geom g, const float* tmp, float* J) {
    const long long n = 3LL * g.nx * g.ny;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = (int)(k % g.nx);
    const long long r = k / g.nx;
    const int j = (int)(r % g.ny), c = (int)(r / g.ny);
    const float* col = tmp + (long long)c * g.ny * g.nx + i;
    const float u = col[(long long)(j == 0 ? g.ny - 1 : j - 1) * g.nx], m = col[(long long)j * g.nx],
                d = col[(long long)(j == g.ny - 1 ? 0 : j + 1) * g.nx];
    J[c * g.cstride + (long long)(j + GY) * g.P + i + GX] = 0.25f * u + 0.5f * m + 0.25f * d;
}

// -------------------------------------------------------- grid utilities
// src is component-major (c, j, i) with nx*ny values per component; writes
// the interior and the periodic images.
__global__ void k_set_grid(const Geom g, float* F, int ncomp, const float* src) {
    const long long n = (long long)g.nx * g.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n * ncomp;
         k += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(k / n);
        const long long r = k - c * n;
        const int j = (int)(r / g.nx), i = (int)(r - (long long)j * g.nx);
        const float v = src[k];
        int ii[2], jj[2], ni = 1, nj = 1;
        ii[0] = i;
        jj[0] = j;
        if (!g.open_x) {  // an open box keeps zero x guards
            if (i < 2) ii[ni++] = i + g.nx;
            else if (i == g.nx - 1) ii[ni++] = -1;
        }
        if (j < 2) jj[nj++] = j + g.ny;
        else if (j == g.ny - 1) jj[nj++] = -1;
        for (int a = 0; a < ni; ++a)
            for (int b = 0; b < nj; ++b) F[c * g.cstride + gidx(g, ii[a], jj[b])] = v;
    }
}

// zero the x guard columns -1, nx, nx+1 (rows -1 .. ny+1) of ncomp components
__global__ void k_zero_x_guards(const Geom g, float* F, int ncomp) {
    const int rows = g.ny + 3;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ncomp * rows * 3;
         k += gridDim.x * blockDim.x) {
        const int c = k / (rows * 3), r = (k / 3) % rows, q = k % 3;
        const int i = q == 0 ? -1 : g.nx + q - 1;
        F[c * g.cstride + gidx(g, i, r - 1)] = 0.f;
    }
}

// ------------------------------------------------------------------ lasers
// Field of a laser pulse at physical (x, y) before polarisation (§3.2: plane
// and Gaussian lasers in the initial fields): envelope sin^2(pi xi / 2 fwhm)
// for 0 <= xi = start - x <= 2 fwhm, carrier cos(omega0 (x - start)), peak
// a0 omega0; the Gaussian beam is the paraxial beam of two dimensions with
// waist W0 at x = focus on y = axis.  FP64.
__device__ double laser_value(const LaserDev& l, double x, double y) {
    const double L = 2.0 * l.fwhm, xi = l.start - x;
    if (!(xi >= 0.0 && xi <= L)) return 0.0;
    const double se = sin(M_PI * xi / L);
    double v = l.a0 * l.omega0 * se * se;
    double phase = l.omega0 * (x - l.start);
    if (l.type == 1) {
        const double z = x - l.focus, r = y - l.axis;
        const double zR = 0.5 * l.omega0 * l.W0 * l.W0;
        const double W = l.W0 * sqrt(1.0 + (z / zR) * (z / zR));
        v *= sqrt(l.W0 / W) * exp(-(r / W) * (r / W));
        phase += 0.5 * l.omega0 * r * r * (z / (z * z + zR * zR)) - 0.5 * atan(z / zR);
    }
    return v * cos(phase);
}

// Adds the pulse to Ey (i, j+1/2), Ez (i, j), By (i+1/2, j), Bz (i+1/2, j+1/2)
// and refreshes those values' guard images (periodic box) -- an open box
// keeps its zero x guards.
__global__ void k_add_laser(const Geom g, float* F, const LaserDev l, const DevState* st) {
    const long long n = (long long)g.nx * g.ny;
    const double x0 = (double)st->win_moves * g.dx;
    const double cp = cos(l.polarization), sp = sin(l.polarization);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < 4 * n;
         k += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(k / n);
        const long long r = k - c * n;
        const int j = (int)(r / g.nx), i = (int)(r - (long long)j * g.nx);
        const bool hx = c >= 2, hy = c == 0 || c == 3;  // half-cell offsets of Ey, Ez, By, Bz
        const double x = x0 + ((double)i + (hx ? 0.5 : 0.0)) * g.dx;
        const double y = ((double)j + (hy ? 0.5 : 0.0)) * g.dy;
        const double pol = c == 0 ? cp : (c == 1 ? sp : (c == 2 ? -sp : cp));
        const int comp = c == 0 ? 1 : (c == 1 ? 2 : (c == 2 ? 4 : 5));  // Ey Ez By Bz
        float* C = F + comp * g.cstride;
        const float v = C[gidx(g, i, j)] + (float)(pol * laser_value(l, x, y));
        int ii[2], jj[2], ni = 1, nj = 1;
        ii[0] = i;
        jj[0] = j;
        if (!g.open_x) {
            if (i < 2) ii[ni++] = i + g.nx;
            else if (i == g.nx - 1) ii[ni++] = -1;
        }
        if (j < 2) jj[nj++] = j + g.ny;
        else if (j == g.ny - 1) jj[nj++] = -1;
        for (int a = 0; a < ni; ++a)
            for (int b = 0; b < nj; ++b) C[gidx(g, ii[a], jj[b])] = v;
    }
}

__global__ void k_get_grid(const Geom g, const float* F, int ncomp, float* dst) {
    const long long n = (long long)g.nx * g.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n * ncomp;
         k += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(k / n);
        const long long r = k - c * n;
        const int j = (int)(r / g.nx), i = (int)(r - (long long)j * g.nx);
        dst[k] = F[c * g.cstride + gidx(g, i, j)];
    }
}

__global__ void k_field_energy(const Geom g, const float* F, double* out_e, double* out_b) {
    __shared__ double sRed[32];
    const long long n = (long long)g.nx * g.ny;
    float we = 0.f, wb = 0.f;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(k / g.nx), i = (int)(k - (long long)j * g.nx);
        const long long o = gidx(g, i, j);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float e = F[c * g.cstride + o], b = F[(3 + c) * g.cstride + o];
            we += e * e;
            wb += b * b;
        }
    }
    const double dxdy = g.dx * g.dy;
    const double se = dev::block_sum((double)we, sRed);
    if (threadIdx.x == 0) atomicAdd(out_e, 0.5 * se * dxdy);
    const double sb = dev::block_sum((double)wb, sRed);
    if (threadIdx.x == 0) atomicAdd(out_b, 0.5 * sb * dxdy);
}

// charge density on nodes by area weighting, accumulated in FP64: one CTA
// per tile, nodes [0, T+1)^2 of the tile in shared memory, then FP64 atomics
struct RhoSpecies {
    const int32_t* cell;
    const float *x, *y;
    const int32_t* off;
    double q;
};
struct RhoParams {
    Geom g;
    int nsp;
    RhoSpecies sp[MAX_SPECIES];
    double* rho;
};

// Charge density on the nodes (area weighting of Fig. 3.3), in FP64.  A CTA
// takes a slice of a tile's particles (tiles holding many are split over
// several CTAs, as in the particle advance).  Each particle adds to its own
// cell the moments 1, x, y and x y as exact integers: fixed-point values
// x 2^38, y 2^38 and x y 2^48 (the product is split exactly into two FP32
// terms with a fused multiply-add), added as 19-, 19- and 16-bit chunks to
// 32-bit shared counters, which cannot overflow for the at most RHO_ROUND
// particles a round accumulates.  The four corner weights follow from the
// moments exactly, (1-x)(1-y) = 1 - x - y + x y, x (1-y) = x - x y,
// (1-x) y = y - x y, in 64-bit integers; each node's sum is scaled to FP64
// once and added to the global rho with an FP64 atomic.  Shared integer
// atomics cost a fraction of FP64 ones, and no FP64 arithmetic is done per
// particle.
constexpr int RHO_THREADS = 256;
constexpr int RHO_ROUND = 8192;  // particles per accumulation round of a CTA
constexpr int RHO_WORDS = 8;     // count, x (2 chunks), y (2 chunks), x y (3 chunks)
constexpr int RHO_CHUNK = 8192;  // particles per CTA (tiles holding more are split)

__device__ __forceinline__ long long rho_moment(const unsigned* sM, int T2, int c, int k0,
                                                int shift) {
    return (long long)sM[k0 * T2 + c] + ((long long)sM[(k0 + 1) * T2 + c] << shift);
}

__global__ void __launch_bounds__(RHO_THREADS) k_rho(const RhoParams prm) {
    extern __shared__ __align__(16) unsigned char smem_r[];
    const Geom& g = prm.g;
    const int T = g.T, W = T + 1, T2 = T * T;
    unsigned* sM = reinterpret_cast<unsigned*>(smem_r);  // [RHO_WORDS][T*T]
    double* sR = reinterpret_cast<double*>(smem_r + (((size_t)RHO_WORDS * T2 * 4 + 15) & ~(size_t)15));
    const int t = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
    const int tx = tile_x(g, t), ty = tile_y(g, t);
    const int ix0 = tx * T, iy0 = ty * T;
    for (int k = tid; k < W * W; k += nth) sR[k] = 0.0;
    for (int s = 0; s < prm.nsp; ++s) {
        const RhoSpecies& S = prm.sp[s];
        const int p0 = S.off[t], nt = S.off[t + 1] - p0;
        const int len = (nt + (int)gridDim.y - 1) / (int)gridDim.y;
        const int c0 = p0 + min((int)blockIdx.y * len, nt);
        const int c1 = p0 + min(((int)blockIdx.y + 1) * len, nt);
        for (int r0 = c0; r0 < c1; r0 += RHO_ROUND) {
            const int r1 = min(r0 + RHO_ROUND, c1);
            for (int k = tid; k < RHO_WORDS * T2; k += nth) sM[k] = 0u;
            __syncthreads();
            for (int p = r0 + tid; p < r1; p += nth) {
                const int c = S.cell[p];
                const int lx = (c & 0xffff) - ix0, ly = (int)((unsigned)c >> 16) - iy0;
                if (c == HOLE || lx < 0 || lx >= T || ly < 0 || ly >= T) continue;
                const float x = S.x[p], y = S.y[p];
                const unsigned long long vx = __float2ull_rn(x * 0x1p38f);  // < 2^38
                const unsigned long long vy = __float2ull_rn(y * 0x1p38f);
                const float pxy = __fmul_rn(x, y);
                const float exy = __fmaf_rn(x, y, -pxy);  // x y = pxy + exy exactly
                long long vxy = (long long)__float2ull_rn(pxy * 0x1p48f) +
                                __float2ll_rn(exy * 0x1p48f);
                if (vxy < 0) vxy = 0;
                const int cc = ly * T + lx;
                atomicAdd(sM + cc, 1u);
                atomicAdd(sM + T2 + cc, (unsigned)(vx & 0x7ffffu));
                atomicAdd(sM + 2 * T2 + cc, (unsigned)(vx >> 19));
                atomicAdd(sM + 3 * T2 + cc, (unsigned)(vy & 0x7ffffu));
                atomicAdd(sM + 4 * T2 + cc, (unsigned)(vy >> 19));
                atomicAdd(sM + 5 * T2 + cc, (unsigned)(vxy & 0xffff));
                atomicAdd(sM + 6 * T2 + cc, (unsigned)((vxy >> 16) & 0xffff));
                atomicAdd(sM + 7 * T2 + cc, (unsigned)(vxy >> 32));
            }
            __syncthreads();
            // node (i, j) of the tile, 0 <= i, j <= T: the (1-x)(1-y) weight of
            // cell (i, j), x (1-y) of cell (i-1, j), (1-x) y of cell (i, j-1)
            // and x y of cell (i-1, j-1), in units of 2^-48
            for (int k = tid; k < W * W; k += nth) {
                const int j = k / W, i = k - j * W;
                long long acc = 0;
                auto moments = [&](int ci, int cj, long long& n, long long& X, long long& Y,
                                   long long& XY) {
                    const int c = cj * T + ci;
                    n = (long long)sM[c] << 48;
                    X = rho_moment(sM, T2, c, 1, 19) << 10;
                    Y = rho_moment(sM, T2, c, 3, 19) << 10;
                    XY = (long long)sM[5 * T2 + c] + ((long long)sM[6 * T2 + c] << 16) +
                         ((long long)sM[7 * T2 + c] << 32);
                };
                long long n, X, Y, XY;
                if (i < T && j < T) {
                    moments(i, j, n, X, Y, XY);
                    acc += n - X - Y + XY;
                }
                if (i > 0 && j < T) {
                    moments(i - 1, j, n, X, Y, XY);
                    acc += X - XY;
                }
                if (i < T && j > 0) {
                    moments(i, j - 1, n, X, Y, XY);
                    acc += Y - XY;
                }
                if (i > 0 && j > 0) {
                    moments(i - 1, j - 1, n, X, Y, XY);
                    acc += XY;
                }
                if (acc) sR[k] += S.q * ((double)acc * 0x1p-48);
            }
            __syncthreads();  // the moments are cleared for the next round
        }
    }
    __syncthreads();
    for (int k = tid; k < W * W; k += nth) {
        const double v = sR[k];
        if (v == 0.0) continue;
        const int ly = k / W, lx = k - ly * W;
        int i = ix0 + lx, j = iy0 + ly;
        i = i >= g.nx ? i - g.nx : i;
        j = j >= g.ny ? j - g.ny : j;
        atomicAdd(&prm.rho[(long long)j * g.nx + i], v);
    }
}

__global__ void k_residuals(const Geom g, const float* F, const float* J, const double* rho,
                            const double* rho_prev, double background, double* out) {
    __shared__ double sRed[32];
    const long long n = (long long)g.nx * g.ny;
    double gmax = 0.0, cmax = 0.0, qsum = 0.0;
    const long long cs = g.cstride;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(k / g.nx), i = (int)(k - (long long)j * g.nx);
        const long long o = gidx(g, i, j);
        const int im = i == 0 ? g.nx - 1 : i - 1, jm = j == 0 ? g.ny - 1 : j - 1;
        const long long oxm = gidx(g, im, j), oym = gidx(g, i, jm);
        const double r = rho[k] + background;
        const double dive = ((double)F[o] - (double)F[oxm]) / g.dx +
                            ((double)F[cs + o] - (double)F[cs + oym]) / g.dy;
        gmax = fmax(gmax, fabs(dive - r));
        qsum += r;
        if (rho_prev) {
            const double divj = ((double)J[o] - (double)J[oxm]) / g.dx +
                                ((double)J[cs + o] - (double)J[cs + oym]) / g.dy;
            cmax = fmax(cmax, fabs((rho[k] - rho_prev[k]) / g.dtd + divj));
        }
    }
    const double a = dev::block_max(gmax, sRed);
    if (threadIdx.x == 0) dev::atomic_max_nonneg(&out[0], a);
    const double b = dev::block_max(cmax, sRed);
    if (threadIdx.x == 0) dev::atomic_max_nonneg(&out[1], b);
    const double c = dev::block_sum(qsum, sRed);
    if (threadIdx.x == 0) atomicAdd(&out[2], c * g.dx * g.dy);
}

// ------------------------------------------------------- particle load
// The initial sort orders particles by tile (§4.1); inside a tile, where the
// method leaves the order free, they are placed in a pseudo-random order
// (key = tile * T^2 + a hash of the input index modulo T^2).  A warp's 32
// particles then fall into many different cells, which keeps the shared-memory
// conflicts of the current deposit low from the first step on (the order a
// simulation reaches after some steps is of this kind anyway: particles keep
// their slot when they change cell).
// phase 0: validate the staged input (out arrays; ocell holds ix, hole holds
//          iy on entry) and count per cell key;
// phase 1: scan the counts into cell offsets, take the tile bookmarks from
//          them and scatter into the particle arrays.
// The slot key hashes the input index with full avalanche (xor-shift and
// multiply rounds): every bit of the index moves every bit of the key.  A
// multiplicative hash kept only some low bits of the index in the key's low
// bits, so particles whose indices differ by a power of two (the same cell
// column of rows a power of two apart, in an input ordered cell by cell)
// shared a key, landed in the same warp and read the same shared-memory bank
// group in the gather (5.6 wavefronts per load instead of about 3.5).
__device__ __forceinline__ unsigned mix32(unsigned h) {
    h ^= h >> 16;
    h *= 0x7feb352du;
    h ^= h >> 15;
    h *= 0x846ca68bu;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ int load_key(const Geom& g, int ix, int iy, int k) {
    const int t = tile_index(g, ix / g.T, iy / g.T);
    const unsigned h = mix32((unsigned)k);
    return t * g.T * g.T + (int)(h % (unsigned)(g.T * g.T));
}

__global__ void k_load_count(const Geom g, SpeciesDev sp, int n, DevState* st) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int ix = sp.ocell[k], iy = sp.hole[k];
        const float x = sp.ox[k], y = sp.oy[k];
        const bool ok = ix >= 0 && ix < g.nx && iy >= 0 && iy < g.ny && x >= 0.f && x < 1.f &&
                        y >= 0.f && y < 1.f && isfinite(sp.oux[k]) && isfinite(sp.ouy[k]) &&
                        isfinite(sp.ouz[k]);
        if (!ok) {
            atomicAdd(&st->load_bad, 1);
            continue;
        }
        atomicAdd(&sp.cursor[load_key(g, ix, iy, k)], 1);
    }
}

__global__ void k_load_scatter(const Geom g, SpeciesDev sp, int n, const int32_t* ids,
                               const int32_t* celloff, int track) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int ix = sp.ocell[k], iy = sp.hole[k];
        const int key = load_key(g, ix, iy, k);
        const int p = celloff[key] + atomicAdd(&sp.cursor[key], 1);
        sp.cell[p] = ix | (iy << 16);
        sp.x[p] = sp.ox[k];
        sp.y[p] = sp.oy[k];
        sp.ux[p] = sp.oux[k];
        sp.uy[p] = sp.ouy[k];
        sp.uz[p] = sp.ouz[k];
        if (track) sp.id[p] = ids ? ids[k] : k;
    }
}

// tile bookmarks = offsets of each tile's first cell key
__global__ void k_tile_from_cells(const int32_t* celloff, int ntiles, int T2, int32_t* off) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t <= ntiles; t += gridDim.x * blockDim.x)
        off[t] = celloff[(long long)t * T2];
}

// exclusive scan of per-tile counts (single CTA)
__global__ void __launch_bounds__(1024) k_scan_counts(const int32_t* cnt, int nt, int32_t* off) {
    __shared__ int sWarp[32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int per = (nt + 1023) / 1024;
    const int t0 = min(tid * per, nt), t1 = min(t0 + per, nt);
    int mysum = 0;
    for (int t = t0; t < t1; ++t) mysum += cnt[t];
    int incl = mysum;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) sWarp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int w = sWarp[lane];
        int wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += v;
        }
        sWarp[lane] = wi - w;
    }
    __syncthreads();
    int run = sWarp[wid] + incl - mysum;
    for (int t = t0; t < t1; ++t) {
        off[t] = run;
        run += cnt[t];
    }
    if (tid == 1023) off[nt] = run;
}

// Exclusive scan of the per-cell counts of a load, in three coalesced passes
// over segments of SCAN_SEG cells: segment sums, their scan (k_scan_counts,
// one CTA), then each segment's own scan plus its offset.
constexpr int SCAN_SEG = 4096;  // cells per CTA of 1024 threads (4 consecutive each)

__device__ __forceinline__ int block_excl_scan_1024(int v, int* sWarp, int* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) sWarp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int w = sWarp[lane];
        int wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += u;
        }
        sWarp[lane] = wi - w;
        if (lane == 31) sWarp[32] = wi;
    }
    __syncthreads();
    *total = sWarp[32];
    return sWarp[wid] + incl - v;
}

__global__ void __launch_bounds__(1024) k_scan_seg_sums(const int32_t* cnt, long long n,
                                                        int32_t* part) {
    __shared__ int sWarp[33];
    const long long k0 = (long long)blockIdx.x * SCAN_SEG + 4 * threadIdx.x;
    int v = 0;
    for (int j = 0; j < 4; ++j)
        if (k0 + j < n) v += cnt[k0 + j];
    int total;
    block_excl_scan_1024(v, sWarp, &total);
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_seg_apply(const int32_t* cnt, long long n,
                                                         const int32_t* partoff, int32_t* off) {
    __shared__ int sWarp[33];
    const long long k0 = (long long)blockIdx.x * SCAN_SEG + 4 * threadIdx.x;
    int c[4];
    for (int j = 0; j < 4; ++j) c[j] = k0 + j < n ? cnt[k0 + j] : 0;
    int total;
    int run = partoff[blockIdx.x] + block_excl_scan_1024(c[0] + c[1] + c[2] + c[3], sWarp, &total);
    for (int j = 0; j < 4; ++j) {
        if (k0 + j < n) off[k0 + j] = run;
        run += c[j];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) off[n] = partoff[gridDim.x];
}

__global__ void k_unpack(const int32_t* cell, int n, int32_t* ix, int32_t* iy) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int c = cell[k];
        if (ix) ix[k] = c & 0xffff;
        if (iy) iy[k] = (int)((unsigned)c >> 16);
    }
}

__global__ void k_off64(const int32_t* off, int n, int64_t* out) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        out[k] = off[k];
}

// The failure path of the bounded waits, on its own: one CTA waits on an
// mbarrier with the helper every kernel uses.  With `arrive` thread 0 arrives
// first and the phase completes; without it nothing ever completes the phase
// (no copy is issued, so none is in flight) and the wait gives up after
// `limit` cycles.  result: 0, or ST_TIMEOUT.
__global__ void k_probe_wait(int arrive, long long limit, unsigned* result) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        dev::mbar_init(&bar, 1);
        dev::fence_mbar_init();
    }
    __syncthreads();
    if (arrive && threadIdx.x == 0) dev::mbar_arrive_expect_tx(&bar, 0);
    const bool ok = dev::mbar_wait_bounded(&bar, 0u, limit);
    const bool out = __syncthreads_or(!ok);
    if (threadIdx.x == 0) *result = out ? ST_TIMEOUT : 0u;
}

__global__ void k_hist_prime(double* he, double* hb, double* hk, DevState* st) {
    const long long n = st->step;
    he[n & (HIST - 1)] = 0.0;
    hb[n & (HIST - 1)] = 0.0;
    hk[n & (HIST - 1)] = 0.0;
}

int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 16) b = 152 * 16;
    return (int)b;
}

}  // namespace

cudaError_t launch_binomial(const Geom& g, float* J, float* tmp, cudaStream_t s) {
    const long long n = 3LL * g.nx * g.ny;
    k_binom_x<<<grid_for(n, 256), 256, 0, s>>>(g, J, tmp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_binom_y<<<grid_for(n, 256), 256, 0, s>>>(g, tmp, J);
    return cudaGetLastError();
}

int yee_tiles(const Geom& g) { return ((g.nx + YX - 1) / YX) * ((g.ny + YY - 1) / YY); }

cudaError_t launch_yee_batch(const YeeBatch& b, cudaStream_t s) {
    if (b.nmembers == 0 || b.total_ytiles == 0) return cudaSuccess;
    k_yee_batch<<<b.total_ytiles, YTHREADS, 0, s>>>(b);
    return cudaGetLastError();
}

static int g_yee_grid = 0;  // persistent CTAs of k_yee_tma (set once)

// Once per process, before any capture: the Yee kernels prefer the largest
// shared-memory carveout (22 KB of static shared memory per CTA).
cudaError_t init_grid_kernels() {
    cudaError_t e = cudaFuncSetAttribute(k_yee, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_yee_batch, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_yee_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)YEE_TMA_SMEM);
    if (e == cudaSuccess && g_yee_grid == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_yee_tma, YTHREADS,
                                                              YEE_TMA_SMEM);
        if (e == cudaSuccess) g_yee_grid = sms * (per_sm > 0 ? per_sm : 1);
    }
    return e;
}

cudaError_t launch_yee(const YeeParams& p, const CUtensorMap* mapF, const CUtensorMap* mapJ,
                       cudaStream_t s) {
    const int nt = yee_tiles(p.g);
    if (mapF && mapJ && g_yee_grid > 0) {
        const int grid = nt < g_yee_grid ? nt : g_yee_grid;
        k_yee_tma<<<grid, YTHREADS, YEE_TMA_SMEM, s>>>(*mapF, *mapJ, p);
        return cudaGetLastError();
    }
    dim3 grid((p.g.nx + YX - 1) / YX, (p.g.ny + YY - 1) / YY);
    k_yee<<<grid, YTHREADS, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_set_grid(const Geom& g, float* F, int ncomp, const float* src,
                            cudaStream_t s) {
    k_set_grid<<<grid_for((long long)g.nx * g.ny * ncomp, 256), 256, 0, s>>>(g, F, ncomp, src);
    return cudaGetLastError();
}

cudaError_t launch_zero_x_guards(const Geom& g, float* F, int ncomp, cudaStream_t s) {
    k_zero_x_guards<<<grid_for((long long)ncomp * (g.ny + 3) * 3, 256), 256, 0, s>>>(g, F, ncomp);
    return cudaGetLastError();
}

cudaError_t launch_add_laser(const Geom& g, float* F, const LaserDev& l, const DevState* st,
                             cudaStream_t s) {
    k_add_laser<<<grid_for(4LL * g.nx * g.ny, 256), 256, 0, s>>>(g, F, l, st);
    return cudaGetLastError();
}

cudaError_t launch_get_grid(const Geom& g, const float* F, int ncomp, float* dst,
                            cudaStream_t s) {
    k_get_grid<<<grid_for((long long)g.nx * g.ny * ncomp, 256), 256, 0, s>>>(g, F, ncomp, dst);
    return cudaGetLastError();
}

cudaError_t launch_field_energy(const Geom& g, const float* F, double* out_e, double* out_b,
                                cudaStream_t s) {
    k_field_energy<<<grid_for((long long)g.nx * g.ny, 256), 256, 0, s>>>(g, F, out_e, out_b);
    return cudaGetLastError();
}

cudaError_t launch_rho(const Geom& g, const SpeciesDev* sp, int nsp, const int32_t* const* off,
                       double* rho, cudaStream_t s) {
    RhoParams p;
    p.g = g;
    p.nsp = nsp;
    for (int k = 0; k < nsp; ++k) {
        p.sp[k].cell = sp[k].cell;
        p.sp[k].x = sp[k].x;
        p.sp[k].y = sp[k].y;
        p.sp[k].off = off[k];
        p.sp[k].q = sp[k].qtilde;
    }
    p.rho = rho;
    if (g.ntiles == 0) return cudaSuccess;
    // slices of at most RHO_CHUNK particles of the fullest species' mean tile
    int64_t nmax = 0;
    for (int k = 0; k < nsp; ++k) nmax = std::max<int64_t>(nmax, sp[k].n);
    const int64_t per_tile = nmax / g.ntiles;
    const int chunks = (int)std::min<int64_t>(std::max<int64_t>((per_tile + RHO_CHUNK - 1) / RHO_CHUNK, 1), 1024);
    const size_t bytes = (((size_t)RHO_WORDS * g.T * g.T * 4 + 15) & ~(size_t)15) +
                         (size_t)(g.T + 1) * (g.T + 1) * sizeof(double);
    k_rho<<<dim3(g.ntiles, chunks), RHO_THREADS, bytes, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_grid_residuals(const Geom& g, const float* F, const float* J,
                                  const double* rho, const double* rho_prev, double background,
                                  double* out, cudaStream_t s) {
    k_residuals<<<grid_for((long long)g.nx * g.ny, 256), 256, 0, s>>>(g, F, J, rho, rho_prev,
                                                                     background, out);
    return cudaGetLastError();
}

cudaError_t launch_load(const Geom& g, SpeciesDev& sp, int track_ids, int64_t n, int32_t* off,
                        DevState* st, cudaStream_t s, int phase, const int32_t* staged_ids,
                        int32_t* celloff) {
    const int nn = (int)n;
    const long long ncell = (long long)g.nx * g.ny;
    if (phase == 0) {
        cudaError_t e = cudaMemsetAsync(sp.cursor, 0, sizeof(int32_t) * ncell, s);
        if (e != cudaSuccess) return e;
        if (nn > 0) k_load_count<<<grid_for(nn, 256), 256, 0, s>>>(g, sp, nn, st);
        return cudaGetLastError();
    }
    // phase 1: cell offsets from the counts (segment sums and their offsets
    // behind the ncell + 1 cell offsets), tile bookmarks, then scatter
    const int nseg = (int)((ncell + SCAN_SEG - 1) / SCAN_SEG);
    int32_t* part = celloff + ncell + 1;
    int32_t* partoff = part + nseg;
    k_scan_seg_sums<<<nseg, 1024, 0, s>>>(sp.cursor, ncell, part);
    k_scan_counts<<<1, 1024, 0, s>>>(part, nseg, partoff);
    k_scan_seg_apply<<<nseg, 1024, 0, s>>>(sp.cursor, ncell, partoff, celloff);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_tile_from_cells<<<grid_for(g.ntiles + 1, 256), 256, 0, s>>>(celloff, g.ntiles, g.T * g.T,
                                                                 off);
    e = cudaMemsetAsync(sp.cursor, 0, sizeof(int32_t) * ncell, s);
    if (e != cudaSuccess) return e;
    if (nn > 0) {
        // One wave of resident CTAs only: the grid-stride loop then sweeps the
        // input in order, so the tiles being written at any time are those of
        // a few hundred thousand consecutive input particles, whose slots the
        // L2 cache holds until their sectors are complete.  A second wave
        // would fill the gaps the first left in every tile long after those
        // sectors went back to memory half-written (each then read back to be
        // merged: about three times the scatter's bytes in DRAM traffic).
        static int resident = 0;
        if (resident == 0) {
            int dev = 0, sms = 0, per = 0;
            e = cudaGetDevice(&dev);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_load_scatter, 256, 0);
            if (e != cudaSuccess) return e;
            resident = sms * (per > 0 ? per : 1);
        }
        const int grid = grid_for(nn, 256) < resident ? grid_for(nn, 256) : resident;
        k_load_scatter<<<grid, 256, 0, s>>>(g, sp, nn, staged_ids, celloff, track_ids);
    }
    return cudaGetLastError();
}

cudaError_t launch_unpack_cells(const int32_t* cell, int64_t n, int32_t* ix, int32_t* iy,
                                cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_unpack<<<grid_for(n, 256), 256, 0, s>>>(cell, (int)n, ix, iy);
    return cudaGetLastError();
}

cudaError_t launch_offsets_to_i64(const int32_t* off, int64_t n, int64_t* out, cudaStream_t s) {
    k_off64<<<grid_for(n, 256), 256, 0, s>>>(off, (int)n, out);
    return cudaGetLastError();
}

cudaError_t launch_probe_wait(int arrive, long long limit, unsigned* result, cudaStream_t s) {
    k_probe_wait<<<1, 64, 0, s>>>(arrive, limit, result);
    return cudaGetLastError();
}

cudaError_t launch_hist_prime(double* he, double* hb, double* hk, DevState* st, cudaStream_t s) {
    k_hist_prime<<<1, 1, 0, s>>>(he, hb, hk, st);
    return cudaGetLastError();
}

}  // namespace pic
