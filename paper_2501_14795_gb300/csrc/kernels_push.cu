// Particle advance: one CTA per tile of T x T cells (§4.1-4.2, Listing 3.1's
// particle loop), for all species of the tile:
//   1. TMA-load the tile's E|B halo, cells [-4, T+4) x [-1, T+2), into shared
//      memory (one 3D box over the six components, mbarrier completion);
//   2. per particle (coalesced SoA loads): linear gather of the six staggered
//      components (Fig. 3.1), Boris push (Eqs. 6-10), move (Eq. 11), the
//      Villasenor-Buneman split into at most three pieces (Figs. 3.4-3.5) and
//      the deposit of each piece's current (Eqs. 13-16 plus the time-averaged
//      Jz) into a shared-memory J tile, cells [-1, T+2), with shared atomics;
//   3. emit the re-sort metadata of §4.3: particles that stay in the tile are
//      written in place; particles that leave are appended (warp-ballot slots)
//      to the tile's section of the out arrays with their old position in the
//      hole list, and counted by destination (8 neighbours);
//   4. flush the J tile once: plain stores to the cells no other tile's halo
//      reaches, red.global.add to the shared ring (update_gc_add);
//   5. FP32 kinetic energy per thread -> FP64 block sum -> one FP64 atomic.
//
// This file is compiled twice: PIC_VARIANT=fast (FMA contraction allowed) and
// PIC_VARIANT=strict (-fmad=false): the strict build evaluates the
// per-particle path in exactly the operation order of the FP32 reference
// (every expression below is written in that order), so cells, offsets and
// momenta are reproducible bit for bit.
#include <cuda.h>

#include "device_util.cuh"
#include "pic_internal.h"

#ifndef PIC_VARIANT
#define PIC_VARIANT fast
#endif
#define PIC_CAT2(a, b) a##b
#define PIC_CAT(a, b) PIC_CAT2(a, b)

namespace pic {
namespace PIC_VARIANT {

template <int T>
struct Tile {
    static constexpr int FW = T + 8;  // TMA box columns: cells -4 .. T+3
    static constexpr int FH = T + 3;  // TMA box rows:    cells -1 .. T+1
    static constexpr int FPLANE = FW * FH;
    static constexpr int FLD = 6 * FPLANE;
    static constexpr int JW = T + 3;  // J tile: cells -1 .. T+1 on both axes
    static constexpr int JPLANE = JW * JW;
    static constexpr int JN = 3 * JPLANE;
    static constexpr size_t OFF_BAR = ((size_t)(FLD + JN) * 4 + 15) & ~(size_t)15;
    static constexpr size_t OFF_CNT = OFF_BAR + 16;
    static constexpr int NCNT = MAX_SPECIES * 9 + 4;
    static constexpr size_t OFF_RED = (OFF_CNT + NCNT * 4 + 7) & ~(size_t)7;
    static constexpr size_t BYTES = OFF_RED + 32 * sizeof(double);
};

__device__ __forceinline__ float interp(const float* F, int fw, int col, int row, float a0,
                                        float a1, float b0, float b1) {
    const float* r0 = F + row * fw + col;
    const float* r1 = r0 + fw;
    return b0 * (a0 * r0[0] + a1 * r0[1]) + b1 * (a0 * r1[0] + a1 * r1[1]);
}

// Current of one straight piece inside local cell (cl, rl) of the J tile
// (indices already shifted by the halo), local start (fx0, fy0), end (fx1, fy1),
// time fraction frac.
template <int JW>
__device__ __forceinline__ void deposit_piece(float* sJx, float* sJy, float* sJz, int cl, int rl,
                                              float fx0, float fy0, float fx1, float fy1,
                                              float frac, float qjx, float qjy, float qvz) {
    const float dxp = fx1 - fx0, dyp = fy1 - fy0;
    const float xm = 0.5f * (fx0 + fx1), ym = 0.5f * (fy0 + fy1);
    const int o = rl * JW + cl;
    const float jxv = qjx * dxp, jyv = qjy * dyp;
    atomicAdd(sJx + o, jxv * (1.f - ym));
    atomicAdd(sJx + o + JW, jxv * ym);
    atomicAdd(sJy + o, jyv * (1.f - xm));
    atomicAdd(sJy + o + 1, jyv * xm);
    // Jz: q vz frac times the mean over the piece of the area weights
    const float sx0 = 1.f - fx0, sx1 = 1.f - fx1;  // a = 0 weights at start / end
    const float sy0 = 1.f - fy0, sy1 = 1.f - fy1;
    const float c = qvz * frac * (1.f / 6.f);
    // W_ab = [S0x_a (2 S0y_b + S1y_b) + S1x_a (S0y_b + 2 S1y_b)] / 6
    const float ay0 = 2.f * sy0 + sy1, by0 = sy0 + 2.f * sy1;  // b = 0
    const float ay1 = 2.f * fy0 + fy1, by1 = fy0 + 2.f * fy1;  // b = 1
    atomicAdd(sJz + o, c * (sx0 * ay0 + sx1 * by0));
    atomicAdd(sJz + o + 1, c * (fx0 * ay0 + fx1 * by0));
    atomicAdd(sJz + o + JW, c * (sx0 * ay1 + sx1 * by1));
    atomicAdd(sJz + o + JW + 1, c * (fx0 * ay1 + fx1 * by1));
}

template <int T>
__global__ void __launch_bounds__(1024) k_push(const __grid_constant__ CUtensorMap fmap,
                                               const PushParams prm) {
    using L = Tile<T>;
    extern __shared__ __align__(128) unsigned char smem[];
    float* sF = reinterpret_cast<float*>(smem);
    float* sJ = sF + L::FLD;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::OFF_BAR);
    int* sLeave = reinterpret_cast<int*>(smem + L::OFF_CNT);  // [MAX_SPECIES]
    int* sDir = sLeave + MAX_SPECIES;                          // [MAX_SPECIES][8]
    double* sRed = reinterpret_cast<double*>(smem + L::OFF_RED);

    const Geom& g = prm.g;
    const int t = blockIdx.x;
    const int tx = t % g.ntx, ty = t / g.ntx;
    const int ix0 = tx * T, iy0 = ty * T;
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31;
    const long long step = *((volatile long long*)&prm.st->step);

    if (tid == 0) {
        dev::mbar_init(bar, 1);
        dev::fence_mbar_init();
    }
    for (int i = tid; i < L::NCNT; i += nth) sLeave[i] = 0;
    __syncthreads();
    if (tid == 0) {
        dev::mbar_arrive_expect_tx(bar, L::FLD * 4);
        // box origin: column ix0 = cell ix0 - GX, row iy0 = cell iy0 - GY
        dev::tma_load_3d(sF, &fmap, ix0, iy0, 0, bar);
    }
    for (int i = tid; i < L::JN; i += nth) sJ[i] = 0.f;
    const bool ok = dev::mbar_wait_bounded(bar, 0);
    if (__syncthreads_or(!ok)) {
        if (tid == 0) dev::set_status(prm.st, ST_TIMEOUT);
        return;
    }

    const float* sEx = sF;
    const float* sEy = sF + L::FPLANE;
    const float* sEz = sF + 2 * L::FPLANE;
    const float* sBx = sF + 3 * L::FPLANE;
    const float* sBy = sF + 4 * L::FPLANE;
    const float* sBz = sF + 5 * L::FPLANE;
    float* sJx = sJ;
    float* sJy = sJ + L::JPLANE;
    float* sJz = sJ + 2 * L::JPLANE;
    const int nx = g.nx, ny = g.ny;
    const float cxs = g.cx, cys = g.cy;
    unsigned bad_bits = 0;
    double ke_tot = 0.0;

    for (int s = 0; s < prm.nsp; ++s) {
        const PushSpecies& S = prm.sp[s];
        const int p0 = S.off[t], p1 = S.off[t + 1];
        const float tem = S.tem, qjx = S.qjx, qjy = S.qjy, qjz = S.qjz;
        float ke = 0.f;
        for (int base = p0; base < p1; base += nth) {
            const int p = base + tid;
            const bool active = p < p1;
            bool write = false;
            int dir = -1;  // -1: stays in this tile; 0..7: leaves towards that neighbour
            int ncell = 0;
            float xn = 0.f, yn = 0.f, vx = 0.f, vy = 0.f, vzm = 0.f;
            if (active) {
                const int c = S.cell[p];
                const float x = S.x[p], y = S.y[p];
                float ux = S.ux[p], uy = S.uy[p], uz = S.uz[p];
                const int ix = c & 0xffff, iy = (int)((unsigned)c >> 16);
                const int lx = ix - ix0, ly = iy - iy0;
                if (c == HOLE || lx < 0 || lx >= T || ly < 0 || ly >= T) {
                    bad_bits |= ST_SORT;  // not in this tile: leave it untouched
                } else {
                    write = true;
                    // ---- gather (Fig. 3.1 staggering) ----
                    const float wx1 = x, wx0 = 1.f - x, wy1 = y, wy0 = 1.f - y;
                    const float xh = x + 0.5f, yh = y + 0.5f;
                    const float fhx = floorf(xh), fhy = floorf(yh);
                    const float hx1 = xh - fhx, hx0 = 1.f - hx1;
                    const float hy1 = yh - fhy, hy0 = 1.f - hy1;
                    const int cn = lx + GX, ch = lx + (int)fhx - 1 + GX;
                    const int rn = ly + GY, rh = ly + (int)fhy - 1 + GY;
                    const float ex = interp(sEx, L::FW, ch, rn, hx0, hx1, wy0, wy1);
                    const float ey = interp(sEy, L::FW, cn, rh, wx0, wx1, hy0, hy1);
                    const float ez = interp(sEz, L::FW, cn, rn, wx0, wx1, wy0, wy1);
                    const float bx = interp(sBx, L::FW, cn, rh, wx0, wx1, hy0, hy1);
                    const float by = interp(sBy, L::FW, ch, rn, hx0, hx1, wy0, wy1);
                    const float bz = interp(sBz, L::FW, ch, rh, hx0, hx1, hy0, hy1);
                    // ---- Boris push, Eqs. 6-10 ----
                    const float umx = ux + tem * ex;
                    const float umy = uy + tem * ey;
                    const float umz = uz + tem * ez;
                    const float gm = sqrtf(1.f + umx * umx + umy * umy + umz * umz);
                    const float gtem = tem / gm;
                    const float btx = gtem * bx, bty = gtem * by, btz = gtem * bz;
                    const float upx = umx + umy * btz - umz * bty;
                    const float upy = umy + umz * btx - umx * btz;
                    const float upz = umz + umx * bty - umy * btx;
                    const float f = 2.f / (1.f + btx * btx + bty * bty + btz * btz);
                    const float sx = f * btx, sy = f * bty, sz = f * btz;
                    const float uqx = umx + upy * sz - upz * sy;
                    const float uqy = umy + upz * sx - upx * sz;
                    const float uqz = umz + upx * sy - upy * sx;
                    ux = uqx + tem * ex;
                    uy = uqy + tem * ey;
                    uz = uqz + tem * ez;
                    // gamma - 1 = |u-|^2 / (gamma + 1), free of cancellation
                    ke += (umx * umx + umy * umy + umz * umz) / (gm + 1.f);
                    // ---- move, Eq. 11 in cell units ----
                    const float gg = sqrtf(1.f + ux * ux + uy * uy + uz * uz);
                    const float rg = 1.f / gg;
                    const float ddx = ux * rg * cxs, ddy = uy * rg * cys;
                    const float vz = uz * rg;
                    vx = ux;
                    vy = uy;
                    vzm = uz;
                    ncell = c;
                    xn = x;
                    yn = y;
                    if (!(fabsf(ddx) < 1.f && fabsf(ddy) < 1.f)) {
                        bad_bits |= ST_PARTICLE;  // keeps its place, new momentum, no current
                    } else {
                        float x1 = x + ddx, y1 = y + ddy;
                        int di = (x1 >= 1.f) - (x1 < 0.f);
                        int dj = (y1 >= 1.f) - (y1 < 0.f);
                        float xnn = x1 - (float)di, ynn = y1 - (float)dj;
                        if (xnn >= 1.f) {  // x1 = -tiny: x1 + 1 rounded to 1
                            xnn = 0.f;
                            di = 0;
                            x1 = 0.f;
                        }
                        if (ynn >= 1.f) {
                            ynn = 0.f;
                            dj = 0;
                            y1 = 0.f;
                        }
                        // ---- Villasenor-Buneman split + deposit ----
                        const float qvz = qjz * vz;
                        const float xbd = di > 0 ? 1.f : 0.f, ybd = dj > 0 ? 1.f : 0.f;
                        const float tcx = di ? (xbd - x) / (x1 - x) : 2.f;
                        const float tcy = dj ? (ybd - y) / (y1 - y) : 2.f;
                        const float t1 = fminf(fminf(tcx, tcy), 1.f);
                        const float t2 = fminf(fmaxf(tcx, tcy), 1.f);
                        float ta = 0.f, xa = x, ya = y;
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const float tb = k == 0 ? t1 : (k == 1 ? t2 : 1.f);
                            if (tb > ta) {
                                const float xe = tb == tcx ? xbd
                                                           : (tb == 1.f ? x1 : x + tb * (x1 - x));
                                const float ye = tb == tcy ? ybd
                                                           : (tb == 1.f ? y1 : y + tb * (y1 - y));
                                const int ci = (di != 0 && tcx <= ta) ? di : 0;
                                const int cj = (dj != 0 && tcy <= ta) ? dj : 0;
                                deposit_piece<L::JW>(sJx, sJy, sJz, lx + ci + 1, ly + cj + 1,
                                                     xa - (float)ci, ya - (float)cj,
                                                     xe - (float)ci, ye - (float)cj, tb - ta, qjx,
                                                     qjy, qvz);
                                xa = xe;
                                ya = ye;
                            }
                            ta = fmaxf(ta, tb);
                        }
                        // ---- new cell and tile ----
                        int nix = ix + di, niy = iy + dj;
                        nix = nix < 0 ? nix + nx : (nix >= nx ? nix - nx : nix);
                        niy = niy < 0 ? niy + ny : (niy >= ny ? niy - ny : niy);
                        ncell = nix | (niy << 16);
                        xn = xnn;
                        yn = ynn;
                        const int nlx = lx + di, nly = ly + dj;
                        int dtx = nlx < 0 ? -1 : (nlx >= T ? 1 : 0);
                        int dty = nly < 0 ? -1 : (nly >= T ? 1 : 0);
                        if (g.ntx == 1) dtx = 0;
                        if (g.nty == 1) dty = 0;
                        if (dtx | dty) {
                            const int d = (dty + 1) * 3 + (dtx + 1);
                            dir = d < 4 ? d : d - 1;
                        }
                    }
                }
            }
            // ---- re-sort metadata: warp-aggregated leaver slots ----
            const unsigned lm = __ballot_sync(0xffffffffu, dir >= 0);
            int slot = 0;
            if (lm) {
                const int leader = __ffs(lm) - 1;
                int wbase = 0;
                if (lane == leader) wbase = atomicAdd(&sLeave[s], __popc(lm));
                wbase = __shfl_sync(0xffffffffu, wbase, leader);
                slot = wbase + __popc(lm & ((1u << lane) - 1u));
            }
            if (write) {
                if (dir < 0) {
                    S.cell[p] = ncell;
                    S.x[p] = xn;
                    S.y[p] = yn;
                    S.ux[p] = vx;
                    S.uy[p] = vy;
                    S.uz[p] = vzm;
                } else {
                    const int q = p0 + slot;
                    S.ocell[q] = ncell;
                    S.ox[q] = xn;
                    S.oy[q] = yn;
                    S.oux[q] = vx;
                    S.ouy[q] = vy;
                    S.ouz[q] = vzm;
                    if (prm.track_ids) S.oid[q] = S.id[p];
                    S.hole[q] = p;
                    S.cell[p] = HOLE;
                    atomicAdd(&sDir[s * 8 + dir], 1);
                }
            }
        }
        ke_tot += (double)ke * S.ke_w;
    }
    __syncthreads();

    // ---- per-tile counts for the re-sort ----
    for (int s = 0; s < prm.nsp; ++s) {
        const PushSpecies& S = prm.sp[s];
        if (tid == 0) {
            const int n = S.off[t + 1] - S.off[t];
            S.leave[t] = sLeave[s];
            S.stay[t] = n - sLeave[s];
        }
        if (tid < 8) S.dirc[t * 8 + tid] = sDir[s * 8 + tid];
    }
    if (bad_bits) dev::set_status(prm.st, bad_bits);

    // ---- kinetic energy: FP64 block sum, one FP64 atomic ----
    const double kb = dev::block_sum(ke_tot, sRed);
    if (tid == 0 && prm.nsp > 0) atomicAdd(&prm.hist_k[step & (HIST - 1)], kb);

    // ---- J flush (update_gc_add) ----
    for (int idx = tid; idx < L::JN; idx += nth) {
        const int comp = idx / L::JPLANE;
        const int rem = idx - comp * L::JPLANE;
        const int r = rem / L::JW, q = rem - r * L::JW;
        const int lx = q - 1, ly = r - 1;
        const float v = sJ[idx];
        const bool deep = lx >= 2 && lx < T - 1 && ly >= 2 && ly < T - 1;
        if (!deep && v == 0.f) continue;
        int i = ix0 + lx, j = iy0 + ly;
        i = i < 0 ? i + nx : (i >= nx ? i - nx : i);
        j = j < 0 ? j + ny : (j >= ny ? j - ny : j);
        float* dst = prm.J + comp * g.cstride + (long long)(j + GY) * g.P + (i + GX);
        if (deep)
            *dst = v;
        else
            atomicAdd(dst, v);
    }
}

// fmap == nullptr: only set the kernel's shared-memory limit (done once per
// process before any launch, so never during a stream capture)
template <int T>
static cudaError_t launch_T(const CUtensorMap* fmap, const PushParams& p, int threads,
                            cudaStream_t s) {
    const size_t bytes = Tile<T>::BYTES;
    if (!fmap)
        return cudaFuncSetAttribute(k_push<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)bytes);
    if (p.g.ntiles == 0) return cudaSuccess;
    k_push<T><<<p.g.ntiles, threads, bytes, s>>>(*fmap, p);
    return cudaGetLastError();
}

}  // namespace PIC_VARIANT

cudaError_t PIC_CAT(launch_push_, PIC_VARIANT)(const CUtensorMap* fmap, const PushParams& p,
                                               int threads, cudaStream_t s) {
    switch (p.g.T) {
        case 8: return PIC_VARIANT::launch_T<8>(fmap, p, threads, s);
        case 16: return PIC_VARIANT::launch_T<16>(fmap, p, threads, s);
        case 32: return PIC_VARIANT::launch_T<32>(fmap, p, threads, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pic
