// Particle advance: CTAs over the tiles of T x T cells (§4.1-4.2, the particle
// loop of Listing 3.1), all species of a tile; a tile holding many particles
// is split over several CTAs (blockIdx.y) that each take a slice of it.
//   1. TMA-load the tile's E|B halo, cells [-4, T+4) x [-1, T+2), into shared
//      memory (one 3D box over the six components, mbarrier completion);
//      particles come in batches of blockDim through NSTAGE stages of bulk
//      copies; warps move through the batches independently and the last
//      warp done with a stage issues its refill;
//   2. per particle (coalesced SoA loads): linear gather of the six staggered
//      components (Fig. 3.1), Boris push (Eqs. 6-10), move (Eq. 11) and the
//      Villasenor-Buneman split into at most three pieces (Figs. 3.4-3.5);
//   3. deposit each piece's current (Eqs. 13-16 plus the time-averaged Jz),
//      computed in FP32, into a J tile, cells [-1, T+2), in shared memory:
//      one tile per pair of warps (T <= 16), holding exact 32-bit fixed-point
//      sums (native integer shared atomics cost the same with up to 4 lanes on
//      one word, float ones grow with every conflicting lane); the scale is
//      bounded so no sum can overflow, and the tiles are converted to FP32
//      once, at the flush;
//   4. emit the re-sort metadata of §4.3: particles that stay in the tile are
//      written in place; particles that leave are appended (warp-ballot slots)
//      to the tile's section of the out arrays with their old position in the
//      hole list, and counted by destination (8 neighbours);
//   5. flush: sum the warps' J tiles; a tile taken by one CTA stores the cells
//      no other tile's halo reaches and adds the shared ring with
//      red.global.add (update_gc_add); a split tile adds everything;
//   6. FP32 kinetic energy per thread -> FP64 block sum -> one FP64 atomic.
//
// This file is compiled twice: PIC_VARIANT=fast (FMA contraction, rsqrt and
// fast division) and PIC_VARIANT=strict (PIC_STRICT_BUILD, -fmad=false, IEEE
// division and square root): the strict build evaluates the per-particle path
// in exactly the operation order of the FP32 reference (every expression below
// is written in that order), so cells, offsets and momenta are reproducible
// bit for bit.
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

constexpr unsigned FULL = 0xffffffffu;

// build-time tuning knobs
#ifndef PIC_NSTAGE
#define PIC_NSTAGE 4
#endif
// Two warps share a fixed-point J tile (half the shared memory of per-warp
// tiles: more CTAs per SM; integer atomics of different warps on one word
// only queue, they do not fail), and the run aggregation is off: with the
// pseudo-random order inside a tile a warp's particles almost never share
// cells, so looking for runs costs more than it saves (measured on GB300:
// -17 % particle-advance time for the two together on the 512^2 Weibel case).
#ifndef PIC_WARPS_PER_JTILE
#define PIC_WARPS_PER_JTILE 2
#endif
#ifndef PIC_AGGREGATE
#define PIC_AGGREGATE 0
#endif
// J tiles of the warp groups: exact 32-bit fixed point (1) or FP32 (0)
#ifndef PIC_J_FIXED
#define PIC_J_FIXED 1
#endif
// At most 512 threads per CTA, one CTA per SM guaranteed: with these bounds
// the compiler gives the periodic particle path 63-64 registers (56 under a
// 1024-thread bound, 51 under a bare 512-thread one), enough to avoid
// recomputing values (measured on GB300: -7 % particle-advance time with the
// flush-to-zero build), and 4 CTAs of 256 threads still fit on an SM.  The
// choice is fragile: small changes outside the particle loop (an early exit
// from the species loop) moved it to 80, and on the periodic kernel explicit
// caps at 64 (__maxnreg__, a (512, 2) bound) measured 8-10 % slower than
// this bound.  Under the same bound the moving-window kernel took 68-69 (3
// CTAs per SM, 8 % slower); it is capped explicitly instead.
constexpr int MAX_PUSH_THREADS = 512;
constexpr int PUSH_WINDOW_REGS = 64;
constexpr int NSTAGE = PIC_NSTAGE;  // particle batches (blockDim particles each) in flight per CTA
constexpr int PAD = 4;     // a batch is copied from a 16-byte aligned start: <= 3 extra
// warps sharing one fixed-point J tile (per-warp tiles: 1)
constexpr int WPT = PIC_WARPS_PER_JTILE;

// Shared-memory layout of one CTA (blocks of `nth` threads):
//   [E|B halo FLD floats][J tiles: one per warp (PW) or one per CTA]
//   [NSTAGE particle stages: 6 arrays x (nth + PAD) 32-bit words]
//   [mbarriers: halo + one per stage][counters][FP64 reduction scratch]
//   [one simulation's parameters (batched launch)]
template <int T, bool PW>
struct Tile {
    static constexpr int FW = T + 8;  // TMA box columns: cells -4 .. T+3
    static constexpr int FH = T + 3;  // TMA box rows:    cells -1 .. T+1
    static constexpr int FPLANE = FW * FH;
    static constexpr int FLD = 6 * FPLANE;
    static constexpr int JW = T + 3;  // J tile: cells -1 .. T+1 on both axes
    static constexpr int JPLANE = JW * JW;
    static constexpr int JN = 3 * JPLANE;
    static constexpr bool PER_WARP = PW;
    // leavers by destination per species, then one release counter per stage
    static constexpr int NCNT = MAX_SPECIES * 8 + NSTAGE;

    static __host__ __device__ size_t j_tiles(int nth) { return PW ? ((nth + 31) / 32 + WPT - 1) / WPT : 1; }
    static __host__ __device__ size_t off_stage(int nth) {
        return ((size_t)FLD * 4 + j_tiles(nth) * JN * 4 + 15) & ~(size_t)15;
    }
    static __host__ __device__ size_t stage_words(int nth) { return 6 * (size_t)(nth + PAD); }
    static __host__ __device__ size_t off_misc(int nth) {
        return off_stage(nth) + NSTAGE * stage_words(nth) * 4;
    }
    static __host__ __device__ size_t off_cnt(int nth) { return off_misc(nth) + 8 * (NSTAGE + 2); }
    static __host__ __device__ size_t off_red(int nth) {
        return (off_cnt(nth) + NCNT * 4 + 7) & ~(size_t)7;
    }
    static __host__ __device__ size_t off_prm(int nth) {
        return (off_red(nth) + 32 * sizeof(double) + 15) & ~(size_t)15;
    }
    static __host__ __device__ size_t bytes(int nth) { return off_red(nth) + 32 * sizeof(double); }
    // batched launch: one simulation's parameters, then the current item index
    static __host__ __device__ size_t bytes_batch(int nth) {
        return off_prm(nth) + sizeof(PushParams) + 16;
    }
};

__device__ __forceinline__ float interp(const float* F, int fw, int col, int row, float a0,
                                        float a1, float b0, float b1) {
    const float* r0 = F + row * fw + col;
    const float* r1 = r0 + fw;
    return b0 * (a0 * r0[0] + a1 * r0[1]) + b1 * (a0 * r1[0] + a1 * r1[1]);
}

// division used outside the bit-reproducible path: IEEE in the strict build
__device__ __forceinline__ float qdiv(float a, float b) {
#ifdef PIC_STRICT_BUILD
    return a / b;
#else
    return __fdividef(a, b);
#endif
}

// Current of one straight piece inside one cell, local start (fx0, fy0), end
// (fx1, fy1), fq = q vz times the piece's time fraction: v[0..1] Jx on the
// faces (i+1/2, j) and (i+1/2, j+1) (Eqs. 13-14), v[2..3] Jy on (i, j+1/2) and
// (i+1, j+1/2) (Eqs. 15-16), v[4..7] Jz on the nodes (i,j), (i+1,j), (i,j+1),
// (i+1,j+1): fq times the mean over the piece of each node's area weight.
// With S0, S1 a node's weights at the start and end, the mean along a straight
// piece is [S0x (2 S0y + S1y) + S1x (S0y + 2 S1y)] / 6; for the row j+1 the
// y-factors are a1 = 2 fy0 + fy1 and b1 = fy0 + 2 fy1, for the row j they are
// 3 - a1 and 3 - b1, and the column i weight is one minus the column i+1
// weight, so each a = 0 value is the row total minus its a = 1 value.
__device__ __forceinline__ void piece_current(float v[8], float fx0, float fy0, float fx1,
                                              float fy1, float fq, float qjx, float qjy) {
    const float dxp = fx1 - fx0, dyp = fy1 - fy0;
    const float xm = 0.5f * (fx0 + fx1), ym = 0.5f * (fy0 + fy1);
    const float jxv = qjx * dxp, jyv = qjy * dyp;
    v[1] = jxv * ym;
    v[0] = jxv - v[1];
    v[3] = jyv * xm;
    v[2] = jyv - v[3];
    const float c = fq * (1.f / 6.f);
    const float a1 = 2.f * fy0 + fy1, b1 = fy0 + 2.f * fy1;  // row j+1
    const float a0 = 3.f - a1, b0 = 3.f - b1;                // row j
    v[5] = c * (fx0 * a0 + fx1 * b0);
    v[4] = c * (a0 + b0) - v[5];
    v[7] = c * (fx0 * a1 + fx1 * b1);
    v[6] = c * (a1 + b1) - v[7];
}

// Offset of value k of piece_current from the piece's cell in the J tile
// (component plane k<2: x, k<4: y, else z).
template <int JW, int JPLANE>
__device__ __forceinline__ int value_offset(int k) {
    const int comp = k < 2 ? 0 : (k < 4 ? 1 : 2);
    const int d = (k == 1 || k == 6) ? JW : (k == 3 || k == 5) ? 1 : (k == 7 ? JW + 1 : 0);
    return comp * JPLANE + d;
}

// Reduce-scatter of eight values over the warp: lane L ends with the warp
// total of value L >> 2 (nine shuffles instead of forty for a full reduction).
__device__ __forceinline__ float warp_reduce_scatter8(const float v[8], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float a[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = b4 ? v[i] : v[4 + i];
        a[i] = (b4 ? v[4 + i] : v[i]) + __shfl_xor_sync(FULL, send, 16);
    }
    float c[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = b3 ? a[i] : a[2 + i];
        c[i] = (b3 ? a[2 + i] : a[i]) + __shfl_xor_sync(FULL, send, 8);
    }
    const float send = b2 ? c[0] : c[1];
    float d = (b2 ? c[1] : c[0]) + __shfl_xor_sync(FULL, send, 4);
    d += __shfl_xor_sync(FULL, d, 2);
    d += __shfl_xor_sync(FULL, d, 1);
    return d;
}

constexpr int AGG_MAX_GROUPS = 8;

// Add one value to the J tile: the fixed-point tiles (PER_WARP) hold exact
// 32-bit sums of values already multiplied by the CTA's scale; the CTA-wide
// tile holds FP32.
template <bool PER_WARP>
__device__ __forceinline__ void tile_add(float* a, float x) {
    if constexpr (PER_WARP && PIC_J_FIXED)
        atomicAdd(reinterpret_cast<int*>(a), __float2int_rn(x));
    else
        atomicAdd(a, x);
}

// Deposit one piece per lane (has == false: nothing) into the J tile `sJw`
// (the warp's own tile when PER_WARP, else the CTA's).  Every lane calls this.
// Lanes holding consecutive particles with the same piece cell form a run
// (a run starts where the cell differs from the previous lane's); when the
// warp has few runs, each run is summed across the warp and added by 8 lanes.
// Runs are exact for any particle order: a cell split over several runs is
// simply added several times.  Otherwise every lane adds its eight values.
template <int JW, int JPLANE, bool PER_WARP>
__device__ __forceinline__ void deposit_warp(bool has, int o, const float v[8], float* sJw,
                                             int lane) {
    unsigned act = 0, heads = 0;
    int ng = AGG_MAX_GROUPS + 1;
    if constexpr (PIC_AGGREGATE) {
        act = __ballot_sync(FULL, has);
        const int prev = __shfl_up_sync(FULL, o, 1);
        const bool head = has && (lane == 0 || prev != o || !((act >> (lane - 1)) & 1u));
        heads = __ballot_sync(FULL, head);
        ng = __popc(heads);
    }
    if (PIC_AGGREGATE && ng <= AGG_MAX_GROUPS && __popc(act) >= 2 * ng) {
        // few runs: sum each run across the warp, 8 lanes add the totals
        const int k = lane >> 2;
        const int voff = value_offset<JW, JPLANE>(k);
        while (heads) {
            const int l = __ffs(heads) - 1;
            heads &= heads - 1u;
            const int nxt = heads ? __ffs(heads) - 1 : 32;
            const unsigned upto = nxt == 32 ? FULL : ((1u << nxt) - 1u);
            const unsigned run = upto & ~((1u << l) - 1u) & act;
            const int ko = __shfl_sync(FULL, o, l);
            const bool mine = (run >> lane) & 1u;
            float s[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) s[i] = mine ? v[i] : 0.f;
            const float tot = warp_reduce_scatter8(s, lane);
            if ((lane & 3) == 0) {
                float* a = sJw + ko + voff;
                if constexpr (PER_WARP && WPT == 1)  // the 8 targets are distinct; one run at a time
                    *reinterpret_cast<int*>(a) += __float2int_rn(tot);
                else if constexpr (PER_WARP)
                    atomicAdd(reinterpret_cast<int*>(a), __float2int_rn(tot));
                else
                    atomicAdd(a, tot);
            }
            if constexpr (PER_WARP && WPT == 1) __syncwarp();
        }
    } else if (has) {
        tile_add<PER_WARP>(sJw + o, v[0]);
        tile_add<PER_WARP>(sJw + o + JW, v[1]);
        tile_add<PER_WARP>(sJw + JPLANE + o, v[2]);
        tile_add<PER_WARP>(sJw + JPLANE + o + 1, v[3]);
        tile_add<PER_WARP>(sJw + 2 * JPLANE + o, v[4]);
        tile_add<PER_WARP>(sJw + 2 * JPLANE + o + 1, v[5]);
        tile_add<PER_WARP>(sJw + 2 * JPLANE + o + JW, v[6]);
        tile_add<PER_WARP>(sJw + 2 * JPLANE + o + JW + 1, v[7]);
    }
}

// One work item: slice `chunk` of tile t of the simulation `prm` (steps 1-6
// above).  The caller has initialised the mbarriers (halo: bar[0], stages:
// bar[1..NSTAGE]); fphase is the parity of the next halo phase and gb counts
// the particle batches taken so far, both carried from item to item.
// Returns false (after flagging the timeout) if a bounded wait ran out.
// OPEN: the simulation has a moving window (box open along x); a separate
// instantiation so that the periodic path carries none of its registers.
template <int T, bool PW, bool OPEN = false>
__device__ __forceinline__ bool push_item(const PushParams& prm, const CUtensorMap* fmap, int t,
                                          int chunk, unsigned& fphase, unsigned& gb) {
    using L = Tile<T, PW>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5;
    float* sF = reinterpret_cast<float*>(smem);
    float* sJ = sF + L::FLD;  // [j_tiles][3][JPLANE]
    float* sStage = reinterpret_cast<float*>(smem + L::off_stage(nth));
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::off_misc(nth));
    uint64_t* sbar = bar + 1;  // one per particle stage
    int* sDir = reinterpret_cast<int*>(smem + L::off_cnt(nth));  // [MAX_SPECIES][8]
    int* sFree = sDir + MAX_SPECIES * 8;  // [NSTAGE]: warps done with the stage's batch
    const int nwarps = nth >> 5;
    double* sRed = reinterpret_cast<double*>(smem + L::off_red(nth));
    float* sJw = sJ + (L::PER_WARP ? (warp / WPT) * L::JN : 0);
    const int jtiles = (int)L::j_tiles(nth);
    const int SW = nth + PAD;  // words per array per stage
    const unsigned stage_bytes = (unsigned)L::stage_words(nth) * 4u;

    const Geom& g = prm.g;
    const int tx = tile_x(g, t), ty = tile_y(g, t);
    const int ix0 = tx * T, iy0 = ty * T;
    const long long step = *((volatile long long*)&prm.st->step);
    // moving window (open box along x): cells are written in the frame of the
    // window after this step's shift; particles leaving the box are removed
    const int wshift = OPEN ? window_shift(step, g) : 0;

    for (int i = tid; i < L::NCNT; i += nth) sDir[i] = 0;
    __syncthreads();
    if (tid == 0) {
        dev::mbar_arrive_expect_tx(bar, L::FLD * 4);
        // box origin: column ix0 = cell ix0 - GX, row iy0 = cell iy0 - GY
        dev::tma_load_3d(sF, fmap, ix0, iy0, 0, bar);
    }
    for (int i = tid; i < jtiles * L::JN; i += nth) sJ[i] = 0.f;
    const bool ok = dev::mbar_wait_bounded(bar, fphase);
    fphase ^= 1u;
    if (__syncthreads_or(!ok)) {
        if (tid == 0) {
            dev::mbar_wait_bounded(bar, fphase ^ 1u);  // the halo copy, once more, before leaving
            dev::set_status(prm.st, ST_TIMEOUT);
        }
        return false;
    }

    const float* sEx = sF;
    const float* sEy = sF + L::FPLANE;
    const float* sEz = sF + 2 * L::FPLANE;
    const float* sBx = sF + 3 * L::FPLANE;
    const float* sBy = sF + 4 * L::FPLANE;
    const float* sBz = sF + 5 * L::FPLANE;
    const int nx = g.nx, ny = g.ny;
    const float cxs = g.cx, cys = g.cy;
    unsigned bad_bits = 0;
    double ke_tot = 0.0;
    // Fixed-point scale of the J tiles.  The current one particle gives to
    // any one node, summed over its pieces, is at most |qtilde| (the pieces
    // partition a move shorter than a cell per step and the weights sum to
    // one), and the WPT warps of a tile take at most 32 particles each per
    // batch, so every tile sum stays below 2^30 with this scale: no overflow
    // is possible.
    float qbound = 0.f;
    for (int s = 0; s < prm.nsp; ++s) {
        const int ns = prm.sp[s].off[t + 1] - prm.sp[s].off[t];
        const int ls = (ns + prm.chunks - 1) / prm.chunks;
        qbound += (float)(((ls + nth - 1) / nth) * 32 * WPT) * fabsf(prm.sp[s].qjz);
    }
    const float qscale = qbound > 0.f ? 1073741824.f / qbound : 1.f;
    const float qinv = 1.f / qscale;

    for (int s = 0; s < prm.nsp; ++s) {
        const PushSpecies& S = prm.sp[s];
        const int p0 = S.off[t];
        const int nt = S.off[t + 1] - p0;
        const int len = (nt + prm.chunks - 1) / prm.chunks;
        const int c0 = p0 + min(chunk * len, nt), c1 = p0 + min((chunk + 1) * len, nt);
        // current constants, times the fixed-point scale for the integer tiles
        const float dsc = (L::PER_WARP && PIC_J_FIXED) ? qscale : 1.f;
        const float tem = S.tem, qjx = S.qjx * dsc, qjy = S.qjy * dsc, qjz = S.qjz * dsc;
        float ke = 0.f;
        // Particle batches come in through a NSTAGE-deep pipeline of bulk copies
        // (one per array, from the 16-byte aligned index below the batch start;
        // the arrays are padded so the copy never leaves their allocation).
        const int nb = (c1 - c0 + nth - 1) / nth;
        auto issue = [&](int b, unsigned gslot) {
            const int a4 = (c0 + b * nth) & ~3;
            float* dst = sStage + (size_t)(gslot % NSTAGE) * L::stage_words(nth);
            uint64_t* sb = sbar + gslot % NSTAGE;
            const unsigned bytes = (unsigned)SW * 4u;
            dev::mbar_arrive_expect_tx(sb, stage_bytes);
            dev::bulk_load(dst, S.cell + a4, bytes, sb);
            dev::bulk_load(dst + SW, S.x + a4, bytes, sb);
            dev::bulk_load(dst + 2 * SW, S.y + a4, bytes, sb);
            dev::bulk_load(dst + 3 * SW, S.ux + a4, bytes, sb);
            dev::bulk_load(dst + 4 * SW, S.uy + a4, bytes, sb);
            dev::bulk_load(dst + 5 * SW, S.uz + a4, bytes, sb);
        };
        // Warps run through the batches independently: the last warp to be
        // done with a stage refills it (no CTA barrier per batch).
        __syncthreads();  // every warp is done with the previous species' stages
        if (tid == 0)
            for (int b = 0; b < min(nb, NSTAGE); ++b) issue(b, gb + b);
        for (int b = 0; b < nb; ++b) {
            const unsigned gcur = gb + b;
            const bool landed = dev::mbar_wait_bounded(sbar + gcur % NSTAGE, (gcur / NSTAGE) & 1u);
            if (!landed) bad_bits |= ST_TIMEOUT;
            const int base = c0 + b * nth;
            const float* sp = sStage + (size_t)(gcur % NSTAGE) * L::stage_words(nth) +
                              (base - (base & ~3)) + tid;
            const int p = base + tid;
            const bool active = p < c1 && landed;
            bool write = false;
            int dir = -1;  // -1: stays in this tile; 0..7: leaves towards that neighbour
            int ncell = 0;
            float xn = 0.f, yn = 0.f, vx = 0.f, vy = 0.f, vzm = 0.f;
            // the move to deposit: start, end, crossings (frame of the start cell)
            bool mv = false;
            float mx0 = 0.f, my0 = 0.f, mx1 = 0.f, my1 = 0.f, mxb = 0.f, myb = 0.f;
            float mtx = 2.f, mty = 2.f, mqvz = 0.f;
            int mdi = 0, mdj = 0, mlx = 0, mly = 0;
            if (active) {
                const int c = __float_as_int(sp[0]);
                const float x = sp[SW], y = sp[2 * SW];
                float ux = sp[3 * SW], uy = sp[4 * SW], uz = sp[5 * SW];
                const int ix = c & 0xffff, iy = (int)((unsigned)c >> 16);
                const int lx = ix - ix0, ly = iy - iy0;
                if (c == HOLE || lx < 0 || lx >= T || ly < 0 || ly >= T) {
                    bad_bits |= ST_SORT;  // not in this tile: leave it untouched
                } else {
                    write = true;
                    // ---- gather (Fig. 3.1 staggering) ----
                    const float wx1 = x, wx0 = 1.f - x, wy1 = y, wy0 = 1.f - y;
                    const float xh = x + 0.5f, yh = y + 0.5f;
                    // floor(xh) for xh in [0.5, 1.5]
                    const bool xup = xh >= 1.f, yup = yh >= 1.f;
                    const float hx1 = xh - (xup ? 1.f : 0.f), hx0 = 1.f - hx1;
                    const float hy1 = yh - (yup ? 1.f : 0.f), hy0 = 1.f - hy1;
                    const int cn = lx + GX, ch = cn - (xup ? 0 : 1);
                    const int rn = ly + GY, rh = rn - (yup ? 0 : 1);
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
#ifdef PIC_STRICT_BUILD
                    const float gm = sqrtf(1.f + umx * umx + umy * umy + umz * umz);
                    const float gtem = tem / gm;
#else
                    const float g2 = 1.f + umx * umx + umy * umy + umz * umz;
                    const float rgm = rsqrtf(g2);
                    const float gtem = tem * rgm;
                    const float gm = g2 * rgm;
#endif
                    const float btx = gtem * bx, bty = gtem * by, btz = gtem * bz;
                    const float upx = umx + umy * btz - umz * bty;
                    const float upy = umy + umz * btx - umx * btz;
                    const float upz = umz + umx * bty - umy * btx;
                    const float f = qdiv(2.f, 1.f + btx * btx + bty * bty + btz * btz);
                    const float sx = f * btx, sy = f * bty, sz = f * btz;
                    const float uqx = umx + upy * sz - upz * sy;
                    const float uqy = umy + upz * sx - upx * sz;
                    const float uqz = umz + upx * sy - upy * sx;
                    ux = uqx + tem * ex;
                    uy = uqy + tem * ey;
                    uz = uqz + tem * ez;
                    // gamma - 1 = |u-|^2 / (gamma + 1), free of cancellation
                    ke += qdiv(umx * umx + umy * umy + umz * umz, gm + 1.f);
                    // ---- move, Eq. 11 in cell units ----
#ifdef PIC_STRICT_BUILD
                    const float gg = sqrtf(1.f + ux * ux + uy * uy + uz * uz);
                    const float rg = 1.f / gg;
#else
                    const float rg = rsqrtf(1.f + ux * ux + uy * uy + uz * uz);
#endif
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
                        // ---- Villasenor-Buneman split: crossing fractions ----
                        mv = true;
                        mx0 = x;
                        my0 = y;
                        mx1 = x1;
                        my1 = y1;
                        mdi = di;
                        mdj = dj;
                        mlx = lx;
                        mly = ly;
                        mqvz = qjz * vz;
                        mxb = di > 0 ? 1.f : 0.f;
                        myb = dj > 0 ? 1.f : 0.f;
                        mtx = di ? qdiv(mxb - x, x1 - x) : 2.f;
                        mty = dj ? qdiv(myb - y, y1 - y) : 2.f;
                        // ---- new cell and tile ----
                        int nix = ix + di - wshift, niy = iy + dj;
                        bool gone = false;
                        if (OPEN)  // left the box (before or by the shift)
                            gone = nix < 0 || nix >= nx - wshift;
                        else
                            nix = nix < 0 ? nix + nx : (nix >= nx ? nix - nx : nix);
                        niy = niy < 0 ? niy + ny : (niy >= ny ? niy - ny : niy);
                        ncell = nix | (niy << 16);
                        xn = xnn;
                        yn = ynn;
                        const int nlx = lx + di - wshift, nly = ly + dj;
                        int dtx = nlx < 0 ? -1 : (nlx >= T ? 1 : 0);
                        int dty = nly < 0 ? -1 : (nly >= T ? 1 : 0);
                        if (g.ntx == 1) dtx = 0;
                        if (g.nty == 1) dty = 0;
                        if (gone) {
                            dir = 8;  // removed: a leaver with no destination
                        } else if (dtx | dty) {
                            const int d = (dty + 1) * 3 + (dtx + 1);
                            dir = d < 4 ? d : d - 1;
                        }
                    }
                }
            }
            // ---- deposit.  A warp none of whose moves crosses a cell edge
            // deposits each move as one piece; otherwise piece by piece over
            // the whole warp (at most three pieces per move, Figs. 3.4-3.5) ----
            if (!__any_sync(FULL, mv && (mdi | mdj))) {
                float v[8];
                const int o = (mly + 1) * L::JW + (mlx + 1);
                piece_current(v, mx0, my0, mx1, my1, mqvz, qjx, qjy);
                deposit_warp<L::JW, L::JPLANE, L::PER_WARP>(mv, o, v, sJw, lane);
            } else {
                const float t1 = fminf(fminf(mtx, mty), 1.f);
                const float t2 = fminf(fmaxf(mtx, mty), 1.f);
                float ta = 0.f, xa = mx0, ya = my0;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float tb = k == 0 ? t1 : (k == 1 ? t2 : 1.f);
                    // a corner crossing leaves the middle piece empty: skip, do not stop
                    const bool has = mv && tb > ta;
                    if (__any_sync(FULL, has)) {
                        float v[8];
                        int o = 0;
                        float xe = xa, ye = ya;
                        if (has) {
                            xe = tb == mtx ? mxb : (tb == 1.f ? mx1 : mx0 + tb * (mx1 - mx0));
                            ye = tb == mty ? myb : (tb == 1.f ? my1 : my0 + tb * (my1 - my0));
                            const int ci = (mdi != 0 && mtx <= ta) ? mdi : 0;
                            const int cj = (mdj != 0 && mty <= ta) ? mdj : 0;
                            o = (mly + cj + 1) * L::JW + (mlx + ci + 1);
                            piece_current(v, xa - (float)ci, ya - (float)cj, xe - (float)ci,
                                          ye - (float)cj, mqvz * (tb - ta), qjx, qjy);
                        } else if constexpr (PIC_AGGREGATE) {
#pragma unroll
                            for (int i = 0; i < 8; ++i) v[i] = 0.f;
                        }
                        deposit_warp<L::JW, L::JPLANE, L::PER_WARP>(has, o, v, sJw, lane);
                        xa = xe;
                        ya = ye;
                    }
                    ta = fmaxf(ta, tb);
                }
            }
            // ---- re-sort metadata: leaver slots in the tile's out section, one
            // global atomic per warp that has leavers (shared by the tile's CTAs) ----
            const unsigned lm = __ballot_sync(FULL, dir >= 0);
            int slot = 0;
            if (lm) {
                const int leader = __ffs(lm) - 1;
                int wbase = 0;
                if (lane == leader) wbase = atomicAdd(&S.leave[t], __popc(lm));
                wbase = __shfl_sync(FULL, wbase, leader);
                slot = wbase + __popc(lm & ((1u << lane) - 1u));
                if (OPEN) {
                    const unsigned rm = __ballot_sync(FULL, dir == 8);
                    if (rm && lane == leader)
                        atomicAdd(reinterpret_cast<unsigned long long*>(&prm.st->removed[s]),
                                  (unsigned long long)__popc(rm));
                }
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
                    S.ocell[q] = dir == 8 ? HOLE : ncell;  // a removed particle goes nowhere
                    S.ox[q] = xn;
                    S.oy[q] = yn;
                    S.oux[q] = vx;
                    S.ouy[q] = vy;
                    S.ouz[q] = vzm;
                    if (prm.track_ids) S.oid[q] = S.id[p];
                    S.hole[q] = p;
                    S.odir[q] = (uint8_t)dir;
                    S.cell[p] = HOLE;
                    if (dir < 8) atomicAdd(&sDir[s * 8 + dir], 1);
                }
            }
            // ---- release the stage; the last warp refills it ----
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                const int st = (int)(gcur % NSTAGE);
                if (atomicAdd(&sFree[st], 1) == nwarps - 1) {
                    atomicExch(&sFree[st], 0);
                    if (b + NSTAGE < nb) {
                        dev::fence_proxy_async_smem();  // our reads before the async overwrite
                        issue(b + NSTAGE, gcur + NSTAGE);
                    }
                }
            }
        }
        gb += nb;
        ke_tot += (double)ke * S.ke_w;
    }
    if (__syncthreads_or(bad_bits & ST_TIMEOUT)) {
        // a wait ran out: wait (bounded) once more for the last copy issued
        // into each stage, so that none is in flight when the CTA leaves.
        // Every batch of every species was issued (releases and refills go on
        // after a wait runs out), so the copies issued are those of the
        // global batch indices below gb, in order.
        if (tid == 0) {
            for (unsigned st = 0; st < (unsigned)NSTAGE; ++st)
                if (gb > st) {
                    const unsigned g = st + ((gb - 1 - st) / NSTAGE) * NSTAGE;
                    dev::mbar_wait_bounded(sbar + st, (g / NSTAGE) & 1u);
                }
            dev::set_status(prm.st, ST_TIMEOUT);
        }
        return false;
    }

    // ---- leavers by destination, for the re-sort's counts ----
    for (int s = 0; s < prm.nsp; ++s)
        if (tid < 8 && sDir[s * 8 + tid]) atomicAdd(&prm.sp[s].dirc[t * 8 + tid], sDir[s * 8 + tid]);
    if (bad_bits) dev::set_status(prm.st, bad_bits);

    // ---- kinetic energy: FP64 block sum, one FP64 atomic ----
    const double kb = dev::block_sum(ke_tot, sRed);
    if (tid == 0 && prm.nsp > 0) atomicAdd(&prm.hist_k[step & (HIST - 1)], kb);

    // ---- J flush (update_gc_add).  A tile taken by one CTA stores the cells
    // no other tile's halo reaches and adds the shared ring; a tile split over
    // several CTAs adds everything (the Yee kernel then clears all of J). ----
    const bool whole = prm.chunks == 1;
    for (int idx = tid; idx < L::JN; idx += nth) {
        const int comp = idx / L::JPLANE;
        const int rem = idx - comp * L::JPLANE;
        const int r = rem / L::JW, q = rem - r * L::JW;
        const int lx = q - 1, ly = r - 1;
        float v;
        if constexpr (L::PER_WARP && PIC_J_FIXED) {
            long long acc = 0;
            for (int w = 0; w < jtiles; ++w)
                acc += reinterpret_cast<const int*>(sJ)[w * L::JN + idx];
            v = (float)acc * qinv;
        } else if constexpr (L::PER_WARP) {
            v = 0.f;
            for (int w = 0; w < jtiles; ++w) v += sJ[w * L::JN + idx];
        } else {
            v = sJ[idx];
        }
        const bool deep = whole && lx >= 2 && lx < T - 1 && ly >= 2 && ly < T - 1;
        if (!deep && v == 0.f) continue;
        int i = ix0 + lx, j = iy0 + ly;
        if (OPEN && (i < 0 || i >= nx)) continue;  // outside the open box: dropped
        i = i < 0 ? i + nx : (i >= nx ? i - nx : i);
        j = j < 0 ? j + ny : (j >= ny ? j - ny : j);
        float* dst = prm.J + comp * g.cstride + (long long)(j + GY) * g.P + (i + GX);
        if (deep)
            *dst = v;
        else
            atomicAdd(dst, v);
    }
    return true;
}

__device__ __forceinline__ void init_barriers(uint64_t* bar) {
    if (threadIdx.x == 0) {
        for (int i = 0; i <= NSTAGE; ++i) dev::mbar_init(bar + i, 1);
        dev::fence_mbar_init();
    }
}

// One simulation: CTA (tile, chunk) = (blockIdx.x, blockIdx.y).  The
// periodic box and the moving window's open box are separate kernels, each
// with the register budget measured best for it (see MAX_PUSH_THREADS).
template <int T, bool PW>
__global__ void __launch_bounds__(MAX_PUSH_THREADS, 1) k_push(const __grid_constant__ CUtensorMap fmap,
                                                             const PushParams prm) {
    extern __shared__ __align__(128) unsigned char smem[];
    init_barriers(reinterpret_cast<uint64_t*>(smem + Tile<T, PW>::off_misc(blockDim.x)));
    unsigned fphase = 0, gb = 0;
    push_item<T, PW, false>(prm, &fmap, blockIdx.x, blockIdx.y, fphase, gb);
}

template <int T, bool PW>
__global__ void __maxnreg__(PUSH_WINDOW_REGS) k_push_window(const __grid_constant__ CUtensorMap fmap,
                                                            const PushParams prm) {
    extern __shared__ __align__(128) unsigned char smem[];
    init_barriers(reinterpret_cast<uint64_t*>(smem + Tile<T, PW>::off_misc(blockDim.x)));
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        // the window decision of this step, for the re-sort and field kernels
        // that follow (no CTA of this launch reads them)
        const int w = window_shift(*((volatile long long*)&prm.st->step), prm.g);
        prm.st->win_shift = w;
        prm.st->win_moves += w;
    }
    unsigned fphase = 0, gb = 0;
    push_item<T, PW, true>(prm, &fmap, blockIdx.x, blockIdx.y, fphase, gb);
}

// Many simulations in one persistent launch: each CTA takes work items
// (member, tile, chunk) from a global counter until the list is exhausted (the
// list is ordered costliest first, so this is greedy longest-first
// balancing); the item's parameters are copied into shared memory and its
// TMA descriptor is read from global memory.
// Two CTAs of 512 threads per SM: the persistent batched kernel keeps the
// 64-register budget of the single-simulation one (without the bound the
// item bookkeeping pushes it past 100 registers and to one CTA per SM).
template <int T, bool PW>
__global__ void __launch_bounds__(MAX_PUSH_THREADS, 2) k_push_batch(const PushBatch pb) {
    using L = Tile<T, PW>;
    extern __shared__ __align__(128) unsigned char smem[];
    init_barriers(reinterpret_cast<uint64_t*>(smem + L::off_misc(blockDim.x)));
    PushParams* sPrm = reinterpret_cast<PushParams*>(smem + L::off_prm(blockDim.x));
    int* sItem = reinterpret_cast<int*>(smem + L::off_prm(blockDim.x) + sizeof(PushParams));
    unsigned fphase = 0, gb = 0;
    while (true) {
        __syncthreads();  // the previous item is done with shared memory
        if (threadIdx.x == 0) *sItem = atomicAdd(pb.next, 1);
        __syncthreads();
        const int it = *sItem;
        if (it >= pb.nitems) return;
        const int4 item = pb.items[it];
        const int4* src = reinterpret_cast<const int4*>(pb.members + item.x);
        int4* dst = reinterpret_cast<int4*>(sPrm);
        for (int i = threadIdx.x; i < (int)(sizeof(PushParams) / 16); i += blockDim.x)
            dst[i] = src[i];
        __syncthreads();
        if (!push_item<T, PW>(*sPrm, pb.tmaps + item.x, item.y, item.z, fphase, gb)) return;
    }
}

// Per-warp J tiles are used for T <= 16 when the CTA's shared memory allows
// (PIC_J_PER_WARP=0 at build time turns them off).
#ifndef PIC_J_PER_WARP
#define PIC_J_PER_WARP 1
#endif
constexpr size_t SMEM_MAX = 227 * 1024;

template <int T, bool PW>
static cudaError_t set_smem_limit() {
    static_assert(sizeof(PushParams) % 16 == 0, "parameters are copied as int4");
    size_t b = Tile<T, PW>::bytes_batch(1024);
    if (b > SMEM_MAX) b = SMEM_MAX;
    cudaError_t e =
        cudaFuncSetAttribute(k_push<T, PW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_push_window<T, PW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_push_batch<T, PW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)b);
}

// fmap == nullptr: only set the kernels' shared-memory limits (done once per
// process before any launch, so never during a stream capture)
template <int T>
static cudaError_t launch_T(const CUtensorMap* fmap, const PushParams& p, int threads,
                            cudaStream_t s) {
    constexpr bool kPW = PIC_J_PER_WARP && T <= 16;
    if (!fmap) {
        cudaError_t e = set_smem_limit<T, false>();
        if (e == cudaSuccess && kPW) e = set_smem_limit<T, kPW>();
        return e;
    }
    if (p.g.ntiles == 0) return cudaSuccess;
    const dim3 grid(p.g.ntiles, p.chunks);
    const bool pw = kPW && !p.fp32_j && Tile<T, kPW>::bytes(threads) <= SMEM_MAX;
    const size_t bytes = pw ? Tile<T, kPW>::bytes(threads) : Tile<T, false>::bytes(threads);
    if (p.g.open_x) {
        if (pw) k_push_window<T, kPW><<<grid, threads, bytes, s>>>(*fmap, p);
        else k_push_window<T, false><<<grid, threads, bytes, s>>>(*fmap, p);
    } else {
        if (pw) k_push<T, kPW><<<grid, threads, bytes, s>>>(*fmap, p);
        else k_push<T, false><<<grid, threads, bytes, s>>>(*fmap, p);
    }
    return cudaGetLastError();
}

template <int T, bool PW>
static cudaError_t launch_batch_TP(const PushBatch& b, int threads, int grid, cudaStream_t s) {
    const size_t bytes = Tile<T, PW>::bytes_batch(threads);
    if (grid <= 0) {
        // persistent: as many CTAs as can be resident at once
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_push_batch<T, PW>, threads,
                                                              bytes);
        if (e != cudaSuccess) return e;
        grid = sms * (per_sm > 0 ? per_sm : 1);
    }
    if (grid > b.nitems) grid = b.nitems;
    k_push_batch<T, PW><<<grid, threads, bytes, s>>>(b);
    return cudaGetLastError();
}

template <int T>
static cudaError_t launch_batch_T(const PushBatch& b, int threads, int grid, cudaStream_t s) {
    constexpr bool kPW = PIC_J_PER_WARP && T <= 16;
    if (b.nitems == 0) return cudaSuccess;
    if (kPW && !b.fp32_j && Tile<T, kPW>::bytes_batch(threads) <= SMEM_MAX)
        return launch_batch_TP<T, kPW>(b, threads, grid, s);
    return launch_batch_TP<T, false>(b, threads, grid, s);
}

}  // namespace PIC_VARIANT

cudaError_t PIC_CAT(launch_push_batch_, PIC_VARIANT)(const PushBatch& b, int T, int threads,
                                                     int grid, cudaStream_t s) {
    switch (T) {
        case 8: return PIC_VARIANT::launch_batch_T<8>(b, threads, grid, s);
        case 16: return PIC_VARIANT::launch_batch_T<16>(b, threads, grid, s);
        case 32: return PIC_VARIANT::launch_batch_T<32>(b, threads, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t PIC_CAT(launch_push_, PIC_VARIANT)(const CUtensorMap* fmap, const PushParams& p,
                                               int threads, cudaStream_t s) {
    if (!fmap) {
        // raise the shared-memory limits of every tile size (a simulation may
        // be re-tiled later)
        cudaError_t e = PIC_VARIANT::launch_T<8>(nullptr, p, threads, s);
        if (e == cudaSuccess) e = PIC_VARIANT::launch_T<16>(nullptr, p, threads, s);
        if (e == cudaSuccess) e = PIC_VARIANT::launch_T<32>(nullptr, p, threads, s);
        return e;
    }
    switch (p.g.T) {
        case 8: return PIC_VARIANT::launch_T<8>(fmap, p, threads, s);
        case 16: return PIC_VARIANT::launch_T<16>(fmap, p, threads, s);
        case 32: return PIC_VARIANT::launch_T<32>(fmap, p, threads, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pic
