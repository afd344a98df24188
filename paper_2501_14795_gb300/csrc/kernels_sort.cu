// Tile re-sort (§4.3, the Jocksch scheme adapted to warp ballots and scans).
//
// After the particle advance every tile t knows: leave[t] leavers appended to out[off_old[t] ...] with their vacated
// positions in hole[off_old[t] ...], and dirc[t][d] leavers per destination.
//   count  (thread per tile): new counts = stayers + incoming from the eight
//            neighbours (step 1 of §4.3);
//   k_scan   (one CTA per species): exclusive scan -> off_new; also advances
//            the step counter and primes the energy history.
//   k_evict  (warp per tile): stayers whose position falls outside the tile's
//            new range are displaced occupants; copy them to the tail of the
//            tile's out section (they are re-inserted into their own tile).
//   k_fill   (warp per tile): target_idx = holes of t inside its new range plus
//            the part of the new range outside the old one; source_idx =
//            leavers of the neighbours heading to t plus t's displaced
//            stayers (steps 2-4); then move source -> target (step 5).
// Only leavers and displaced particles move; a particle's bytes are read and
// written once more.  No per-particle global atomics: slots come from warp
// ballots.  Every step has a single-simulation kernel and a batched one that
// flattens the tiles of many simulations into one grid; both call the same
// per-tile bodies.
#include "device_util.cuh"
#include "pic_internal.h"

namespace pic {

namespace {

// neighbour of tile (tx, ty) displaced by direction d (0..7 over the 3x3
// stencil without its centre)
__device__ __forceinline__ void dir_delta(int d, int& dx, int& dy) {
    const int k = d < 4 ? d : d + 1;
    dx = k % 3 - 1;
    dy = k / 3 - 1;
}

// member m of a batch whose items start at start[m] (start[nmembers] = total)
__device__ __forceinline__ int find_member(const int* start, int n, int g) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Moving-window injection into tile t this step: particles per tile row of
// cells (k * kept lattice columns), the first kept lattice column and the
// tile's total (0 unless the window shifted this step and t is in the last
// tile column).
struct Injection {
    int per_row, a0, total;
};
__device__ __forceinline__ Injection injection(const SortParams& prm, const SortSpecies& S, int t) {
    Injection r{0, 0, 0};
    const Geom& g = prm.g;
    if (!g.open_x || S.inj_k == 0 || tile_x(g, t) != g.ntx - 1) return r;
    if (!*((volatile int*)&prm.st->win_shift)) return r;
    const long long gcol = *((volatile long long*)&prm.st->win_moves) + g.nx - 1;
    r.a0 = inject_first(gcol, S.inj_k, S.inj_x0, g.dx);
    r.per_row = S.inj_k * (S.inj_k - r.a0);
    r.total = r.per_row * g.T;
    return r;
}

// Write injected particle m of tile t (rows of cells, then lattice rows b,
// then kept lattice columns a) at slot `to`.
__device__ __forceinline__ void inject_particle(const SortParams& prm, const SortSpecies& S,
                                                int t, const Injection& inj, int m, int to) {
    const Geom& g = prm.g;
    const int k = S.inj_k, na = k - inj.a0;
    const int r = m / inj.per_row, rem = m - r * inj.per_row;
    const int b = rem / na, a = inj.a0 + rem % na;
    const int iy = tile_y(g, t) * g.T + r;
    S.cell[to] = (g.nx - 1) | (iy << 16);
    S.x[to] = (float)(((double)a + 0.5) / (double)k);
    S.y[to] = (float)(((double)b + 0.5) / (double)k);
    S.ux[to] = S.inj_u[0];
    S.uy[to] = S.inj_u[1];
    S.uz[to] = S.inj_u[2];
    if (prm.track_ids) S.id[to] = -1;
}

__device__ __forceinline__ void copy_particle(const SortSpecies& S, int from_out, int to_main,
                                              int track) {
    S.cell[to_main] = S.ocell[from_out];
    S.x[to_main] = S.ox[from_out];
    S.y[to_main] = S.oy[from_out];
    S.ux[to_main] = S.oux[from_out];
    S.uy[to_main] = S.ouy[from_out];
    S.uz[to_main] = S.ouz[from_out];
    if (track) S.id[to_main] = S.oid[from_out];
}

// two particles from the out arrays: all loads, then all stores
__device__ __forceinline__ void copy_two(const SortSpecies& S, int f0, int t0, int f1, int t1,
                                         int track) {
    const int c0 = S.ocell[f0], c1 = S.ocell[f1];
    const float x0 = S.ox[f0], x1 = S.ox[f1], y0 = S.oy[f0], y1 = S.oy[f1];
    const float a0 = S.oux[f0], a1 = S.oux[f1], b0 = S.ouy[f0], b1 = S.ouy[f1];
    const float z0 = S.ouz[f0], z1 = S.ouz[f1];
    int i0 = 0, i1 = 0;
    if (track) {
        i0 = S.oid[f0];
        i1 = S.oid[f1];
    }
    S.cell[t0] = c0;
    S.cell[t1] = c1;
    S.x[t0] = x0;
    S.x[t1] = x1;
    S.y[t0] = y0;
    S.y[t1] = y1;
    S.ux[t0] = a0;
    S.ux[t1] = a1;
    S.uy[t0] = b0;
    S.uy[t1] = b1;
    S.uz[t0] = z0;
    S.uz[t1] = z1;
    if (track) {
        S.id[t0] = i0;
        S.id[t1] = i1;
    }
}

constexpr int SCAN_THREADS = 1024;

// Step 1 of §4.3 for tile t of species s: the tile's new count = its stayers
// (old count - leavers) + the leavers of the eight neighbours heading here;
// kept in off_new[t] for the scan.  Also clears the idle parity's counters
// for the next step.  Returns the tile's leavers.
__device__ __forceinline__ int count_tile(const SortParams& prm, int s, int t) {
    const SortSpecies& S = prm.sp[s];
    const Geom& g = prm.g;
    const int tx = tile_x(g, t), ty = tile_y(g, t);
    const int lv = S.leave[t];
    int c = S.off_old[t + 1] - S.off_old[t] - lv;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        int ddx, ddy;
        dir_delta(d, ddx, ddy);
        if ((g.ntx == 1 && ddx) || (g.nty == 1 && ddy)) continue;
        const int sx = dev::wrapi(tx - ddx, g.ntx), sy = dev::wrapi(ty - ddy, g.nty);
        c += S.dirc[tile_index(g, sx, sy) * 8 + d];
    }
    c += injection(prm, S, t).total;
    S.off_new[t] = c;
    S.leave_next[t] = 0;
#pragma unroll
    for (int d = 0; d < 8; ++d) S.dirc_next[t * 8 + d] = 0;
    return lv;
}

__global__ void k_count(const SortParams prm) {
    const int s = blockIdx.y;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    int lv = t < prm.g.ntiles ? count_tile(prm, s, t) : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lv += __shfl_xor_sync(0xffffffffu, lv, o);
    if ((threadIdx.x & 31) == 0 && lv)
        atomicAdd(reinterpret_cast<unsigned long long*>(&prm.st->leavers_acc[s]),
                  (unsigned long long)lv);
}

// batched: thread per tile of the flattened tile list of all members
__global__ void k_count_batch(const SortBatch b) {
    const int s = blockIdx.y;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    if (gt >= b.total_tiles) return;
    const int m = find_member(b.tile_start, b.nmembers, gt);
    const SortParams& P = b.members[m];
    if (s >= P.nsp) return;
    const int lv = count_tile(P, s, gt - b.tile_start[m]);
    if (lv)
        atomicAdd(reinterpret_cast<unsigned long long*>(&P.st->leavers_acc[s]),
                  (unsigned long long)lv);
}

// In-place exclusive scan of the counts in off_new of species s by the whole
// CTA, 4096 tiles per round with coalesced loads; off_new[ntiles] = total,
// which must equal the particle count.  With `advance`, thread 0 also moves
// the simulation to time level n+1 and primes that level's history slots.
__device__ __forceinline__ void scan_species(const SortParams& prm, int s, bool advance) {
    __shared__ int sWarp[32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (advance && tid == 0) {
        const long long n = prm.st->step + 1;
        prm.hist_e[n & (HIST - 1)] = 0.0;
        prm.hist_b[n & (HIST - 1)] = 0.0;
        prm.hist_k[n & (HIST - 1)] = 0.0;
        prm.st->step = n;
    }
    if (s >= prm.nsp) return;
    const SortSpecies& S = prm.sp[s];
    const int nt = prm.g.ntiles;
    int carry = 0;
    for (int base = 0; base < nt; base += 4 * SCAN_THREADS) {
        const int i0 = base + 4 * tid;
        int v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = i0 + k < nt ? S.off_new[i0 + k] : 0;
        const int mine = v[0] + v[1] + v[2] + v[3];
        int incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) sWarp[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            const int w = sWarp[lane];
            int wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += u;
            }
            sWarp[lane] = wi;  // inclusive prefix of the warp sums
        }
        __syncthreads();
        int run = carry + (wid ? sWarp[wid - 1] : 0) + incl - mine;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (i0 + k < nt) S.off_new[i0 + k] = run;
            run += v[k];
        }
        carry += sWarp[31];
        __syncthreads();  // sWarp is rewritten by the next round
    }
    __shared__ int sBad;
    const int lim = prm.g.open_x ? S.cap : S.n;
    if (tid == 0) {
        S.off_new[nt] = carry;
        bool bad;
        if (prm.g.open_x) {
            // the count changes by the removed and injected particles
            const Injection inj = injection(prm, S, tile_index(prm.g, prm.g.ntx - 1, 0));
            const long long want =
                prm.st->np[s] - prm.st->removed[s] + (long long)inj.total * prm.g.nty;
            bad = carry != want || carry > S.cap;
            prm.st->np[s] = min(carry, S.cap);
            prm.st->removed[s] = 0;
        } else {
            bad = carry != S.n;
        }
        if (bad) dev::set_status(prm.st, ST_SORT);
        sBad = bad;
    }
    __syncthreads();
    // inconsistent counts: the bookmarks are clamped to the arrays so that no
    // later kernel reads or writes outside them (the sticky status stops the run)
    if (sBad)
        for (int i = tid; i <= nt; i += SCAN_THREADS) S.off_new[i] = min(S.off_new[i], lim);
    if (tid == 0) {
        prm.st->leavers_sp[s] = prm.st->leavers_acc[s];
        prm.st->leavers_acc[s] = 0;
    }
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan(const SortParams prm) {
    scan_species(prm, blockIdx.x, blockIdx.x == 0);
}

// batched: CTA (member, species)
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_batch(const SortBatch b) {
    scan_species(b.members[blockIdx.x], blockIdx.y, blockIdx.y == 0);
}

// Warp-per-tile bodies: a warp takes one tile; slots come from the warp's
// ballots (register counters), so no CTA barrier or shared atomic is needed.
// The re-sort moves about two per cent of the particles a step and is bound
// by memory latency, not bandwidth: each body issues its independent loads in
// one round (the tile's bookmarks with its neighbours' in the fill, four
// positions per lane in the eviction, sources and holes together) so that a
// tile costs few dependent round trips.
constexpr int SORT_WARPS = 4;
// entries per list (sources, targets) a warp keeps in shared memory; a tile
// needing more uses the global index arrays
constexpr int FILL_LIST = 256;
constexpr int EVICT_UNROLL = 4;  // positions per lane and round in the eviction

__device__ __forceinline__ void evict_tile(const SortParams& prm, int s, int t, int lane) {
    const SortSpecies& S = prm.sp[s];
    // the tile's old and new bookmarks and leaver count (lanes 0-4) and its
    // leavers by direction (lanes 8-15), one round of loads
    int hv = 0;
    if (lane < 5)
        hv = lane < 2 ? S.off_old[t + lane] : (lane < 4 ? S.off_new[t + lane - 2] : S.leave[t]);
    else if (lane >= 8 && lane < 16)
        hv = S.dirc[t * 8 + lane - 8];
    const int p0 = __shfl_sync(0xffffffffu, hv, 0), p1 = __shfl_sync(0xffffffffu, hv, 1);
    const int r0 = __shfl_sync(0xffffffffu, hv, 2), r1 = __shfl_sync(0xffffffffu, hv, 3);
    const int lv = __shfl_sync(0xffffffffu, hv, 4);
    const int lim = prm.g.open_x ? S.cap : S.n;
    if (r0 < 0 || r1 < r0 || r1 > lim || p1 - p0 < lv) {
        if (lane == 0) dev::set_status(prm.st, ST_SORT);
        return;
    }
    // positions of the old range outside the new one: [p0, min(r0,p1)) and [max(r1,p0), p1)
    const int a1 = min(r0, p1), b0 = max(r1, p0);
    const int na = max(a1 - p0, 0), nb = max(p1 - b0, 0);
    const int tot = na + nb;
    const unsigned lt = (1u << lane) - 1u;
    int count = 0;
    bool overflow = false;
    for (int base = 0; base < tot; base += 32 * EVICT_UNROLL) {
        int p[EVICT_UNROLL], c[EVICT_UNROLL];
#pragma unroll
        for (int u = 0; u < EVICT_UNROLL; ++u) {
            const int k = base + 32 * u + lane;
            p[u] = k < tot ? (k < na ? p0 + k : b0 + (k - na)) : -1;
            c[u] = p[u] >= 0 ? S.cell[p[u]] : HOLE;
        }
        // slots for the stayers among them, then every copy's loads before its stores
        int q[EVICT_UNROLL];
#pragma unroll
        for (int u = 0; u < EVICT_UNROLL; ++u) {
            const bool take = c[u] != HOLE;
            const unsigned m = __ballot_sync(0xffffffffu, take);
            q[u] = take ? p0 + lv + count + __popc(m & lt) : -1;
            if (q[u] >= p1) {
                overflow = true;
                q[u] = -1;
            }
            count += __popc(m);
        }
        float x[EVICT_UNROLL], y[EVICT_UNROLL], ux[EVICT_UNROLL], uy[EVICT_UNROLL],
            uz[EVICT_UNROLL];
        int id[EVICT_UNROLL];
#pragma unroll
        for (int u = 0; u < EVICT_UNROLL; ++u)
            if (q[u] >= 0) {
                x[u] = S.x[p[u]];
                y[u] = S.y[p[u]];
                ux[u] = S.ux[p[u]];
                uy[u] = S.uy[p[u]];
                uz[u] = S.uz[p[u]];
                if (prm.track_ids) id[u] = S.id[p[u]];
            }
#pragma unroll
        for (int u = 0; u < EVICT_UNROLL; ++u)
            if (q[u] >= 0) {
                S.ocell[q[u]] = c[u];
                S.ox[q[u]] = x[u];
                S.oy[q[u]] = y[u];
                S.oux[q[u]] = ux[u];
                S.ouy[q[u]] = uy[u];
                S.ouz[q[u]] = uz[u];
                if (prm.track_ids) S.oid[q[u]] = id[u];
            }
    }
    if (lane == 0) S.evict[t] = min(count, p1 - p0 - lv);

    // The tile's leavers as one list per direction of motion (the
    // neighbours' fills read the run heading to them directly): out indices
    // in lsort[p0 ...], runs starting at ldir[t][d], the total at ldir[t][8].
    const int d8 = lane - 8;
    int pre = d8 >= 0 && d8 < 8 ? hv : 0;  // inclusive prefix of the counts over lanes 8-15
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, pre, o);
        if (d8 >= o) pre += v;
    }
    const int total = __shfl_sync(0xffffffffu, pre, 15);
    if (d8 >= 0 && d8 < 8) S.ldir[t * 9 + d8] = pre - hv;
    if (lane == 0) S.ldir[t * 9 + 8] = total;
    int start[8], run[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        start[k] = __shfl_sync(0xffffffffu, pre - hv, 8 + k);
        run[k] = 0;
    }
    if (total > lv) overflow = true;
    for (int base = 0; base < lv; base += 32) {
        const int k = base + lane;
        const int dk = k < lv ? (int)S.odir[p0 + k] : 8;  // 8: removed, or past the end
#pragma unroll
        for (int dd = 0; dd < 8; ++dd) {
            const unsigned m = __ballot_sync(0xffffffffu, dk == dd);
            if (dk == dd) {
                const int pos = start[dd] + run[dd] + __popc(m & lt);
                if (pos < min(total, lv)) S.lsort[p0 + pos] = p0 + k;
                else overflow = true;
            }
            run[dd] += __popc(m);
        }
    }
    int got = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) got += run[k];
    if (got != total) overflow = true;
    if (overflow) dev::set_status(prm.st, ST_SORT);
}

__global__ void __launch_bounds__(32 * SORT_WARPS) k_evict(const SortParams prm) {
    const int t = blockIdx.x * SORT_WARPS + (threadIdx.x >> 5);
    if (t < prm.g.ntiles) evict_tile(prm, blockIdx.y, t, threadIdx.x & 31);
}

// batched: warp per tile of the flattened tile list of all members
__global__ void __launch_bounds__(32 * SORT_WARPS) k_evict_batch(const SortBatch b) {
    const int gt = blockIdx.x * SORT_WARPS + (threadIdx.x >> 5);
    if (gt >= b.total_tiles) return;
    const int m = find_member(b.tile_start, b.nmembers, gt);
    const SortParams& P = b.members[m];
    if ((int)blockIdx.y < P.nsp) evict_tile(P, blockIdx.y, gt - b.tile_start[m], threadIdx.x & 31);
}

// `wl`: this warp's shared lists, 2 * FILL_LIST ints (sources, then targets).
__device__ __forceinline__ void fill_tile(const SortParams& prm, int s, int t, int lane, int* wl) {
    const SortSpecies& S = prm.sp[s];
    const Geom& g = prm.g;
    const int tx = tile_x(g, t), ty = tile_y(g, t);
    const unsigned lt = (1u << lane) - 1u;
    // one round of loads: the tile's bookmarks, leavers and evictions (lanes
    // 0-5) and, for each of the eight directions of motion d (lanes 8-15),
    // the run of leavers heading here from the tile the motion comes from:
    // its out section, the run's start (ldir) and length (dirc).  These are
    // the sources k_count summed into the new count.
    int hv = 0;
    if (lane < 6)
        hv = lane < 2 ? S.off_old[t + lane]
                      : (lane < 4 ? S.off_new[t + lane - 2] : (lane == 4 ? S.leave[t] : S.evict[t]));
    const int d = lane - 8;
    int q0 = 0, nl = 0;
    if (d >= 0 && d < 8) {
        int ddx, ddy;
        dir_delta(d, ddx, ddy);
        if (!((g.ntx == 1 && ddx) || (g.nty == 1 && ddy))) {
            const int src = tile_index(g, dev::wrapi(tx - ddx, g.ntx), dev::wrapi(ty - ddy, g.nty));
            q0 = S.off_old[src] + S.ldir[src * 9 + d];
            nl = S.dirc[src * 8 + d];
        }
    }
    const int p0 = __shfl_sync(0xffffffffu, hv, 0), p1 = __shfl_sync(0xffffffffu, hv, 1);
    const int r0 = __shfl_sync(0xffffffffu, hv, 2), r1 = __shfl_sync(0xffffffffu, hv, 3);
    const int lvt = __shfl_sync(0xffffffffu, hv, 4), ev = __shfl_sync(0xffffffffu, hv, 5);
    const int cap = r1 - r0;
    const int lim = g.open_x ? S.cap : S.n;
    if (r0 < 0 || r1 < r0 || r1 > lim || lvt + ev > p1 - p0) {
        if (lane == 0) dev::set_status(prm.st, ST_SORT);
        return;
    }
    // particles to place: incoming = new count - stayers, plus displaced stayers
    const int need = cap - (p1 - p0 - lvt) + ev;
    if (need == 0) return;
    // the lists: in shared memory when they fit, else in the global index arrays
    int* lsrc = need <= FILL_LIST ? wl : S.isrc + r0;
    int* ltgt = need <= FILL_LIST ? wl + FILL_LIST : S.fslot + r0;
    int nsrc = 0, ntgt = 0;
    bool overflow = false;

    // source_idx: the eight runs heading here, as one concatenated list
    int pre = nl;  // inclusive prefix over lanes 8-15
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, pre, o);
        if (d >= o) pre += v;
    }
    const int total = __shfl_sync(0xffffffffu, pre, 15);
    int ex[8], qq[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        ex[k] = __shfl_sync(0xffffffffu, pre - nl, 8 + k);
        qq[k] = __shfl_sync(0xffffffffu, q0, 8 + k);
    }
    // position in lsort of entry e: in the last run starting at or before it
    // (runs of length 0 share their start with the next one)
    auto sorted_pos = [&](int e) {
        int q = qq[0], x = ex[0];  // selects, not an indexed array: stays in registers
#pragma unroll
        for (int j = 1; j < 8; ++j)
            if (ex[j] <= e) {
                q = qq[j];
                x = ex[j];
            }
        return q + (e - x);
    };
    if (total > need) overflow = true;
    // target_idx: holes of this tile inside its new range.  Sources and holes
    // are read in the same rounds, two chunks of 32 each, so that all their
    // loads are in flight together.
    const int rounds = max(total, lvt);
    for (int base = 0; base < rounds; base += 64) {
        const int e0 = base + lane, e1 = e0 + 32;
        const int src0 = e0 < total ? S.lsort[sorted_pos(e0)] : 0;
        const int src1 = e1 < total ? S.lsort[sorted_pos(e1)] : 0;
        const int h0 = e0 < lvt ? S.hole[p0 + e0] : -1;
        const int h1 = e1 < lvt ? S.hole[p0 + e1] : -1;
        if (e0 < total && e0 < need) lsrc[e0] = src0;
        if (e1 < total && e1 < need) lsrc[e1] = src1;
        const bool hk0 = h0 >= r0 && h0 < r1, hk1 = h1 >= r0 && h1 < r1;
        const unsigned g0 = __ballot_sync(0xffffffffu, hk0);
        const unsigned g1 = __ballot_sync(0xffffffffu, hk1);
        if (hk0) {
            const int slot = ntgt + __popc(g0 & lt);
            if (slot < need) ltgt[slot] = h0;
            else overflow = true;
        }
        if (hk1) {
            const int slot = ntgt + __popc(g0) + __popc(g1 & lt);
            if (slot < need) ltgt[slot] = h1;
            else overflow = true;
        }
        ntgt += __popc(g0) + __popc(g1);
    }
    nsrc = total;
    // sources: this tile's displaced stayers ...
    for (int base = 0; base < ev; base += 32) {
        const int i = base + lane;
        if (i < ev) {
            const int slot = nsrc + i;
            if (slot < need) lsrc[slot] = p0 + lvt + i;
            else overflow = true;
        }
    }
    nsrc += ev;
    // ... plus the particles the moving window injects here (negative: -1 - m)
    const Injection inj = injection(prm, S, t);
    for (int base = 0; base < inj.total; base += 32) {
        const int i = base + lane;
        if (i < inj.total) {
            const int slot = nsrc + i;
            if (slot < need) lsrc[slot] = -1 - i;
            else overflow = true;
        }
    }
    nsrc += inj.total;
    // targets: the part of the new range outside the old one
    {
        const int a1 = min(p0, r1), b0 = max(p1, r0);
        const int na = max(a1 - r0, 0), nb2 = max(r1 - b0, 0);
        const int tot = na + nb2;
        for (int base = 0; base < tot; base += 32) {
            const int k = base + lane;
            if (k < tot) {
                const int slot = ntgt + k;
                const int pos = k < na ? r0 + k : b0 + (k - na);
                if (slot < need) ltgt[slot] = pos;
                else overflow = true;
            }
        }
        ntgt += tot;
    }
    __syncwarp();
    if (nsrc != ntgt || nsrc != need || nsrc > cap || overflow) {
        if (lane == 0) dev::set_status(prm.st, ST_SORT);
        return;
    }
    // move source -> target, two particles per lane and round with all their
    // loads issued before the stores
    for (int k = lane; k < nsrc; k += 64) {
        const bool two = k + 32 < nsrc;
        const int src0 = lsrc[k], to0 = ltgt[k];
        const int src1 = two ? lsrc[k + 32] : -1;
        const int to1 = two ? ltgt[k + 32] : 0;
        if (src0 >= 0 && src1 >= 0) {
            copy_two(S, src0, to0, src1, to1, prm.track_ids);
        } else {
            if (src0 >= 0) copy_particle(S, src0, to0, prm.track_ids);
            else inject_particle(prm, S, t, inj, -1 - src0, to0);
            if (two) {
                if (src1 >= 0) copy_particle(S, src1, to1, prm.track_ids);
                else inject_particle(prm, S, t, inj, -1 - src1, to1);
            }
        }
    }
}

__global__ void __launch_bounds__(32 * SORT_WARPS) k_fill(const SortParams prm) {
    __shared__ int sList[SORT_WARPS][2 * FILL_LIST];
    const int w = threadIdx.x >> 5;
    const int t = blockIdx.x * SORT_WARPS + w;
    if (t < prm.g.ntiles) fill_tile(prm, blockIdx.y, t, threadIdx.x & 31, sList[w]);
}

__global__ void __launch_bounds__(32 * SORT_WARPS) k_fill_batch(const SortBatch b) {
    __shared__ int sList[SORT_WARPS][2 * FILL_LIST];
    const int w = threadIdx.x >> 5;
    const int gt = blockIdx.x * SORT_WARPS + w;
    if (gt >= b.total_tiles) return;
    const int m = find_member(b.tile_start, b.nmembers, gt);
    const SortParams& P = b.members[m];
    if ((int)blockIdx.y < P.nsp)
        fill_tile(P, blockIdx.y, gt - b.tile_start[m], threadIdx.x & 31, sList[w]);
}

}  // namespace

cudaError_t launch_scan(const SortParams& p, cudaStream_t s) {
    if (p.nsp > 0 && p.g.ntiles > 0) {
        k_count<<<dim3((p.g.ntiles + 255) / 256, p.nsp), 256, 0, s>>>(p);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_scan<<<p.nsp > 0 ? p.nsp : 1, SCAN_THREADS, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_evict(const SortParams& p, int, cudaStream_t s) {
    if (p.nsp == 0 || p.g.ntiles == 0) return cudaSuccess;
    k_evict<<<dim3((p.g.ntiles + SORT_WARPS - 1) / SORT_WARPS, p.nsp), 32 * SORT_WARPS, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_fill(const SortParams& p, int, cudaStream_t s) {
    if (p.nsp == 0 || p.g.ntiles == 0) return cudaSuccess;
    k_fill<<<dim3((p.g.ntiles + SORT_WARPS - 1) / SORT_WARPS, p.nsp), 32 * SORT_WARPS, 0, s>>>(p);
    return cudaGetLastError();
}

// count, scan, evict and fill over all members of a batch (four launches)
cudaError_t launch_sort_batch(const SortBatch& b, cudaStream_t s) {
    if (b.nmembers == 0) return cudaSuccess;
    const int nsp = b.max_nsp > 0 ? b.max_nsp : 1;
    cudaError_t e;
    if (b.total_tiles > 0) {
        k_count_batch<<<dim3((b.total_tiles + 255) / 256, nsp), 256, 0, s>>>(b);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_scan_batch<<<dim3(b.nmembers, nsp), SCAN_THREADS, 0, s>>>(b);
    if ((e = cudaGetLastError()) != cudaSuccess || b.total_tiles == 0) return e;
    const dim3 grid((b.total_tiles + SORT_WARPS - 1) / SORT_WARPS, nsp);
    k_evict_batch<<<grid, 32 * SORT_WARPS, 0, s>>>(b);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_fill_batch<<<grid, 32 * SORT_WARPS, 0, s>>>(b);
    return cudaGetLastError();
}

}  // namespace pic
