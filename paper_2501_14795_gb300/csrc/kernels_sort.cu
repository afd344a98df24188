// Tile re-sort (§4.3, the Jocksch scheme adapted to warp ballots and scans).
//
// After the particle advance every tile t knows: stay[t] particles still in
// place, leave[t] leavers appended to out[off_old[t] ...] with their vacated
// positions in hole[off_old[t] ...], and dirc[t][d] leavers per destination.
//   k_scan   (one CTA per species): new counts stay + incoming from the eight
//            neighbours (step 1 of §4.3), exclusive scan -> off_new; also
//            advances the step counter and primes the energy history.
//   k_evict  (CTA per tile): stayers whose position falls outside the tile's
//            new range are displaced occupants; copy them to the tail of the
//            tile's out section (they are re-inserted into their own tile).
//   k_fill   (CTA per tile): target_idx = holes of t inside its new range plus
//            the part of the new range outside the old one; source_idx =
//            leavers of the neighbours heading to t plus t's displaced
//            stayers (steps 2-4); then move source -> target (step 5).
// Only leavers and displaced particles move; a particle's bytes are read and
// written once more.  No per-particle global atomics: slots come from warp
// ballots and CTA-local counters.
#include "device_util.cuh"
#include "pic_internal.h"

namespace pic {

namespace {

__device__ __forceinline__ int tile_of(int c, int T, int ntx) {
    const int ix = c & 0xffff, iy = (int)((unsigned)c >> 16);
    return (iy / T) * ntx + ix / T;
}

// neighbour of tile (tx, ty) displaced by direction d (0..7 over the 3x3
// stencil without its centre)
__device__ __forceinline__ void dir_delta(int d, int& dx, int& dy) {
    const int k = d < 4 ? d : d + 1;
    dx = k % 3 - 1;
    dy = k / 3 - 1;
}

// warp-aggregated slot in a CTA counter; every lane of the warp must call it
__device__ __forceinline__ int warp_slot(bool take, int* counter) {
    const unsigned m = __ballot_sync(0xffffffffu, take);
    if (!m) return 0;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(counter, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    return base + __popc(m & ((1u << lane) - 1u));
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

constexpr int SCAN_THREADS = 1024;

__global__ void __launch_bounds__(SCAN_THREADS) k_scan(const SortParams prm) {
    __shared__ int sWarp[32];
    __shared__ long long sLeavers[32];
    const int s = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (s == 0 && tid == 0) {
        // advance the time level and prime the history slots of level n+1
        const long long n = prm.st->step + 1;
        prm.hist_e[n & (HIST - 1)] = 0.0;
        prm.hist_b[n & (HIST - 1)] = 0.0;
        prm.hist_k[n & (HIST - 1)] = 0.0;
        prm.st->step = n;
    }
    if (s >= prm.nsp) return;
    const SortSpecies& S = prm.sp[s];
    const Geom& g = prm.g;
    const int nt = g.ntiles;
    const int per = (nt + SCAN_THREADS - 1) / SCAN_THREADS;
    const int t0 = min(tid * per, nt), t1 = min(t0 + per, nt);

    // pass 1: new count of each of my tiles (kept in off_new[t]) and their sum
    int mysum = 0;
    long long myleave = 0;
    for (int t = t0; t < t1; ++t) {
        const int tx = t % g.ntx, ty = t / g.ntx;
        int c = S.off_old[t + 1] - S.off_old[t] - S.leave[t];  // stayers
        myleave += S.leave[t];
        S.leave_next[t] = 0;  // counters of the next step (other parity)
#pragma unroll
        for (int d = 0; d < 8; ++d) S.dirc_next[t * 8 + d] = 0;
        for (int d = 0; d < 8; ++d) {
            int ddx, ddy;
            dir_delta(d, ddx, ddy);
            if (g.ntx == 1 && ddx) continue;
            if (g.nty == 1 && ddy) continue;
            const int sx = dev::wrapi(tx - ddx, g.ntx), sy = dev::wrapi(ty - ddy, g.nty);
            c += S.dirc[(sy * g.ntx + sx) * 8 + d];
        }
        S.off_new[t] = c;
        mysum += c;
    }
    // exclusive block scan of the per-thread sums
    int incl = mysum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    long long lv = myleave;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lv += __shfl_xor_sync(0xffffffffu, lv, o);
    if (lane == 31) sWarp[wid] = incl;
    if (lane == 0) sLeavers[wid] = lv;
    __syncthreads();
    if (wid == 0) {
        const int w = sWarp[lane];
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += v;
        }
        sWarp[lane] = wi - w;  // exclusive prefix of the warp sums
    }
    __syncthreads();
    // pass 2: each thread rewrites only its own tiles' entries
    int run = sWarp[wid] + incl - mysum;
    for (int t = t0; t < t1; ++t) {
        const int c = S.off_new[t];
        S.off_new[t] = run;
        run += c;
    }
    if (tid == SCAN_THREADS - 1) {
        // the last thread's running sum is the grand total
        S.off_new[nt] = run;
        if (run != S.n) dev::set_status(prm.st, ST_SORT);
    }
    if (tid == 0) {
        long long tot = 0;
        for (int w = 0; w < SCAN_THREADS / 32; ++w) tot += sLeavers[w];
        prm.st->leavers_sp[s] = tot;
    }
}

__global__ void k_evict(const SortParams prm) {
    __shared__ int sCount;
    const int t = blockIdx.x, s = blockIdx.y;
    const SortSpecies& S = prm.sp[s];
    const int p0 = S.off_old[t], p1 = S.off_old[t + 1];
    const int r0 = S.off_new[t], r1 = S.off_new[t + 1];
    const int lv = S.leave[t];
    if (r0 < 0 || r1 < r0 || r1 > S.n || p1 - p0 < lv) {
        if (threadIdx.x == 0) dev::set_status(prm.st, ST_SORT);
        return;
    }
    if (threadIdx.x == 0) sCount = 0;
    __syncthreads();
    // positions of the old range outside the new one: [p0, min(r0,p1)) and [max(r1,p0), p1)
    const int a1 = min(r0, p1), b0 = max(r1, p0);
    const int na = max(a1 - p0, 0), nb = max(p1 - b0, 0);
    const int tot = na + nb;
    bool overflow = false;
    for (int base = 0; base < tot; base += blockDim.x) {
        const int k = base + threadIdx.x;
        int p = -1;
        bool take = false;
        if (k < tot) {
            p = k < na ? p0 + k : b0 + (k - na);
            take = S.cell[p] != HOLE;
        }
        const int slot = warp_slot(take, &sCount);
        if (take) {
            const int q = p0 + lv + slot;
            if (q < p1) {
                S.ocell[q] = S.cell[p];
                S.ox[q] = S.x[p];
                S.oy[q] = S.y[p];
                S.oux[q] = S.ux[p];
                S.ouy[q] = S.uy[p];
                S.ouz[q] = S.uz[p];
                if (prm.track_ids) S.oid[q] = S.id[p];
            } else {
                overflow = true;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) S.evict[t] = min(sCount, p1 - p0 - lv);
    if (overflow) dev::set_status(prm.st, ST_SORT);
}

__global__ void k_fill(const SortParams prm) {
    __shared__ int sSrc, sTgt;
    const int t = blockIdx.x, s = blockIdx.y;
    const SortSpecies& S = prm.sp[s];
    const Geom& g = prm.g;
    const int T = g.T;
    const int tx = t % g.ntx, ty = t / g.ntx;
    const int p0 = S.off_old[t], p1 = S.off_old[t + 1];
    const int r0 = S.off_new[t], r1 = S.off_new[t + 1];
    const int cap = r1 - r0;
    if (r0 < 0 || r1 < r0 || r1 > S.n || S.leave[t] + S.evict[t] > p1 - p0) {
        if (threadIdx.x == 0) dev::set_status(prm.st, ST_SORT);
        return;
    }
    if (threadIdx.x == 0) {
        sSrc = 0;
        sTgt = 0;
    }
    __syncthreads();
    bool overflow = false;

    // source_idx: neighbours' leavers heading here (distinct neighbour tiles only)
    int nbs[8];
    int nnb = 0;
    for (int d = 0; d < 8; ++d) {
        int ddx, ddy;
        dir_delta(d, ddx, ddy);
        const int nb = dev::wrapi(ty + ddy, g.nty) * g.ntx + dev::wrapi(tx + ddx, g.ntx);
        bool dup = nb == t;
        for (int k = 0; k < nnb; ++k) dup |= nbs[k] == nb;
        if (!dup) nbs[nnb++] = nb;
    }
    for (int k = 0; k < nnb; ++k) {
        const int nb = nbs[k];
        const int q0 = S.off_old[nb], nl = S.leave[nb];
        for (int base = 0; base < nl; base += blockDim.x) {
            const int i = base + threadIdx.x;
            const bool take = i < nl && tile_of(S.ocell[q0 + i], T, g.ntx) == t;
            const int slot = warp_slot(take, &sSrc);
            if (take) {
                if (slot < cap) S.isrc[r0 + slot] = q0 + i;
                else overflow = true;
            }
        }
    }
    // ... plus this tile's displaced stayers
    {
        const int q0 = p0 + S.leave[t], ne = S.evict[t];
        for (int base = 0; base < ne; base += blockDim.x) {
            const int i = base + threadIdx.x;
            const bool take = i < ne;
            const int slot = warp_slot(take, &sSrc);
            if (take) {
                if (slot < cap) S.isrc[r0 + slot] = q0 + i;
                else overflow = true;
            }
        }
    }
    // target_idx: holes of this tile inside its new range ...
    {
        const int nl = S.leave[t];
        for (int base = 0; base < nl; base += blockDim.x) {
            const int i = base + threadIdx.x;
            int h = -1;
            if (i < nl) h = S.hole[p0 + i];
            const bool take = i < nl && h >= r0 && h < r1;
            const int slot = warp_slot(take, &sTgt);
            if (take) {
                if (slot < cap) S.fslot[r0 + slot] = h;
                else overflow = true;
            }
        }
    }
    // ... plus the part of the new range outside the old one
    {
        const int a1 = min(p0, r1), b0 = max(p1, r0);
        const int na = max(a1 - r0, 0), nb = max(r1 - b0, 0);
        const int tot = na + nb;
        for (int base = 0; base < tot; base += blockDim.x) {
            const int k = base + threadIdx.x;
            const bool take = k < tot;
            const int slot = warp_slot(take, &sTgt);
            if (take) {
                const int pos = k < na ? r0 + k : b0 + (k - na);
                if (slot < cap) S.fslot[r0 + slot] = pos;
                else overflow = true;
            }
        }
    }
    __syncthreads();
    const int m = sSrc;
    if (m != sTgt || m > cap) {
        if (threadIdx.x == 0) dev::set_status(prm.st, ST_SORT);
        return;
    }
    if (overflow) dev::set_status(prm.st, ST_SORT);
    // move source -> target
    for (int k = threadIdx.x; k < m; k += blockDim.x)
        copy_particle(S, S.isrc[r0 + k], S.fslot[r0 + k], prm.track_ids);
}

}  // namespace

cudaError_t launch_scan(const SortParams& p, cudaStream_t s) {
    k_scan<<<p.nsp > 0 ? p.nsp : 1, SCAN_THREADS, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_evict(const SortParams& p, int threads, cudaStream_t s) {
    if (p.nsp == 0 || p.g.ntiles == 0) return cudaSuccess;
    k_evict<<<dim3(p.g.ntiles, p.nsp), threads, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_fill(const SortParams& p, int threads, cudaStream_t s) {
    if (p.nsp == 0 || p.g.ntiles == 0) return cudaSuccess;
    k_fill<<<dim3(p.g.ntiles, p.nsp), threads, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace pic
