// Internal declarations shared by the host runtime (pic_host.cu) and the
// kernel translation units.  Not part of the public ABI (include/pic.h).
//
// Device data layout (one simulation):
//   * Grid arrays (E|B: 6 components, J: 3 components) are float32, each
//     component R = ny + 3 rows of P = nx + 8 floats.  Cell (i, j) lives at
//     row j + GY, column i + GX (GX = 4, GY = 1), so every component has guard
//     cells i in [-4, nx+4), j in [-1, ny+2).  Guards i = -1, nx, nx+1 and
//     j = -1, ny, ny+1 hold periodic images (update_gc_copy of Listing 3.1);
//     the others are never written and stay zero.  With the moving window the
//     box is open along x and the guards i = -1, nx, nx+1 hold zeros instead.  The column shift of 4 makes
//     the TMA box of a tile start on a 16-byte boundary (x multiple of 4).
//   * E|B are double-buffered (read one, write the other each step) and so is
//     J, because the fused Yee kernel reads neighbours across CTAs.
//   * Particles of a species are structure-of-arrays in one contiguous range
//     sorted by tile (§4.1): cell (int32, ix | iy << 16), x, y, ux, uy, uz
//     (float32), optional id; tile t owns [off[t], off[t+1]) (int32 offsets,
//     double-buffered across the re-sort).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pic {

constexpr int GX = 4;            // guard columns left of cell 0
constexpr int GY = 1;            // guard rows below cell 0
constexpr int HIST = 1 << 16;    // energy-history ring length (time levels)
constexpr int32_t HOLE = -1;     // cell value of a slot vacated by a leaver
constexpr int MAX_SPECIES = 4;

// device status bits (sticky)
constexpr unsigned ST_PARTICLE = 1u;  // moved >= 1 cell, non-finite, or out of its tile
constexpr unsigned ST_TIMEOUT = 2u;   // bounded wait ran out
constexpr unsigned ST_SORT = 4u;      // re-sort counts inconsistent

struct DevState {
    unsigned status;
    unsigned pad;
    long long step;      // time level n of the current fields
    long long leavers_sp[MAX_SPECIES];  // particles that changed tile in the last step
    long long leavers_acc[MAX_SPECIES]; // running sum of the current step (k_count -> k_scan)
    int load_bad;        // pic_load_particles validation failures
    int win_shift;       // moving window: 1 if the step being taken shifts it (set by the push)
    long long win_moves; // moving window: cells moved so far (after the step's shift)
    long long np[MAX_SPECIES];       // particles per species (moving window: changes)
    long long removed[MAX_SPECIES];  // particles that left the open box this step
};

struct SpeciesDev {
    // particle arrays (capacity >= n)
    int32_t* cell;
    float *x, *y, *ux, *uy, *uz;
    int32_t* id;
    // leaver / eviction staging ("out") arrays, same capacity
    int32_t* ocell;
    float *ox, *oy, *oux, *ouy, *ouz;
    int32_t* oid;
    int32_t* hole;    // positions vacated by leavers, per source tile
    uint8_t* odir;    // each leaver's direction (0-7; 8: left the open box), out-array order
    int32_t* lsort;   // each tile's leavers' out indices sorted by direction
    int32_t* fslot;   // fill lists: target positions ...
    int32_t* isrc;    // ... and source indices into the out arrays
    int32_t* off[2];  // ntiles + 1 bookmarks (tile_offset), ping-pong
    int32_t* leave[2];  // per tile: particles that left (ping-pong; the scan clears the idle one)
    int32_t* dirc[2];   // per tile x 8 directions: leavers by destination (ping-pong)
    int32_t* evict;   // per tile: stayers displaced by the new bookmarks
    int32_t* ldir;    // per tile x 9: start of each direction's run in lsort (8: total)
    int32_t* cursor;  // per cell scratch for the initial load (nx*ny)
    int64_t n;        // particles
    int64_t cap;      // capacity of the particle arrays
    // per-species constants (computed in double on the host, rounded once)
    float tem;        // (q/m) dt / 2
    float qjx, qjy;   // qtilde dx/dt, qtilde dy/dt
    float qjz;        // qtilde
    double ke_w;      // kinetic-energy weight qtilde/(q/m) dx dy
    double qtilde;
    // moving-window injection (inj_k = 0: none) and requested capacity
    int inj_k;
    float inj_u[3];
    double inj_x0;
    int64_t want_cap;
};

struct Geom {
    int nx, ny, T, ntx, nty, ntiles;
    int P, R;          // pitch (floats) and rows of a grid component
    long long cstride; // R * P
    float cx, cy;      // dt/dx, dt/dy
    float hdt_dx, hdt_dy, dt_dx, dt_dy, dt;
    double dx, dy, dtd;
    int open_x;        // moving window: box open along x (else periodic)
    int pad_g;
};

// Order of the tiles in the tile-sorted arrays (the bookmarks are indexed by
// it).  A periodic box takes them row by row, t = ty * ntx + tx.  The moving
// window's open box takes them column by column from its right edge,
// t = (ntx - 1 - tx) * nty + ty: the plasma (a step profile, filled beyond
// its edge) enters at the right edge, and its edge walks left through the
// tiles, one cell per shift.  The tiles around the edge change their counts
// on every shift, which moves the ranges of all tiles after them in the
// arrays; in this order those are the tiles to the left of the edge, still
// empty, instead of the whole plasma.  The tile column that receives the
// injected plasma comes first and hands its left cell column to the next
// tile column on each shift, which keeps the counts of the filled tiles
// balanced.
__host__ __device__ inline int tile_index(const Geom& g, int tx, int ty) {
    return g.open_x ? (g.ntx - 1 - tx) * g.nty + ty : ty * g.ntx + tx;
}
__host__ __device__ inline int tile_x(const Geom& g, int t) {
    return g.open_x ? g.ntx - 1 - t / g.nty : t % g.ntx;
}
__host__ __device__ inline int tile_y(const Geom& g, int t) {
    return g.open_x ? t % g.nty : t / g.ntx;
}

// Moving window (the last steps of Listing 3.1; the window moves at c = 1).
// Cells moved after k steps, M(k) = floor(k dt / dx + 1e-9), in IEEE double
// with the operation order of the host and the tests.
__host__ __device__ inline long long window_moves(long long k, double dt, double dx) {
#ifdef __CUDA_ARCH__
    return (long long)floor(__dadd_rn(__ddiv_rn(__dmul_rn((double)k, dt), dx), 1e-9));
#else
    return (long long)floor((double)k * dt / dx + 1e-9);
#endif
}
// 1 if the step from time level n to n+1 ends with a shift of the window
__host__ __device__ inline int window_shift(long long n, const Geom& g) {
    return (int)(window_moves(n + 1, g.dtd, g.dx) - window_moves(n, g.dtd, g.dx));
}
// Injection into the new last column (global cell index gcol) of a moving
// window: lattice sub-indices a >= first of a k x k lattice keep the
// particles at physical x = (gcol + (a + 1/2)/k) dx >= x0 (a step profile).
// Returns the first kept a (k if none).
__host__ __device__ inline int inject_first(long long gcol, int k, double x0, double dx) {
    int a = 0;
#ifdef __CUDA_ARCH__
    while (a < k && __dmul_rn(__dadd_rn((double)gcol, __ddiv_rn(__dadd_rn((double)a, 0.5), (double)k)),
                              dx) < x0)
        ++a;
#else
    while (a < k && ((double)gcol + ((double)a + 0.5) / (double)k) * dx < x0) ++a;
#endif
    return a;
}

// ---- parameters passed by value to the kernels ------------------------------
struct PushSpecies {
    const int32_t* off;
    int32_t *cell, *id, *ocell, *oid, *hole, *leave, *dirc;
    uint8_t* odir;
    float *x, *y, *ux, *uy, *uz, *ox, *oy, *oux, *ouy, *ouz;
    float tem, qjx, qjy, qjz;
    double ke_w;
};

struct alignas(16) PushParams {
    Geom g;
    float* J;              // this step's current buffer (base of component 0)
    int chunks;            // CTAs per tile (gridDim.y): each takes a slice of the tile's particles
    int nsp;
    int track_ids;
    int fp32_j;            // FP32 J tiles instead of the fixed-point ones (PIC_FP32_J)
    PushSpecies sp[MAX_SPECIES];
    double* hist_k;        // kinetic-energy history ring
    DevState* st;
};

struct SortSpecies {
    const int32_t* off_old;
    int32_t* off_new;
    int32_t *cell, *id, *ocell, *oid, *hole, *fslot, *isrc, *leave, *dirc, *evict;
    int32_t *leave_next, *dirc_next;  // cleared here for the next step
    const uint8_t* odir;
    int32_t *lsort, *ldir;
    float *x, *y, *ux, *uy, *uz, *ox, *oy, *oux, *ouy, *ouz;
    int n;       // particles (fixed count; with the moving window see DevState::np)
    int cap;     // capacity of the particle arrays
    // moving-window injection (inj_k = 0: none): k x k cold lattice per cell at
    // physical x >= inj_x0 with momentum inj_u
    int inj_k;
    float inj_u[3];
    double inj_x0;
};

struct SortParams {
    Geom g;
    int nsp;
    int track_ids;
    SortSpecies sp[MAX_SPECIES];
    double *hist_e, *hist_b, *hist_k;
    DevState* st;
};

struct YeeParams {
    Geom g;
    const float* Fin;   // E|B at n (6 components)
    float* Fout;        // E|B at n+1
    const float* J;     // current of this step
    float* Jnext;       // next step's current buffer: its shared ring is zeroed here
    int zero_all;       // zero all of Jnext (tiles split over several CTAs flush with atomics)
    double *hist_e, *hist_b;
    DevState* st;
};

// ---- batched launches: many simulations, one grid per kernel -----------------
// Parameter blocks of every member live in device memory; work items are
// flattened over the members.
struct PushBatch {
    const PushParams* members;  // one per member (current parity)
    const CUtensorMap* tmaps;   // each member's E|B map (current parity), 64-byte aligned
    const int4* items;          // (member, tile, chunk, 0), costliest first
    int nitems;
    int* next;                  // work-item counter, zero at launch
    int fp32_j;                 // the members' PIC_FP32_J setting (shared by all)
};

struct SortBatch {
    const SortParams* members;
    const int* tile_start;      // nmembers + 1 prefix of the members' tile counts
    int nmembers;
    int total_tiles;
    int max_nsp;
};

struct YeeBatch {
    const YeeParams* members;
    const int* ytile_start;     // nmembers + 1 prefix of the members' Yee-tile counts
    int nmembers;
    int total_ytiles;
};

// ---- launchers (defined in the kernel translation units) ---------------------
// particle advance, fast (FMA) and strict (no contraction) builds
cudaError_t launch_push_fast(const CUtensorMap* fmap, const PushParams& p, int threads,
                             cudaStream_t s);
cudaError_t launch_push_strict(const CUtensorMap* fmap, const PushParams& p, int threads,
                               cudaStream_t s);

// batched particle advance; grid = number of persistent CTAs (0: all that fit at once)
cudaError_t launch_push_batch_fast(const PushBatch& b, int T, int threads, int grid,
                                   cudaStream_t s);
cudaError_t launch_push_batch_strict(const PushBatch& b, int T, int threads, int grid,
                                     cudaStream_t s);
// batched re-sort and field advance
cudaError_t launch_sort_batch(const SortBatch& b, cudaStream_t s);
cudaError_t launch_yee_batch(const YeeBatch& b, cudaStream_t s);
int yee_tiles(const Geom& g);

// one pass of the binomial current filter on J (tmp: 3 nx ny floats); 2 kernels
cudaError_t launch_binomial(const Geom& g, float* J, float* tmp, cudaStream_t s);
cudaError_t launch_scan(const SortParams& p, cudaStream_t s);
cudaError_t launch_evict(const SortParams& p, int threads, cudaStream_t s);
cudaError_t launch_fill(const SortParams& p, int threads, cudaStream_t s);
// field advance; with both tensor maps (E|B of the input parity: 3D box 40 x
// 19 x 3; J: box 36 x 17 x 3) the persistent TMA kernel, else one CTA per tile
cudaError_t launch_yee(const YeeParams& p, const CUtensorMap* mapF, const CUtensorMap* mapJ,
                       cudaStream_t s);
cudaError_t init_grid_kernels();  // kernel attributes, once before any capture

// grid utilities
cudaError_t launch_set_grid(const Geom& g, float* F, int ncomp, const float* src, cudaStream_t s);
cudaError_t launch_get_grid(const Geom& g, const float* F, int ncomp, float* dst, cudaStream_t s);
cudaError_t launch_field_energy(const Geom& g, const float* F, double* out_e, double* out_b,
                                cudaStream_t s);
cudaError_t launch_rho(const Geom& g, const SpeciesDev* sp, int nsp, const int32_t* const* off,
                       double* rho, cudaStream_t s);
cudaError_t launch_grid_residuals(const Geom& g, const float* F, const float* J,
                                  const double* rho, const double* rho_prev, double background,
                                  double* out /* [gauss_max, cont_max, charge_sum] */,
                                  cudaStream_t s);
// Initial sort of a staged species into tiles, in a pseudo-random order inside
// each tile.  The input is staged in the out arrays: ix in ocell, iy in hole,
// x..uz in ox..ouz; ids (optional) in `staged_ids`.  phase 0 validates and
// counts per key (sp.cursor holds nx*ny counters), phase 1 scans the counts into
// `celloff` (scratch of nx*ny + 2 + 2 ceil(nx*ny / 4096) ints: the cell offsets,
// then the scan's segment sums and their offsets), writes the tile bookmarks
// `off` and scatters into the particle arrays.
cudaError_t launch_load(const Geom& g, SpeciesDev& sp, int track_ids, int64_t n, int32_t* off,
                        DevState* st, cudaStream_t s, int phase, const int32_t* staged_ids,
                        int32_t* celloff);
cudaError_t launch_unpack_cells(const int32_t* cell, int64_t n, int32_t* ix, int32_t* iy,
                                cudaStream_t s);
cudaError_t launch_offsets_to_i64(const int32_t* off, int64_t n, int64_t* out, cudaStream_t s);
cudaError_t launch_hist_prime(double* hist_e, double* hist_b, double* hist_k, DevState* st,
                              cudaStream_t s);
// one CTA waiting on an mbarrier that completes (arrive) or never does;
// *result = 0 or ST_TIMEOUT (device word)
cudaError_t launch_probe_wait(int arrive, long long limit, unsigned* result, cudaStream_t s);

// Laser pulse of the initial conditions (§3.2), added to E|B (6 components)
// with its guard images; x of node column 0 is (moves + 0) dx with moves read
// from st->win_moves.
struct LaserDev {
    int type;           // 0 plane, 1 Gaussian
    double start, fwhm, a0, omega0, polarization, W0, focus, axis;
};
cudaError_t launch_add_laser(const Geom& g, float* F, const LaserDev& l, const DevState* st,
                             cudaStream_t s);
// zero the x guard columns (-1, nx, nx+1) of ncomp components (open box)
cudaError_t launch_zero_x_guards(const Geom& g, float* F, int ncomp, cudaStream_t s);

}  // namespace pic
