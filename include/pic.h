/*
 * pic.h -- C ABI of the GB300 (sm_103a) particle-in-cell library.
 *
 * One simulation = one periodic 2D electromagnetic PIC box (Guidotti 2021,
 * §3.1-3.2): fields E, B on a Yee grid (Fig. 3.1), particles sorted by tiles
 * of T x T cells (§4.1, Figs. 4.2-4.3), advanced by the loop of Listing 3.1:
 * zero J; gather E and B at each particle, Boris push (Eqs. 6-10), move
 * (Eq. 11), charge-conserving current deposit (Eqs. 12-16); guard-cell
 * reduction of J; Yee advance B/2, E, B/2 (Eqs. 19-20); guard-cell copy.  The
 * particles are re-sorted into tiles every step (§4.3).
 *
 * Units are the normalised units of Eqs. 21-22 (c = 1).  Conventions:
 *   node (i,j) at (i dx, j dy); a particle in cell (ix,iy) with offset (x,y)
 *   in [0,1)^2 sits at ((ix+x) dx, (iy+y) dy).
 *   Ex at (i+1/2, j), Ey at (i, j+1/2), Ez at (i, j);
 *   Bx at (i, j+1/2), By at (i+1/2, j), Bz at (i+1/2, j+1/2);
 *   J co-located with E; rho on nodes.
 *   Field arrays exchanged through this ABI are float32, component-major:
 *   three blocks of ny rows of nx values (element (c, j, i) at
 *   c*nx*ny + j*nx + i), at the Yee locations above.
 *
 * Ownership: the library owns all of its device memory from pic_init until
 * pic_destroy.  Every buffer a caller passes is owned by the caller; the
 * library copies from it (load/set) or into it (get) before the call returns
 * (get/diagnostics synchronise the simulation's stream; load/set copy on the
 * stream and synchronise it before returning).  "on_device" = 1 means the
 * caller's pointers are CUDA device pointers (any device memory of the current
 * device), 0 means host memory.
 *
 * Errors: every call returns a pic_status.  Errors raised on the device
 * (a particle moving a cell or more in one step, a non-finite momentum, a
 * bounded wait that ran out, an inconsistent re-sort) set sticky bits in a
 * per-simulation status word; pic_step does not wait for the device, so they
 * are reported by the next call that synchronises (pic_sync, pic_get_*,
 * pic_diagnostics), and by every later call until pic_clear_status.  No call
 * aborts the process or traps the GPU.  pic_last_error gives a message.
 *
 * Threading: a handle is not thread-safe; all work is ordered on the CUDA
 * stream given to pic_init.
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pic_sim pic_sim; /* opaque */

typedef enum {
    PIC_OK = 0,
    PIC_EINVAL = 1,     /* bad argument, size or configuration */
    PIC_ECFL = 2,       /* dt violates the Courant condition of Eq. 1 */
    PIC_ENOMEM = 3,     /* device or host allocation failed */
    PIC_ECUDA = 4,      /* a CUDA runtime call failed */
    PIC_EOVERFLOW = 5,  /* re-sort bookkeeping inconsistent (counts do not add up) */
    PIC_EPARTICLE = 6,  /* a particle tried to move one cell or more in a step, or
                           its momentum or position is not finite */
    PIC_ETIMEOUT = 7    /* a bounded device-side wait ran out */
} pic_status;

#define PIC_MAX_SPECIES 4

/* config flags */
#define PIC_STRICT_FP 1u  /* per-particle path without fused multiply-add, in the
                             operation order of the FP32 reference, so that cells
                             and offsets are reproducible bit for bit */
#define PIC_TRACK_IDS 2u  /* carry an int32 particle id through the re-sort */
#define PIC_TIMING 4u     /* record CUDA events around each particle-advance launch */
#define PIC_NO_GRAPH 8u   /* launch kernels one by one instead of a CUDA graph */
#define PIC_FP32_J 16u    /* deposit the current into FP32 shared-memory tiles (float
                             atomics, rounded sums) instead of the default exact 32-bit
                             fixed-point tiles; slower, and free of the fixed-point
                             quantum: the default quantum is 64 B |qtilde| / 2^30 per
                             contribution, B the particle batches of blockDim in a CTA
                             item (chunk is capped so that B <= 64) */

typedef struct {
    double q_over_m; /* charge-to-mass ratio (electrons: -1) */
    double density;  /* n_s, number density in units of n0 (> 0) */
    double ppc;      /* particles per cell; each particle carries the charge
                        density qtilde = sign(q/m) * density / ppc */
} pic_species_cfg;

typedef struct {
    int nx, ny;       /* cells; multiples of tile, 8 <= n <= 32768 */
    double dx, dy, dt;/* dt must satisfy Eq. 1: dt < (1/dx^2 + 1/dy^2)^-1/2 */
    int tile;         /* T in {8, 16, 32}; 0 = 16 */
    int threads;      /* threads per tile in the particle kernels: 64..512, multiple
                         of 32; 0 = 256 */
    int chunk;        /* particles per CTA in the particle kernels: a tile holding more
                         is split over several CTAs (16..1<<20); 0 = 8192 */
    int n_species;    /* 1..PIC_MAX_SPECIES */
    pic_species_cfg species[PIC_MAX_SPECIES];
    double background;/* fixed neutralising ion charge density (enters rho only) */
    unsigned flags;   /* PIC_STRICT_FP | PIC_TRACK_IDS | PIC_TIMING | PIC_NO_GRAPH |
                         PIC_FP32_J */
} pic_config;

typedef struct {
    int64_t step;          /* time level n of E and B */
    double time;           /* n dt */
    double w_e, w_b;       /* field energies 1/2 sum(E^2) dx dy, 1/2 sum(B^2) dx dy at n (FP64 sums) */
    double w_k;            /* kinetic energy sum (gamma(u-) - 1) m n_s/ppc dx dy of the last
                              particle push, i.e. at time level n-1 (NaN before the first step) */
    double gauss_max;      /* max over nodes of |div E - rho| at n (FP64), rho including the background
                              (NaN with the moving window) */
    double continuity_max; /* max over nodes of |(rho^n - rho^(n-1))/dt + div J^(n-1/2)| if the previous
                              pic_diagnostics call was at n-1 and no state was loaded since, else NaN
                              (always NaN with the moving window) */
    double charge_total;   /* sum over nodes of rho dx dy (FP64) */
    int64_t n_particles[PIC_MAX_SPECIES];
    int64_t leavers;       /* particles that changed tile in the last step (all species) */
    uint32_t status_bits;  /* sticky device status: 1 = particle, 2 = timeout, 4 = re-sort */
    int64_t window_moves;  /* cells the moving window has moved (0 without it) */
} pic_diag;

/* Create a simulation.  Validates the configuration (Eq. 1 for dt, tile
 * divisibility, sizes) and allocates the grid.  `cuda_stream` is a cudaStream_t
 * (NULL = the legacy default stream).  Fields start at zero, no particles.
 * Returns PIC_EINVAL / PIC_ECFL / PIC_ENOMEM / PIC_ECUDA; *out is NULL on error. */
pic_status pic_init(const pic_config* cfg, void* cuda_stream, pic_sim** out);

/* Load (replace) the particles of one species: n particles given as seven
 * arrays (cell ix, iy as int32; offsets x, y in [0,1) and momenta ux, uy, uz as
 * float32), plus an optional int32 id array (used when PIC_TRACK_IDS is set;
 * NULL = ids 0..n-1).  The library copies them and sorts them into tiles
 * (§4.1: one contiguous array with a tile_offset bookmark array).  Rejects
 * cells outside the grid, offsets outside [0,1) and non-finite values with
 * PIC_EINVAL (nothing is changed then).  n may be 0. */
pic_status pic_load_particles(pic_sim* sim, int species, int64_t n, const int32_t* ix,
                              const int32_t* iy, const float* x, const float* y,
                              const float* ux, const float* uy, const float* uz,
                              const int32_t* id, int on_device);

/* Set E and B (each 3*nx*ny float32 values in the ABI field layout) at the
 * current time level.  Either pointer may be NULL to leave that field as is. */
pic_status pic_set_fields(pic_sim* sim, const float* E, const float* B, int on_device);

/* Advance nsteps >= 0 time steps (Listing 3.1, with the current filter and
 * the moving window when they are set).  Asynchronous: enqueues the work on
 * the stream and returns. */
pic_status pic_step(pic_sim* sim, int nsteps);

/* The current filter of Listing 3.1 (applied after the guard-cell reduction
 * of J and before the field advance): `passes` passes (0 = off, at most 64)
 * of the binomial stencil (1/4, 1/2, 1/4) along x and then along y on each
 * component's periodic lattice; each pass multiplies the Fourier mode
 * (kx, ky) by cos^2(kx dx/2) cos^2(ky dy/2).  Replaces an installed denoiser
 * (and pic_set_denoiser replaces it).  Synchronises. */
pic_status pic_set_binomial_filter(pic_sim* sim, int passes);

/* ---- Moving window and lasers (the steps around the loop of Listing 3.1) ----
 * With the moving window the simulation box follows the plasma at the speed of
 * light (§3.2): after k steps it has moved M(k) = floor(k dt/dx + 1e-9) cells,
 * and a step whose M grows ends, after the field update, with the three
 * window steps of Listing 3.1: E and B shift one cell left (the new last
 * column is zero), the particles shift one cell left (those leaving the box
 * are removed), and new particles are inserted in the last column.  The box
 * is then open along x: E and B are zero outside 0 <= i < nx, current
 * deposited outside is dropped, and a particle leaving through either x edge
 * is removed (y stays periodic).  Particle counts change: pic_get_particles
 * and pic_diagnostics report the current ones.  Injection per species: a
 * cold k x k lattice per cell at offsets ((a+1/2)/k, (b+1/2)/k) with momentum
 * (ux, uy, uz), keeping the particles at physical x = (g + (a+1/2)/k) dx >=
 * x_start, g the column's global cell index (a step density profile); k = 0
 * injects nothing.  Each injected particle carries the species' charge
 * density qtilde, so the injected density is k*k*|qtilde| (the species'
 * density when k*k = ppc); injected particles carry id -1.  The filters of
 * the current-filter slot and batches are periodic and refuse a moving window. */
typedef struct {
    int k;            /* injected lattice k x k per cell (0..64), 0 = none */
    double x_start;   /* plasma at physical x >= x_start */
    float ux, uy, uz; /* momentum of the injected (cold) particles */
    int64_t capacity; /* particle slots to reserve for the species (>= any count reached;
                         the loaded count if larger); exceeding it stops the re-sort with
                         PIC_EOVERFLOW */
} pic_inject;

/* Turn the moving window on.  `inject` holds n_species entries (NULL: no
 * injection).  Must be called before any particles are loaded.  Zeroes the x
 * guard cells of E and B.  PIC_EINVAL if particles are loaded, a filter is
 * installed, the simulation is in a batch or a parameter is out of range. */
pic_status pic_set_moving_window(pic_sim* sim, const pic_inject* inject);

#define PIC_LASER_PLANE 0
#define PIC_LASER_GAUSSIAN 1

/* A laser pulse moving towards +x (§3.2, lasers of the input file).  Field
 * envelope sin^2(pi xi / (2 fwhm)) for 0 <= xi = start - x <= 2 fwhm (full
 * width at half maximum fwhm), carrier cos(omega0 (x - start)), peak field
 * a0 omega0; E at angle `polarization` from y towards z (Ey = cos f, Ez = sin
 * f) and B = x_hat x E (By = -sin f, Bz = cos f), each at its Yee location.
 * Gaussian: the paraxial beam of two dimensions with waist W0 at x = focus on
 * y = axis: amplitude sqrt(W0/W(z)) exp(-r^2/W(z)^2), W(z) = W0 sqrt(1 +
 * (z/zR)^2), zR = omega0 W0^2/2, extra phase omega0 r^2 z/(2(z^2 + zR^2)) -
 * atan(z/zR)/2, z = x - focus, r = y - axis.  x is physical (the window's
 * position included). */
typedef struct {
    int type;            /* PIC_LASER_PLANE or PIC_LASER_GAUSSIAN */
    double start;        /* x of the pulse front */
    double fwhm;         /* > 0 */
    double a0;           /* normalised vector potential */
    double omega0;       /* carrier frequency (= wavenumber, c = 1), > 0 */
    double polarization; /* radians */
    double W0, focus, axis; /* Gaussian only; W0 > 0 */
} pic_laser;

/* Add a laser pulse to the current E and B (computed in FP64 on the device,
 * added in FP32).  Synchronises. */
pic_status pic_add_laser(pic_sim* sim, const pic_laser* laser);

/* Copy a grid quantity into the caller's buffer: which = 0 E, 1 B (3*nx*ny
 * values each, at time level n), 2 J (the current deposited by the last step,
 * at n-1/2, 3*nx*ny values), 3 rho (nx*ny values at nodes, including the
 * background; computed from the particles now).  Synchronises the stream. */
pic_status pic_get_fields(pic_sim* sim, int which, float* out, int on_device);

/* Copy one species' particles out, in the library's current (tile-sorted)
 * order.  Each non-NULL array receives n_particles values; id is filled only
 * with PIC_TRACK_IDS.  tile_offset, if non-NULL, receives the ntiles+1
 * bookmark array of §4.1 (int64; tile t owns particles
 * [tile_offset[t], tile_offset[t+1]), with t = ty*(nx/T) + tx in a periodic
 * box and t = (nx/T - 1 - tx)*(ny/T) + ty with a moving window: tile columns
 * from the right edge, where the plasma enters).  Synchronises. */
pic_status pic_get_particles(pic_sim* sim, int species, int32_t* ix, int32_t* iy, float* x,
                             float* y, float* ux, float* uy, float* uz, int32_t* id,
                             int64_t* tile_offset, int on_device);

/* Number of particles of a species (host value, no synchronisation; with the
 * moving window the count as of the last synchronising call). */
int64_t pic_num_particles(const pic_sim* sim, int species);

/* Number of tiles (nx/T)*(ny/T). */
int64_t pic_num_tiles(const pic_sim* sim);

/* The failure path of the library's bounded device waits, on its own (every
 * wait of its kernels on an mbarrier gives up after about 2e9 clock cycles,
 * about a second, drains the copies it had issued and reports PIC_ETIMEOUT
 * instead of hanging).  One CTA waits on an mbarrier with the same helper:
 * with arrive != 0 the phase completes first (PIC_OK); with arrive == 0
 * nothing completes it and the wait gives up after limit_cycles
 * (1..4e9; PIC_ETIMEOUT).  No copy is in flight either way, and the context
 * stays usable.  Synchronises `cuda_stream`. */
pic_status pic_probe_bounded_wait(int arrive, int64_t limit_cycles, void* cuda_stream);

/* Diagnostics at the current time level (see pic_diag).  Synchronises; FP64
 * reductions on the device. */
pic_status pic_diagnostics(pic_sim* sim, pic_diag* out);

/* Energy history kept on the device for the last 65536 time levels: w_e[k],
 * w_b[k] at time level first+k, w_k[k] from the push at time level first+k.
 * Any output pointer may be NULL.  Levels not (or no longer) recorded give NaN.
 * Synchronises. */
pic_status pic_get_history(pic_sim* sim, int64_t first, int64_t count, double* w_e,
                           double* w_b, double* w_k);

/* Wait for the stream; return the sticky device status as a pic_status (with
 * the moving window also refreshes the particle counts). */
pic_status pic_sync(pic_sim* sim);

/* Clear the sticky device status bits. */
pic_status pic_clear_status(pic_sim* sim);

/* Timing of the particle-advance launches (PIC_TIMING): sum of their CUDA
 * event durations in ms and their count since the last reset.  Synchronises. */
pic_status pic_timing(pic_sim* sim, double* advance_ms, int64_t* advance_launches, int reset);

/* The same events split by stage of the step loop (Listing 3.1; PIC_TIMING):
 * stage_ms[0] the particle advance (gather, push, move, deposit, leaver
 * emission), stage_ms[1] the tile re-sort (§4.3: count, scan, evict, fill),
 * stage_ms[2] the rest of the step after the re-sort's fill.  The current
 * filter (if any) and the field advance (Eqs. 19-20) depend on the deposit
 * and the scan only, and run on a side stream beside the eviction and the
 * fill: stage_ms[2] is the part of them not hidden under the re-sort.  Each is
 * summed over the steps since the last reset (CUDA events on the
 * simulation's stream), and their count is in *steps.  Synchronises. */
pic_status pic_timing_stages(pic_sim* sim, double stage_ms[3], int64_t* steps, int reset);

/* Number of kernels this simulation has launched (graph nodes included). */
int64_t pic_kernel_launches(const pic_sim* sim);

/* Message for the last error on this handle ("" if none); valid until the next call. */
const char* pic_last_error(const pic_sim* sim);

/* Free everything.  NULL is accepted. */
void pic_destroy(pic_sim* sim);

/* ---- Batches: many independent simulations stepped together --------------
 * The paper steps one simulation; a batch advances many independent ones (any
 * mix of grid sizes, particle counts and tile sizes) with one kernel per stage
 * of Listing 3.1 for all of them: the particle advance of every member in one
 * persistent launch per (tile size, threads) group over a work list of
 * (member, tile, slice) items, the re-sort over all members' tiles, the field
 * advance over all members' field tiles; each step is a captured CUDA graph.
 * Each member computes exactly what pic_step computes for it alone. */
typedef struct pic_batch pic_batch;

/* Create n simulations with the configurations cfgs[0..n-1], all on
 * `cuda_stream`; out[0..n-1] receive the handles (all NULL on error).  Each is
 * an ordinary pic_sim (load particles, set fields, read diagnostics through
 * the calls above).  Errors as pic_init, for the first failing member. */
pic_status pic_init_batch(const pic_config* cfgs, int n, void* cuda_stream, pic_sim** out);

/* Group n existing simulations into a batch stepped on `cuda_stream`.  Every
 * member must have been created on that same stream (so single-simulation
 * calls on a member stay ordered with the batch's steps), none may belong to
 * another batch, and all must share the PIC_STRICT_FP and PIC_FP32_J settings.  The caller
 * keeps ownership of the members and must destroy the batch before them.
 * Returns PIC_EINVAL (message through pic_batch_last_error), PIC_ENOMEM,
 * PIC_ECUDA. */
pic_status pic_batch_create(pic_sim* const* members, int n, void* cuda_stream, pic_batch** out);

/* Advance every member nsteps time steps (asynchronous, like pic_step).
 * Members reloaded, re-tiled or stepped on their own since the last call are
 * picked up (the step graphs are rebuilt). */
pic_status pic_batch_step(pic_batch* batch, int nsteps);

/* Wait for the stream; return the first member's non-OK sticky status
 * (PIC_OK if none), its index in *member if member is non-NULL (-1 if none). */
pic_status pic_batch_sync(pic_batch* batch, int* member);

/* Number of kernels the batch has launched, and per step. */
int64_t pic_batch_kernel_launches(const pic_batch* batch, int* per_step);

const char* pic_batch_last_error(const pic_batch* batch);

/* Free the batch (not its members).  NULL is accepted. */
void pic_batch_destroy(pic_batch* batch);

/* ---- Autotuner ---------------------------------------------------------------
 * Pick the tile size T in {8, 16, 32} (those dividing nx and ny) and the
 * threads per CTA in {64, 128, 256, 512} of the particle kernels for a loaded
 * simulation by timing `steps` steps (CUDA events, after two warm-up steps) of
 * each candidate on its own particles and fields.  The simulation's state
 * (particles, fields, energy history, step count) is saved before and put
 * back afterwards, so tuning does not advance the physics; the particles'
 * order inside a tile may change.  The winner is applied to the simulation and
 * cached for the process, keyed by (nx, ny, loaded particles per cell, species,
 * PIC_STRICT_FP, device); a later call with the same key applies the cached
 * choice without timing unless `force` is non-zero.  tile, threads and
 * step_ms (the winner's mean step time; 0 for a cached choice) may be NULL.
 * Synchronises.  Needs free device memory for one copy of the particles. */
pic_status pic_autotune(pic_sim* sim, int steps, int force, int* tile, int* threads,
                        double* step_ms);

/* Change the tile size T of a loaded simulation in place (re-sorts the
 * particles into the new tiles); `threads` > 0 also sets the threads per CTA.
 * Synchronises.  PIC_EINVAL if T is not in {8, 16, 32} or does not divide
 * the grid. */
pic_status pic_set_tiling(pic_sim* sim, int tile, int threads);

/* ---- Learned current denoiser -----------------------------------------------
 * The paper smooths the deposited current with a binomial filter placed after
 * the guard-cell reduction of J and before the field advance (Listing 3.1).
 * The denoiser is a learned alternative for that slot: a small convolutional
 * encoder-decoder that maps the current of a low-ppc run to that of a
 * high-ppc run.  Architecture (3 levels, 3x3 kernels with periodic padding,
 * ReLU, 2x2 mean pooling, nearest upsampling, additive skips s1, s2):
 *   c1 3->32, c2 32->32 (s1), pool, c3 32->64, c4 64->64 (s2), pool,
 *   c5 64->128, c6 128->128, up, c7 128->64 (+s2), c8 64->64, up,
 *   c9 64->32 (+s1), c10 32->32, c11 32->3;  out = x + c11(...),
 * with x = J / scale and the denoised current scale * out.  Activations and
 * weights are bfloat16 on the tensor cores with FP32 accumulation; the
 * parameters have an FP32 master copy trained with Adam (beta1 0.9, beta2
 * 0.999, eps 1e-8) on the mean-squared error of the normalised output.
 * Parameter vector (FP32, pic_denoiser_num_params() values): per layer in
 * order c1..c11 the weights [ky][kx][cin][cout] (tap offset (ky-1, kx-1)),
 * then the bias [cout].  Currents are exchanged as `batch` consecutive
 * samples in the field layout of the header comment (3 x ny x nx FP32 each).
 * A handle is not thread-safe; its work is ordered on `cuda_stream`, and while
 * it is installed in a simulation it also runs on that simulation's stream.
 * The thin first layer c1 runs on a CUDA-core kernel (fused with the input
 * scaling) when a pass has fewer than 2^18 pixels, else on the tensor cores;
 * the output layer c11 runs on the tensor cores as one GEMM per input row with
 * its nine taps side by side (an mma.sync kernel below 128-pixel rows).  Convolutions whose rows are multiples of 128
 * pixels and with at least 17 output channels run on the tcgen05 kernel when
 * the launch is large (>= 200 work units of 2 x 128 pixels), else on an
 * mma.sync kernel; the two layers that read a 2x upsampled input (c7, c9)
 * run as four 2x2 convolutions of the coarse grid (tcgen05) whenever its rows
 * are multiples of 128 pixels, with the 3x3 taps summed per output parity
 * (each sum rounded to bfloat16 once).  The environment variable
 * PIC_DENOISER_TC, read at creation, selects the tcgen05 kernels whenever
 * the shape allows, the end layers included (=always, used by the tests), or
 * never (=never).  The network's kernels are launched with programmatic
 * dependent launch (each waits for the previous one before it reads its
 * inputs); PIC_NN_PDL=0, read once per process, launches them plainly.
 * Low-wavenumber restoration (off unless pic_denoiser_set_low_k_restore sets
 * n > 0 passes): after the network, out <- out + L^n (J_in - out), where L is
 * one pass of the periodic binomial smoothing (1/4, 1/2, 1/4) along x and
 * along y, which multiplies the Fourier mode (mx, my) of the nx x ny lattice
 * by cos^2(pi mx / nx) cos^2(pi my / ny).  It hands back the long-wavelength
 * part of the correction the network made: a network trained on the mean
 * squared error shrinks a weak coherent mode together with the noise, and the
 * growth of that mode is what the simulation has to get right.  Applied by
 * pic_denoiser_forward and in the current-filter slot, not in training. */
typedef struct pic_denoiser pic_denoiser;

#define PIC_LOW_K_MAX_PASSES 64

int64_t pic_denoiser_num_params(void);

/* nx a multiple of 64, ny of 32 (two 2x poolings onto 16x8 convolution
 * tiles), ny <= 65535; batch_max >= 1 samples per call; scale > 0 the current
 * normalisation.  Parameters start at zero (the network is the identity). */
pic_status pic_denoiser_create(int nx, int ny, int batch_max, double scale, void* cuda_stream,
                               pic_denoiser** out);

/* Replace / read the parameter vector (resets the Adam moments). */
pic_status pic_denoiser_set_params(pic_denoiser* d, const float* params, int on_device);
pic_status pic_denoiser_get_params(pic_denoiser* d, float* params, int on_device);

/* J_out = the denoised J_in (batch samples).  J_out may equal J_in.  Synchronises. */
pic_status pic_denoiser_forward(pic_denoiser* d, const float* J_in, float* J_out, int batch,
                                int on_device);

/* Passes n of the low-wavenumber restoration (0: off, the default; at most
 * PIC_LOW_K_MAX_PASSES, else PIC_EINVAL).  A simulation that has already
 * stepped with d keeps the setting it had in its captured step graphs: call
 * pic_set_denoiser again after a change (that rebuilds them).  The
 * restoration uses the gradient buffers as scratch. */
pic_status pic_denoiser_set_low_k_restore(pic_denoiser* d, int passes);

/* Loss (mean squared error of the normalised output against J_target / scale)
 * and, if grads is non-NULL, its gradient with respect to the parameter
 * vector.  Synchronises. */
pic_status pic_denoiser_grad(pic_denoiser* d, const float* J_in, const float* J_target, int batch,
                             double* loss, float* grads, int on_device);

/* pic_denoiser_grad followed by one Adam step with learning rate lr. */
pic_status pic_denoiser_train_step(pic_denoiser* d, const float* J_in, const float* J_target,
                                   int batch, float lr, double* loss, int on_device);

/* Install d (NULL: remove) in the current-filter slot of sim: every later
 * pic_step applies the network to J in place between the deposit and the
 * field advance (the continuity residual of pic_diagnostics then measures the
 * filtered current).  d must match the grid.  Simulations with a filter of
 * their own cannot be stepped in a batch (see pic_batch_set_denoiser). */
pic_status pic_set_denoiser(pic_sim* sim, pic_denoiser* d);

/* Install d (NULL: remove) in the current-filter slot of every member of a
 * batch: each pic_batch_step gathers the members' currents after the re-sort,
 * runs the network over them as one batch of samples (groups of at most the
 * batch_max d was created with), applies d's low-wavenumber restoration and
 * writes the currents back before the field advance.  Every member must have
 * the network's grid (PIC_EINVAL otherwise, message through
 * pic_batch_last_error).  A member gets what pic_set_denoiser would give it
 * alone, up to the order of a convolution's FP32 sums: which kernel runs a
 * layer depends on the pixels of the pass (CUDA cores for the thin first
 * layer below 2^18 pixels, else implicit GEMMs; mma.sync or tcgen05 by shape
 * and size), and each sums in its own order.  d must stay alive while installed; kernel
 * timeouts show in the first member's status.  Synchronises. */
pic_status pic_batch_set_denoiser(pic_batch* batch, pic_denoiser* d);

const char* pic_denoiser_last_error(const pic_denoiser* d);
void pic_denoiser_destroy(pic_denoiser* d);

/* Kernel-level probes on caller device buffers (bfloat16 NHWC tensors as
 * uint16 bit patterns, channel counts padded to a multiple of 16; FP32
 * weights [ky][kx][cin][cout]).  Synchronise `cuda_stream`.
 *   pic_nn_conv3x3: a = bf16(relu?(conv(x) + bias)), y = bf16(a + skip) if
 *     skip is non-NULL; cout in {32, 64, 128}; H % 8 == 0, W % 16 == 0.
 *   pic_nn_conv3x3_dgrad: dx (FP32 NHWC, cin channels) = input gradient of
 *     the convolution for the output gradient dz; cin in {32, 64, 128}.
 *   pic_nn_conv3x3_wgrad: dw (FP32 [3][3][cin][cout], overwritten) = weight
 *     gradient; B*H*W a multiple of 64.  Runs the tcgen05 kernel when W is a
 *     multiple of 16 and H of its tile height (256 pixels, 128 when cin or
 *     cout is 128, over the widest of 64, 32, 16 columns that divides W),
 *     else the mma.sync kernel.
 *   pic_nn_low_k_restore: the denoiser's low-wavenumber restoration on FP32
 *     currents [B][3][H][W]: out <- out + L^passes (raw - out) (B <= 4096,
 *     H <= 65535, B H W <= 2^28; passes 0..PIC_LOW_K_MAX_PASSES); raw and out must not overlap; allocates
 *     and frees its own scratch (3 B H W floats). */
pic_status pic_nn_conv3x3(const void* x, int B, int H, int W, int cin, int cout, const float* w,
                          const float* bias, int relu, const void* skip, void* a_out, void* y_out,
                          void* cuda_stream);
pic_status pic_nn_conv3x3_dgrad(const void* dz, int B, int H, int W, int cin, int cout,
                                const float* w, float* dx, void* cuda_stream);
pic_status pic_nn_conv3x3_wgrad(const void* x, const void* dz, int B, int H, int W, int cin,
                                int cout, float* dw, void* cuda_stream);
pic_status pic_nn_low_k_restore(const float* raw, float* out, int B, int H, int W, int passes,
                                void* cuda_stream);

/* ---- Allocation-free tile sort ---------------------------------------------
 * The paper has no counterpart: this entry point is for callers that cannot
 * call cudaMalloc (host callbacks, allocator hooks, plugins whose host
 * application owns every device allocation, processes that pre-carved all of
 * device memory into their own pool).  It sorts n caller-owned device particle
 * arrays (same seven arrays and validity rules as pic_load_particles) by tile
 * into caller-owned device output arrays of n values each, and writes the
 * (nx/tile)*(ny/tile)+1 tile_offset bookmarks (int64, device), the same
 * counting sort pic_load_particles performs; order inside a tile is
 * unspecified.  It allocates nothing: its scratch is a fixed device array of
 * PIC_NOALLOC_MAX_TILES + 64 int32 (256 KB + 256 B) that every GPU loading the
 * library holds until exit.  Every call looks up that array's address on the
 * current device.  Calls share the array: two calls whose work overlaps on
 * the GPU race and give wrong results.  Synchronises `cuda_stream` (a
 * cudaStream_t, NULL = default) twice, so it cannot be called during a stream
 * capture.  n = 0 is valid (all bookmarks zero).
 * Returns PIC_EINVAL for a bad size or tile, more than PIC_NOALLOC_MAX_TILES
 * tiles, or an invalid particle (outputs then unspecified); PIC_ECUDA on a
 * CUDA error. */
#define PIC_NOALLOC_MAX_TILES 65536
pic_status pic_tile_sort_noalloc(int nx, int ny, int tile, int64_t n, const int32_t* ix,
                                 const int32_t* iy, const float* x, const float* y,
                                 const float* ux, const float* uy, const float* uz,
                                 int32_t* ix_out, int32_t* iy_out, float* x_out, float* y_out,
                                 float* ux_out, float* uy_out, float* uz_out,
                                 int64_t* tile_offset, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* PIC_H */
