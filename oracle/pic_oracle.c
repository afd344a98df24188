/*
 * Plain, slow CPU oracle of one time step of the 2D electromagnetic
 * particle-in-cell (PIC) method of Guidotti 2021 ("Accelerating
 * Particle-Mesh Algorithms with FPGAs and OmpSs@OpenCL"), §3.1-3.2.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker, not the product: only
 * the test-suite, the smoke check and the CPU-baseline leg of the benchmark may
 * build, load or call it.  It shares no code, header, table or constant with
 * the CUDA library and includes nothing from it.
 *
 * The file is compiled twice:
 *   REAL=double, SFX=_f64 : the FP64 oracle (the reference result);
 *   REAL=float,  SFX=_f32 : the same plain code in the thesis's own precision
 *                           (all its implementations are FP32, §5.2), used
 *                           where floating point decides an integer (a
 *                           particle's new cell, hence its tile).
 * Both are built with -ffp-contract=off so that no multiply-add is fused.
 *
 * Conventions (normalised units of Eqs. 21-22: c = 1, omega_n = 1):
 *   node (i,j) sits at (i*dx, j*dy); a particle in cell (ix,iy) with offset
 *   (x,y) in [0,1)^2 sits at ((ix+x)dx, (iy+y)dy).  Yee locations (Fig. 3.1):
 *   Ex (i+1/2, j)   Ey (i, j+1/2)   Ez (i, j)
 *   Bx (i, j+1/2)   By (i+1/2, j)   Bz (i+1/2, j+1/2)
 *   J is co-located with E, rho sits on nodes.  A field array holds its three
 *   components one after the other, each ny rows of nx values (row = j), with
 *   every index taken modulo nx, ny (periodic box).  With open_x != 0 (the box
 *   of the moving window, the last steps of Listing 3.1) the box is open along
 *   x instead: E and B are zero outside 0 <= i < nx, current deposited outside
 *   is dropped and particles whose cell leaves 0 <= ix < nx are flagged gone.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef REAL
#define REAL double
#define SFX _f64
#define REAL_IS_DOUBLE 1
#endif

#define CAT2(a, b) a##b
#define CAT(a, b) CAT2(a, b)
#define FN(name) CAT(name, SFX)
#define R(v) ((REAL)(v))

#ifdef REAL_IS_DOUBLE
#define RSQRT(v) sqrt(v)
#define RFLOOR(v) floor(v)
#define RABS(v) fabs(v)
#else
#define RSQRT(v) sqrtf(v)
#define RFLOOR(v) floorf(v)
#define RABS(v) fabsf(v)
#endif

/* status bits, shared meaning with the Python wrapper in oracle.py */
#define ORC_EPARTICLE 1 /* displacement of one cell or more, or non-finite */

static int wrap(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

/* Linear interpolation of one staggered component from the four values at
 * columns (i0, i0+1) and rows (j0, j0+1) with weights (a0, a1) along x and
 * (b0, b1) along y (§3.1: "interpolate linearly ... from the cell where the
 * particle is located and all its adjacent cells"). */
/* value of one component at column i, row j: periodic, or zero outside the
 * box along x when open_x */
static REAL at(const REAL *F, int nx, int ny, int open_x, int i, int j) {
    if (open_x && (i < 0 || i >= nx)) return R(0);
    return F[(size_t)wrap(j, ny) * nx + wrap(i, nx)];
}

static REAL interp(const REAL *F, int nx, int ny, int open_x, int i0, int j0,
                   REAL a0, REAL a1, REAL b0, REAL b1) {
    return b0 * (a0 * at(F, nx, ny, open_x, i0, j0) +
                 a1 * at(F, nx, ny, open_x, i0 + 1, j0)) +
           b1 * (a0 * at(F, nx, ny, open_x, i0, j0 + 1) +
                 a1 * at(F, nx, ny, open_x, i0 + 1, j0 + 1));
}

/* Field at a particle (§3.1, Fig. 3.1).  A component sampled on nodes along
 * an axis takes the weights (1-x, x) on cells (ix, ix+1); a component sampled
 * half a cell up takes xh = x + 1/2, columns ix + floor(xh) - 1 and +1, with
 * weights (1-w, w), w = xh - floor(xh). */
void FN(orc_gather)(int nx, int ny, int open_x, const REAL *E, const REAL *B,
                    int ix, int iy, REAL x, REAL y, REAL *Ep, REAL *Bp) {
    size_t nc = (size_t)nx * ny;
    REAL wx1 = x, wx0 = R(1) - x;
    REAL wy1 = y, wy0 = R(1) - y;
    REAL xh = x + R(0.5), yh = y + R(0.5);
    REAL fhx = RFLOOR(xh), fhy = RFLOOR(yh);
    REAL hx1 = xh - fhx, hx0 = R(1) - hx1;
    REAL hy1 = yh - fhy, hy0 = R(1) - hy1;
    int ihx = ix + (int)fhx - 1, ihy = iy + (int)fhy - 1;

    Ep[0] = interp(E + 0 * nc, nx, ny, open_x, ihx, iy, hx0, hx1, wy0, wy1);
    Ep[1] = interp(E + 1 * nc, nx, ny, open_x, ix, ihy, wx0, wx1, hy0, hy1);
    Ep[2] = interp(E + 2 * nc, nx, ny, open_x, ix, iy, wx0, wx1, wy0, wy1);
    Bp[0] = interp(B + 0 * nc, nx, ny, open_x, ix, ihy, wx0, wx1, hy0, hy1);
    Bp[1] = interp(B + 1 * nc, nx, ny, open_x, ihx, iy, hx0, hx1, wy0, wy1);
    Bp[2] = interp(B + 2 * nc, nx, ny, open_x, ihx, ihy, hx0, hx1, hy0, hy1);
}

/* Boris push, Eqs. 6-10, with tem = (q/m) dt / 2.  gamma_t of Eq. 10 is taken
 * as gamma(u-), which equals gamma(u+) because the rotation keeps |u|.
 * u is updated in place; returns gamma(u-). */
REAL FN(orc_boris)(REAL *u, const REAL *Ep, const REAL *Bp, REAL tem) {
    REAL umx = u[0] + tem * Ep[0]; /* Eq. 6 */
    REAL umy = u[1] + tem * Ep[1];
    REAL umz = u[2] + tem * Ep[2];
    REAL gm = RSQRT(R(1) + umx * umx + umy * umy + umz * umz);
    REAL gtem = tem / gm;
    REAL tx = gtem * Bp[0], ty = gtem * Bp[1], tz = gtem * Bp[2]; /* Eq. 10 */
    REAL upx = umx + umy * tz - umz * ty;                          /* Eq. 7 */
    REAL upy = umy + umz * tx - umx * tz;
    REAL upz = umz + umx * ty - umy * tx;
    REAL f = R(2) / (R(1) + tx * tx + ty * ty + tz * tz);
    REAL sx = f * tx, sy = f * ty, sz = f * tz;
    REAL uqx = umx + upy * sz - upz * sy; /* Eq. 8 */
    REAL uqy = umy + upz * sx - upx * sz;
    REAL uqz = umz + upx * sy - upy * sx;
    u[0] = uqx + tem * Ep[0]; /* Eq. 9 */
    u[1] = uqy + tem * Ep[1];
    u[2] = uqz + tem * Ep[2];
    return gm;
}

/* Current of one straight sub-move that stays inside cell (ci,cj), from local
 * (xa,ya) to (xb,yb) during the fraction f of the step.  Jx and Jy are the
 * Villasenor-Buneman fluxes of Eqs. 13-16, written with the local origin at the
 * cell corner instead of the cell centre (their 0.5 - y - dy/2 is 1 - ym here,
 * ym the mid-point of the sub-move).  Jz (not in the thesis, which works in the
 * plane) is q v_z times the time average of the area weight of each corner
 * node along the sub-move. */
/* add v to component C at column i, row j: periodic, or dropped outside the
 * box along x when open_x */
static void add_at(REAL *C, int nx, int ny, int open_x, int i, int j, REAL v) {
    if (open_x && (i < 0 || i >= nx)) return;
    C[(size_t)wrap(j, ny) * nx + wrap(i, nx)] += v;
}

static void deposit_piece(REAL *J, int nx, int ny, int open_x, int ci, int cj,
                          REAL xa, REAL ya, REAL xb, REAL yb, REAL f,
                          REAL qjx, REAL qjy, REAL qvz) {
    size_t nc = (size_t)nx * ny;
    REAL *Jx = J, *Jy = J + nc, *Jz = J + 2 * nc;
    REAL ddx = xb - xa, ddy = yb - ya;
    REAL xm = R(0.5) * (xa + xb), ym = R(0.5) * (ya + yb);
    add_at(Jx, nx, ny, open_x, ci, cj, qjx * ddx * (R(1) - ym));
    add_at(Jx, nx, ny, open_x, ci, cj + 1, qjx * ddx * ym);
    add_at(Jy, nx, ny, open_x, ci, cj, qjy * ddy * (R(1) - xm));
    add_at(Jy, nx, ny, open_x, ci + 1, cj, qjy * ddy * xm);

    REAL s0x[2] = {R(1) - xa, xa}, s1x[2] = {R(1) - xb, xb};
    REAL s0y[2] = {R(1) - ya, ya}, s1y[2] = {R(1) - yb, yb};
    for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
            REAL w = (s0x[a] * s0y[b] + s1x[a] * s1y[b]) / R(3) +
                     (s0x[a] * s1y[b] + s1x[a] * s0y[b]) / R(6);
            add_at(Jz, nx, ny, open_x, ci + a, cj + b, qvz * f * w);
        }
}

/* Charge-conserving deposit of the straight move from (x0,y0) to (x1,y1),
 * both given in the frame of the starting cell (ix,iy), so x1 in (-1,2).  The
 * move is cut where it crosses x = 0 or 1 and y = 0 or 1 into at most three
 * sub-moves that each stay inside one cell (the 4-, 7- and 10-boundary cases
 * of Figs. 3.4-3.5). */
void FN(orc_deposit_move)(int nx, int ny, int open_x, REAL *J, int ix, int iy,
                          REAL x0, REAL y0, REAL x1, REAL y1, REAL qjx,
                          REAL qjy, REAL qvz) {
    int di = (x1 >= R(1)) - (x1 < R(0));
    int dj = (y1 >= R(1)) - (y1 < R(0));
    REAL xbd = di > 0 ? R(1) : R(0), ybd = dj > 0 ? R(1) : R(0);
    REAL tx = R(2), ty = R(2); /* fraction of the move at each crossing */
    if (di != 0) tx = (xbd - x0) / (x1 - x0);
    if (dj != 0) ty = (ybd - y0) / (y1 - y0);

    REAL brk[4];
    int nb = 0;
    brk[nb++] = R(0);
    if (tx <= R(1) && ty <= R(1)) {
        brk[nb++] = tx < ty ? tx : ty;
        brk[nb++] = tx < ty ? ty : tx;
    } else if (tx <= R(1)) {
        brk[nb++] = tx;
    } else if (ty <= R(1)) {
        brk[nb++] = ty;
    }
    brk[nb++] = R(1);

    for (int k = 0; k + 1 < nb; ++k) {
        REAL ta = brk[k], tb = brk[k + 1];
        int cx = (di != 0 && tx <= ta) ? di : 0; /* crossed x before ta */
        int cy = (dj != 0 && ty <= ta) ? dj : 0;
        /* points at the two ends; a crossing point lies exactly on its line */
        REAL xa = (ta == tx) ? xbd : x0 + ta * (x1 - x0);
        REAL ya = (ta == ty) ? ybd : y0 + ta * (y1 - y0);
        REAL xb = (tb == tx) ? xbd : (tb == R(1) ? x1 : x0 + tb * (x1 - x0));
        REAL yb = (tb == ty) ? ybd : (tb == R(1) ? y1 : y0 + tb * (y1 - y0));
        deposit_piece(J, nx, ny, open_x, ix + cx, iy + cy, xa - (REAL)cx,
                      ya - (REAL)cy, xb - (REAL)cx, yb - (REAL)cy, tb - ta,
                      qjx, qjy, qvz);
    }
}

/* The particle loop of Listing 3.1 for one species: for every particle,
 * interpolate E and B, Boris push (Eqs. 6-10), move (Eq. 11) and deposit the
 * current of the move (Eqs. 12-16).  Particles are updated in place; J must be
 * zeroed by the caller (current_zero) and is accumulated periodically (which is
 * update_gc_add).  ke_sum receives sum(gamma(u-) - 1) in double.  Returns
 * ORC_EPARTICLE if a particle tried to move one cell or more in a step (the
 * Courant condition of Eq. 1 rules that out); such a particle is left where it
 * was, with its new momentum, and deposits nothing.  With open_x, gone[p] is
 * set to 1 for a particle whose new cell lies outside 0 <= ix < nx (it has
 * left the box; the caller removes it), else 0; its cell index is then left
 * unwrapped. */
/* The particles [p0, p1) of orc_advance below, their current added into J;
 * returns the status bits and adds sum(gamma(u-) - 1) to *ke. */
static int FN(advance_range)(int nx, int ny, int open_x, double dx, double dy,
                             double dt, double q_over_m, double qtilde,
                             int64_t p0, int64_t p1, int32_t *ix, int32_t *iy,
                             REAL *x, REAL *y, REAL *ux, REAL *uy, REAL *uz,
                             const REAL *E, const REAL *B, REAL *J,
                             uint8_t *gone, double *ke_sum) {
    REAL tem = (REAL)(0.5 * q_over_m * dt);
    REAL cx = (REAL)(dt / dx), cy = (REAL)(dt / dy);
    REAL qjx = (REAL)(qtilde * dx / dt), qjy = (REAL)(qtilde * dy / dt);
    REAL qjz = (REAL)qtilde;
    int status = 0;
    double ke = 0.0;
    for (int64_t p = p0; p < p1; ++p) {
        REAL Ep[3], Bp[3], u[3] = {ux[p], uy[p], uz[p]};
        FN(orc_gather)(nx, ny, open_x, E, B, ix[p], iy[p], x[p], y[p], Ep, Bp);
        if (gone) gone[p] = 0;
        REAL gm = FN(orc_boris)(u, Ep, Bp, tem);
        ke += (double)gm - 1.0;
        ux[p] = u[0];
        uy[p] = u[1];
        uz[p] = u[2];

        /* Eq. 11 in cell units */
        REAL g = RSQRT(R(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        REAL rg = R(1) / g;
        REAL ddx = u[0] * rg * cx, ddy = u[1] * rg * cy;
        REAL vz = u[2] * rg;
        if (!(RABS(ddx) < R(1) && RABS(ddy) < R(1))) {
            status |= ORC_EPARTICLE;
            continue;
        }
        REAL x0 = x[p], y0 = y[p];
        REAL x1 = x0 + ddx, y1 = y0 + ddy;
        int di = (x1 >= R(1)) - (x1 < R(0));
        int dj = (y1 >= R(1)) - (y1 < R(0));
        REAL xn = x1 - (REAL)di, yn = y1 - (REAL)dj;
        /* x1 just below 0: x1 + 1 rounds up to 1.  The particle then stays in
         * its cell at offset 0 and its move ends on the boundary. */
        if (xn >= R(1)) {
            xn = R(0);
            di = 0;
            x1 = R(0);
        }
        if (yn >= R(1)) {
            yn = R(0);
            dj = 0;
            y1 = R(0);
        }
        FN(orc_deposit_move)(nx, ny, open_x, J, ix[p], iy[p], x0, y0, x1, y1,
                             qjx, qjy, qjz * vz);
        x[p] = xn;
        y[p] = yn;
        if (open_x) {
            ix[p] = ix[p] + di;
            if (ix[p] < 0 || ix[p] >= nx) gone[p] = 1;
        } else {
            ix[p] = wrap(ix[p] + di, nx);
        }
        iy[p] = wrap(iy[p] + dj, ny);
    }
    *ke_sum += ke;
    return status;
}

int FN(orc_advance)(int nx, int ny, int open_x, double dx, double dy, double dt,
                    double q_over_m, double qtilde, int64_t n, int32_t *ix,
                    int32_t *iy, REAL *x, REAL *y, REAL *ux, REAL *uy,
                    REAL *uz, const REAL *E, const REAL *B, REAL *J,
                    uint8_t *gone, double *ke_sum) {
    *ke_sum = 0.0;
    return FN(advance_range)(nx, ny, open_x, dx, dy, dt, q_over_m, qtilde, 0, n,
                             ix, iy, x, y, ux, uy, uz, E, B, J, gone, ke_sum);
}

/* The same particle loop spread over `nthreads` threads, the thesis's CPU
 * scheme (§4.2, OpenMP): each thread takes a contiguous block of the
 * tile-sorted particles (whole groups of tiles), deposits into a private
 * current array, and the private arrays are added into J afterwards in
 * thread order.  Every particle's update is the same arithmetic as in
 * orc_advance, so positions and momenta are identical bit for bit; J and the
 * kinetic-energy sum differ only by the order of the additions.  Built
 * without OpenMP it runs the blocks one after another.  Returns -1 if the
 * private arrays cannot be allocated. */
int FN(orc_advance_par)(int nx, int ny, int open_x, double dx, double dy,
                        double dt, double q_over_m, double qtilde, int64_t n,
                        int32_t *ix, int32_t *iy, REAL *x, REAL *y, REAL *ux,
                        REAL *uy, REAL *uz, const REAL *E, const REAL *B,
                        REAL *J, uint8_t *gone, double *ke_sum, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    size_t ncell = (size_t)3 * nx * ny;
    REAL *Jt = (REAL *)calloc((size_t)nthreads * ncell, sizeof(REAL));
    double *ket = (double *)calloc((size_t)nthreads, sizeof(double));
    int *stt = (int *)calloc((size_t)nthreads, sizeof(int));
    if (!Jt || !ket || !stt) {
        free(Jt);
        free(ket);
        free(stt);
        return -1;
    }
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static, 1)
#endif
    for (int t = 0; t < nthreads; ++t) {
        int64_t p0 = n * t / nthreads, p1 = n * (t + 1) / nthreads;
        stt[t] = FN(advance_range)(nx, ny, open_x, dx, dy, dt, q_over_m, qtilde,
                                   p0, p1, ix, iy, x, y, ux, uy, uz, E, B,
                                   Jt + (size_t)t * ncell, gone, &ket[t]);
    }
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static)
#endif
    for (int64_t c = 0; c < (int64_t)ncell; ++c)
        for (int t = 0; t < nthreads; ++t) J[c] += Jt[(size_t)t * ncell + c];
    int status = 0;
    double ke = 0.0;
    for (int t = 0; t < nthreads; ++t) {
        status |= stt[t];
        ke += ket[t];
    }
    *ke_sum = ke;
    free(Jt);
    free(ket);
    free(stt);
    return status;
}

/* Yee advance of Listing 3.1 (§3.1, Eqs. 19-20 on the staggered grid of
 * Fig. 3.1): B by dt/2, E by dt with J, B by dt/2.  Periodic, or with zero
 * fields outside the box along x when open_x.  The x-neighbours are read
 * through at() with the row index unwrapped; the values read are the same. */
static void yee_b(int nx, int ny, int open_x, REAL *E, REAL *B, REAL hdt_dx,
                  REAL hdt_dy) {
    size_t nc = (size_t)nx * ny;
    REAL *Ex = E, *Ey = E + nc, *Ez = E + 2 * nc;
    REAL *Bx = B, *By = B + nc, *Bz = B + 2 * nc;
    for (int j = 0; j < ny; ++j) {
        int jp = wrap(j + 1, ny);
        for (int i = 0; i < nx; ++i) {
            size_t c = (size_t)j * nx + i;
            size_t cyp = (size_t)jp * nx + i;
            REAL ez_xp = at(Ez, nx, ny, open_x, i + 1, j);
            REAL ey_xp = at(Ey, nx, ny, open_x, i + 1, j);
            Bx[c] -= hdt_dy * (Ez[cyp] - Ez[c]);
            By[c] += hdt_dx * (ez_xp - Ez[c]);
            Bz[c] -= hdt_dx * (ey_xp - Ey[c]) - hdt_dy * (Ex[cyp] - Ex[c]);
        }
    }
}

static void yee_e(int nx, int ny, int open_x, REAL *E, const REAL *B,
                  const REAL *J, REAL dt, REAL dt_dx, REAL dt_dy) {
    size_t nc = (size_t)nx * ny;
    REAL *Ex = E, *Ey = E + nc, *Ez = E + 2 * nc;
    const REAL *Bx = B, *By = B + nc, *Bz = B + 2 * nc;
    const REAL *Jx = J, *Jy = J + nc, *Jz = J + 2 * nc;
    for (int j = 0; j < ny; ++j) {
        int jm = wrap(j - 1, ny);
        for (int i = 0; i < nx; ++i) {
            size_t c = (size_t)j * nx + i;
            size_t cym = (size_t)jm * nx + i;
            REAL bz_xm = at(Bz, nx, ny, open_x, i - 1, j);
            REAL by_xm = at(By, nx, ny, open_x, i - 1, j);
            Ex[c] += dt_dy * (Bz[c] - Bz[cym]) - dt * Jx[c];
            Ey[c] += -dt_dx * (Bz[c] - bz_xm) - dt * Jy[c];
            Ez[c] += dt_dx * (By[c] - by_xm) - dt_dy * (Bx[c] - Bx[cym]) -
                     dt * Jz[c];
        }
    }
}

void FN(orc_yee)(int nx, int ny, int open_x, double dx, double dy, double dt,
                 REAL *E, REAL *B, const REAL *J) {
    REAL hdt_dx = (REAL)(0.5 * dt / dx), hdt_dy = (REAL)(0.5 * dt / dy);
    yee_b(nx, ny, open_x, E, B, hdt_dx, hdt_dy);
    yee_e(nx, ny, open_x, E, B, J, (REAL)dt, (REAL)(dt / dx), (REAL)(dt / dy));
    yee_b(nx, ny, open_x, E, B, hdt_dx, hdt_dy);
}

/* Charge density on the nodes by area weighting (Fig. 3.3): a particle gives
 * qtilde*(1-x)(1-y), qtilde*x(1-y), qtilde*(1-x)y and qtilde*xy to the four
 * corners of its cell.  Accumulated into rho. */
void FN(orc_rho)(int nx, int ny, double qtilde, int64_t n, const int32_t *ix,
                 const int32_t *iy, const REAL *x, const REAL *y, REAL *rho) {
    REAL q = (REAL)qtilde;
    for (int64_t p = 0; p < n; ++p) {
        int i0 = wrap(ix[p], nx), i1 = wrap(ix[p] + 1, nx);
        int j0 = wrap(iy[p], ny), j1 = wrap(iy[p] + 1, ny);
        REAL a1 = x[p], a0 = R(1) - x[p], b1 = y[p], b0 = R(1) - y[p];
        rho[(size_t)j0 * nx + i0] += q * a0 * b0;
        rho[(size_t)j0 * nx + i1] += q * a1 * b0;
        rho[(size_t)j1 * nx + i0] += q * a0 * b1;
        rho[(size_t)j1 * nx + i1] += q * a1 * b1;
    }
}

#ifdef REAL_IS_DOUBLE
/* Tile re-sort (§4.3) by its plain definition: a stable counting sort of the
 * particles by the row-major index of the T x T tile that holds their cell.
 * perm[k] = old index of the particle that goes to position k; counts[t] =
 * particles in tile t; offsets has ntiles+1 entries (exclusive scan, the
 * thesis's tile_offset bookmark array). */
void orc_tile_sort(int nx, int ny, int T, int64_t n, const int32_t *ix,
                   const int32_t *iy, int64_t *perm, int64_t *counts,
                   int64_t *offsets) {
    int ntx = nx / T, nty = ny / T;
    int64_t nt = (int64_t)ntx * nty;
    memset(counts, 0, sizeof(int64_t) * nt);
    for (int64_t p = 0; p < n; ++p)
        counts[(int64_t)(iy[p] / T) * ntx + ix[p] / T] += 1;
    offsets[0] = 0;
    for (int64_t t = 0; t < nt; ++t) offsets[t + 1] = offsets[t] + counts[t];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (nt > 0 ? nt : 1));
    memcpy(fill, offsets, sizeof(int64_t) * nt);
    for (int64_t p = 0; p < n; ++p) {
        int64_t t = (int64_t)(iy[p] / T) * ntx + ix[p] / T;
        perm[fill[t]++] = p;
    }
    free(fill);
    (void)nty;
}
#endif
