"""Pins of the CPU oracle's primitives against what the mathematics fixes.

Each test checks one oracle function against something other than itself: a
closed form, an invariant, a brute-force restatement in a different form, or a
library routine.  Tolerances are round-off level for FP64.
"""
import math

import numpy as np
import pytest

DX, DY, DT = 0.1, 0.1, 0.05

# Yee locations (Fig. 3.1) as (x, y) shifts in cells for Ex, Ey, Ez, Bx, By, Bz
STAGGER_E = [(0.5, 0.0), (0.0, 0.5), (0.0, 0.0)]
STAGGER_B = [(0.0, 0.5), (0.5, 0.0), (0.5, 0.5)]


def _bilinear_on_shifted_lattice(F, sx, sy, X, Y):
    """Generic bilinear interpolation of samples F[j, i] located at
    (i + sx, j + sy) (cell units) at the point (X, Y), periodic."""
    ny, nx = F.shape
    u, v = X - sx, Y - sy
    i0, j0 = math.floor(u), math.floor(v)
    fu, fv = u - i0, v - j0
    val = 0.0
    for dj, wv in ((0, 1 - fv), (1, fv)):
        for di, wu in ((0, 1 - fu), (1, fu)):
            val += wu * wv * F[(j0 + dj) % ny, (i0 + di) % nx]
    return val


def test_gather_matches_shifted_lattice_bilinear(orc):
    rng = np.random.default_rng(5)
    nx, ny = 7, 5
    E = rng.standard_normal((3, ny, nx))
    B = rng.standard_normal((3, ny, nx))
    for _ in range(200):
        ix, iy = int(rng.integers(0, nx)), int(rng.integers(0, ny))
        x, y = float(rng.random()), float(rng.random())
        if _ % 10 == 0:
            x, y = 0.5, 0.0  # exactly on a half-stagger boundary
        Ep, Bp = orc.gather(E, B, ix, iy, x, y)
        for c in range(3):
            want_e = _bilinear_on_shifted_lattice(E[c], *STAGGER_E[c], ix + x, iy + y)
            want_b = _bilinear_on_shifted_lattice(B[c], *STAGGER_B[c], ix + x, iy + y)
            assert Ep[c] == pytest.approx(want_e, abs=1e-13)
            assert Bp[c] == pytest.approx(want_b, abs=1e-13)


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-13), (np.float32, 2e-6)])
def test_gather_reproduces_uniform_and_linear_fields(orc, dtype, tol):
    """Linear interpolation is exact for fields linear in space: with each
    component sampled at its own Yee location, the value at the particle must
    be the linear function at the particle (away from the periodic seam)."""
    nx, ny = 16, 16
    rng = np.random.default_rng(7)
    coef = rng.standard_normal((6, 3))
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    E = np.zeros((3, ny, nx))
    B = np.zeros((3, ny, nx))
    for c in range(3):
        sx, sy = STAGGER_E[c]
        E[c] = coef[c, 0] + coef[c, 1] * (ii + sx) + coef[c, 2] * (jj + sy)
        sx, sy = STAGGER_B[c]
        B[c] = coef[3 + c, 0] + coef[3 + c, 1] * (ii + sx) + coef[3 + c, 2] * (jj + sy)
    E, B = E.astype(dtype), B.astype(dtype)
    for _ in range(100):
        ix, iy = int(rng.integers(3, 12)), int(rng.integers(3, 12))
        x, y = float(np.float32(rng.random())), float(np.float32(rng.random()))
        Ep, Bp = orc.gather(E, B, ix, iy, x, y)
        X, Y = ix + x, iy + y
        for c in range(3):
            assert Ep[c] == pytest.approx(coef[c, 0] + coef[c, 1] * X + coef[c, 2] * Y, abs=tol * 30)
            assert Bp[c] == pytest.approx(coef[3 + c, 0] + coef[3 + c, 1] * X + coef[3 + c, 2] * Y,
                                          abs=tol * 30)
    # uniform field: every component returns its constant
    Eu = np.ones((3, ny, nx), dtype) * np.array([1.5, -2.0, 0.25], dtype)[:, None, None]
    Ep, Bp = orc.gather(Eu, Eu, 3, 4, 0.3, 0.9)
    np.testing.assert_allclose(Ep, [1.5, -2.0, 0.25], rtol=tol)


def test_boris_keeps_speed_in_pure_magnetic_field(orc):
    rng = np.random.default_rng(1)
    for _ in range(200):
        u = rng.standard_normal(3) * rng.choice([0.01, 1.0, 30.0])
        Bp = rng.standard_normal(3) * 3
        u1, gm = orc.boris(u, np.zeros(3), Bp, -0.5 * DT)
        assert np.linalg.norm(u1) == pytest.approx(np.linalg.norm(u), rel=1e-14)
        assert gm == pytest.approx(math.sqrt(1 + u @ u), rel=1e-15)


def test_boris_rotation_angle_and_sense(orc):
    """In a pure B field the Boris step rotates u_perp by exactly
    2 atan(|q/m| B dt / (2 gamma)) about B, in the sense of (q/m) u x B."""
    for qm in (-1.0, 1.0, -0.3):
        for Bz in (0.2, 1.0, 5.0):
            u = np.array([0.3, -0.1, 0.7])
            tem = 0.5 * qm * DT
            u1, gm = orc.boris(u, np.zeros(3), np.array([0.0, 0.0, Bz]), tem)
            theta = 2 * math.atan(abs(tem) * Bz / gm)
            # dw/dt = -i (q/m) Bz w / gamma for w = ux + i uy
            w0 = complex(u[0], u[1])
            w1 = w0 * complex(math.cos(theta), -math.copysign(1.0, qm * Bz) * math.sin(theta))
            assert u1[0] == pytest.approx(w1.real, abs=1e-14)
            assert u1[1] == pytest.approx(w1.imag, abs=1e-14)
            assert u1[2] == pytest.approx(u[2], abs=1e-15)


def test_boris_pure_electric_field(orc):
    """B = 0: u(n+1/2) = u(n-1/2) + (q/m) E dt (Eqs. 6 and 9)."""
    u = np.array([0.1, 0.2, -0.3])
    Ep = np.array([0.5, -1.0, 2.0])
    for qm in (-1.0, 0.5):
        u1, _ = orc.boris(u, Ep, np.zeros(3), 0.5 * qm * DT)
        np.testing.assert_allclose(u1, u + qm * Ep * DT, rtol=0, atol=1e-15)


# ------------------------------------------------------------------ deposit

def _rho_single(orc, nx, ny, ix, iy, x, y, q=1.0):
    sp = orc.SpeciesState(-1.0, q, np.array([ix], np.int32), np.array([iy], np.int32),
                          np.array([x]), np.array([y]), np.zeros(1), np.zeros(1), np.zeros(1))
    return orc.rho_nodes(nx, ny, [sp], np.float64, 0.0)


def _final_cell(ix, iy, x1, y1, nx, ny):
    di = int(x1 >= 1) - int(x1 < 0)
    dj = int(y1 >= 1) - int(y1 < 0)
    return (ix + di) % nx, (iy + dj) % ny, x1 - di, y1 - dj


MOVES = [
    # (x0, y0, x1, y1) in the frame of the start cell: same-cell, 7- and 10-boundary cases
    (0.3, 0.4, 0.6, 0.7),     # same cell (4 boundaries)
    (0.8, 0.4, 1.3, 0.5),     # crosses x = 1 (7 boundaries)
    (0.2, 0.1, 0.4, -0.35),   # crosses y = 0
    (0.9, 0.85, 1.2, 1.4),    # crosses x = 1 and y = 1 (10 boundaries)
    (0.05, 0.9, -0.45, 1.05), # crosses x = 0 and y = 1
    (0.1, 0.1, -0.3, -0.2),   # crosses both at the lower sides
    (0.5, 0.5, 1.0, 0.5),     # ends exactly on x = 1
    (0.5, 0.5, 0.5, 0.0),     # ends exactly on y = 0 (no crossing)
    (0.6, 0.6, 1.2, 1.2),     # passes exactly through the corner
    (0.0, 0.0, 0.0, 0.0),     # no motion
]


@pytest.mark.parametrize("move", MOVES)
def test_deposit_satisfies_discrete_continuity(orc, move):
    """Eq. 12 on the grid: (rho1 - rho0)/dt + div J = 0 at every node."""
    nx, ny = 6, 5
    ix, iy = 2, 3
    q = 0.7
    x0, y0, x1, y1 = move
    J = np.zeros((3, ny, nx))
    orc.deposit_move(J, ix, iy, x0, y0, x1, y1, q * DX / DT, q * DY / DT, q * 0.3)
    rho0 = _rho_single(orc, nx, ny, ix, iy, x0, y0, q)
    fx, fy, xn, yn = _final_cell(ix, iy, x1, y1, nx, ny)
    rho1 = _rho_single(orc, nx, ny, fx, fy, xn, yn, q)
    res = (rho1 - rho0) / DT + orc.div_j(J, DX, DY)
    assert np.max(np.abs(res)) < 1e-12
    # total current equals q times the velocity (Eq. 3 with J = q v)
    assert J[0].sum() * 1 == pytest.approx(q * (x1 - x0) * DX / DT, abs=1e-13)
    assert J[1].sum() == pytest.approx(q * (y1 - y0) * DY / DT, abs=1e-13)
    assert J[2].sum() == pytest.approx(q * 0.3, abs=1e-14)


def test_deposit_random_moves_continuity(orc):
    rng = np.random.default_rng(11)
    nx, ny = 4, 4
    for _ in range(500):
        ix, iy = int(rng.integers(0, nx)), int(rng.integers(0, ny))
        x0, y0 = rng.random(2)
        x1, y1 = x0 + rng.uniform(-0.99, 0.99), y0 + rng.uniform(-0.99, 0.99)
        J = np.zeros((3, ny, nx))
        orc.deposit_move(J, ix, iy, x0, y0, x1, y1, DX / DT, DY / DT, 0.0)
        rho0 = _rho_single(orc, nx, ny, ix, iy, x0, y0)
        fx, fy, xn, yn = _final_cell(ix, iy, x1, y1, nx, ny)
        rho1 = _rho_single(orc, nx, ny, fx, fy, xn, yn)
        res = (rho1 - rho0) / DT + orc.div_j(J, DX, DY)
        assert np.max(np.abs(res)) < 1e-12


@pytest.mark.parametrize("move", MOVES[:6])
def test_deposit_is_additive_under_subdivision(orc, move):
    """The current of a straight move equals the sum of the currents of its
    pieces (each piece deposited from its own start cell), Jz included with
    the time fraction carried by the velocity factor."""
    nx, ny = 6, 6
    ix, iy = 2, 2
    x0, y0, x1, y1 = move
    vz = 0.4
    J = np.zeros((3, ny, nx))
    orc.deposit_move(J, ix, iy, x0, y0, x1, y1, DX / DT, DY / DT, vz)
    K = 13
    Jsum = np.zeros_like(J)
    for k in range(K):
        ta, tb = k / K, (k + 1) / K
        xa, ya = x0 + ta * (x1 - x0), y0 + ta * (y1 - y0)
        xb, yb = x0 + tb * (x1 - x0), y0 + tb * (y1 - y0)
        ci, cj = math.floor(xa), math.floor(ya)
        orc.deposit_move(Jsum, ix + ci, iy + cj, xa - ci, ya - cj, xb - ci, yb - cj,
                         DX / DT, DY / DT, vz / K)
    np.testing.assert_allclose(Jsum, J, atol=1e-13)


def test_deposit_jz_is_time_average_of_area_weights(orc):
    """Jz at the four corners of a same-cell move equals q vz times the mean of
    the area weights along the move (numerical quadrature)."""
    nx, ny = 4, 4
    x0, y0, x1, y1 = 0.15, 0.8, 0.7, 0.3
    J = np.zeros((3, ny, nx))
    orc.deposit_move(J, 1, 1, x0, y0, x1, y1, 0.0, 0.0, 1.0)
    t = (np.arange(20000) + 0.5) / 20000
    X, Y = x0 + t * (x1 - x0), y0 + t * (y1 - y0)
    want = {(1, 1): np.mean((1 - X) * (1 - Y)), (2, 1): np.mean(X * (1 - Y)),
            (1, 2): np.mean((1 - X) * Y), (2, 2): np.mean(X * Y)}
    for (i, j), w in want.items():
        assert J[2, j, i] == pytest.approx(w, abs=1e-9)


# ---------------------------------------------------------------------- Yee

def _mode_amplitude(F, kx, ky, sx, sy, trig):
    ny, nx = F.shape
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    ph = kx * (ii + sx) * DX + ky * (jj + sy) * DY
    basis = trig(ph)
    return float(np.sum(F * basis) / np.sum(basis * basis))


@pytest.mark.parametrize("mx,my,pol", [(1, 0, "TE"), (0, 2, "TE"), (3, 1, "TM"), (1, 1, "TE"), (2, 0, "TM")])
def test_yee_vacuum_mode_obeys_leapfrog_recurrence(orc, mx, my, pol):
    """With J = 0, E at integer steps obeys E(n+1) - 2E(n) + E(n-1) = -dt^2 K^2
    E(n) exactly for a Fourier mode, with K^2 = sum (2/dx_i sin(k_i dx_i/2))^2.
    This fixes the signs and the staggering of every curl term."""
    nx, ny = 32, 16
    kx, ky = 2 * np.pi * mx / (nx * DX), 2 * np.pi * my / (ny * DY)
    K2 = (2 / DX * np.sin(kx * DX / 2)) ** 2 + (2 / DY * np.sin(ky * DY / 2)) ** 2
    E = np.zeros((3, ny, nx))
    B = np.zeros((3, ny, nx))
    J = np.zeros((3, ny, nx))
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    if pol == "TM":
        E[2] = np.sin(kx * ii * DX + ky * jj * DY)
        series = []
        for n in range(200):
            series.append(_mode_amplitude(E[2], kx, ky, 0.0, 0.0, np.sin))
            orc.yee(E, B, J, DX, DY, DT)
    else:
        # E = (-Ky, Kx) sin(phase) at the Ex and Ey locations, K_i = 2/dx_i sin(k_i dx_i/2):
        # the discrete div E of this field is exactly zero
        Kx, Ky = 2 / DX * np.sin(kx * DX / 2), 2 / DY * np.sin(ky * DY / 2)
        E[0] = -Ky * np.sin(kx * (ii + 0.5) * DX + ky * jj * DY)
        E[1] = Kx * np.sin(kx * ii * DX + ky * (jj + 0.5) * DY)
        series = []
        ref = 0 if abs(ky) > 0 else 1
        sref = STAGGER_E[ref]
        for n in range(200):
            series.append(_mode_amplitude(E[ref], kx, ky, sref[0], sref[1], np.sin))
            orc.yee(E, B, J, DX, DY, DT)
    a = np.array(series)
    res = a[2:] - (2 - DT * DT * K2) * a[1:-1] + a[:-2]
    assert np.max(np.abs(res)) < 1e-12 * np.max(np.abs(a))
    assert np.max(np.abs(a)) > 0.5 * abs(a[0])
    # div B stays zero
    # div B at cell centres (i+1/2, j+1/2): Bx sits at (i, j+1/2), By at (i+1/2, j)
    divb = (np.roll(B[0], -1, axis=1) - B[0]) / DX + (np.roll(B[1], -1, axis=0) - B[1]) / DY
    assert np.max(np.abs(divb)) < 1e-12


def test_yee_dispersion_number():
    """The vacuum dispersion sin(w dt/2)/dt = sin(k dx/2)/dx for k = 2 pi/6.4
    gives w = 0.981452 (exact light line: 0.981748)."""
    k = 2 * np.pi / 6.4
    w = 2 / DT * np.arcsin(DT / DX * np.sin(k * DX / 2))
    assert w == pytest.approx(0.981452, abs=2e-6)
    assert k == pytest.approx(0.981748, abs=2e-6)


# ------------------------------------------------------------------ rho, sort

def test_rho_weights_sum_to_charge_and_lattice_is_uniform(orc):
    from paper_2501_14795_gb300 import workloads as wl
    nx, ny, k = 8, 6, 4
    ix, iy, x, y, _, _ = wl.lattice(nx, ny, k)
    sp = orc.SpeciesState(-1.0, -1.0 / (k * k), ix, iy, x.astype(np.float64), y.astype(np.float64),
                          np.zeros(ix.size), np.zeros(ix.size), np.zeros(ix.size))
    rho = orc.rho_nodes(nx, ny, [sp], np.float64, background=1.0)
    assert np.max(np.abs(rho)) < 1e-14
    rng = np.random.default_rng(3)
    for _ in range(20):
        r = _rho_single(orc, nx, ny, int(rng.integers(0, nx)), int(rng.integers(0, ny)),
                        rng.random(), rng.random(), 0.37)
        assert r.sum() == pytest.approx(0.37, abs=1e-15)
        assert np.count_nonzero(r) <= 4


def test_tile_sort_equals_stable_argsort(orc):
    rng = np.random.default_rng(2)
    nx, ny, T = 64, 32, 8
    n = 5000
    ix = rng.integers(0, nx, n).astype(np.int32)
    iy = rng.integers(0, ny, n).astype(np.int32)
    perm, counts, offsets = orc.tile_sort(nx, ny, T, ix, iy)
    tid = (iy // T) * (nx // T) + ix // T
    np.testing.assert_array_equal(perm, np.argsort(tid, kind="stable"))
    np.testing.assert_array_equal(counts, np.bincount(tid, minlength=(nx // T) * (ny // T)))
    np.testing.assert_array_equal(offsets[1:], np.cumsum(counts))
    assert offsets[0] == 0
    # empty input
    perm, counts, offsets = orc.tile_sort(nx, ny, T, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert perm.size == 0 and counts.sum() == 0 and np.all(offsets == 0)


def test_cfl_limit_number():
    """Eq. 1: dt < (1/dx^2 + 1/dy^2)^(-1/2) = 0.0707 for dx = dy = 0.1."""
    lim = (1 / DX ** 2 + 1 / DY ** 2) ** -0.5
    assert lim == pytest.approx(0.0707107, abs=1e-6)
    assert DT < lim


def test_oracle_never_writes_into_its_inputs(orc):
    """Both precisions copy the particle and field arrays they are given: a
    run must leave the caller's arrays (shared with the GPU side) untouched."""
    from paper_2501_14795_gb300 import workloads as wl
    sp = wl.random_particles(16, 16, 500, u_max=0.6, seed=3)
    E, B = wl.random_fields(16, 16, amp=0.2, seed=4)
    E0, B0, a0 = E.copy(), B.copy(), [a.copy() for a in sp.arrays()]
    for dt in (np.float32, np.float64):
        o = orc.OracleSim(16, 16, DX, DY, DT, 8,
                          [orc.SpeciesState(sp.q_over_m, sp.qtilde, *sp.arrays())],
                          dtype=dt, E=E, B=B)
        o.step(2)
    np.testing.assert_array_equal(E, E0)
    np.testing.assert_array_equal(B, B0)
    for a, b in zip(a0, sp.arrays()):
        np.testing.assert_array_equal(a, b)


from oracle import binomial_filter  # noqa: E402


def test_binomial_filter_closed_form_response():
    """One pass multiplies the mode (mx, my) by cos^2(pi mx/nx) cos^2(pi my/ny);
    the sum is kept (k = 0) and the Nyquist mode in x is removed."""
    nx, ny = 16, 12
    y, x = np.mgrid[0:ny, 0:nx]
    for mx, my, passes in ((1, 0, 1), (3, 2, 1), (2, 5, 3), (0, 0, 2)):
        f = np.cos(2 * np.pi * (mx * x / nx + my * y / ny) + 0.3)
        J = np.stack([f, 2 * f, -f])
        got = binomial_filter(J, passes)
        gain = (np.cos(np.pi * mx / nx) ** 2 * np.cos(np.pi * my / ny) ** 2) ** passes
        np.testing.assert_allclose(got, gain * J, atol=1e-12)
    rng = np.random.Generator(np.random.PCG64(5))
    J = rng.standard_normal((3, ny, nx))
    assert abs(binomial_filter(J, 2).sum() - J.sum()) < 1e-12
    nyq = np.cos(np.pi * x)[None].repeat(3, 0)
    assert np.max(np.abs(binomial_filter(nyq, 1))) < 1e-12


def test_binomial_filter_is_the_3x3_stencil():
    rng = np.random.Generator(np.random.PCG64(6))
    J = rng.standard_normal((3, 7, 9))
    w = np.array([1.0, 2.0, 1.0]) / 4
    want = np.zeros_like(J)
    for c in range(3):
        for j in range(7):
            for i in range(9):
                want[c, j, i] = sum(w[a] * w[b] * J[c, (j + b - 1) % 7, (i + a - 1) % 9]
                                    for a in range(3) for b in range(3))
    np.testing.assert_allclose(binomial_filter(J, 1), want, atol=1e-13)


def test_rho_of_an_fp32_state_equals_its_fp64_evaluation():
    """The charge density of FP32 particles (Fig. 3.3 area weights) does not
    depend on the precision the state is stored in: the FP32 offsets are exact
    doubles."""
    import numpy as np
    import oracle as orc
    rng = np.random.default_rng(5)
    n, nx, ny = 2000, 16, 8
    sp = orc.SpeciesState(-1.0, -0.25, rng.integers(0, nx, n).astype(np.int32),
                          rng.integers(0, ny, n).astype(np.int32),
                          rng.random(n).astype(np.float32), rng.random(n).astype(np.float32),
                          np.zeros(n, np.float32), np.zeros(n, np.float32), np.zeros(n, np.float32))
    r32 = orc.rho_nodes(nx, ny, [sp], np.float64, 0.0)
    r64 = orc.rho_nodes(nx, ny, [sp.astype(np.float64)], np.float64, 0.0)
    np.testing.assert_array_equal(r32, r64)
    assert abs(r64.sum() + 0.25 * n) < 1e-9
