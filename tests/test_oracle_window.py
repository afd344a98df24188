"""Pins of the oracle's moving window, injection and lasers (CPU only).

Each pin checks the oracle against something other than itself: exact
rational arithmetic for the window position, the invariance of a cold plasma
at rest under the window's relabelling, the Yee scheme's own group velocity
and energy conservation for a plane pulse, and the diffraction of a Gaussian
beam down to its waist (a property of the propagation, not of the formula
that launches it)."""
from fractions import Fraction

import numpy as np
import pytest

import oracle as orc
from oracle import window as W


def test_window_moves_matches_exact_rational():
    for dt, dx in ((0.05, 0.1), (0.045, 0.1), (0.03, 0.05), (0.07, 0.1)):
        r = Fraction(str(dt)) / Fraction(str(dx))
        for k in range(0, 2000):
            assert W.window_moves(k, dt, dx) == (k * r.numerator) // r.denominator, (dt, dx, k)


def _lattice_plasma(nx, ny, k, x_start, dx, dtype):
    sub = (np.arange(k) + 0.5) / k
    ix, iy, x, y = [], [], [], []
    for j in range(ny):
        for i in range(nx):
            for b in range(k):
                for a in range(k):
                    if (i + (a + 0.5) / k) * dx >= x_start:
                        ix.append(i), iy.append(j), x.append(sub[a]), y.append(sub[b])
    n = len(ix)
    f = lambda v: np.asarray(v, np.float32).astype(dtype)
    z = np.zeros(n, dtype)
    return orc.SpeciesState(-1.0, -1.0 / (k * k), np.asarray(ix, np.int32), np.asarray(iy, np.int32),
                            f(x), f(y), z, z.copy(), z.copy())


def _physical_set(sp, moves, dx, dy):
    X = (sp.ix.astype(np.float64) + moves + sp.x.astype(np.float64)) * dx
    Y = (sp.iy.astype(np.float64) + sp.y.astype(np.float64)) * dy
    return sorted(zip(np.round(X, 9), np.round(Y, 9)))


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_cold_plasma_at_rest_is_invariant_under_the_window(dtype):
    """A cold plasma at rest carries no current, so the fields stay zero; the
    window only relabels it: at every step the box holds exactly the lattice
    particles whose physical position lies inside the window and at or beyond
    the plasma edge (removal at the left edge and injection at the right edge
    must balance that exactly, including the part-filled column at the edge)."""
    nx, ny, k, dx, dy, dt = 32, 8, 3, 0.1, 0.1, 0.05
    x_start = (nx // 2 + 0.4) * dx       # plasma edge inside a cell: a part-filled column
    sp = _lattice_plasma(nx, ny, k, x_start, dx, dtype)
    sim = orc.OracleSim(nx, ny, dx, dy, dt, 8, [sp], dtype=dtype,
                        window=[W.Inject(k=k, x_start=x_start)])
    for n in range(1, 41):
        sim.step(1)
        assert sim.moves == W.window_moves(n, dt, dx)
        assert not np.any(sim.E) and not np.any(sim.B) and not np.any(sim.J)
        want = _lattice_plasma(nx + sim.moves, ny, k, x_start, dx, dtype)
        inside = want.ix >= sim.moves
        want.keep(inside)
        want.ix = want.ix - sim.moves
        got = sim.species[0]
        assert got.n == want.n
        assert _physical_set(got, sim.moves, dx, dy) == _physical_set(want, sim.moves, dx, dy)
        assert not np.any(got.ux) and not np.any(got.uy) and not np.any(got.uz)
    assert sim.moves == 20 and sim.status == 0


def test_open_box_drops_the_current_outside_and_removes_the_particle():
    """A particle leaving through x = 0 of the open box deposits only its part
    of the move inside the box and is removed."""
    nx, ny, dx, dy, dt = 16, 8, 0.1, 0.1, 0.05
    x0, y0, ux = 0.2, 0.5, -0.9
    sp = orc.SpeciesState(-1.0, -1.0, np.array([0], np.int32), np.array([3], np.int32),
                          np.array([x0]), np.array([y0]), np.array([ux]), np.zeros(1), np.zeros(1))
    E = np.zeros((3, ny, nx))
    J = np.zeros_like(E)
    st, _ = orc.advance(sp, E, E.copy(), J, dx, dy, dt, open_x=True)
    assert st == 0 and sp.n == 0
    g = np.sqrt(1 + ux * ux)
    x1 = x0 + ux / g * dt / dx
    assert x1 < 0
    want = np.zeros_like(J)     # the inside piece alone, from x0 to the box edge
    orc.deposit_move(want, 0, 3, x0, y0, 0.0, y0, -1.0 * dx / dt, -1.0 * dy / dt, 0.0)
    np.testing.assert_allclose(J, want, rtol=0, atol=1e-15)
    assert J[0, 3, 0] != 0 and not np.any(J[0, :, nx - 1])


def _centroid(E, B, dx, x_origin=0.0):
    u = (E ** 2).sum(axis=(0, 1)) + (B ** 2).sum(axis=(0, 1))
    x = x_origin + np.arange(E.shape[2]) * dx
    return (u * x).sum() / u.sum(), u.sum()


def test_plane_pulse_moves_at_the_yee_group_velocity_and_keeps_its_energy():
    nx, ny, dx, dy, dt = 512, 8, 0.05, 0.05, 0.025
    l = W.Laser("plane", start=12.0, fwhm=2.0, a0=0.01, omega0=10.0)
    E, B = W.laser_fields(nx, ny, dx, dy, l)
    J = np.zeros_like(E)
    c0, u0 = _centroid(E, B, dx)
    n = 200
    for _ in range(n):
        orc.yee(E, B, J, dx, dy, dt)
    c1, u1 = _centroid(E, B, dx)
    vg = W.yee_group_velocity(10.0, dx, dt)
    assert (c1 - c0) / (n * dt) == pytest.approx(vg, rel=1e-3)
    assert vg < 0.99                           # the pin can tell v_g from c
    assert u1 / u0 == pytest.approx(1.0, abs=1e-3)


def test_plane_pulse_in_the_moving_window_slides_back_at_c_minus_v_g():
    nx, ny, dx, dy, dt = 512, 8, 0.05, 0.05, 0.025
    l = W.Laser("plane", start=20.0, fwhm=2.0, a0=0.01, omega0=10.0)
    E, B = W.laser_fields(nx, ny, dx, dy, l)
    sim = orc.OracleSim(nx, ny, dx, dy, dt, 8, [], E=E, B=B, window=[])
    c0, u0 = _centroid(sim.E, sim.B, dx)
    n = 400
    sim.step(n)
    assert sim.moves == W.window_moves(n, dt, dx) == 200
    c1, u1 = _centroid(sim.E, sim.B, dx, sim.moves * dx)     # physical coordinates
    vg = W.yee_group_velocity(10.0, dx, dt)
    assert (c1 - c0) / (n * dt) == pytest.approx(vg, rel=2e-3)
    assert u1 / u0 == pytest.approx(1.0, abs=2e-3)


def test_polarisation_rotates_e_in_the_y_z_plane_with_b_equal_x_cross_e():
    nx, ny, dx, dy = 64, 8, 0.05, 0.05
    a = W.Laser("plane", start=2.5, fwhm=0.8, a0=0.5, omega0=8.0, polarization=0.0)
    b = W.Laser("plane", start=2.5, fwhm=0.8, a0=0.5, omega0=8.0, polarization=np.pi / 2)
    Ea, Ba = W.laser_fields(nx, ny, dx, dy, a)
    Eb, Bb = W.laser_fields(nx, ny, dx, dy, b)
    # a plane wave does not depend on y: Ez (i, j) = Ey (i, j + 1/2) of the rotated pulse
    np.testing.assert_allclose(Eb[2], Ea[1], atol=1e-12)
    np.testing.assert_allclose(Bb[1], -Ba[2], atol=1e-12)     # B = x_hat x E
    assert np.max(np.abs(Ea[1])) == pytest.approx(0.5 * 8.0, rel=1e-2)
    assert not np.any(Ea[0]) and not np.any(Ba[0])


def test_gaussian_beam_diffracts_down_to_its_waist_at_the_focus():
    """Launched a Rayleigh length before its focus, the pulse's transverse rms
    width (of E^2 + B^2) is W(-zR)/2 = W0/sqrt(2); after the Yee scheme has
    carried it zR forward it is W0/2."""
    om, W0, dx = 10.0, 2.0, 0.05
    zR = 0.5 * om * W0 * W0
    dy, dt = dx, 0.6 * dx
    nx, ny = 512, 480
    Ly = ny * dy
    front = 0.5 * nx * dx
    l = W.Laser("gaussian", start=front, fwhm=2.0, a0=0.01, omega0=om, W0=W0,
                focus=front - 2.0 + zR, axis=Ly / 2)
    E, B = W.laser_fields(nx, ny, dx, dy, l)
    J = np.zeros_like(E)

    def width():
        u = (E ** 2).sum(axis=(0, 2)) + (B ** 2).sum(axis=(0, 2))
        y = (np.arange(ny) + 0.5) * dy - Ly / 2
        m = (u * y).sum() / u.sum()
        return np.sqrt((u * (y - m) ** 2).sum() / u.sum())

    assert width() == pytest.approx(W0 / np.sqrt(2), rel=5e-3)
    for _ in range(int(round(zR / dt))):
        orc.yee(E, B, J, dx, dy, dt)
    assert width() == pytest.approx(W0 / 2, rel=2e-2)


@pytest.mark.parametrize("window", [False, True])
def test_tile_order_bookmarks_count_each_tile_by_brute_force(window):
    """Tile t of the order owns off[t+1] - off[t] particles: those whose tile
    coordinates are (t % ntx, t // ntx) in rows, or (ntx - 1 - t // nty,
    t % nty) in the window's columns from the right edge."""
    nx, ny, T = 48, 32, 8
    ntx, nty = nx // T, ny // T
    rng = np.random.default_rng(21)
    ix = rng.integers(0, nx, 500).astype(np.int32)
    iy = rng.integers(0, ny, 500).astype(np.int32)
    off = orc.tile_offsets_in_order(nx, ny, T, ix, iy, window=window)
    assert off[0] == 0 and off[-1] == ix.size and off.size == ntx * nty + 1
    for t in range(ntx * nty):
        tx, ty = (ntx - 1 - t // nty, t % nty) if window else (t % ntx, t // ntx)
        n = sum(1 for a, b in zip(ix, iy) if a // T == tx and b // T == ty)
        assert off[t + 1] - off[t] == n
