"""GPU (CUDA, through the C ABI) versus the CPU oracle.

* strict build (PIC_STRICT_FP): cells, offsets, momenta and tile_offset equal
  the FP32 oracle bit for bit after a step from an identical state;
* fast build: momenta within 2e-6 |u|, offsets within 1e-6 cell of the FP64
  oracle, cells equal except where the FP64 position lies within 1e-5 cell of a
  cell boundary;
* J, E, B within a tolerance derived from FP32 accumulation (see
  ``J_RTOL``): each J value sums O(10) FP32 contributions, each carrying a few
  ulp (6e-8) of relative error, hence |dJ| <= 5e-6 max|J|;
* multi-step, full-size and edge cases.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2501_14795_gb300 import pic
from paper_2501_14795_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

J_RTOL = 5e-6     # max |J_gpu - J_fp64| / max |J_fp64|
F_RTOL = 2e-6     # same for E and B after one Yee step
U_RTOL = 2e-6     # |u_gpu - u_fp64| / (|u| + 1e-3)
X_ATOL = 1e-6     # offsets, in cells
NEAR = 1e-5       # cells within this of a boundary may round either way


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_14795_gb300 import build
    build.build_library()
    oracle.build_oracle()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _gpu(w, flags=pic.PIC_TRACK_IDS, tile=None, threads=256, E=None, B=None, chunk=0):
    sim = pic.Simulation.from_workload(w, tile=tile, threads=threads, flags=flags, device=True,
                                       chunk=chunk)
    if E is not None or B is not None:
        pic.pic_set_fields(sim.h, None if E is None else _dev(E.reshape(-1)),
                           None if B is None else _dev(B.reshape(-1)))
    return sim


def _oracle(w, dtype, E=None, B=None, T=None):
    sps = []
    for s in w.species:
        st = oracle.SpeciesState(s.q_over_m, s.qtilde, *s.arrays())
        st.pid = np.arange(s.n, dtype=np.int64)
        sps.append(st)
    E = w.E0 if E is None else E
    B = w.B0 if B is None else B
    o = oracle.OracleSim(w.nx, w.ny, w.dx, w.dy, w.dt, T or w.tile, sps, dtype=dtype,
                         background=w.background, E=E, B=B)
    for st in o.species:
        st.pid = np.arange(st.n, dtype=np.int64)
    return o


def _by_id(d):
    o = np.argsort(d["id"], kind="stable")
    return {k: (v[o] if k not in ("tile_offset",) else v) for k, v in d.items()}


def _oracle_by_id(sp):
    o = np.argsort(sp.pid)
    return dict(ix=sp.ix[o], iy=sp.iy[o], x=sp.x[o], y=sp.y[o], ux=sp.ux[o], uy=sp.uy[o],
                uz=sp.uz[o])


def _tile_ids(ix, iy, nx, T):
    return (iy // T) * (nx // T) + ix // T


def _random_case(nx, ny, T, n, seed, u_max=0.6, amp=0.2):
    sp = wl.random_particles(nx, ny, n, u_max=u_max, seed=seed)
    E, B = wl.random_fields(nx, ny, amp=amp, seed=seed + 100)
    return wl.Workload("random", nx, ny, 0.1, 0.1, 0.05, T, 1, [sp]), E, B


CASES = [(48, 32, 16, 5003), (64, 64, 8, 20011), (32, 64, 32, 7001), (16, 16, 8, 999),
         (16, 32, 16, 1500)]


@pytest.mark.parametrize("chunk", [0, 64])
@pytest.mark.parametrize("nx,ny,T,n", CASES)
def test_strict_step_is_bit_exact_with_fp32_oracle(nx, ny, T, n, chunk):
    """chunk = 64 splits every tile over several CTAs (shared leaver counters,
    all-atomic J flush); chunk = 0 keeps one CTA per tile at these sizes."""
    w, E, B = _random_case(nx, ny, T, n, seed=nx + ny + T)
    with _gpu(w, pic.PIC_STRICT_FP | pic.PIC_TRACK_IDS, tile=T, E=E, B=B, chunk=chunk) as sim:
        sim.step(1)
        got = sim.particles(0, ids=True)
        Jg = sim.fields(pic.FIELD_J)
        Eg = sim.fields(pic.FIELD_E)
        Bg = sim.fields(pic.FIELD_B)
    o32 = _oracle(w, np.float32, E, B, T)
    o32.step(1)
    ref = _oracle_by_id(o32.species[0])
    g = _by_id(got)
    for k in ("ix", "iy", "x", "y", "ux", "uy", "uz"):
        np.testing.assert_array_equal(g[k], ref[k], err_msg=k)
    np.testing.assert_array_equal(got["tile_offset"], o32.tile_offsets())
    # every particle lies in the range of its tile, and each tile holds the same ids
    tid = _tile_ids(got["ix"], got["iy"], nx, T)
    off = got["tile_offset"]
    for t in range(len(off) - 1):
        assert np.all(tid[off[t]:off[t + 1]] == t)
    sp = o32.species[0]
    otid = _tile_ids(sp.ix, sp.iy, nx, T)
    for t in range(len(off) - 1):
        assert set(got["id"][off[t]:off[t + 1]]) == set(sp.pid[otid == t])
    # grid quantities against FP64
    o64 = _oracle(w, np.float64, E, B, T)
    o64.step(1)
    assert np.max(np.abs(Jg - o64.J)) <= J_RTOL * np.max(np.abs(o64.J))
    assert np.max(np.abs(Eg - o64.E)) <= F_RTOL * np.max(np.abs(o64.E))
    assert np.max(np.abs(Bg - o64.B)) <= F_RTOL * np.max(np.abs(o64.B))


@pytest.mark.parametrize("nx,ny,T,n", CASES[:3])
@pytest.mark.parametrize("threads,chunk", [(128, 0), (256, 0), (512, 0), (256, 100)])
def test_fast_step_matches_fp64_oracle(nx, ny, T, n, threads, chunk):
    w, E, B = _random_case(nx, ny, T, n, seed=7 * nx + T)
    with _gpu(w, pic.PIC_TRACK_IDS, tile=T, threads=threads, E=E, B=B, chunk=chunk) as sim:
        sim.step(1)
        got = _by_id(sim.particles(0, ids=True))
        Jg = sim.fields(pic.FIELD_J)
        off = sim.particles(0)["tile_offset"]
    o = _oracle(w, np.float64, E, B, T)
    o.step(1)
    ref = _oracle_by_id(o.species[0])
    u_ref = np.stack([ref["ux"], ref["uy"], ref["uz"]])
    u_got = np.stack([got["ux"], got["uy"], got["uz"]])
    du = np.linalg.norm(u_got - u_ref, axis=0)
    assert np.all(du <= U_RTOL * (np.linalg.norm(u_ref, axis=0) + 1e-3))
    same = (got["ix"] == ref["ix"]) & (got["iy"] == ref["iy"])
    near = ((np.minimum(ref["x"], 1 - ref["x"]) < NEAR) | (np.minimum(ref["y"], 1 - ref["y"]) < NEAR))
    assert np.all(same | near), f"{np.count_nonzero(~same)} cells differ away from boundaries"
    assert np.all(np.abs(got["x"][same] - ref["x"][same]) <= X_ATOL)
    assert np.all(np.abs(got["y"][same] - ref["y"][same]) <= X_ATOL)
    assert np.max(np.abs(Jg - o.J)) <= J_RTOL * np.max(np.abs(o.J))
    # counts per tile follow the cells bit for bit
    counts = np.bincount(_tile_ids(got["ix"], got["iy"], nx, T), minlength=len(off) - 1)
    np.testing.assert_array_equal(np.diff(off), counts)


def test_graph_and_direct_launch_agree():
    """Graph replay and one-by-one launches run the same kernels: identical
    after one step; after five, equal to round-off (J is summed with atomics
    in no fixed order, so later steps are reproducible to round-off only)."""
    w, E, B = _random_case(48, 32, 16, 4000, seed=5)
    outs = {}
    for nsteps in (1, 5):
        for extra in (0, pic.PIC_NO_GRAPH):
            with _gpu(w, pic.PIC_STRICT_FP | pic.PIC_TRACK_IDS | extra, tile=16, E=E, B=B) as sim:
                sim.step(nsteps)
                outs[nsteps, extra] = (_by_id(sim.particles(0, ids=True)), sim.fields(pic.FIELD_E))
    a, b = outs[1, 0][0], outs[1, pic.PIC_NO_GRAPH][0]
    for k in ("ix", "iy", "x", "y", "ux", "uy", "uz"):
        np.testing.assert_array_equal(a[k], b[k])
    a, b = outs[5, 0], outs[5, pic.PIC_NO_GRAPH]
    _assert_close_states(a[0], b[0], 48, 32)
    np.testing.assert_allclose(a[1], b[1], rtol=0, atol=1e-5 * np.max(np.abs(b[1])))


def _assert_close_states(a, b, nx, ny, pos_tol=1e-5, u_tol=1e-5):
    """Same particles (by id) within round-off: unwrapped positions and momenta."""
    np.testing.assert_array_equal(a["id"], b["id"])
    dx = (a["ix"] + a["x"].astype(np.float64)) - (b["ix"] + b["x"].astype(np.float64))
    dy = (a["iy"] + a["y"].astype(np.float64)) - (b["iy"] + b["y"].astype(np.float64))
    dx = (dx + nx / 2) % nx - nx / 2
    dy = (dy + ny / 2) % ny - ny / 2
    assert np.max(np.abs(dx)) < pos_tol and np.max(np.abs(dy)) < pos_tol
    for k in ("ux", "uy", "uz"):
        assert np.max(np.abs(a[k].astype(np.float64) - b[k])) < u_tol


@pytest.mark.parametrize("chunk", [0, 256])
def test_two_stream_100_steps_tracks_fp64_oracle(chunk):
    """The two-stream workload (64x64, 4x4 ppc, drift +-0.2, u_th 0.1), 100
    steps: particle positions agree within 1e-4 cell and the energy histories
    within 1e-3 of the total (chunk = 256: every tile split over 16 CTAs)."""
    w = wl.two_stream()
    with _gpu(w, pic.PIC_TRACK_IDS, chunk=chunk) as sim:
        sim.step(100)
        got = _by_id(sim.particles(0, ids=True))
        he, hb, hk = sim.history(0, 101)
        d = sim.diagnostics()
    o = _oracle(w, np.float64)
    WE, WB = [], []
    for _ in range(100):
        e, b = o.energies()
        WE.append(e)
        WB.append(b)
        o.step(1)
    e, b = o.energies()
    WE.append(e)
    WB.append(b)
    ref = _oracle_by_id(o.species[0])
    dxp = (got["ix"] + got["x"].astype(np.float64)) - (ref["ix"] + ref["x"])
    dyp = (got["iy"] + got["y"].astype(np.float64)) - (ref["iy"] + ref["y"])
    dxp = (dxp + 32) % 64 - 32
    dyp = (dyp + 32) % 64 - 32
    assert np.max(np.abs(dxp)) < 1e-4 and np.max(np.abs(dyp)) < 1e-4
    tot = np.array(o.ke_history) + np.array(WE[:-1]) + np.array(WB[:-1])
    scale = float(np.max(tot))
    assert np.max(np.abs(he - np.array(WE))) < 1e-3 * scale
    assert np.max(np.abs(hb - np.array(WB))) < 1e-3 * scale
    assert np.max(np.abs(hk[:100] - np.array(o.ke_history))) < 1e-3 * scale
    assert math.isnan(hk[100])
    assert d["status_bits"] == 0


def test_diagnostics_energies_gauss_and_continuity():
    w = wl.thermal_seeded(nx=64, ny=64, k=4, u_th=0.2, amp=1e-3, tile=16)
    with _gpu(w, 0) as sim:
        d0 = sim.diagnostics()
        E0 = sim.fields(pic.FIELD_E)
        sim.step(1)
        d1 = sim.diagnostics()
        sim.step(1)
        d2 = sim.diagnostics()
        E2 = sim.fields(pic.FIELD_E)
        rho2 = sim.fields(pic.FIELD_RHO)
        J2 = sim.fields(pic.FIELD_J)
    assert d0["w_e"] == pytest.approx(oracle.field_energy(E0, 0.1, 0.1), rel=1e-6)
    assert d2["w_e"] == pytest.approx(oracle.field_energy(E2, 0.1, 0.1), rel=1e-6)
    assert math.isnan(d0["continuity_max"]) and math.isnan(d0["w_k"])
    scale = np.max(np.abs(J2)) / 0.1
    for d in (d1, d2):
        assert d["continuity_max"] < 1e-5 * scale
    # Gauss's law residual does not drift (charge-conserving deposit)
    assert abs(d2["gauss_max"] - d0["gauss_max"]) < 1e-5
    # the FP64 residual agrees with a numpy evaluation of the fetched arrays
    g = np.max(np.abs(oracle.div_e(E2, 0.1, 0.1) - rho2))
    assert d2["gauss_max"] == pytest.approx(g, abs=1e-5)
    assert abs(d2["charge_total"]) < 1e-6 * w.nx * w.ny * 0.01


def _full_size_checks(w, steps, tile, threads=256, sample=2000):
    """Run `steps` steps at full size in the bench launch configuration (with
    particle ids), then one more step on a fetched state; sampled particles
    that stay in their tile are found again by id and checked one by one
    against the oracle's per-particle push, and whole-grid properties
    (sortedness, counts, continuity, Gauss drift) on everything."""
    with _gpu(w, pic.PIC_TRACK_IDS, tile=tile, threads=threads) as sim:
        d0 = sim.diagnostics()
        sim.step(steps)
        before = sim.particles(0, ids=True)
        E = sim.fields(pic.FIELD_E)
        B = sim.fields(pic.FIELD_B)
        d1 = sim.diagnostics()
        sim.step(1)
        after = sim.particles(0, ids=True)
        d2 = sim.diagnostics()
        J = sim.fields(pic.FIELD_J)
    nx, T = w.nx, tile
    n = w.n_particles
    assert after["tile_offset"][-1] == n
    for st in (before, after):
        tid = _tile_ids(st["ix"], st["iy"], nx, T)
        counts = np.bincount(tid, minlength=len(st["tile_offset"]) - 1)
        np.testing.assert_array_equal(np.diff(st["tile_offset"]), counts)
        assert np.all(np.diff(tid) >= 0)
    # the ids are a permutation of 0..n-1: where each particle is after the step
    assert np.array_equal(np.sort(after["id"]), np.arange(n, dtype=np.int32))
    where = np.empty(n, np.int64)
    where[after["id"]] = np.arange(n)
    rng = np.random.default_rng(0)
    idx = rng.choice(n, size=min(sample, n), replace=False)
    s = w.species[0]
    sub = oracle.SpeciesState(s.q_over_m, s.qtilde, before["ix"][idx].copy(), before["iy"][idx].copy(),
                              before["x"][idx].astype(np.float64), before["y"][idx].astype(np.float64),
                              before["ux"][idx].astype(np.float64), before["uy"][idx].astype(np.float64),
                              before["uz"][idx].astype(np.float64))
    Jtmp = np.zeros((3, w.ny, w.nx))
    st, _ = oracle.advance(sub, E.astype(np.float64), B.astype(np.float64), Jtmp, w.dx, w.dy, w.dt)
    assert st == 0
    t_old = _tile_ids(before["ix"][idx], before["iy"][idx], nx, T)
    t_new = _tile_ids(sub.ix, sub.iy, nx, T)
    keep = t_old == t_new
    keep &= (np.minimum(sub.x, 1 - sub.x) > NEAR) & (np.minimum(sub.y, 1 - sub.y) > NEAR)
    assert keep.sum() > 0.5 * len(idx)
    k = where[before["id"][idx][keep]]
    np.testing.assert_array_equal(after["ix"][k], sub.ix[keep])
    np.testing.assert_array_equal(after["iy"][k], sub.iy[keep])
    assert np.max(np.abs(after["x"][k] - sub.x[keep])) <= X_ATOL
    assert np.max(np.abs(after["y"][k] - sub.y[keep])) <= X_ATOL
    u_ref = np.stack([sub.ux[keep], sub.uy[keep], sub.uz[keep]])
    u_got = np.stack([after["ux"][k], after["uy"][k], after["uz"][k]])
    assert np.all(np.linalg.norm(u_got - u_ref, axis=0) <= U_RTOL * (np.linalg.norm(u_ref, axis=0) + 1e-3))
    # whole-grid invariants
    assert d2["continuity_max"] < 1e-5 * np.max(np.abs(J)) / w.dx
    assert abs(d2["gauss_max"] - d0["gauss_max"]) < 1e-4
    assert d2["status_bits"] == 0 and d1["status_bits"] == 0
    return d0, d2


def test_full_size_weibel_512():
    """Weibel workload at full size: 512x512 cells, 2 x 8x8 ppc (33.5M
    particles), 16x16 tiles, 256 threads per tile."""
    w = wl.weibel()
    _full_size_checks(w, steps=20, tile=16)


def test_full_size_thermal_2048():
    """Large thermal workload: 2048x2048 cells, 4x4 ppc (67.1M particles),
    seeded Ex mode, 16x16 tiles."""
    w = wl.thermal_seeded()
    _full_size_checks(w, steps=5, tile=16, sample=4000)


# ------------------------------------------------------------------ edge cases

def test_empty_species_and_single_tile_crowding():
    nx = ny = 32
    # species 0: everything in tile 0 (ragged: all other tiles empty); species 1: empty
    rng = np.random.default_rng(1)
    n = 3000
    sp0 = wl.Species(-1.0, -1 / 16, rng.integers(0, 8, n).astype(np.int32),
                     rng.integers(0, 8, n).astype(np.int32), rng.random(n, dtype=np.float32),
                     rng.random(n, dtype=np.float32),
                     *(rng.uniform(-0.5, 0.5, (3, n)).astype(np.float32)))
    sp1 = wl.Species(1.0, 1 / 16, *(np.zeros(0, t) for t in (np.int32, np.int32, np.float32,
                                                             np.float32, np.float32, np.float32,
                                                             np.float32)))
    w = wl.Workload("crowd", nx, ny, 0.1, 0.1, 0.05, 8, 1, [sp0, sp1], background=0.0)
    E, B = wl.random_fields(nx, ny, amp=0.1, seed=9)
    with _gpu(w, pic.PIC_STRICT_FP | pic.PIC_TRACK_IDS, tile=8, E=E, B=B) as sim:
        sim.step(1)
        got1 = _by_id(sim.particles(0, ids=True))
        sim.step(2)
        got3 = _by_id(sim.particles(0, ids=True))
        assert pic.pic_num_particles(sim.h, 1) == 0
        p1 = sim.particles(1)
        assert np.all(p1["tile_offset"] == 0)
    o = _oracle(w, np.float32, E, B, 8)
    o.step(1)
    ref = _oracle_by_id(o.species[0])
    for k in ("ix", "iy", "x", "y", "ux", "uy", "uz"):
        np.testing.assert_array_equal(got1[k], ref[k], err_msg=k)
    o.step(2)
    ref = _oracle_by_id(o.species[0])
    ref["id"] = np.sort(o.species[0].pid).astype(np.int32)
    _assert_close_states(got3, ref, nx, ny)


def test_boundary_offsets_and_two_species():
    """Particles exactly on cell corners and at the largest offset below 1, an
    electron and a positron species (opposite q/m and charge)."""
    nx = ny = 16
    one_m = np.float32(np.nextafter(np.float32(1), np.float32(0)))
    xs = np.array([0, 0, one_m, one_m, 0.5, 0.25], np.float32)
    ys = np.array([0, one_m, 0, one_m, 0.5, 0.0], np.float32)
    m = xs.size
    ix = np.array([0, 15, 7, 8, 3, 12], np.int32)
    iy = np.array([0, 15, 8, 7, 12, 3], np.int32)
    u = np.array([[0.3, -0.3, 0.4, -0.4, 0.0, 0.2], [0.2, -0.1, -0.3, 0.3, 0.0, -0.2],
                  [0.1, 0.0, 0.0, 0.0, 0.5, 0.0]], np.float32)
    el = wl.Species(-1.0, -1 / 8, ix, iy, xs, ys, *u.copy())
    po = wl.Species(1.0, 1 / 8, iy.copy(), ix.copy(), ys.copy(), xs.copy(), *(-u).copy())
    w = wl.Workload("edges", nx, ny, 0.1, 0.1, 0.05, 8, 1, [el, po], background=0.0)
    E, B = wl.random_fields(nx, ny, amp=0.3, seed=2)
    with _gpu(w, pic.PIC_STRICT_FP | pic.PIC_TRACK_IDS, tile=8, E=E, B=B) as sim:
        sim.step(1)
        gots = [_by_id(sim.particles(s, ids=True)) for s in range(2)]
        Jg = sim.fields(pic.FIELD_J)
        sim.step(3)
        gots4 = [_by_id(sim.particles(s, ids=True)) for s in range(2)]
    o = _oracle(w, np.float32, E, B, 8)
    o.step(1)
    for s in range(2):
        ref = _oracle_by_id(o.species[s])
        for k in ("ix", "iy", "x", "y", "ux", "uy", "uz"):
            np.testing.assert_array_equal(gots[s][k], ref[k], err_msg=f"species {s} {k}")
    o64 = _oracle(w, np.float64, E, B, 8)
    o64.step(1)
    assert np.max(np.abs(Jg - o64.J)) <= J_RTOL * np.max(np.abs(o64.J))
    o64.step(3)
    for s in range(2):
        ref = _oracle_by_id(o64.species[s])
        ref["id"] = np.arange(m, dtype=np.int32)
        _assert_close_states(gots4[s], ref, nx, ny)
    assert m == 6


def test_restart_roundtrip_is_exact():
    w = wl.two_stream(nx=32, ny=32, k=2, tile=8)
    with _gpu(w, pic.PIC_STRICT_FP | pic.PIC_TRACK_IDS, tile=8) as a:
        a.step(7)
        st = a.particles(0, ids=True)
        E = a.fields(pic.FIELD_E)
        B = a.fields(pic.FIELD_B)
        a.step(1)
        ref = _by_id(a.particles(0, ids=True))
    sp = wl.Species(-1.0, w.species[0].qtilde, st["ix"], st["iy"], st["x"], st["y"], st["ux"],
                    st["uy"], st["uz"])
    w2 = wl.Workload("restart", 32, 32, 0.1, 0.1, 0.05, 8, 1, [sp], E0=E, B0=B)
    with pic.Simulation.from_workload(w2, tile=8, flags=pic.PIC_STRICT_FP | pic.PIC_TRACK_IDS) as b:
        # carry the ids over
        pic.pic_load_particles(b.h, 0, st["ix"], st["iy"], st["x"], st["y"], st["ux"], st["uy"],
                               st["uz"], id=st["id"])
        b.step(1)
        got = _by_id(b.particles(0, ids=True))
    for k in ("ix", "iy", "x", "y", "ux", "uy", "uz", "id"):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)


def test_invalid_loads_are_rejected_and_state_kept():
    w = wl.two_stream(nx=16, ny=16, k=2, tile=8)
    with _gpu(w, pic.PIC_TRACK_IDS, tile=8) as sim:
        before = sim.particles(0)
        s = w.species[0]
        for field, bad in (("x", 1.0), ("ix", 16), ("uy", np.nan), ("iy", -1), ("y", -0.25)):
            arrs = {k: v.copy() for k, v in zip(("ix", "iy", "x", "y", "ux", "uy", "uz"), s.arrays())}
            arrs[field][5] = bad
            with pytest.raises(pic.PicError) as ei:
                pic.pic_load_particles(sim.h, 0, *arrs.values())
            assert ei.value.status == 1
        after = sim.particles(0)
        for k in ("ix", "x", "ux"):
            np.testing.assert_array_equal(before[k], after[k])
        with pytest.raises(pic.PicError):
            pic.pic_load_particles(sim.h, 3, *s.arrays())


def test_non_finite_field_raises_particle_status_not_a_fault():
    """A non-finite field value makes the pushed particles' momenta non-finite:
    they are reported through the sticky status (PIC_EPARTICLE), stay where they
    were, and the context stays usable."""
    w = wl.two_stream(nx=16, ny=16, k=2, tile=8)
    E = np.zeros((3, 16, 16), np.float32)
    E[0, 5, 5] = np.inf
    with _gpu(w, 0, tile=8, E=E) as sim:
        sim.step(1)
        with pytest.raises(pic.PicError) as ei:
            pic.pic_sync(sim.h)
        assert ei.value.status == 6
        # the affected particles keep their non-finite momenta: reload them
        pic.pic_clear_status(sim.h)
        pic.pic_set_fields(sim.h, np.zeros(3 * 256, np.float32), np.zeros(3 * 256, np.float32))
        pic.pic_load_particles(sim.h, 0, *w.species[0].arrays())
        sim.step(1)
        pic.pic_sync(sim.h)
        assert sim.particles(0)["tile_offset"][-1] == w.n_particles


def test_timing_events_and_launch_count():
    w = wl.two_stream(nx=64, ny=64, k=2, tile=16)
    with _gpu(w, pic.PIC_TIMING, tile=16) as sim:
        sim.step(10)
        ms, cnt = pic.pic_timing(sim.h, reset=True)
        assert cnt == 10 and ms > 0
        # per step: advance, count, scan, evict, fill, Yee
        assert pic.pic_kernel_launches(sim.h) == 60


@pytest.mark.parametrize("passes", [1, 3])
def test_binomial_filter_matches_oracle(passes):
    """The current filter slot with the binomial filter: J after the filter,
    E and B after the field advance against the FP64 oracle with the same
    filter; 20 more steps keep the energies together."""
    w, E, B = _random_case(64, 32, 16, 9000, seed=77)
    with _gpu(w, pic.PIC_TRACK_IDS, tile=16, E=E, B=B) as sim:
        pic.pic_set_binomial_filter(sim.h, passes)
        sim.step(1)
        Jg = sim.fields(pic.FIELD_J)
        Eg = sim.fields(pic.FIELD_E)
        Bg = sim.fields(pic.FIELD_B)
        sim.step(20)
        d = sim.diagnostics()
    o = _oracle(w, np.float64, E, B, 16)
    o.filter_passes = passes
    o.step(1)
    assert np.abs(Jg - o.J).max() <= J_RTOL * np.abs(o.J).max()
    assert np.abs(Eg - o.E).max() <= F_RTOL * np.abs(o.E).max()
    assert np.abs(Bg - o.B).max() <= F_RTOL * np.abs(o.B).max()
    o.step(20)
    assert d["status_bits"] == 0
    we, wb = o.energies()
    assert d["w_e"] == pytest.approx(we, rel=2e-3)
    assert d["w_b"] == pytest.approx(wb, rel=2e-3)


def test_electron_positron_weibel_follows_the_oracle():
    """Two mobile species of opposite charge (the thesis's Weibel shape) on a
    small grid: 10 steps against the FP64 oracle; the pair plasma stays
    neutral and charge-conserving."""
    w = wl.weibel_pair(nx=64, ny=64, k=4, tile=16)
    with _gpu(w, 0) as sim:
        sim.diagnostics()
        sim.step(10)
        d = sim.diagnostics()
        sim.step(1)
        d2 = sim.diagnostics()
    o = _oracle(w, np.float64)
    o.step(10)
    we, wb = o.energies()
    assert d["status_bits"] == 0 and d["n_particles"][:2] == [w.species[0].n, w.species[1].n]
    assert d["w_e"] == pytest.approx(we, rel=1e-3, abs=1e-9)
    assert d["w_k"] == pytest.approx(o.ke_history[-1], rel=1e-5)
    assert abs(d["charge_total"]) < 1e-9
    assert d2["continuity_max"] < 1e-4


@pytest.mark.parametrize("nx,ny,T,n", [(1040, 528, 16, 2_000_003), (160, 48, 16, 30_011)])
def test_load_sorts_ragged_lattices_like_the_oracle(nx, ny, T, n):
    """The load path's per-cell count scan runs over segments of 4096 cells:
    on 1040 x 528 (549,120 cells, 134 segments and a ragged last one) and
    160 x 48 (7,680 cells, two segments) the tile bookmarks equal the oracle's
    bit for bit and every input particle is in its tile's range, unchanged."""
    w, _, _ = _random_case(nx, ny, T, n, seed=nx + ny)
    with _gpu(w, pic.PIC_TRACK_IDS, tile=T) as sim:
        got = sim.particles(0, ids=True)
    s = w.species[0]
    np.testing.assert_array_equal(got["tile_offset"],
                                  oracle.tile_offsets_in_order(nx, ny, T, s.ix, s.iy))
    tid = _tile_ids(got["ix"], got["iy"], nx, T)
    off = got["tile_offset"]
    assert np.all(np.repeat(np.arange(off.size - 1), np.diff(off)) == tid)
    d = _by_id(got)
    assert np.array_equal(d["id"], np.arange(n))
    for k, v in zip(("ix", "iy", "x", "y", "ux", "uy", "uz"), s.arrays()):
        np.testing.assert_array_equal(d[k], v)
