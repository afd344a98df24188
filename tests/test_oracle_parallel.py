"""The oracle's threaded particle loop (the thesis's CPU scheme, §4.2: blocks
of tile-sorted particles over threads, each with a private current array added
afterwards) against the plain single-threaded loop: it is used as the timed CPU
baseline and to speed up long oracle runs, so it must give the same particles
bit for bit and the same current up to the order of the additions."""
import numpy as np
import pytest

from paper_2501_14795_gb300 import workloads as wl


def _sim(orc, w, threads, dtype=np.float64):
    sps = [orc.SpeciesState(s.q_over_m, s.qtilde, *s.arrays()) for s in w.species]
    return orc.OracleSim(w.nx, w.ny, w.dx, w.dy, w.dt, w.tile, sps, dtype=dtype,
                         background=w.background, E=w.E0, B=w.B0, threads=threads)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("threads", [2, 3, 8])
def test_threaded_loop_gives_identical_particles(orc, threads, dtype):
    w = wl.thermal_seeded(nx=32, ny=32, k=4, u_th=0.3, amp=1e-2, tile=8)
    a = _sim(orc, w, 1, dtype)
    b = _sim(orc, w, threads, dtype)
    for _ in range(6):
        # from the same fields (the threaded run's differ by round-off after a
        # step, through J), the particles must come out identical
        b.E[...] = a.E
        b.B[...] = a.B
        a.step(1)
        b.step(1)
        # same particle arrays (in the same tile-sorted order), bit for bit
        for k in ("ix", "iy", "x", "y", "ux", "uy", "uz"):
            np.testing.assert_array_equal(getattr(b.species[0], k), getattr(a.species[0], k))
        # the current: private arrays added in another order, round-off apart;
        # the fields follow from it and stay round-off apart too
        eps = np.finfo(dtype).eps
        assert np.max(np.abs(b.J - a.J)) <= 64 * eps * np.max(np.abs(a.J))
        assert abs(b.ke_history[-1] - a.ke_history[-1]) <= 1e-12 * abs(a.ke_history[-1])
        np.testing.assert_allclose(b.E, a.E, rtol=0, atol=64 * eps * np.max(np.abs(a.E)))


def test_threaded_loop_with_more_threads_than_particles(orc):
    w = wl.random_particles(16, 16, 5, seed=3)
    work = wl.Workload("random", 16, 16, 0.1, 0.1, 0.05, 8, 1, [w])
    a = _sim(orc, work, 1)
    b = _sim(orc, work, 16)
    a.step(2)
    b.step(2)
    for k in ("ix", "iy", "x", "y", "ux", "uy", "uz"):
        np.testing.assert_array_equal(getattr(b.species[0], k), getattr(a.species[0], k))
