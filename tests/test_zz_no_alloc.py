"""The allocation-free tile sort (pic_tile_sort_noalloc), for callers that
cannot allocate device memory, against the library's own tile sort
(pic_load_particles followed by pic_get_particles), through the C ABI.

Collected last on purpose (file name): it shares a fixed device scratch array
across calls, and must give the same result as the allocating path on two
calls in a row, whether run alone in a fresh process or after every other
test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _sorted_by_tile(ix, iy, x, y, ux, uy, uz, off, nx, T):
    """Per tile, the particles in a canonical order (lexicographic), so two
    valid sorts that differ only inside tiles compare equal."""
    rows = np.stack([ix.astype(np.float64), iy, x, y, ux, uy, uz], axis=1)
    parts = []
    for t in range(len(off) - 1):
        blk = rows[off[t]:off[t + 1]]
        parts.append(blk[np.lexsort(blk.T[::-1])])
    return np.concatenate(parts) if parts else rows[:0]


@pytest.mark.parametrize("case", [(64, 48, 16, 30011, 1), (128, 128, 8, 100003, 2)])
def test_noalloc_sort_matches_library_sort_on_two_calls(case):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_14795_gb300 import build, pic
    from paper_2501_14795_gb300 import workloads as wl
    build.build_library()
    nx, ny, T, n, seed = case
    for call in range(2):
        sp = wl.random_particles(nx, ny, n - 7 * call, u_max=0.5, seed=seed + 10 * call)
        arrs = sp.arrays()
        dev_in = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]
        dev_out = [torch.empty_like(t) for t in dev_in]
        off = torch.empty((nx // T) * (ny // T) + 1, dtype=torch.int64, device="cuda")
        pic.pic_tile_sort_noalloc(nx, ny, T, *dev_in, *dev_out, off)
        got = [t.cpu().numpy() for t in dev_out]
        got_off = off.cpu().numpy()
        # the allocating path: load into a simulation, read back sorted
        cfg = pic.make_config(nx, ny, 0.1, 0.1, 0.05, [(sp.q_over_m, sp.qtilde)], tile=T)
        with pic.Simulation(cfg) as sim:
            pic.pic_load_particles(sim.h, 0, *arrs)
            ref = sim.particles(0)
        np.testing.assert_array_equal(got_off, ref["tile_offset"])
        a = _sorted_by_tile(*got, got_off, nx, T)
        b = _sorted_by_tile(ref["ix"], ref["iy"], ref["x"], ref["y"], ref["ux"], ref["uy"],
                            ref["uz"], ref["tile_offset"], nx, T)
        np.testing.assert_array_equal(a, b)
