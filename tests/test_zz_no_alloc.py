"""The allocation-free tile sort (pic_tile_sort_noalloc), for callers that
cannot allocate device memory, through the C ABI: its bookmarks against the
oracle's counting sort, its particles against the library's own tile sort
(pic_load_particles followed by pic_get_particles), and its refusals.

Collected last on purpose (file name): it shares a fixed device scratch array
across calls, and must give the same result as the allocating path on two
calls in a row, after a call that stopped early on a validation failure, and
whether run alone in a fresh process or after every other test."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_14795_gb300 import build
    build.build_library()
    oracle.build_oracle()
    return torch


def _sorted_by_tile(ix, iy, x, y, ux, uy, uz, off):
    """Per tile, the particles in a canonical order (lexicographic), so two
    valid sorts that differ only inside tiles compare equal."""
    rows = np.stack([ix.astype(np.float64), iy, x, y, ux, uy, uz], axis=1)
    parts = []
    for t in range(len(off) - 1):
        blk = rows[off[t]:off[t + 1]]
        parts.append(blk[np.lexsort(blk.T[::-1])])
    return np.concatenate(parts) if parts else rows[:0]


def _noalloc(torch, nx, ny, T, arrs):
    from paper_2501_14795_gb300 import pic
    dev_in = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]
    dev_out = [torch.empty_like(t) for t in dev_in]
    off = torch.full(((nx // T) * (ny // T) + 1,), -1, dtype=torch.int64, device="cuda")
    pic.pic_tile_sort_noalloc(nx, ny, T, *dev_in, *dev_out, off)
    return [t.cpu().numpy() for t in dev_out], off.cpu().numpy()


def _check_against_oracle_and_library(torch, nx, ny, T, sp):
    from paper_2501_14795_gb300 import pic
    arrs = sp.arrays()
    got, got_off = _noalloc(torch, nx, ny, T, arrs)
    # bookmarks: the oracle's counting sort by tile id (the plain definition)
    np.testing.assert_array_equal(got_off, oracle.tile_offsets_in_order(nx, ny, T, sp.ix, sp.iy))
    # every particle in the range of its tile
    tid = (got[1] // T) * (nx // T) + got[0] // T
    np.testing.assert_array_equal(np.repeat(np.arange(len(got_off) - 1), np.diff(got_off)), tid)
    # the same particles per tile as the library's own (allocating) sort
    cfg = pic.make_config(nx, ny, 0.1, 0.1, 0.05, [(sp.q_over_m, sp.qtilde)], tile=T)
    with pic.Simulation(cfg) as sim:
        pic.pic_load_particles(sim.h, 0, *arrs)
        ref = sim.particles(0)
    np.testing.assert_array_equal(got_off, ref["tile_offset"])
    a = _sorted_by_tile(*got, got_off)
    b = _sorted_by_tile(ref["ix"], ref["iy"], ref["x"], ref["y"], ref["ux"], ref["uy"], ref["uz"],
                        ref["tile_offset"])
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("case", [(64, 48, 16, 30011, 1), (128, 128, 8, 100003, 2)])
def test_noalloc_sort_matches_oracle_and_library_sort_on_two_calls(torch_cuda, case):
    from paper_2501_14795_gb300 import workloads as wl
    nx, ny, T, n, seed = case
    for call in range(2):
        sp = wl.random_particles(nx, ny, n - 7 * call, u_max=0.5, seed=seed + 10 * call)
        _check_against_oracle_and_library(torch_cuda, nx, ny, T, sp)


@pytest.mark.parametrize("bad", ["nan_momentum", "cell_outside", "offset_one"])
def test_noalloc_rejects_invalid_particle_then_sorts_cleanly(torch_cuda, bad):
    """A call that stops at the validation step (PIC_EINVAL) leaves counts in
    the shared array; the next valid call clears them and sorts exactly."""
    from paper_2501_14795_gb300 import pic
    from paper_2501_14795_gb300 import workloads as wl
    nx, ny, T = 64, 64, 16
    sp = wl.random_particles(nx, ny, 20011, u_max=0.5, seed=77)
    arrs = [np.array(a, copy=True) for a in sp.arrays()]
    if bad == "nan_momentum":
        arrs[5][1234] = np.nan
    elif bad == "cell_outside":
        arrs[0][99] = nx
    else:
        arrs[3][4321] = np.float32(1.0)
    with pytest.raises(pic.PicError) as ei:
        _noalloc(torch_cuda, nx, ny, T, arrs)
    assert ei.value.status == pic.PIC_EINVAL
    _check_against_oracle_and_library(torch_cuda, nx, ny, T,
                                      wl.random_particles(nx, ny, 20011, u_max=0.5, seed=78))


def test_noalloc_rejects_more_tiles_than_its_scratch(torch_cuda):
    """4096 x 4096 cells in 8 x 8 tiles is 262,144 tiles, above
    PIC_NOALLOC_MAX_TILES (65,536): refused before anything runs."""
    from paper_2501_14795_gb300 import pic
    from paper_2501_14795_gb300 import workloads as wl
    sp = wl.random_particles(4096, 4096, 1000, u_max=0.5, seed=5)
    with pytest.raises(pic.PicError) as ei:
        _noalloc(torch_cuda, 4096, 4096, 8, sp.arrays())
    assert ei.value.status == pic.PIC_EINVAL
    # the largest accepted grid: 65,536 tiles exactly
    sp = wl.random_particles(2048, 2048, 50000, u_max=0.5, seed=6)
    _check_against_oracle_and_library(torch_cuda, 2048, 2048, 8, sp)


def test_noalloc_empty_input_gives_zero_bookmarks(torch_cuda):
    from paper_2501_14795_gb300 import workloads as wl
    sp = wl.random_particles(32, 32, 0, u_max=0.5, seed=9)
    _, off = _noalloc(torch_cuda, 32, 32, 16, sp.arrays())
    np.testing.assert_array_equal(off, np.zeros(5, np.int64))
