"""The denoiser in the current-filter slot of a batch (pic_batch_set_denoiser):
all members' currents go through the network as one batch of samples.

* exactness: each member's filtered current after one batched step equals,
  bit for bit, pic_denoiser_forward (with the same low-wavenumber
  restoration) applied to that member's unfiltered current, run as the same
  group of samples.  The members' particles sit away from their tile's edge
  rows and columns and move a fortieth of a cell, so the deposit touches only
  cells that the particle advance stores rather than adds (no float atomics),
  and the strict build makes each particle's contribution independent of the
  warp it lands in (the fast build contracts multiply-adds differently in the
  single-piece path and in the piece loop, and the load's slot atomics decide
  the order inside a tile, so a few values may differ by a quantum between
  runs): the unfiltered current is the same in every run.  Cases: 4 members of
  256^2 in one group (the large batch takes the tcgen05 kernel where a single
  sample would not), and 3 members of 128 x 64 in groups of 2 and 1;
* a network of another grid is refused.

The speed test (ensembles of two-stream draws at 256^2, 4 ppc + the batched
denoiser against the plain 64-ppc runs) is in test_gpu_denoiser_speed.py.
"""
import numpy as np
import pytest

from paper_2501_14795_gb300 import denoise as dn
from paper_2501_14795_gb300 import pic
from paper_2501_14795_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_14795_gb300 import build
    build.build_library()


def _interior_workload(nx, ny, n, seed, T=16):
    """n particles in cells 3..T-4 of their tile along both axes, |u| < 0.05
    (a move of at most 0.025 cells per step): every current value lands in a
    cell that no other tile's halo reaches."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ix = (rng.integers(0, nx // T, n) * T + rng.integers(3, T - 3, n)).astype(np.int32)
    iy = (rng.integers(0, ny // T, n) * T + rng.integers(3, T - 3, n)).astype(np.int32)
    x = rng.random(n, dtype=np.float32)
    y = rng.random(n, dtype=np.float32)
    u = rng.uniform(-0.05, 0.05, (3, n)).astype(np.float32)
    sp = wl.Species(-1.0, -1.0 / 4, ix, iy, x, y, u[0].copy(), u[1].copy(), u[2].copy())
    return wl.Workload(f"interior_{nx}x{ny}_{seed}", nx, ny, 0.1, 0.1, 0.05, T, 1, [sp])


def _network(nx, ny, batch_max, restore):
    """Random parameters, the last layer included (a zero last layer would
    make the network the identity)."""
    params = dn.init_params(dn.SEED_DENOISER + 31).astype(np.float32)
    rng = np.random.Generator(np.random.PCG64(17))
    last = 9 * 32 * 3
    params[-(last + 3):-3] = rng.uniform(-0.05, 0.05, last).astype(np.float32)
    net = pic.Denoiser(nx, ny, batch_max, 0.05)
    net.set_params(params)
    net.set_low_k_restore(restore)
    return net


def _sim(w):
    return pic.Simulation.from_workload(w, device=True, flags=pic.PIC_STRICT_FP)


def _raw_current(w):
    with _sim(w) as sim:
        sim.step(1)
        assert sim.diagnostics()["status_bits"] == 0
        return sim.fields(pic.FIELD_J).astype(np.float32)


@pytest.mark.parametrize("nx,ny,members,batch_max", [(256, 256, 4, 4), (128, 64, 3, 2)])
def test_batched_filter_equals_the_forward_pass_of_each_group(nx, ny, members, batch_max):
    ws = [_interior_workload(nx, ny, 4 * nx * ny // 2, seed=100 + k) for k in range(members)]
    raw = [_raw_current(w) for w in ws]
    # the construction makes the unfiltered current reproducible
    assert np.array_equal(raw[0], _raw_current(ws[0]))
    net = _network(nx, ny, batch_max, restore=2)
    sims = [_sim(w) for w in ws]
    try:
        with pic.Batch(sims) as b:
            b.set_denoiser(net)
            b.step(1)
            b.sync()
            got = [s.fields(pic.FIELD_J) for s in sims]
        for s in sims:
            assert s.diagnostics()["status_bits"] == 0
        for g0 in range(0, members, batch_max):
            grp = np.stack(raw[g0:g0 + batch_max])
            want = net.forward(grp)
            for j in range(grp.shape[0]):
                k = g0 + j
                assert not np.array_equal(got[k], raw[k])  # the network changed the current
                assert np.array_equal(got[k], want[j]), f"member {k}: max diff " \
                    f"{np.max(np.abs(got[k] - want[j]))}"
    finally:
        for s in sims:
            s.close()
        net.close()


def test_batch_refuses_a_network_of_another_grid():
    ws = [_interior_workload(128, 64, 1000, seed=200 + k) for k in range(2)]
    sims = [pic.Simulation.from_workload(w, device=True) for w in ws]
    net = pic.Denoiser(64, 64, 2, 1.0)
    try:
        with pic.Batch(sims) as b:
            with pytest.raises(pic.PicError) as e:
                b.set_denoiser(net)
            assert e.value.status == pic.PIC_EINVAL
            b.step(1)  # still steps without a filter
            b.sync()
    finally:
        for s in sims:
            s.close()
        net.close()
