"""What the denoiser buys in speed at the learned-denoiser workload's grid
(256^2 two-stream runs): an ensemble of 16 draws stepped at 4 ppc with the
network in the current-filter slot (one batch, the network over all 16
currents at once, low-wavenumber restoration of 4 passes) against the same
16 draws stepped plainly at 64 ppc, the faster of one batch and 16 runs one
after another.  Mean step time per simulation from CUDA events around 20
steps after 3; the 4-ppc + denoiser ensemble must be faster.  The figures
are printed.

A single 256^2 run is too small to fill the GPU: its network pass is a
chain of 13 launches that each run a few microseconds (0.86x of the 64-ppc
step, see the launch lists), so the speed of the learned stand-in shows on
ensembles, and on single runs from 512^2 up.
"""
import numpy as np
import pytest

from paper_2501_14795_gb300 import denoise as dn
from paper_2501_14795_gb300 import pic

pytestmark = pytest.mark.gpu

SIDE = 256
MEMBERS = 16
WARM, STEPS = 3, 20


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_14795_gb300 import build
    build.build_library()


def _timed(step, n):
    import torch
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    step(n)
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def _ensemble(k):
    return [pic.Simulation.from_workload(dn.workload(d, SIDE, SIDE, k, STEPS), device=True)
            for d in dn.draws(MEMBERS, offset=700)]


def _batched_ms(sims, net=None):
    with pic.Batch(sims) as b:
        if net is not None:
            b.set_denoiser(net)
        b.step(WARM)
        ms = _timed(b.step, STEPS)
        b.sync()
    for s in sims:
        assert s.diagnostics()["status_bits"] == 0
    return ms / STEPS / MEMBERS


def _sequential_ms(sims):
    for s in sims:
        s.step(WARM)
    ms = sum(_timed(s.step, STEPS) for s in sims)
    return ms / STEPS / MEMBERS


def test_four_ppc_with_batched_denoiser_is_faster_than_sixty_four_ppc():
    sims = _ensemble(8)
    try:
        seq64 = _sequential_ms(sims)
    finally:
        for s in sims:
            s.close()
    sims = _ensemble(8)
    try:
        bat64 = _batched_ms(sims)
    finally:
        for s in sims:
            s.close()
    net = pic.Denoiser(SIDE, SIDE, MEMBERS, 0.03)
    net.set_params(dn.init_params(dn.SEED_DENOISER + 7).astype(np.float32))
    net.set_low_k_restore(4)
    sims = _ensemble(2)
    try:
        den4 = _batched_ms(sims, net)
    finally:
        for s in sims:
            s.close()
        net.close()
    base = min(seq64, bat64)
    print(f"{MEMBERS} draws at {SIDE}^2, ms per simulation-step: 64 ppc one after another "
          f"{seq64:.4f}, 64 ppc batched {bat64:.4f}; 4 ppc + batched denoiser {den4:.4f}: "
          f"speedup {base / den4:.2f}x")
    assert den4 < base
