"""What batching buys: the 64 simulations of the batched workload (grids drawn
from 64^2..512^2, 4, 16 or 64 ppc, counter-streaming drifts) stepped as one
batch (one captured graph per step: one particle-advance launch over all
members' work items, one launch per re-sort stage, one field launch) against
the same simulations stepped one after another, each with its own step
graph.  Mean step time of the whole ensemble from CUDA events around 10 steps
after 3; the batch must be faster.  The figures are printed."""
import pytest

from paper_2501_14795_gb300 import pic
from paper_2501_14795_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

MEMBERS, WARM, STEPS = 64, 3, 10


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
    return e0.elapsed_time(e1) / n


def test_batch_of_64_is_faster_than_its_members_one_after_another():
    members = [wl.batch_member(s) for s in range(MEMBERS)]
    n = sum(w.n_particles for w in members)
    sims = [pic.Simulation.from_workload(w, tile=16, device=True) for w in members]
    try:
        def seq(k):
            for _ in range(k):
                for s in sims:
                    s.step(1)
        seq(WARM)
        seq_ms = _timed(seq, STEPS)
        with pic.Batch(sims) as b:
            b.step(WARM)
            bat_ms = _timed(b.step, STEPS)
            b.sync()
        for s in sims:
            assert s.diagnostics()["status_bits"] == 0
    finally:
        for s in sims:
            s.close()
    print(f"{MEMBERS} simulations, {n} particles: one after another {seq_ms:.3f} ms per step "
          f"({n / seq_ms / 1e6:.3e} p/s), one batch {bat_ms:.3f} ms ({n / bat_ms / 1e6:.3e} p/s): "
          f"{seq_ms / bat_ms:.2f}x")
    assert bat_ms < seq_ms
