"""Failure detection without a GPU fault (the bounded device waits).

Every wait of the library's kernels on an mbarrier (TMA halo and particle
copies, tensor-core products) gives up after a bounded number of cycles, waits
once more (bounded) for the copies it had issued, sets a status bit and
returns; the host reports PIC_ETIMEOUT.  The probe runs that helper on a
barrier that nothing completes (no copy is issued, so none is in flight):
the wait runs out, the status comes back, and the context stays usable.
"""
import time

import pytest

from paper_2501_14795_gb300 import pic
from paper_2501_14795_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

PIC_ETIMEOUT = 7


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_14795_gb300 import build
    build.build_library()


def test_bounded_wait_completes_when_the_phase_does():
    assert pic.pic_probe_bounded_wait(1, 2_000_000) == 0


def test_bounded_wait_runs_out_and_the_context_stays_usable():
    t0 = time.perf_counter()
    assert pic.pic_probe_bounded_wait(0, 2_000_000) == PIC_ETIMEOUT   # about a millisecond
    assert time.perf_counter() - t0 < 5.0
    assert pic.pic_probe_bounded_wait(1, 2_000_000) == 0
    w = wl.two_stream(nx=64, ny=32, k=2, u_th=0.1, drift=0.2, tile=16, seed=9)
    with pic.Simulation.from_workload(w, device=True) as sim:
        sim.step(5)
        d = sim.diagnostics()
    assert d["status_bits"] == 0 and d["n_particles"][0] == w.n_particles


def test_allocation_failures_report_enomem_and_keep_the_state(monkeypatch):
    """PIC_FAULT=alloc (host-side injection) makes every device allocation of a
    simulation fail: creating one reports PIC_ENOMEM; a load that needs more
    capacity reports PIC_ENOMEM and keeps the loaded particles; with the
    variable cleared both work again."""
    import numpy as np
    w = wl.two_stream(nx=64, ny=32, k=2, u_th=0.1, drift=0.2, tile=16, seed=9)
    monkeypatch.setenv("PIC_FAULT", "alloc")
    with pytest.raises(pic.PicError) as ei:
        pic.Simulation.from_workload(w, device=True)
    assert ei.value.status == 3
    monkeypatch.delenv("PIC_FAULT")
    with pic.Simulation.from_workload(w, device=True) as sim:
        s = w.species[0]
        twice = [np.concatenate([a, a]) for a in s.arrays()]
        monkeypatch.setenv("PIC_FAULT", "alloc")
        with pytest.raises(pic.PicError) as ei:
            pic.pic_load_particles(sim.h, 0, *twice)
        assert ei.value.status == 3
        monkeypatch.delenv("PIC_FAULT")
        assert pic.pic_num_particles(sim.h, 0) == s.n
        sim.step(3)
        assert sim.diagnostics()["status_bits"] == 0
        pic.pic_load_particles(sim.h, 0, *twice)
        assert pic.pic_num_particles(sim.h, 0) == 2 * s.n
