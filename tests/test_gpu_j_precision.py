"""Precision of the deposited current (§3.1 deposit, Eqs. 13-16, accumulated in
FP32 per the precision split): one step of the fast build from the same state
as the FP64 oracle, on states shaped like the thesis-style workloads, with
the default exact 32-bit fixed-point J tiles and with PIC_FP32_J (FP32 tiles
with float atomics).

The fixed-point tiles sum exactly, but each FP32 contribution is first
rounded to the tiles' quantum q = 64 B |qtilde| / 2^30 (B: particle batches of
blockDim in a CTA item, at most 64; 64 = 32 lanes x 2 warps per tile and
batch), so a J value carries at most n q / 2 of rounding for its n
contributions.  The FP32 tiles round every addition instead (relative 2^-24
per addition), in an order the float atomics leave to the hardware, so their
error differs from run to run.  Both errors are printed.  The FP32 tiles meet
the particle-advance parity tolerance, 5e-6 of max|J| (measured 0.35-1e-6 on
the thermal and two-stream states, 1.2-2.1e-6 on the start of the Weibel
workload, where J is the small residue of cancelling streams and the FP32
sums round at the scale of the streams), and are closer to the oracle than
the fixed-point tiles; the fixed-point tiles meet their quantum bound,
whatever the chunk (an item holds at most 64 batches), plus the same 5e-6 of
max|J| for the FP32 additions of the tile ring into the global J."""
import math

import numpy as np
import pytest

import oracle
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
    oracle.build_oracle()


CASES = {
    "thermal_128": lambda: wl.thermal_seeded(nx=128, ny=128, k=4, u_th=0.2, amp=1e-3, tile=16),
    "weibel_128": lambda: wl.weibel(nx=128, ny=128, k=8, tile=16),
    "two_stream_64": lambda: wl.two_stream(),
}


def _oracle_J(w):
    sps = [oracle.SpeciesState(s.q_over_m, s.qtilde, *s.arrays()) for s in w.species]
    o = oracle.OracleSim(w.nx, w.ny, w.dx, w.dy, w.dt, w.tile, sps, background=w.background,
                         E=w.E0, B=w.B0)
    o.step(1)
    return o.J


def _contributions_bound(w):
    """At most three pieces per particle reach a J value, from particles
    starting in the 3 x 3 cells around it: 3 x the largest such count."""
    s = w.species[0]
    cnt = np.zeros((w.ny, w.nx))
    np.add.at(cnt, (s.iy, s.ix), 1)
    around = sum(np.roll(np.roll(cnt, a, 0), b, 1) for a in (-1, 0, 1) for b in (-1, 0, 1))
    return 3 * around.max()


@pytest.mark.parametrize("case", sorted(CASES))
def test_deposited_current_precision_fixed_point_and_fp32(case):
    w = CASES[case]()
    J64 = _oracle_J(w)
    scale = np.max(np.abs(J64))
    errs = {}
    for name, flags, chunk in (("fixed", 0, 0), ("fixed_chunk_2^20", 0, 1 << 20),
                               ("fp32", pic.PIC_FP32_J, 0)):
        with pic.Simulation.from_workload(w, tile=16, threads=256, flags=flags, device=True,
                                          chunk=chunk) as sim:
            sim.step(1)
            Jg = sim.fields(pic.FIELD_J)
            assert sim.diagnostics()["status_bits"] == 0
        errs[name] = float(np.max(np.abs(Jg - J64)))
    per_tile = w.n_particles / ((w.nx // 16) * (w.ny // 16))
    B_default = math.ceil(min(per_tile, 8192) / 256)
    B_capped = math.ceil(min(per_tile, 64 * 256) / 256)
    qt = abs(w.species[0].qtilde)
    n = _contributions_bound(w)
    # J units of the library: qtilde times a velocity (|v| < c = 1) per cell
    bound = {"fixed": n * 64 * B_default * qt / 2**30 / 2,
             "fixed_chunk_2^20": n * 64 * B_capped * qt / 2**30 / 2}
    print(f"{case}: max|J| {scale:.4e}; max|dJ|/max|J|: " +
          ", ".join(f"{k} {v / scale:.2e}" for k, v in errs.items()) +
          f"; fixed-point bound {bound['fixed'] / scale:.2e} (B = {B_default}), "
          f"capped chunk {bound['fixed_chunk_2^20'] / scale:.2e} (B = {B_capped})")
    assert errs["fp32"] <= 5e-6 * scale
    assert errs["fp32"] < errs["fixed"]
    for k in ("fixed", "fixed_chunk_2^20"):
        assert errs[k] <= bound[k] + 5e-6 * scale
