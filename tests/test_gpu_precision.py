"""The precision split: particle state and deposit in FP32, the global energy
and charge-conservation reductions in FP64 on the GPU.  Each reduced quantity
is compared, on the same state, with the FP64 oracle's evaluation (numpy FP64
over the fetched FP32 arrays for grid quantities; the FP32 oracle's push,
bit-identical to the strict build, accumulated in FP64 for the kinetic
energy), and its error is printed per quantity (run with -s to see them).
Bounds: the FP64 sums lose no more than the FP32 rounding of one thread's
partial (a few cells or particles: below 4e-7 relative, where an all-FP32
sum of the 65,536 cells would lose about 1e-7 x sqrt(cells) = 3e-5), and
the residual maxima agree with numpy's FP64 evaluation to 1e-9."""
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


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def test_fp64_reductions_against_the_fp64_oracle_per_quantity():
    w = wl.thermal_seeded(nx=256, ny=256, k=4, u_th=0.2, amp=1e-2, tile=16)
    dx, dy, dt = w.dx, w.dy, w.dt
    with pic.Simulation.from_workload(w, flags=pic.PIC_STRICT_FP | pic.PIC_TRACK_IDS) as sim:
        sim.step(20)
        state = sim.particles(0, ids=True)
        E0, B0 = sim.fields(pic.FIELD_E), sim.fields(pic.FIELD_B)
        d0 = sim.diagnostics()
        rho0 = sim.fields(pic.FIELD_RHO)
        sim.step(1)
        d1 = sim.diagnostics()
        E1, B1 = sim.fields(pic.FIELD_E), sim.fields(pic.FIELD_B)
        J1 = sim.fields(pic.FIELD_J)
        rho1 = sim.fields(pic.FIELD_RHO)
    errs = {}
    # field energies of level 21: FP64 sums over the FP32 fields
    errs["W_E"] = _rel(d1["w_e"], oracle.field_energy(E1, dx, dy))
    errs["W_B"] = _rel(d1["w_b"], oracle.field_energy(B1, dx, dy))
    # kinetic energy of the push from level 20: the FP32 oracle's push of the
    # same particles is bit-identical to the strict build; it accumulates in FP64
    s = w.species[0]
    sp = oracle.SpeciesState(s.q_over_m, s.qtilde, state["ix"], state["iy"], state["x"],
                             state["y"], state["ux"], state["uy"], state["uz"])
    o = oracle.OracleSim(w.nx, w.ny, dx, dy, dt, w.tile, [sp], dtype=np.float32,
                         background=w.background, E=E0, B=B0)
    o.step(1)
    errs["W_K"] = _rel(d1["w_k"], o.ke_history[-1])
    # charge and the residuals of level 21, in FP64: rho from the oracle's
    # particles (bit-identical to the GPU's), E and J the fetched FP32 arrays
    rho_np = oracle.rho_nodes(w.nx, w.ny, [o.species[0].astype(np.float64)], np.float64,
                              w.background)
    rho_prev = oracle.rho_nodes(w.nx, w.ny, [sp.astype(np.float64)], np.float64, w.background)
    assert np.max(np.abs(rho_np - rho1)) < 1e-6 and np.max(np.abs(rho_prev - rho0)) < 1e-6
    qscale = np.max(np.abs(rho_np - w.background))
    errs["charge_total"] = abs(d1["charge_total"] - float(rho_np.sum()) * dx * dy) / (
        abs(s.qtilde) * s.n * dx * dy)
    gauss = np.max(np.abs(oracle.div_e(E1, dx, dy) - rho_np))
    errs["gauss_max"] = abs(d1["gauss_max"] - gauss) / qscale
    cont = np.max(np.abs((rho_np - rho_prev) / dt + oracle.div_j(J1, dx, dy)))
    jscale = np.max(np.abs(J1)) / dx
    errs["continuity_max"] = abs(d1["continuity_max"] - cont) / jscale
    print("\nFP64 reductions vs FP64 evaluation, relative errors:",
          {k: float(f"{v:.2e}") for k, v in errs.items()},
          f"(continuity residual itself {d1['continuity_max'] / jscale:.2e} of max|div J| scale)")
    assert errs["W_E"] < 4e-7 and errs["W_B"] < 4e-7   # per-thread FP32 partials of 2 cells
    assert errs["W_K"] < 1e-6           # per-thread FP32 partials of <= 16 particles, FP64 after
    assert errs["charge_total"] < 1e-9
    # the residual maxima: FP64 on both sides, over the same values
    assert errs["gauss_max"] < 1e-9 and errs["continuity_max"] < 1e-9
    assert d1["continuity_max"] < 1e-5 * jscale
    assert abs(d1["gauss_max"] - d0["gauss_max"]) < 1e-5 * qscale
