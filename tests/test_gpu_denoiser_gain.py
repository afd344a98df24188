"""What the trained denoiser gains over the method without it (GPU).

Pairs come from 64-ppc two-stream runs (current of all particles vs current of
the fixed 1/16 subsample with 16x charge, at the same step); the network is
trained on the GPU by the library's own forward/backward kernels and Adam, and
evaluated on pairs from draws it never saw:
* the denoised subsample current is much closer to the 64-ppc current than the
  raw subsample current (mean squared error at most half);
* in the filter slot of a true 4-ppc run it keeps the run stable and its
  current's continuity residual is reported (the network does not conserve
  charge exactly: the residual is finite and non-zero).
"""
import numpy as np
import pytest

from oracle import denoiser as D
from paper_2501_14795_gb300 import denoise as dn
from paper_2501_14795_gb300 import pic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_14795_gb300 import build
    build.build_library()


def test_trained_denoiser_beats_the_raw_low_ppc_current():
    nx = ny = 128
    Jn, Jc = dn.make_pairs(dn.draws(3), nx, ny, steps=300, every=5)
    Vn, Vc = dn.make_pairs(dn.draws(1, offset=500), nx, ny, steps=300, every=20)
    scale = float(Jc.pow(2).mean().sqrt())
    with pic.Denoiser(nx, ny, 8, scale) as net:
        net.set_params(D.flatten(D.init_params(7)).astype(np.float32))
        raw0, den0 = dn.mse_gain(net, Vn, Vc, 8)
        assert den0 == pytest.approx(raw0, rel=1e-6)      # untrained: the identity
        losses = dn.train(net, Jn, Jc, 400, 8, lr=1e-3, lr_min=1e-4, seed=1)
        raw, den = dn.mse_gain(net, Vn, Vc, 8)
        assert np.mean(losses[-50:]) < 0.5 * losses[0]
        assert den < 0.5 * raw, (raw, den)

        w = dn.workload(dn.draws(1, offset=500)[0], nx, ny, k=2, steps=100)
        we, ms, diag, _ = dn.field_energy_run(w, 100, net)
        assert diag["status_bits"] == 0
        assert np.all(np.isfinite(we)) and ms > 0
        assert np.isfinite(diag["continuity_max"]) and diag["continuity_max"] > 0
