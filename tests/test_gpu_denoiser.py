"""The denoiser's GPU kernels against the CPU oracle (``oracle/denoiser.py``).

Both sides round to bfloat16 at the same points (conv inputs, weights, stored
activations, dz), so they differ only by FP32 vs FP64 accumulation:
* convolution forward: the bfloat16 outputs agree to one bfloat16 step
  (2^-7 relative), nearly all exactly;
* input and weight gradients (FP32 outputs): within 1e-5 of the largest value
  (a sum of at most 9*128 or a few 10^4 products, FP32 accumulation);
* whole network: loss to 1e-3 relative, every parameter gradient within a few
  percent of its tensor's largest entry (rounding flips of the activations
  propagate), most much closer;
* Adam: the GPU's parameters after one step equal p - lr g / (|g| + eps);
* in the current-filter slot: the identity network changes nothing, a
  trained-looking one runs and its continuity residual is reported.
"""
import numpy as np
import pytest

from oracle import denoiser as D
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


def _rng(s):
    return np.random.Generator(np.random.PCG64(s))


def _bf16_tensor(a):
    """numpy FP64 values (already bfloat16-representable) -> CUDA bfloat16 tensor."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).cuda()


def _f32(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _np(t):
    import torch
    return t.float().cpu().numpy().astype(np.float64) if t.dtype == torch.bfloat16 else \
        t.cpu().numpy().astype(np.float64)


def _pad(x, c):
    out = np.zeros(x.shape[:-1] + (c,))
    out[..., :x.shape[-1]] = x
    return out


# rows of 32 run on the mma.sync kernel, rows of 128 on the tcgen05 kernel
SHAPES = [(2, 16, 32), (1, 8, 128)]


@pytest.mark.parametrize("B,H,W", SHAPES)
@pytest.mark.parametrize("cin,cout,relu,skip", [(3, 32, True, False), (32, 32, True, True),
                                                 (32, 64, True, False), (64, 128, True, False),
                                                 (128, 128, True, False), (128, 64, True, True),
                                                 (64, 32, False, False), (64, 64, True, True)])
def test_conv_forward_matches_oracle(cin, cout, relu, skip, B, H, W):
    import torch
    rng = _rng(cin * 1000 + cout)
    x = D.bf16(rng.standard_normal((B, H, W, cin)))
    w = rng.uniform(-1, 1, (3, 3, cin, cout)) * np.sqrt(3.0 / (9 * cin))
    b = rng.uniform(-0.1, 0.1, cout)
    s = D.bf16(rng.standard_normal((B, H, W, cout))) if skip else None
    cpad = (cin + 15) // 16 * 16
    xt = _bf16_tensor(_pad(x, cpad))
    a = torch.empty((B, H, W, cout), dtype=torch.bfloat16, device="cuda")
    y = torch.empty_like(a) if skip else None
    pic.pic_nn_conv3x3(xt, _f32(w), _f32(b), a, relu=relu,
                       skip=_bf16_tensor(s) if skip else None, y_out=y)
    z = D.conv3x3(x, D.bf16(w), b.astype(np.float32).astype(np.float64))
    ref_a = D.bf16(np.maximum(z, 0) if relu else z)
    got_a = _np(a)
    step = np.abs(ref_a) * 2.0 ** -7 + 1e-30
    assert np.all(np.abs(got_a - ref_a) <= step + 1e-6)
    assert np.mean(got_a == ref_a) > 0.99
    if skip:
        ref_y = D.bf16(got_a + s)          # the same rounding applied to the GPU's own a
        np.testing.assert_array_equal(_np(y), ref_y)


@pytest.mark.parametrize("B,H,W", SHAPES)
@pytest.mark.parametrize("cin,cout", [(32, 3), (32, 32), (32, 64), (64, 64), (64, 128),
                                      (128, 128), (128, 64)])
def test_conv_input_gradient_matches_oracle(cin, cout, B, H, W):
    import torch
    rng = _rng(cin * 7 + cout)
    dz = D.bf16(rng.standard_normal((B, H, W, cout)))
    w = rng.uniform(-1, 1, (3, 3, cin, cout)) * 0.1
    dx = torch.empty((B, H, W, cin), dtype=torch.float32, device="cuda")
    pic.pic_nn_conv3x3_dgrad(_bf16_tensor(_pad(dz, (cout + 15) // 16 * 16)), _f32(w), dx)
    ref = D.conv3x3_dgrad(dz, D.bf16(w))
    got = _np(dx)
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))


@pytest.mark.parametrize("B,H,W", [(2, 16, 32), (1, 8, 128), (3, 16, 16)])
@pytest.mark.parametrize("cin,cout", [(3, 32), (32, 32), (32, 64), (64, 64), (64, 128),
                                      (128, 128), (128, 64), (64, 32), (32, 3)])
def test_conv_weight_gradient_matches_oracle(cin, cout, B, H, W):
    """Tiles of 64, 32 and 16 columns (the widest dividing W), several tiles
    per CTA and the circular edge on both axes."""
    import torch
    rng = _rng(cin * 13 + cout)
    x = D.bf16(rng.standard_normal((B, H, W, cin)))
    dz = D.bf16(rng.standard_normal((B, H, W, cout)))
    dw = torch.empty((3, 3, cin, cout), dtype=torch.float32, device="cuda")
    pic.pic_nn_conv3x3_wgrad(_bf16_tensor(_pad(x, (cin + 15) // 16 * 16)),
                             _bf16_tensor(_pad(dz, (cout + 15) // 16 * 16)), dw)
    ref, _ = D.conv3x3_wgrad(x, dz)
    got = _np(dw)
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))


def _params(seed):
    p = D.init_params(seed)
    rng = _rng(seed + 1)
    p["c11.w"] = rng.uniform(-0.05, 0.05, p["c11.w"].shape)
    for name, *_ in D.LAYERS:
        p[name + ".b"] = rng.uniform(-0.05, 0.05, p[name + ".b"].shape)
    return p


def _flat32(p):
    return D.flatten(p).astype(np.float32)


def _currents(seed, B, ny, nx):
    rng = _rng(seed)
    Jc = np.zeros((B, 3, ny, nx))
    yy, xx = np.mgrid[0:ny, 0:nx]
    for b in range(B):
        for c in range(3):
            Jc[b, c] = np.sin(2 * np.pi * (rng.integers(1, 3) * xx / nx + rng.random())) * \
                np.cos(2 * np.pi * (rng.integers(1, 3) * yy / ny + rng.random()))
    Jn = Jc + 0.5 * rng.standard_normal(Jc.shape)
    return Jn.astype(np.float32), Jc.astype(np.float32)


def _nhwc(J):
    return np.transpose(J, (0, 2, 3, 1)).astype(np.float64)


@pytest.mark.parametrize("ny,nx,tc", [(32, 64, None), (32, 256, None), (32, 256, "always"),
                                      (32, 512, "always"), (32, 64, "never")])
def test_network_loss_and_gradients_match_oracle(ny, nx, tc, monkeypatch):
    """tc: PIC_DENOISER_TC=always puts every 128-wide row layer on the tcgen05
    kernels (at nx = 256 c9, at nx = 512 c7 and c9 as four 2x2 convolutions of
    the coarse grid), =never keeps every layer (the weight gradients included)
    on the mma.sync kernels."""
    if tc:
        monkeypatch.setenv("PIC_DENOISER_TC", tc)
    B, scale = 2, 0.5
    Jn, Jc = _currents(5, B, ny, nx)
    p = _params(41)
    flat = _flat32(p)
    with pic.Denoiser(nx, ny, B, scale) as net:
        net.set_params(flat)
        g = np.empty(D.n_params(), np.float32)
        loss = net.grad(Jn, Jc, g)
        out = net.forward(Jn)
    p32 = D.unflatten(flat.astype(np.float64))
    L, gref, oref = D.loss_and_grads(p32, _nhwc(Jn) / scale, _nhwc(Jc) / scale, rnd=D.bf16)
    assert abs(loss - L) <= 1e-3 * L
    np.testing.assert_allclose(_nhwc(out), oref * scale, rtol=0, atol=2e-2 * np.max(np.abs(oref)))
    gg = D.unflatten(g.astype(np.float64))
    worst = 0.0
    for k in gref:
        scale_k = np.max(np.abs(gref[k])) + 1e-12
        err = np.max(np.abs(gg[k] - gref[k])) / scale_k
        rel2 = np.linalg.norm(gg[k] - gref[k]) / (np.linalg.norm(gref[k]) + 1e-30)
        worst = max(worst, err)
        assert err < 5e-2 and rel2 < 2e-2, (k, err, rel2)


def test_adam_step_on_the_gpu():
    B, ny, nx = 1, 32, 64
    Jn, Jc = _currents(6, B, ny, nx)
    flat = _flat32(_params(42))
    with pic.Denoiser(nx, ny, B, 1.0) as net:
        net.set_params(flat)
        g = np.empty(D.n_params(), np.float32)
        net.grad(Jn, Jc, g)
        net.train_step(Jn, Jc, lr=1e-3)
        after = net.params()
    g64 = g.astype(np.float64)
    want = flat - 1e-3 * g64 / (np.abs(g64) + 1e-8)
    np.testing.assert_allclose(after, want, rtol=0, atol=2e-6 * np.max(np.abs(flat)) + 1e-7)


def test_training_reduces_the_loss():
    B, ny, nx = 4, 32, 64
    Jn, Jc = _currents(7, B, ny, nx)
    p = D.init_params(43)
    with pic.Denoiser(nx, ny, B, 1.0) as net:
        net.set_params(_flat32(p))
        first = net.grad(Jn, Jc)
        for _ in range(60):
            last = net.train_step(Jn, Jc, lr=2e-3)
        last = net.grad(Jn, Jc)
    assert last < 0.5 * first, (first, last)


def test_identity_network_in_the_filter_slot_changes_nothing():
    w = wl.two_stream(nx=64, ny=32, k=2, u_th=0.1, drift=0.2, tile=16, seed=9)
    with pic.Simulation.from_workload(w, device=True) as a, \
            pic.Simulation.from_workload(w, device=True) as b, \
            pic.Denoiser(64, 32, 1, 0.01) as net:
        pic.pic_set_denoiser(b.h, net.d)      # parameters zero: the identity
        a.step(20)
        b.step(20)
        da, db = a.diagnostics(), b.diagnostics()
        assert db["status_bits"] == 0
        np.testing.assert_allclose(db["w_e"], da["w_e"], rtol=1e-4, atol=1e-12)
        np.testing.assert_allclose(db["w_k"], da["w_k"], rtol=1e-6)
        net.set_params(_flat32(_params(44)))
        b.step(5)
        d2 = b.diagnostics()
        assert d2["status_bits"] == 0 and np.isfinite(d2["w_e"])
        pic.pic_set_denoiser(b.h, None)
        b.step(1)
        assert b.diagnostics()["status_bits"] == 0


# ---- low-wavenumber restoration after the network ---------------------------

@pytest.mark.parametrize("passes,H,W", [(0, 24, 40), (1, 24, 40), (2, 24, 40), (5, 70, 300),
                                         (64, 8, 12)])
def test_low_k_restore_kernels_match_oracle(passes, H, W):
    """out + L^n (raw - out) on ragged lattices (not multiples of the kernels'
    tiles; 8 x 12 with 64 passes wraps the halo several times), FP32 on the GPU
    (the (2n+1)-tap binomial kernel) against the FP64 oracle (n passes of the
    3-point stencil)."""
    B = 2
    rng = _rng(60 + passes)
    raw = rng.normal(size=(B, 3, H, W))
    out = rng.normal(size=(B, 3, H, W))
    r, o = _f32(raw), _f32(out)
    pic.pic_nn_low_k_restore(r, o, passes)
    want = D.low_k_restore(raw.astype(np.float32), out.astype(np.float32), passes)
    np.testing.assert_allclose(_np(o), want, rtol=0, atol=2e-6 * np.max(np.abs(want)))


def _bias_only(b):
    """parameters whose network output is x + b (per component): all zero but c11's bias"""
    p = D.unflatten(np.zeros(D.n_params()))
    p["c11.b"] = np.asarray(b, np.float64)
    return _flat32(p)


def test_restoration_gives_back_a_uniform_correction():
    """A network that only adds a constant per component moves the k = 0 mode
    alone, which the restoration gives back whole: out = x for n >= 1, and
    out = x + scale * b without it (host buffers, and device in place)."""
    import torch
    B, ny, nx, scale = 2, 32, 64, 0.5
    Jn, _ = _currents(8, B, ny, nx)
    Jn = Jn.astype(np.float32)
    b = np.array([0.3, -0.2, 0.1])
    with pic.Denoiser(nx, ny, B, scale) as net:
        net.set_params(_bias_only(b))
        plain = net.forward(Jn)
        np.testing.assert_allclose(plain, Jn + scale * b[None, :, None, None], rtol=0, atol=1e-6)
        net.set_low_k_restore(3)
        back = net.forward(Jn)
        np.testing.assert_allclose(back, Jn, rtol=0, atol=2e-6)
        t = _f32(Jn)
        net.forward(t, t)                  # in place on the device
        np.testing.assert_allclose(_np(t), Jn, rtol=0, atol=2e-6)
        with pytest.raises(pic.PicError):
            net.set_low_k_restore(-1)
        with pytest.raises(pic.PicError):
            net.set_low_k_restore(65)
        torch.cuda.synchronize()


def test_restoration_in_the_filter_slot():
    """In the current-filter slot, the constant-adding network with the
    restoration steps like the unfiltered simulation; without it, it does not."""
    w = wl.two_stream(nx=64, ny=32, k=2, u_th=0.1, drift=0.2, tile=16, seed=9)
    with pic.Simulation.from_workload(w, device=True) as a, \
            pic.Simulation.from_workload(w, device=True) as b, \
            pic.Simulation.from_workload(w, device=True) as c, \
            pic.Denoiser(64, 32, 1, 0.1) as net, pic.Denoiser(64, 32, 1, 0.1) as net0:
        net.set_params(_bias_only([0.5, -0.5, 0.25]))
        net.set_low_k_restore(2)
        net0.set_params(_bias_only([0.5, -0.5, 0.25]))
        pic.pic_set_denoiser(b.h, net.d)
        pic.pic_set_denoiser(c.h, net0.d)
        for s in (a, b, c):
            s.step(20)
        da, db, dc = a.diagnostics(), b.diagnostics(), c.diagnostics()
        assert db["status_bits"] == 0 and dc["status_bits"] == 0
        np.testing.assert_allclose(db["w_e"], da["w_e"], rtol=1e-4, atol=1e-12)
        np.testing.assert_allclose(db["w_k"], da["w_k"], rtol=1e-6)
        assert abs(dc["w_e"] - da["w_e"]) > 1e-2 * da["w_e"]
