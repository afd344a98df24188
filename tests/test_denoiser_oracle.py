"""Pins of the denoiser oracle (CPU, FP64) against what mathematics fixes:
brute-force sums, an FFT circular correlation, adjoint identities, central
finite differences of the whole network's loss, closed forms of Adam, and the
bfloat16 rounding on hand-computed bit patterns."""
import numpy as np
import pytest

from oracle import denoiser as D


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


# ------------------------------------------------------------ bfloat16

def test_bf16_rounding_hand_computed():
    u = 2.0 ** -7      # spacing of bfloat16 numbers in [1, 2)
    cases = [
        (1.0, 1.0),
        (1.0 + u / 2, 1.0),                    # tie -> even (1.0)
        (1.0 + u + u / 2, 1.0 + 2 * u),        # tie -> even (1 + 2u)
        (1.0 + u / 2 + 2.0 ** -20, 1.0 + u),   # just above the tie
        (1.0 + u / 2 - 2.0 ** -20, 1.0),       # just below
        (-(1.0 + u + u / 2), -(1.0 + 2 * u)),
        (3.140625, 3.140625),                  # exactly representable (0x4049)
        (0.0, 0.0),
    ]
    for x, want in cases:
        assert D.bf16(np.array([x]))[0] == want, x


def test_bf16_is_the_nearest_of_its_neighbours():
    x = (_rng(1).standard_normal(20000) * 10.0 ** _rng(2).integers(-5, 5, 20000)).astype(np.float32)
    r = D.bf16(x)
    bits = x.view(np.uint32)
    lo = (bits & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)
    hi = ((bits & np.uint32(0xFFFF0000)) + np.uint32(0x10000)).view(np.float32).astype(np.float64)
    xd = x.astype(np.float64)
    assert np.all((r == lo) | (r == hi))
    assert np.all(np.abs(r - xd) <= np.minimum(np.abs(lo - xd), np.abs(hi - xd)) + 0.0)


# ------------------------------------------------------------ convolution

def test_conv3x3_brute_force():
    rng = _rng(3)
    B, H, W, Ci, Co = 2, 5, 4, 3, 2
    x = rng.standard_normal((B, H, W, Ci))
    w = rng.standard_normal((3, 3, Ci, Co))
    b = rng.standard_normal(Co)
    z = D.conv3x3(x, w, b)
    for bb in range(B):
        for y in range(H):
            for xx in range(W):
                for o in range(Co):
                    s = b[o]
                    for ky in range(3):
                        for kx in range(3):
                            for i in range(Ci):
                                s += x[bb, (y + ky - 1) % H, (xx + kx - 1) % W, i] * w[ky, kx, i, o]
                    assert abs(z[bb, y, xx, o] - s) < 1e-12


def test_conv3x3_against_fft_correlation():
    rng = _rng(4)
    B, H, W, Ci, Co = 1, 12, 10, 4, 3
    x = rng.standard_normal((B, H, W, Ci))
    w = rng.standard_normal((3, 3, Ci, Co))
    z = D.conv3x3(x, w)
    for o in range(Co):
        acc = np.zeros((H, W))
        for i in range(Ci):
            K = np.zeros((H, W))
            for ky in range(3):
                for kx in range(3):
                    K[(1 - ky) % H, (1 - kx) % W] = w[ky, kx, i, o]
            acc += np.real(np.fft.ifft2(np.fft.fft2(x[0, :, :, i]) * np.fft.fft2(K)))
        np.testing.assert_allclose(z[0, :, :, o], acc, atol=1e-11)


def test_dgrad_is_the_adjoint_of_conv():
    rng = _rng(5)
    x = rng.standard_normal((2, 6, 8, 5))
    w = rng.standard_normal((3, 3, 5, 7))
    dz = rng.standard_normal((2, 6, 8, 7))
    lhs = np.sum(D.conv3x3(x, w) * dz)
    rhs = np.sum(x * D.conv3x3_dgrad(dz, w))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_wgrad_is_the_gradient_of_the_pairing():
    rng = _rng(6)
    x = rng.standard_normal((2, 6, 8, 5))
    w = rng.standard_normal((3, 3, 5, 7))
    b = rng.standard_normal(7)
    dz = rng.standard_normal((2, 6, 8, 7))
    dw, db = D.conv3x3_wgrad(x, dz)
    # <conv(x; w, b), dz> is linear in (w, b): it equals <w, dw> + <b, db>
    lhs = np.sum(D.conv3x3(x, w, b) * dz)
    assert abs(lhs - (np.sum(w * dw) + np.sum(b * db))) < 1e-10 * abs(lhs)
    # and a single weight's derivative is a brute-force sum
    ky, kx, i, o = 2, 0, 3, 5
    s = sum(x[bb, (y + ky - 1) % 6, (xx + kx - 1) % 8, i] * dz[bb, y, xx, o]
            for bb in range(2) for y in range(6) for xx in range(8))
    assert abs(dw[ky, kx, i, o] - s) < 1e-11


def test_pool_and_upsample_adjoints():
    rng = _rng(7)
    x = rng.standard_normal((2, 8, 6, 3))
    d = rng.standard_normal((2, 4, 3, 3))
    assert abs(np.sum(D.pool2(x) * d) - np.sum(x * D.pool2_back(d))) < 1e-12
    x2 = rng.standard_normal((2, 4, 3, 3))
    d2 = rng.standard_normal((2, 8, 6, 3))
    assert abs(np.sum(D.up2(x2) * d2) - np.sum(x2 * D.up2_back(d2))) < 1e-12
    np.testing.assert_allclose(D.pool2(D.up2(x2)), x2)


# ------------------------------------------------------------ network

def _trained_looking_params(seed):
    p = D.init_params(seed)
    rng = _rng(seed + 1)
    p["c11.w"] = rng.uniform(-0.1, 0.1, p["c11.w"].shape)
    for name, *_ in D.LAYERS:
        p[name + ".b"] = rng.uniform(-0.05, 0.05, p[name + ".b"].shape)
    return p


def test_untrained_network_is_the_identity():
    p = D.init_params(11)
    x = _rng(12).standard_normal((2, 8, 8, 3))
    out, _ = D.forward(p, x)
    np.testing.assert_array_equal(out, x)


def test_flatten_round_trip_and_parameter_count():
    p = D.init_params(13)
    flat = D.flatten(p)
    assert flat.size == D.n_params()
    q = D.unflatten(flat)
    for k in p:
        np.testing.assert_array_equal(q[k], p[k])
    # 3x3 kernels of the 3-32-32 | 64-64 | 128-128 | 64-64 | 32-32-3 network
    want = sum(9 * ci * co + co for _, ci, co, *_ in D.LAYERS)
    assert want == D.n_params() == 426307


def test_network_gradient_matches_central_differences():
    """Every layer's weight and bias gradient (incl. the skips and the
    pool/upsample adjoints) against central differences of the FP64 loss."""
    p = _trained_looking_params(21)
    rng = _rng(22)
    x = rng.standard_normal((2, 16, 16, 3))
    t = x + 0.3 * rng.standard_normal((2, 16, 16, 3))
    L0, g, _ = D.loss_and_grads(p, x, t)
    h = 1e-6
    errs = []
    for name, shape in D.param_shapes():
        # entries with a non-zero gradient (a ReLU can switch a channel off)
        live = np.argwhere(np.abs(g[name]) > 1e-9)
        assert len(live) > len(g[name].reshape(-1)) // 4, name
        for j in rng.choice(len(live), min(4, len(live)), replace=False):
            idx = tuple(int(v) for v in live[j])
            q = {k: v.copy() for k, v in p.items()}
            q[name][idx] += h
            Lp = D.mse(D.forward(q, x)[0], t)[0]
            q[name][idx] -= 2 * h
            Lm = D.mse(D.forward(q, x)[0], t)[0]
            fd = (Lp - Lm) / (2 * h)
            an = g[name][idx]
            errs.append(abs(fd - an) / max(abs(fd), abs(an), 1e-7))
    errs = np.array(errs)
    assert np.median(errs) < 1e-6, errs
    assert np.max(errs) < 1e-3, errs


def test_backward_with_bf16_rounding_stays_close_to_fp64():
    p = _trained_looking_params(31)
    rng = _rng(32)
    x = rng.standard_normal((1, 8, 8, 3))
    t = x + 0.3 * rng.standard_normal((1, 8, 8, 3))
    _, g64, o64 = D.loss_and_grads(p, x, t)
    _, g16, o16 = D.loss_and_grads(p, x, t, rnd=D.bf16)
    assert np.max(np.abs(o16 - o64)) < 2e-2 * np.max(np.abs(o64))
    for k in g64:
        scale = np.max(np.abs(g64[k])) + 1e-12
        assert np.max(np.abs(g16[k] - g64[k])) < 0.1 * scale, k


# ------------------------------------------------------------ Adam

def test_adam_first_step_is_lr_times_sign():
    p = {"a": np.array([1.0, -2.0, 3.0, 0.5])}
    g = {"a": np.array([0.3, -4.0, 1e-3, -2.5])}
    opt = D.Adam(p, lr=0.01)
    q = opt.step({k: v.copy() for k, v in p.items()}, g)
    want = p["a"] - 0.01 * g["a"] / (np.abs(g["a"]) + 1e-8)
    np.testing.assert_allclose(q["a"], want, rtol=0, atol=1e-15)


def test_adam_converges_on_a_quadratic():
    c = np.array([1.5, -0.5, 2.0])
    a = np.array([1.0, 10.0, 0.1])
    p = {"x": np.zeros(3)}
    opt = D.Adam(p, lr=0.05)
    for _ in range(3000):
        g = {"x": 2 * a * (p["x"] - c)}
        p = opt.step(p, g)
    np.testing.assert_allclose(p["x"], c, atol=1e-3)


def test_library_parameter_layout_and_init_match_the_oracle():
    """The library's flat parameter vector (layer order, [ky][kx][cin][cout]
    weights then biases) and its seeded initialisation recipe agree with the
    oracle's, so parameters pass between them unchanged."""
    from paper_2501_14795_gb300 import denoise as dn
    assert dn.LAYERS == [(ci, co, lv) for _, ci, co, lv, _, _ in D.LAYERS]
    np.testing.assert_array_equal(dn.init_params(5), D.flatten(D.init_params(5)).astype(np.float32))
    assert dn.forward_flops(256, 256) == sum(2.0 * 65536 / 4 ** lv * 9 * ci * co
                                              for _, ci, co, lv, _, _ in D.LAYERS)


def _mode(H, W, mx, my):
    y, x = np.mgrid[0:H, 0:W]
    return np.cos(2 * np.pi * (mx * x / W + my * y / H) + 0.3)


@pytest.mark.parametrize("passes", [1, 3, 8])
def test_low_k_restore_gives_back_each_mode_by_the_closed_form_factor(passes):
    """raw - den a Fourier mode (mx, my) per component: the restoration adds it
    back times cos^2(pi mx / W)^n cos^2(pi my / H)^n (the response of n passes
    of the binomial stencil), on top of an arbitrary den."""
    H, W = 12, 20
    rng = np.random.default_rng(3)
    den = rng.normal(size=(2, 3, H, W))
    modes = [(1, 0), (3, 2), (7, 5)]
    diff = np.stack([_mode(H, W, mx, my) for mx, my in modes])
    raw = den + np.stack([diff, 2.0 * diff])
    out = D.low_k_restore(raw, den, passes)
    for c, (mx, my) in enumerate(modes):
        f = (np.cos(np.pi * mx / W) ** 2 * np.cos(np.pi * my / H) ** 2) ** passes
        for b, amp in enumerate((1.0, 2.0)):
            np.testing.assert_allclose(out[b, c] - den[b, c], amp * f * diff[c], rtol=0, atol=1e-12)


def test_low_k_restore_special_cases():
    H, W = 8, 16
    rng = np.random.default_rng(4)
    den = rng.normal(size=(3, H, W))
    raw = rng.normal(size=(3, H, W))
    # no passes: the network's output unchanged
    np.testing.assert_array_equal(D.low_k_restore(raw, den, 0), den)
    # a uniform difference is the k = 0 mode: given back whole
    np.testing.assert_allclose(D.low_k_restore(den + 0.7, den, 5), den + 0.7, rtol=0, atol=1e-12)
    # the Nyquist checkerboard along x is removed by one pass
    chk = np.broadcast_to((-1.0) ** np.arange(W), (3, H, W))
    np.testing.assert_allclose(D.low_k_restore(den + chk, den, 1), den, rtol=0, atol=1e-12)
