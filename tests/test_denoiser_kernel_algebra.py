"""CPU checks (FP64) of the exact identities the denoiser's tensor-core
kernels are built on, against the oracle's primitives:

* a 3x3 circular convolution of the nearest 2x upsampling of x equals, for
  each parity (a, b) of the output pixel (2i + a, 2j + b), a 2x2 convolution
  of x over the pixels (i + u, j + v), u in {a - 1, a}, v in {b - 1, b},
  whose weights are the sums of the 3x3 taps (dy, dx) with
  floor((a + dy) / 2) = u and floor((b + dx) / 2) = v (the upsampling
  layers' sixteen combined taps);
* the weight gradient with the kx taps side by side: for output row r and
  patch column q, sum over q of patch[r + ky][q][ci] dz[r][q - kx][co] equals
  the oracle's dW[ky][kx][ci][co] (dz shifted right by kx pixels, zero
  outside the row's tile; here the tile is the whole circular row);
* the output layer as one GEMM per input row with the nine taps in N: the sum
  over taps of D_{y+ky-1}[x + kx - 1][(ky, kx, co)], D_r[p][(tap, co)] =
  sum over ci of a[r][p][ci] w[tap][ci][co], equals the convolution.

A wrong tap table, a swapped parity or a shift of the wrong sign fails one of
them."""
import numpy as np

from oracle import denoiser as D


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _taps(a, uu):
    """Offsets dy whose upsampled row lands on coarse row i + u for parity a,
    u = a - 1 + uu."""
    u = a - 1 + uu
    return [dy for dy in (-1, 0, 1) if (a + dy) // 2 == u]


def test_tap_table_partitions_the_three_offsets():
    for a in (0, 1):
        got = sorted(_taps(a, 0) + _taps(a, 1))
        assert got == [-1, 0, 1]
    assert _taps(0, 0) == [-1] and _taps(0, 1) == [0, 1]
    assert _taps(1, 0) == [-1, 0] and _taps(1, 1) == [1]


def test_upsampled_conv_is_four_2x2_convolutions_of_the_coarse_grid():
    rng = _rng(3)
    B, Hc, Wc, Ci, Co = 2, 5, 7, 4, 3
    x = rng.standard_normal((B, Hc, Wc, Ci))
    w = rng.standard_normal((3, 3, Ci, Co))
    want = D.conv3x3(D.up2(x), w)
    got = np.zeros_like(want)
    for a in (0, 1):
        for b in (0, 1):
            acc = np.zeros((B, Hc, Wc, Co))
            for uu in (0, 1):
                for vv in (0, 1):
                    u, v = a - 1 + uu, b - 1 + vv
                    wc = sum(w[dy + 1, dx + 1] for dy in _taps(a, uu) for dx in _taps(b, vv))
                    xs = np.roll(x, shift=(-u, -v), axis=(1, 2))   # xs[i, j] = x[i + u, j + v]
                    acc += (xs.reshape(-1, Ci) @ wc).reshape(B, Hc, Wc, Co)
            got[:, a::2, b::2, :] = acc
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.max(np.abs(want)))


def test_weight_gradient_with_the_kx_taps_in_n():
    rng = _rng(5)
    B, H, W, Ci, Co = 2, 6, 8, 3, 4
    x = rng.standard_normal((B, H, W, Ci))
    dz = rng.standard_normal((B, H, W, Co))
    want, _ = D.conv3x3_wgrad(x, dz)
    got = np.zeros_like(want)
    for ky in range(3):
        xr = np.roll(x, shift=-(ky - 1), axis=1)             # rows y + ky - 1
        for kx in range(3):
            # patch column q = x + kx - 1 (circular); dz shifted right by kx
            # pixels is dz at column q - kx + 1 = x
            dzs = np.roll(dz, shift=kx - 1, axis=2)           # dzs[..., q, :] = dz[..., q - kx + 1, :]
            got[ky, kx] = xr.reshape(-1, Ci).T @ dzs.reshape(-1, Co)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.max(np.abs(want)))


def test_output_layer_as_one_gemm_per_row_with_the_taps_in_n():
    rng = _rng(7)
    B, H, W, Ci, Co = 1, 6, 9, 5, 3
    a = rng.standard_normal((B, H, W, Ci))
    w = rng.standard_normal((3, 3, Ci, Co))
    want = D.conv3x3(a, w)
    wn = np.concatenate([w[ky, kx] for ky in range(3) for kx in range(3)], axis=1)  # [ci][(tap, co)]
    Dr = (a.reshape(-1, Ci) @ wn).reshape(B, H, W, 9, Co)   # D_r[p][(tap, co)] per input row
    got = np.zeros_like(want)
    for ky in range(3):
        for kx in range(3):
            # input row y + ky - 1 and column x + kx - 1 of D, the tap's column block
            got += np.roll(Dr[..., 3 * ky + kx, :], shift=(-(ky - 1), -(kx - 1)), axis=(1, 2))
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.max(np.abs(want)))
