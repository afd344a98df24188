"""Plain CPU oracle of the learned current denoiser (numpy, FP64).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and ``bench.py``'s CPU legs,
never by the product library, and sharing no code with it.

The network is the small convolutional encoder-decoder applied to the
deposited current in the filter slot of the time loop (Listing 3.1: after the
guard-cell reduction of J, before the field solve), where the thesis applies
its binomial filter (Eq. 18 reading: a smoothing of J before the field
advance).  Everything here follows the textbook definitions:

* 3x3 convolution with periodic (circular) padding, written as a
  cross-correlation: z[b,y,x,o] = sum_{ky,kx,i} x[b,(y+ky-1)%H,(x+kx-1)%W,i]
  w[ky,kx,i,o] + bias[o] (arrays are NHWC, weights [ky][kx][cin][cout]);
* its input gradient (the adjoint: correlation with the flipped kernel) and
  its weight and bias gradients (sums of input x output-gradient products);
* ReLU, 2x2 mean pooling, 2x2 nearest upsampling and their adjoints;
* mean-squared-error loss and the Adam update (Kingma & Ba 2015, Algorithm 1,
  with the bias-corrected moments).

Precision: the GPU stores activations and the gradients it feeds to the tensor
cores as bfloat16 and accumulates in FP32.  ``forward``/``backward`` take a
rounding function ``rnd`` applied at exactly those storage points (``bf16`` to
mirror the GPU, ``ident`` for plain FP64 maths); everything else is FP64.

The optional low-wavenumber restoration after the network,
den + L^n (raw - den) with L the binomial current filter, is ``low_k_restore``.

Pins (``tests/test_denoiser_oracle.py``): brute-force loops on tiny inputs,
an FFT circular correlation, adjoint identities <A x, y> = <x, A^T y>, central
finite differences of the whole network's loss in FP64, the first Adam step
(-lr sign(g)) and Adam's convergence on a quadratic, the bfloat16 rounding
against hand-computed bit patterns; the restoration against the closed-form
response of a Fourier mode, a uniform difference (given back whole) and the
Nyquist checkerboard (removed by one pass).
"""
from __future__ import annotations

import numpy as np

# ------------------------------------------------------------ architecture
# (name, cin, cout, level, relu, skip source).  Level 0 is full resolution,
# each level halves both sides; "pool" / "up" mark resolution changes.
LAYERS = [
    ("c1", 3, 32, 0, True, None),
    ("c2", 32, 32, 0, True, None),      # -> s1
    ("c3", 32, 64, 1, True, None),      # after pool
    ("c4", 64, 64, 1, True, None),      # -> s2
    ("c5", 64, 128, 2, True, None),     # after pool
    ("c6", 128, 128, 2, True, None),
    ("c7", 128, 64, 1, True, "c4"),     # after up; + s2
    ("c8", 64, 64, 1, True, None),
    ("c9", 64, 32, 0, True, "c2"),      # after up; + s1
    ("c10", 32, 32, 0, True, None),
    ("c11", 32, 3, 0, False, None),     # residual: out = x + z11
]
POOL_AFTER = {"c2", "c4"}
UP_AFTER = {"c6", "c8"}


def param_shapes():
    out = []
    for name, ci, co, *_ in LAYERS:
        out.append((name + ".w", (3, 3, ci, co)))
        out.append((name + ".b", (co,)))
    return out


def n_params():
    return sum(int(np.prod(s)) for _, s in param_shapes())


def unflatten(flat):
    flat = np.asarray(flat, np.float64)
    p, k = {}, 0
    for name, shape in param_shapes():
        n = int(np.prod(shape))
        p[name] = flat[k:k + n].reshape(shape)
        k += n
    assert k == flat.size
    return p


def flatten(p):
    return np.concatenate([np.asarray(p[name], np.float64).reshape(-1) for name, _ in param_shapes()])


def init_params(seed):
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases; the last layer
    starts at zero so the untrained network is the identity."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = {}
    for name, ci, co, *_ in LAYERS:
        bound = np.sqrt(6.0 / (9 * ci))
        w = rng.uniform(-bound, bound, (3, 3, ci, co))
        if name == "c11":
            w[...] = 0.0
        p[name + ".w"] = w
        p[name + ".b"] = np.zeros(co)
    return p


# ------------------------------------------------------------ rounding

def ident(x):
    return np.asarray(x, np.float64)


def bf16(x):
    """Round to the nearest bfloat16 (ties to even) via the float32 bit
    pattern: add 0x7fff plus the lowest kept bit, drop the low 16 bits."""
    f = np.ascontiguousarray(np.asarray(x, np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


# ------------------------------------------------------------ primitives

def conv3x3(x, w, b=None):
    """Circular 3x3 cross-correlation, NHWC; np.roll + matrix products."""
    x = np.asarray(x, np.float64)
    B, H, W, Ci = x.shape
    Co = w.shape[3]
    z = np.zeros((B, H, W, Co))
    for ky in range(3):
        for kx in range(3):
            xs = np.roll(x, shift=(-(ky - 1), -(kx - 1)), axis=(1, 2))  # xs[y,x] = x[y+ky-1, x+kx-1]
            z += (xs.reshape(-1, Ci) @ w[ky, kx]).reshape(B, H, W, Co)
    if b is not None:
        z += b
    return z


def conv3x3_dgrad(dz, w):
    """Input gradient of conv3x3: dx[y,x,i] = sum dz[y-ky+1, x-kx+1, o] w[ky,kx,i,o]."""
    dz = np.asarray(dz, np.float64)
    B, H, W, Co = dz.shape
    Ci = w.shape[2]
    dx = np.zeros((B, H, W, Ci))
    for ky in range(3):
        for kx in range(3):
            ds = np.roll(dz, shift=(ky - 1, kx - 1), axis=(1, 2))   # ds[y,x] = dz[y-ky+1, x-kx+1]
            dx += (ds.reshape(-1, Co) @ w[ky, kx].T).reshape(B, H, W, Ci)
    return dx


def conv3x3_wgrad(x, dz):
    """Weight and bias gradients: dw[ky,kx,i,o] = sum x[y+ky-1,x+kx-1,i] dz[y,x,o]."""
    x = np.asarray(x, np.float64)
    dz = np.asarray(dz, np.float64)
    Ci, Co = x.shape[3], dz.shape[3]
    dw = np.zeros((3, 3, Ci, Co))
    dzf = dz.reshape(-1, Co)
    for ky in range(3):
        for kx in range(3):
            xs = np.roll(x, shift=(-(ky - 1), -(kx - 1)), axis=(1, 2))
            dw[ky, kx] = xs.reshape(-1, Ci).T @ dzf
    return dw, dzf.sum(axis=0)


def pool2(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool2_back(d):
    return np.repeat(np.repeat(d, 2, axis=1), 2, axis=2) / 4.0


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_back(d):
    B, H, W, C = d.shape
    return d.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def mse(out, target):
    d = np.asarray(out, np.float64) - np.asarray(target, np.float64)
    return float(np.mean(d * d)), 2.0 * d / d.size


# ------------------------------------------------------------ network

def forward(p, x, rnd=ident):
    """x: normalised noisy current (B, H, W, 3).  Returns (out, cache), out =
    x + z11.  Stored tensors (conv outputs after ReLU and skip, pooled and
    upsampled tensors, the conv input) pass through ``rnd``."""
    cache = {"x": np.asarray(x, np.float64)}
    h = rnd(x)
    cache["in.c1"] = h
    acts = {}
    for name, ci, co, lev, relu, skip in LAYERS:
        w = rnd(p[name + ".w"])
        z = conv3x3(h, w, p[name + ".b"])
        if name == "c11":
            out = cache["x"] + z
            cache["out"] = out
            break
        a = rnd(np.maximum(z, 0.0)) if relu else rnd(z)
        cache["a." + name] = a
        y = rnd(a + acts[skip]) if skip else a
        acts[name] = y
        h = y
        if name in POOL_AFTER:
            h = rnd(pool2(h))
        elif name in UP_AFTER:
            h = up2(h)
        nxt = LAYERS[[l[0] for l in LAYERS].index(name) + 1][0]
        cache["in." + nxt] = h
    return cache["out"], cache


def backward(p, cache, dout, rnd=ident):
    """Gradients of the loss given dL/dout (FP64 except the operands the GPU
    feeds to its tensor cores: dz is rounded with ``rnd``)."""
    g = {}
    names = [l[0] for l in LAYERS]
    skip_of = {l[0]: l[5] for l in LAYERS}
    relu_of = {l[0]: l[4] for l in LAYERS}
    dskip = {}
    dy = np.asarray(dout, np.float64)       # gradient w.r.t. the output of the current layer
    for k in range(len(LAYERS) - 1, -1, -1):
        name = names[k]
        if name == "c11":
            dzr = dy
        else:
            if name in dskip:                # this layer's output also feeds a skip
                dy = dy + dskip.pop(name)
            dzr = dy * (cache["a." + name] > 0) if relu_of[name] else dy
            if skip_of[name]:
                dskip[skip_of[name]] = dy    # y = a + skip: the skip gets dy
        dz = rnd(dzr)
        dw, _ = conv3x3_wgrad(cache["in." + name], dz)
        g[name + ".w"] = dw
        g[name + ".b"] = dzr.reshape(-1, dzr.shape[-1]).sum(axis=0)
        if k == 0:
            break
        dh = conv3x3_dgrad(dz, rnd(p[name + ".w"]))
        prev = names[k - 1]
        if prev in POOL_AFTER:
            dh = pool2_back(dh)
        elif prev in UP_AFTER:
            dh = up2_back(dh)
        dy = dh
    return g


def loss_and_grads(p, x, target, rnd=ident):
    out, cache = forward(p, x, rnd)
    L, dout = mse(out, target)
    return L, backward(p, cache, dout, rnd), out


# ------------------------------------------------------------ restoration

def low_k_restore(raw, den, passes):
    """Low-wavenumber restoration after the network: den + L^passes (raw - den),
    L one pass of the periodic binomial smoothing of the time loop's current
    filter (``binomial_filter``: (1/4, 1/2, 1/4) along x, then along y).
    Arrays [..., 3, H, W] (field layout); FP64.  passes = 0 means no
    restoration (the network's output), not L^0 = identity."""
    from .oracle import binomial_filter
    raw = np.asarray(raw, np.float64)
    den = np.asarray(den, np.float64)
    if passes == 0:
        return den.copy()
    diff = (raw - den).reshape((-1,) + raw.shape[-3:])
    back = np.stack([binomial_filter(v, passes) for v in diff]).reshape(raw.shape)
    return den + back


# ------------------------------------------------------------ Adam

class Adam:
    """Kingma & Ba (2015), Algorithm 1, with bias-corrected moments."""

    def __init__(self, p, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = {k: np.zeros_like(v) for k, v in p.items()}
        self.v = {k: np.zeros_like(v) for k, v in p.items()}
        self.t = 0

    def step(self, p, g):
        self.t += 1
        for k in p:
            self.m[k] = self.b1 * self.m[k] + (1 - self.b1) * g[k]
            self.v[k] = self.b2 * self.v[k] + (1 - self.b2) * g[k] * g[k]
            mh = self.m[k] / (1 - self.b1 ** self.t)
            vh = self.v[k] / (1 - self.b2 ** self.t)
            p[k] = p[k] - self.lr * mh / (np.sqrt(vh) + self.eps)
        return p
