"""Training pairs, training loop and in-loop evaluation of the current denoiser.

Pairs follow the "matched physics" reading: one high-ppc (8x8 lattice, 64
ppc) two-stream run per draw; at sampled steps the current of that step is
deposited twice from the same particles and fields: by all particles (the
target) and by a fixed 1/16 subsample carrying 16x the charge (the input,
statistically a 4-ppc deposit).  The subsample is the 2x2 sub-lattice of
sites (a, b) in {2, 5}^2 of each cell's 8x8 lattice, so it has the 4-ppc
lattice's beam pattern.  Everything runs through the library's C ABI on the
GPU; torch only gathers device buffers.

The two-stream draws: drift ~ U[0.1, 0.4], thermal spread u_th ~ U[0.02, 0.1],
one seed per draw; training and evaluation seeds are disjoint.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np

from . import pic
from . import workloads as wl

SEED_DENOISER = (wl.SEED_BASE + 5) * 1000
SUB_SITES = (2, 5)      # sub-lattice of the 8x8 lattice kept in the 1/16 subsample

# (cin, cout, level) of the convolutions c1..c11 (the library's network)
LAYERS = [(3, 32, 0), (32, 32, 0), (32, 64, 1), (64, 64, 1), (64, 128, 2), (128, 128, 2),
          (128, 64, 1), (64, 64, 1), (64, 32, 0), (32, 32, 0), (32, 3, 0)]


def init_params(seed):
    """Flat FP32 parameter vector in the library's layout: He-uniform weights
    (bound sqrt(6 / (9 cin))), zero biases, and a zero last layer, so that the
    untrained network is the identity."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for li, (ci, co, _) in enumerate(LAYERS):
        bound = math.sqrt(6.0 / (9 * ci))
        w = rng.uniform(-bound, bound, (3, 3, ci, co))
        if li == len(LAYERS) - 1:
            w[...] = 0.0
        parts += [w.reshape(-1), np.zeros(co)]
    return np.concatenate(parts).astype(np.float32)


def forward_flops(nx, ny, batch=1):
    """Multiply-adds x 2 of one forward pass (real channel counts)."""
    return sum(2.0 * batch * (nx >> lv) * (ny >> lv) * 9 * ci * co for ci, co, lv in LAYERS)


@dataclass
class Draw:
    seed: int
    drift: float
    u_th: float


def draws(n, offset=0):
    """n two-stream draws with seeds SEED_DENOISER + offset + i."""
    out = []
    for i in range(n):
        s = SEED_DENOISER + offset + i
        rng = np.random.Generator(np.random.PCG64(s))
        out.append(Draw(s, float(rng.uniform(0.1, 0.4)), float(rng.uniform(0.02, 0.1))))
    return out


def workload(d: Draw, nx=256, ny=256, k=8, steps=600):
    return wl.two_stream(nx=nx, ny=ny, k=k, u_th=d.u_th, drift=d.drift, tile=16, steps=steps,
                         seed=d.seed)


def _subsample_species_cfg(cfg, factor):
    """Configuration whose particles carry `factor` times the charge."""
    import copy
    c = copy.deepcopy(cfg)
    c.species[0].density = cfg.species[0].density * factor
    c.flags = 0
    return c


def make_pairs(ds, nx=256, ny=256, steps=600, every=3, first=0, stream=None):
    """(J_sub, J_full) device tensors [N, 3, ny, nx] for every draw in ds:
    the step's current from the 1/16 subsample (charge x16) and from all 64
    ppc, at steps first, first+every, ... < steps."""
    import torch
    k = 8
    outs_n, outs_c = [], []
    dev = torch.device("cuda")
    for d in ds:
        w = workload(d, nx, ny, k, steps)
        main = pic.Simulation.from_workload(w, flags=pic.PIC_TRACK_IDS, device=True, stream=stream)
        sub = pic.Simulation(_subsample_species_cfg(main.cfg, 16.0), stream)
        n = w.n_particles
        bufs = {key: torch.empty(n, dtype=torch.int32 if key in ("ix", "iy", "id") else torch.float32,
                                 device=dev) for key in ("ix", "iy", "x", "y", "ux", "uy", "uz", "id")}
        E = torch.empty(3 * nx * ny, dtype=torch.float32, device=dev)
        B = torch.empty_like(E)
        try:
            for step in range(steps):
                if step >= first and (step - first) % every == 0:
                    pic.pic_get_particles(main.h, 0, **bufs)
                    site = bufs["id"] % (k * k)
                    a, b = site % k, site // k
                    keep = ((a == SUB_SITES[0]) | (a == SUB_SITES[1])) & \
                        ((b == SUB_SITES[0]) | (b == SUB_SITES[1]))
                    arrs = [bufs[key][keep].contiguous() for key in ("ix", "iy", "x", "y", "ux", "uy", "uz")]
                    pic.pic_load_particles(sub.h, 0, *arrs)
                    pic.pic_get_fields(main.h, pic.FIELD_E, E)
                    pic.pic_get_fields(main.h, pic.FIELD_B, B)
                    pic.pic_set_fields(sub.h, E, B)
                    sub.step(1)
                    main.step(1)
                    Jn = torch.empty(3 * nx * ny, dtype=torch.float32, device=dev)
                    Jc = torch.empty_like(Jn)
                    pic.pic_get_fields(sub.h, pic.FIELD_J, Jn)
                    pic.pic_get_fields(main.h, pic.FIELD_J, Jc)
                    outs_n.append(Jn.view(3, ny, nx))
                    outs_c.append(Jc.view(3, ny, nx))
                else:
                    main.step(1)
            pic.pic_sync(main.h)
        finally:
            main.close()
            sub.close()
    return torch.stack(outs_n), torch.stack(outs_c)


def train(net: pic.Denoiser, Jn, Jc, iters, batch, lr=1e-3, lr_min=1e-4, seed=0, log_every=0):
    """Adam on random mini-batches (cosine learning-rate decay); returns the
    loss of every step."""
    import torch
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    N = Jn.shape[0]
    losses = []
    for it in range(iters):
        idx = torch.randint(0, N, (batch,), generator=g).to(Jn.device)
        xb = Jn.index_select(0, idx).contiguous()
        yb = Jc.index_select(0, idx).contiguous()
        a = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * it / max(iters - 1, 1)))
        losses.append(pic.pic_denoiser_train_step(net.d, xb, yb, batch, a))
        if log_every and it % log_every == 0:
            print(f"iter {it} loss {losses[-1]:.4g} lr {a:.2e}", flush=True)
    return losses


def mse_gain(net: pic.Denoiser, Jn, Jc, batch):
    """Mean squared error against the high-ppc current of the raw subsample
    current and of the denoised one, over all pairs."""
    import torch
    raw = den = 0.0
    out = torch.empty_like(Jn[:batch])
    N = Jn.shape[0]
    for s in range(0, N, batch):
        b = min(batch, N - s)
        xb = Jn[s:s + b].contiguous()
        o = out[:b]
        pic.pic_denoiser_forward(net.d, xb, o, b)
        raw += float(((xb - Jc[s:s + b]) ** 2).sum())
        den += float(((o - Jc[s:s + b]) ** 2).sum())
    return raw / Jn.numel(), den / Jn.numel()


def spectral_gain(net: pic.Denoiser, Jn, Jc, batch, edges=(1, 2, 4, 8, 16, 32, 64, 182)):
    """Shell-by-shell comparison of the raw subsample current and of the
    network's output (with the net's current restoration setting) against the
    high-ppc current, over all pairs: per shell of |m| (Fourier index radius,
    lo <= |m| < hi) the gain sum Re(F(out) conj F(Jc)) / sum |F(Jc)|^2 (1: the
    coherent part passes unchanged; below 1: it is shrunk) and the error
    power sum |F(out) - F(Jc)|^2 / sum |F(Jc)|^2."""
    import torch
    N, _, H, W = Jn.shape
    dev = Jn.device
    ky = torch.fft.fftfreq(H, 1.0 / H, device=dev, dtype=torch.float64)
    kx = torch.fft.rfftfreq(W, 1.0 / W, device=dev, dtype=torch.float64)
    m = torch.sqrt(ky[:, None] ** 2 + kx[None, :] ** 2)
    masks = [(m >= lo) & (m < hi) for lo, hi in zip(edges[:-1], edges[1:])]
    z = lambda: torch.zeros(len(masks), dtype=torch.float64, device=dev)
    auto, cr_n, cr_d, er_n, er_d = z(), z(), z(), z(), z()
    out = torch.empty_like(Jn[:batch])
    for s in range(0, N, batch):
        b = min(batch, N - s)
        xb = Jn[s:s + b].contiguous()
        o = out[:b]
        pic.pic_denoiser_forward(net.d, xb, o, b)
        Fc = torch.fft.rfft2(Jc[s:s + b].double())
        Fn = torch.fft.rfft2(xb.double())
        Fd = torch.fft.rfft2(o.double())
        for i, mk in enumerate(masks):
            c = Fc[..., mk]
            auto[i] += (c.abs() ** 2).sum()
            cr_n[i] += (Fn[..., mk] * c.conj()).real.sum()
            cr_d[i] += (Fd[..., mk] * c.conj()).real.sum()
            er_n[i] += ((Fn[..., mk] - c).abs() ** 2).sum()
            er_d[i] += ((Fd[..., mk] - c).abs() ** 2).sum()
    a = auto.cpu().numpy()
    rows = []
    for i, (lo, hi) in enumerate(zip(edges[:-1], edges[1:])):
        rows.append({"shell": [lo, hi], "gain_raw": float(cr_n[i] / auto[i]),
                     "gain_out": float(cr_d[i] / auto[i]), "err_raw": float(er_n[i] / auto[i]),
                     "err_out": float(er_d[i] / auto[i]), "power": float(a[i])})
    return rows


def field_energy_run(w, steps, net=None, stream=None, modes=False, binomial=0):
    """W_E(t) history (t = 0..steps) of a run (with the denoiser `net` or
    `binomial` passes of the binomial filter in the current-filter slot), its
    mean step time (ms, CUDA
    events around the stepping; None with modes=True, whose per-step field
    reads would be timed too) and the diagnostics of one further step (with
    its current's continuity residual); with modes=True also |E_x(m)|^2 of the
    k_y = 0 Fourier modes m = 0..nx/2 after every step (t = 1..steps)."""
    import torch
    sim = pic.Simulation.from_workload(w, device=True, stream=stream)
    try:
        if net is not None:
            pic.pic_set_denoiser(sim.h, net.d)
        elif binomial:
            pic.pic_set_binomial_filter(sim.h, binomial)
        spec = None
        if modes:
            E = torch.empty((3, w.ny, w.nx), dtype=torch.float32, device="cuda")
            rows = []
            for _ in range(steps):
                sim.step(1)
                pic.pic_get_fields(sim.h, pic.FIELD_E, E.view(-1))
                rows.append(torch.fft.rfft(E[0].double().mean(dim=0)).abs().pow(2))
            spec = torch.stack(rows).cpu().numpy()
            we, _, _ = sim.history(0, steps + 1)
            d = _continuity_diag(sim)
            return np.asarray(we), None, d, spec
        sim.step(2)  # builds both graphs
        pic.pic_sync(sim.h)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        s = torch.cuda.current_stream()
        e0.record(s)
        sim.step(steps - 2)
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / (steps - 2)
        we, _, _ = sim.history(0, steps + 1)
        d = _continuity_diag(sim)
    finally:
        sim.close()
    return np.asarray(we), ms, d, None


def _continuity_diag(sim):
    """Diagnostics after one more step, with the continuity residual of that
    step's (possibly filtered) current."""
    sim.diagnostics()
    sim.step(1)
    return sim.diagnostics()


def _smooth(v, w):
    if w <= 1:
        return v
    k = np.ones(w) / w
    pad = np.concatenate([np.full(w // 2, v[0]), v, np.full(w - 1 - w // 2, v[-1])])
    return np.convolve(pad, k, mode="valid")


def _fit_window(lv, floor_steps, lo, hi, smooth):
    """Indices of the exponential-growth stretch of a log-amplitude history:
    the longest contiguous run, before the (smoothed) global maximum, where the
    smoothed value lies between lo above the early noise level (median of the
    first floor_steps values) and hi below the maximum."""
    ls = _smooth(lv, smooth)
    ks = int(np.argmax(ls))
    floor = float(np.median(ls[:floor_steps]))
    top = float(ls[ks])
    ok = [(floor + lo <= ls[j] <= top - hi) for j in range(ks + 1)]
    best, cur = (0, -1), None
    for j, o in enumerate(ok):
        if o:
            cur = (cur[0], j) if cur else (j, j)
            if cur[1] - cur[0] > best[1] - best[0]:
                best = cur
        else:
            cur = None
    return best


def mode_growth_rate(power, dt, m, floor_steps=20, lo=1.5, hi=1.0, smooth=9, band=1):
    """Growth rate of the field amplitude in the band of Fourier modes
    m-band..m+band (power |E_m|^2 at steps 1..): least-squares slope of
    ln|E| over the longest stretch between lo e-folds above the early noise
    level and hi e-folds below the saturation maximum (smoothed over `smooth`
    steps to place the window)."""
    lo_m, hi_m = max(1, m - band), min(power.shape[1] - 1, m + band)
    lv = 0.5 * np.log(np.maximum(power[:, lo_m:hi_m + 1].sum(axis=1), 1e-300))
    j0, j1 = _fit_window(lv, floor_steps, lo, hi, smooth)
    if j1 - j0 < 5:
        return float("nan"), (j0, j1)
    t = (np.arange(j0, j1 + 1) + 1) * dt
    return float(np.polyfit(t, lv[j0:j1 + 1], 1)[0]), (j0, j1)


def growth_rate(we, dt, floor_steps=20, lo=1.5, hi=1.0, smooth=9):
    """Field-amplitude growth rate from the field-energy history W_E(t) (t = 0,
    dt, ...): the slope of ln W_E / 2 over the same window as
    mode_growth_rate."""
    lv = 0.5 * np.log(np.maximum(np.asarray(we[1:], np.float64), 1e-300))
    j0, j1 = _fit_window(lv, floor_steps, lo, hi, smooth)
    if j1 - j0 < 5:
        return float("nan"), (j0, j1)
    t = (np.arange(j0, j1 + 1) + 1) * dt
    return float(np.polyfit(t, lv[j0:j1 + 1], 1)[0]), (j0, j1)


def kinetic_growth_rate(drift, u_th, L, m_max=None):
    """Largest growth rate over the box's modes k = 2 pi m / L of two
    counter-streaming Maxwellian beams (density 1/2 each, velocities +-drift,
    thermal velocity u_th; non-relativistic): roots of
    1 + sum_beams (1/2) / (k u_th)^2 (1 + zeta Z(zeta)) = 0,
    zeta = (omega - k v) / (sqrt(2) k u_th), Z the plasma dispersion function."""
    from scipy import optimize, special

    def Z(z):
        return 1j * math.sqrt(math.pi) * special.wofz(z)

    def disp(w, k):
        s = 1.0 + 0j
        for v in (drift, -drift):
            z = (w - k * v) / (math.sqrt(2.0) * k * u_th)
            s += (0.5 / (k * k * u_th * u_th)) * (1 + z * Z(z))
        return s

    best = 0.0
    m_max = m_max or int(L * 2.0 / (2 * math.pi * max(drift, 1e-3))) + 2
    for m in range(1, m_max + 1):
        k = 2 * math.pi * m / L
        if k * drift > 2.0:
            break

        def f(v):
            r = disp(v[0] + 1j * v[1], k)
            return [r.real, r.imag]

        for g0 in (0.05, 0.2, 0.4):
            try:
                sol, info, ok, _ = optimize.fsolve(f, [0.0, g0], full_output=True)
            except Exception:
                continue
            if ok == 1 and abs(complex(*f(sol))) < 1e-8 and sol[1] > best:
                best = float(sol[1])
    return best
