"""Seeded synthetic plasmas shaped like the thesis's workloads (§5.1).

This module only draws inputs: particle positions on a quiet-start lattice,
Maxwellian momenta plus drifts, and optional seeded initial fields.  It holds
none of the method's arithmetic, so it may feed both the CUDA library and the
CPU oracle with identical arrays.  All randomness comes from
``numpy.random.Generator(PCG64(seed))``.

Units are those of Eqs. 21-22 (c = 1, omega_p = 1 for the total electron
density n0 = 1).  A particle is (ix, iy, x, y, ux, uy, uz): int32 cell, FP32
offset in [0,1)^2, FP32 momentum u = gamma v.  Every particle of a species
carries the charge density ``qtilde = sign(q) n_s / ppc_s``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20210


@dataclass
class Species:
    q_over_m: float
    qtilde: float
    ix: np.ndarray
    iy: np.ndarray
    x: np.ndarray
    y: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    uz: np.ndarray

    @property
    def n(self) -> int:
        return int(self.ix.size)

    def arrays(self):
        return (self.ix, self.iy, self.x, self.y, self.ux, self.uy, self.uz)


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    dx: float
    dy: float
    dt: float
    tile: int
    steps: int
    species: list
    background: float = 1.0          # fixed neutralising ion density
    E0: np.ndarray | None = None     # (3, ny, nx) float32 at the Yee locations, or None = 0
    B0: np.ndarray | None = None
    meta: dict = field(default_factory=dict)
    window: list | None = None       # moving window: one injection dict (or None) per species
    lasers: list = field(default_factory=list)   # laser pulses (keyword dicts) added at start

    @property
    def n_particles(self) -> int:
        return sum(s.n for s in self.species)


def lattice(nx: int, ny: int, k: int):
    """k x k particles per cell at offsets ((a+1/2)/k, (b+1/2)/k).

    Returns (ix, iy, x, y, a, b) with particles ordered cell by cell (row-major
    over cells), and inside a cell by (b, a)."""
    sub = (np.arange(k, dtype=np.float64) + 0.5) / k
    ix = np.repeat(np.tile(np.arange(nx, dtype=np.int32), ny), k * k)
    iy = np.repeat(np.repeat(np.arange(ny, dtype=np.int32), nx), k * k)
    a = np.tile(np.tile(np.arange(k, dtype=np.int32), k), nx * ny)
    b = np.tile(np.repeat(np.arange(k, dtype=np.int32), k), nx * ny)
    x = sub[a].astype(np.float32)
    y = sub[b].astype(np.float32)
    return ix, iy, x, y, a, b


def _maxwellian(rng, n, u_th):
    if u_th == 0.0:
        return np.zeros(n, np.float64)
    return rng.normal(0.0, u_th, n)


def _f32(a):
    return np.ascontiguousarray(a, np.float32)


def displace_x(ix, x, shift_cells, nx):
    """Move particles by ``shift_cells`` (float64, cell units) along x, keeping
    cell + offset form with the offset in [0,1)."""
    pos = ix.astype(np.float64) + x.astype(np.float64) + shift_cells
    cell = np.floor(pos)
    off = (pos - cell).astype(np.float32)
    up = off >= np.float32(1.0)
    off[up] = 0.0
    cell[up] += 1
    return np.mod(cell, nx).astype(np.int32), off


def two_stream(nx=64, ny=64, k=4, u_th=0.1, drift=0.2, dx=0.1, dy=0.1, dt=0.05,
               tile=16, steps=100, seed=SEED_BASE + 1) -> Workload:
    """Electrons on fixed ions, Maxwellian u_th per axis, and two interleaved
    counter-streaming beams: lattice sites with even (a+b) drift +drift along
    x, odd ones -drift.  Zero initial fields."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ix, iy, x, y, a, b = lattice(nx, ny, k)
    n = ix.size
    sgn = np.where((a + b) % 2 == 0, 1.0, -1.0)
    ux = _maxwellian(rng, n, u_th) + drift * sgn
    uy = _maxwellian(rng, n, u_th)
    uz = _maxwellian(rng, n, u_th)
    sp = Species(-1.0, -1.0 / (k * k), ix, iy, x, y, _f32(ux), _f32(uy), _f32(uz))
    return Workload("two_stream", nx, ny, dx, dy, dt, tile, steps, [sp],
                    meta=dict(ppc=k * k, u_th=u_th, drift=drift, seed=seed))


def weibel(nx=512, ny=512, k=8, u_drift=0.6, u_th=0.05, dx=0.1, dy=0.1, dt=0.05,
           tile=16, steps=500, seed=SEED_BASE + 2) -> Workload:
    """Two electron populations, each k x k per cell with density 1/2, sharing
    lattice positions and drifting +-u_drift along z, on fixed ions.  Both have
    q/m = -1 and the same charge per particle, so they form one species of
    2 k^2 particles per cell (population 1 first in every cell)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ix, iy, x, y, _, _ = lattice(nx, ny, k)
    n1 = ix.size
    k2 = k * k
    # interleave the two populations cell by cell: [pop1 cell0, pop2 cell0, pop1 cell1, ...]
    idx1 = np.arange(nx * ny, dtype=np.int64)[:, None] * k2 + np.arange(k2)[None, :]
    src = np.stack([idx1, idx1], axis=1).reshape(-1)
    pop = np.tile(np.repeat(np.array([0, 1], np.int8), k2), nx * ny)
    n = 2 * n1
    ux = _maxwellian(rng, n, u_th)
    uy = _maxwellian(rng, n, u_th)
    uz = _maxwellian(rng, n, u_th) + np.where(pop == 0, u_drift, -u_drift)
    sp = Species(-1.0, -0.5 / k2, ix[src], iy[src], x[src], y[src], _f32(ux), _f32(uy), _f32(uz))
    return Workload("weibel", nx, ny, dx, dy, dt, tile, steps, [sp],
                    meta=dict(ppc=2 * k2, u_th=u_th, u_drift=u_drift, seed=seed))


def weibel_pair(nx=512, ny=512, k=10, u_drift=0.6, u_th=0.05, dx=0.1, dy=0.1, dt=0.05,
                tile=16, steps=500, seed=SEED_BASE + 6) -> Workload:
    """The thesis's own Weibel shape (§5.1): electrons and positrons, k x k per
    cell each (k = 10: 26.2M per species on 512^2, the thesis's 25M per species
    on 500^2 cells rounded to a tile-divisible grid), density 1 each, electrons
    drifting +u_drift and positrons -u_drift along z, thermal spread u_th; a
    neutral pair plasma, no fixed background."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ix, iy, x, y, _, _ = lattice(nx, ny, k)
    n = ix.size
    sps = []
    for qm, drift in ((-1.0, u_drift), (1.0, -u_drift)):
        ux = _maxwellian(rng, n, u_th)
        uy = _maxwellian(rng, n, u_th)
        uz = _maxwellian(rng, n, u_th) + drift
        sps.append(Species(qm, qm / (k * k), ix.copy(), iy.copy(), x.copy(), y.copy(), _f32(ux),
                           _f32(uy), _f32(uz)))
    return Workload("weibel_pair", nx, ny, dx, dy, dt, tile, steps, sps, background=0.0,
                    meta=dict(ppc=2 * k * k, u_th=u_th, u_drift=u_drift, seed=seed))


def thermal_seeded(nx=2048, ny=2048, k=4, u_th=0.2, amp=1e-3, mode=1, dx=0.1, dy=0.1,
                   dt=0.05, tile=16, steps=200, seed=SEED_BASE + 3) -> Workload:
    """Thermal electrons on fixed ions with a seeded longitudinal mode:
    Ex(x_{i+1/2}) = amp sin(kx x) with kx = 2 pi mode / L_x, and every electron
    displaced along x by xi = amp sin(kx x0) (so that div E = rho holds to first
    order for n0 = 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ix, iy, x, y, _, _ = lattice(nx, ny, k)
    n = ix.size
    Lx = nx * dx
    kx = 2.0 * np.pi * mode / Lx
    x0 = (ix.astype(np.float64) + x.astype(np.float64)) * dx
    xi = amp * np.sin(kx * x0)
    ix2, x2 = displace_x(ix, x, xi / dx, nx)
    ux = _maxwellian(rng, n, u_th)
    uy = _maxwellian(rng, n, u_th)
    uz = _maxwellian(rng, n, u_th)
    sp = Species(-1.0, -1.0 / (k * k), ix2, iy, x2, y, _f32(ux), _f32(uy), _f32(uz))
    E0 = np.zeros((3, ny, nx), np.float32)
    xh = (np.arange(nx, dtype=np.float64) + 0.5) * dx
    E0[0, :, :] = (amp * np.sin(kx * xh))[None, :].astype(np.float32)
    return Workload("thermal_seeded", nx, ny, dx, dy, dt, tile, steps, [sp], E0=E0,
                    meta=dict(ppc=k * k, u_th=u_th, amp=amp, kx=kx, seed=seed))


def cold_oscillation(nx=64, ny=4, k=4, amp=1e-3, mode=1, dx=0.1, dy=0.1, dt=0.05,
                     tile=4, steps=400, seed=SEED_BASE + 9) -> Workload:
    """Cold electrons (u = 0) with the same Gauss-consistent displacement and
    Ex seed as ``thermal_seeded``: a standing Langmuir oscillation."""
    w = thermal_seeded(nx=nx, ny=ny, k=k, u_th=0.0, amp=amp, mode=mode, dx=dx, dy=dy,
                       dt=dt, tile=tile, steps=steps, seed=seed)
    w.name = "cold_oscillation"
    return w


def batch_member(s: int, steps=300, dt=0.05, dx=0.1, dy=0.1) -> Workload:
    """Simulation s of the batched workload: grid side drawn from
    {64,128,256,512}, ppc from {4,16,64}, counter-streaming drift ux ~ U[0.1,0.5]
    on two interleaved beams, u_th = 0.05, seed 20210*1000 + s."""
    seed = SEED_BASE * 1000 + s
    rng = np.random.Generator(np.random.PCG64(seed))
    side = int(rng.choice([64, 128, 256, 512]))
    k = int(rng.choice([2, 4, 8]))
    drift = float(rng.uniform(0.1, 0.5))
    w = two_stream(nx=side, ny=side, k=k, u_th=0.05, drift=drift, dx=dx, dy=dy, dt=dt,
                   tile=16, steps=steps, seed=seed + 7)
    w.name = f"batch_{s}"
    w.meta.update(side=side)
    return w


def random_particles(nx, ny, n, u_max=0.5, seed=0, q_over_m=-1.0, qtilde=-1.0 / 16):
    """Uniformly random cells, offsets and momenta (|u_i| < u_max): an
    unstructured workload for parity tests (ragged tiles, arbitrary moves)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ix = rng.integers(0, nx, n, dtype=np.int32)
    iy = rng.integers(0, ny, n, dtype=np.int32)
    x = rng.random(n, dtype=np.float32)
    y = rng.random(n, dtype=np.float32)
    u = rng.uniform(-u_max, u_max, (3, n)).astype(np.float32)
    return Species(q_over_m, qtilde, ix, iy, x, y, u[0].copy(), u[1].copy(), u[2].copy())


def random_fields(nx, ny, amp=0.1, seed=1):
    rng = np.random.Generator(np.random.PCG64(seed))
    E = (amp * rng.standard_normal((3, ny, nx))).astype(np.float32)
    B = (amp * rng.standard_normal((3, ny, nx))).astype(np.float32)
    return E, B


def laser_wakefield(nx=128, ny=64, k=2, dx=0.1, dy=0.1, dt=0.05, tile=16, steps=200,
                    x_start=None, a0=1.0, omega0=10.0, fwhm=1.0, kind="gaussian", W0=1.5,
                    capacity_margin=1.25, seed=SEED_BASE + 7) -> Workload:
    """A laser pulse entering a cold plasma in a moving window (the steps around
    the loop of Listing 3.1; §3.2 lasers and moving window): cold electrons on
    a k x k quiet-start lattice per cell at physical x >= x_start (half the
    box), the ions immobile (they carry no current; they would enter only
    rho, which a moving-window run does not report, so no background is set);
    a Gaussian (or plane) pulse focused on the plasma edge, its front 5 % of
    the box behind it; the window injects the same lattice at its right edge.
    Deterministic (no random draws)."""
    del seed
    Lx = nx * dx
    if x_start is None:
        x_start = 0.5 * Lx
    ix, iy, x, y, a, _ = lattice(nx, ny, k)
    keep = (ix.astype(np.float64) + (a.astype(np.float64) + 0.5) / k) * dx >= x_start
    n = int(keep.sum())
    z = np.zeros(n, np.float32)
    sp = Species(-1.0, -1.0 / (k * k), ix[keep], iy[keep], x[keep], y[keep], z, z.copy(), z.copy())
    cap = int(capacity_margin * nx * ny * k * k) + 1024
    laser = dict(kind=kind, start=x_start - 0.05 * Lx, fwhm=fwhm, a0=a0, omega0=omega0,
                 W0=W0, focus=x_start, axis=0.5 * ny * dy)
    return Workload("laser_wakefield", nx, ny, dx, dy, dt, tile, steps, [sp], background=0.0,
                    window=[dict(k=k, x_start=x_start, capacity=cap)], lasers=[laser],
                    meta=dict(ppc=k * k, x_start=x_start, a0=a0, omega0=omega0, kind=kind))

