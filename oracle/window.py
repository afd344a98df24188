"""Moving window, particle injection and lasers of the plain CPU oracle (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The time loop of Listing 3.1 ends, when the moving window is enabled, with
three steps: shift E and B one cell to the left, shift the particles one cell
to the left, insert new particles.  §3.2 adds that the window follows the
plasma at the speed of light, moving one cell to the right at the end of a
step, and that the input file can add plane and Gaussian lasers to the
initial fields.  The thesis gives no formulas for any of these; the readings
taken here (the same ones the CUDA library implements) are:

* Window position: after k steps the window has moved M(k) = floor(k dt / dx
  + 1e-9) cells (speed c = 1; at most one cell per step because dt < dx by
  Eq. 1).  A step whose M grows shifts the window by one cell after the field
  update.
* The box of a moving-window run is open along x: E and B are zero outside
  0 <= i < nx, current falling outside is dropped, a particle whose cell
  leaves the box is removed (y stays periodic).
* Shift: E, B <- values one column to the right; the new last column is zero.
  Particles: ix <- ix - 1, those reaching ix < 0 are removed.
* Injection: the new last column (global cell index g = M + nx - 1) receives,
  per injecting species, a cold k x k lattice per cell at offsets
  ((a + 1/2)/k, (b + 1/2)/k) with momentum u_inj, keeping the particles whose
  physical position (g + (a + 1/2)/k) dx is at or beyond x_start (a step
  density profile).  Injected particles carry no id (-1).
* Lasers (plane, Gaussian) are added to the initial E and B as a pulse moving
  towards +x: field envelope sin^2(pi xi / 2 fwhm) for 0 <= xi = start - x
  <= 2 fwhm (its full width at half maximum is fwhm), carrier cos(omega0 (x -
  start)), peak field a0 omega0, E at the polarisation angle theta from y
  towards z (Ey = cos(theta) f, Ez = sin(theta) f) and B = x_hat x E (Bz =
  cos(theta) f, By = -sin(theta) f), each component evaluated at its own Yee
  location.  The Gaussian beam is the paraxial beam of two dimensions with
  waist W0 at x = focus on the axis y = axis: amplitude sqrt(W0/W(z))
  exp(-r^2/W(z)^2), W(z) = W0 sqrt(1 + (z/zR)^2), zR = omega0 W0^2/2, and an
  extra phase omega0 r^2 z / (2 (z^2 + zR^2)) - atan(z/zR)/2 (z = x - focus,
  r = y - axis).  No longitudinal component is added (paraxial fields).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def window_moves(k: int, dt: float, dx: float) -> int:
    """Cells the window has moved after k steps (speed c = 1)."""
    return int(np.floor(k * dt / dx + 1e-9))


@dataclass
class Inject:
    """Cold plasma entering at the right edge of a moving window."""
    k: int                 # k x k particles per cell (k*k = the species' ppc)
    x_start: float = 0.0   # plasma at physical x >= x_start
    ux: float = 0.0
    uy: float = 0.0
    uz: float = 0.0


def injected_offsets(g: int, inj: Inject, dx: float):
    """Lattice sub-indices a (along x) kept in the column of global cell index
    g: those with (g + (a + 1/2)/k) dx >= x_start."""
    a = np.arange(inj.k)
    keep = np.array([(g + (float(ai) + 0.5) / inj.k) * dx >= inj.x_start for ai in a])
    return a[keep]


def inject_column(sp, inj: Inject, nx: int, ny: int, g: int, dx: float, dtype):
    """Append the injected particles of column nx - 1 (global index g)."""
    a = injected_offsets(g, inj, dx)
    if a.size == 0:
        return
    k = inj.k
    sub = (np.arange(k, dtype=np.float64) + 0.5) / k
    iy = np.repeat(np.arange(ny, dtype=np.int32), k * a.size)
    bb = np.tile(np.repeat(np.arange(k), a.size), ny)
    aa = np.tile(np.tile(a, k), ny)
    n = iy.size
    sp.append(np.full(n, nx - 1, np.int32), iy, sub[aa].astype(np.float32).astype(dtype),
              sub[bb].astype(np.float32).astype(dtype),
              np.full(n, inj.ux, np.float32).astype(dtype),
              np.full(n, inj.uy, np.float32).astype(dtype),
              np.full(n, inj.uz, np.float32).astype(dtype))


def shift_window(sim) -> None:
    """The last three steps of Listing 3.1: shift E and B one cell left (zero
    new column), shift the particles left (removing those leaving the box),
    insert the new plasma column."""
    for F in (sim.E, sim.B):
        F[:, :, :-1] = F[:, :, 1:]
        F[:, :, -1] = 0
    sim.moves += 1
    g = sim.moves + sim.nx - 1
    for sp, inj in zip(sim.species, sim.window):
        sp.ix = np.ascontiguousarray(sp.ix - 1, np.int32)
        sp.keep(sp.ix >= 0)
        if inj is not None:
            inject_column(sp, inj, sim.nx, sim.ny, g, sim.dx, sim.dtype)


@dataclass
class Laser:
    """A laser pulse added to the initial fields (see the module docstring)."""
    kind: str = "plane"        # "plane" or "gaussian"
    start: float = 0.0         # x of the pulse front
    fwhm: float = 1.0          # full width at half maximum of the field envelope
    a0: float = 1.0            # normalised vector potential (peak field a0 omega0)
    omega0: float = 10.0       # carrier frequency = wavenumber (c = 1)
    polarization: float = 0.0  # angle of E from y towards z (radians)
    W0: float = 1.0            # Gaussian: waist
    focus: float = 0.0         # Gaussian: x of the focal plane
    axis: float = 0.0          # Gaussian: y of the beam axis


def laser_envelope(x, start, fwhm):
    L = 2.0 * fwhm
    xi = start - np.asarray(x, np.float64)
    return np.where((xi >= 0.0) & (xi <= L), np.sin(np.pi * xi / L) ** 2, 0.0)


def laser_profile(l: Laser, x, y):
    """Transverse field before polarisation at physical (x, y) (broadcast)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    env = laser_envelope(x, l.start, l.fwhm)
    E0 = l.a0 * l.omega0
    if l.kind == "plane":
        return E0 * env * np.cos(l.omega0 * (x - l.start)) + 0.0 * y
    if l.kind != "gaussian":
        raise ValueError(l.kind)
    z = x - l.focus
    r = y - l.axis
    zR = 0.5 * l.omega0 * l.W0 * l.W0
    W = l.W0 * np.sqrt(1.0 + (z / zR) ** 2)
    curv = z / (z * z + zR * zR)          # 1 / R(z)
    gouy = np.arctan(z / zR)
    amp = np.sqrt(l.W0 / W) * np.exp(-(r / W) ** 2)
    phase = l.omega0 * (x - l.start) + 0.5 * l.omega0 * r * r * curv - 0.5 * gouy
    return E0 * env * amp * np.cos(phase)


def laser_fields(nx, ny, dx, dy, laser: Laser, x_origin: float = 0.0):
    """(E, B), each (3, ny, nx) FP64 at the Yee locations of Fig. 3.1, of one
    laser; x_origin = physical x of node column 0."""
    xn = x_origin + np.arange(nx) * dx
    xh = x_origin + (np.arange(nx) + 0.5) * dx
    yn = np.arange(ny) * dy
    yh = (np.arange(ny) + 0.5) * dy
    c, s = np.cos(laser.polarization), np.sin(laser.polarization)
    E = np.zeros((3, ny, nx))
    B = np.zeros((3, ny, nx))
    E[1] = c * laser_profile(laser, xn[None, :], yh[:, None])    # Ey (i, j+1/2)
    E[2] = s * laser_profile(laser, xn[None, :], yn[:, None])    # Ez (i, j)
    B[1] = -s * laser_profile(laser, xh[None, :], yn[:, None])   # By (i+1/2, j)
    B[2] = c * laser_profile(laser, xh[None, :], yh[:, None])    # Bz (i+1/2, j+1/2)
    return E, B


def yee_group_velocity(k: float, dx: float, dt: float) -> float:
    """Group velocity along x of the 1D Yee scheme (Eqs. 19-20) at wavenumber
    k: from sin(w dt/2)/dt = sin(k dx/2)/dx, dw/dk = cos(k dx/2)/cos(w dt/2)."""
    s = dt / dx * np.sin(0.5 * k * dx)
    return float(np.cos(0.5 * k * dx) / np.sqrt(1.0 - s * s))
