"""ctypes wrapper and plain simulation driver for the C oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).  The arithmetic of the
method lives in ``pic_oracle.c``; this module only moves arrays in and out and
computes grid diagnostics by their plain definitions with numpy in FP64.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

ORC_EPARTICLE = 1


def _openmp_flag() -> list:
    """["-fopenmp"] when gcc can build and link OpenMP code here, else [] (the
    threaded particle loop then runs its blocks one after another)."""
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.c")
        with open(src, "w") as f:
            f.write("#include <omp.h>\nint main(void){return omp_get_max_threads() < 1;}\n")
        r = subprocess.run(["gcc", "-fopenmp", src, "-o", os.path.join(d, "t")],
                           capture_output=True)
    return ["-fopenmp"] if r.returncode == 0 else []


def build_oracle(force: bool = False) -> str:
    """Compile the oracle (both precisions) into oracle/liboracle.so."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    objs = []
    omp = _openmp_flag()
    flags = ["-O2", "-fPIC", "-ffp-contract=off", "-fno-fast-math", "-std=c11", *omp]
    for real, sfx, extra in (("double", "_f64", ["-DREAL_IS_DOUBLE"]),
                             ("float", "_f32", [])):
        obj = os.path.join(_HERE, f"_pic_oracle{sfx}.o")
        cmd = ["gcc", *flags, f"-DREAL={real}", f"-DSFX={sfx}", *extra,
               "-c", _SRC, "-o", obj]
        subprocess.run(cmd, check=True)
        objs.append(obj)
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-shared", *omp, "-o", tmp, *objs, "-lm"], check=True)
    os.replace(tmp, _LIB)
    for o in objs:
        os.remove(o)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build_oracle()
        _lib = C.CDLL(_LIB)
        _declare(_lib)
    return _lib


_P = C.c_void_p
_I = C.c_int
_I64 = C.c_int64
_D = C.c_double


def _declare(L):
    for sfx, real in (("_f64", C.c_double), ("_f32", C.c_float)):
        getattr(L, "orc_gather" + sfx).argtypes = [_I, _I, _I, _P, _P, _I, _I, real, real, _P, _P]
        getattr(L, "orc_gather" + sfx).restype = None
        getattr(L, "orc_boris" + sfx).argtypes = [_P, _P, _P, real]
        getattr(L, "orc_boris" + sfx).restype = real
        getattr(L, "orc_deposit_move" + sfx).argtypes = [_I, _I, _I, _P, _I, _I, real, real, real, real, real, real, real]
        getattr(L, "orc_deposit_move" + sfx).restype = None
        getattr(L, "orc_advance" + sfx).argtypes = [_I, _I, _I, _D, _D, _D, _D, _D, _I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]
        getattr(L, "orc_advance" + sfx).restype = _I
        getattr(L, "orc_advance_par" + sfx).argtypes = [_I, _I, _I, _D, _D, _D, _D, _D, _I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _I]
        getattr(L, "orc_advance_par" + sfx).restype = _I
        getattr(L, "orc_yee" + sfx).argtypes = [_I, _I, _I, _D, _D, _D, _P, _P, _P]
        getattr(L, "orc_yee" + sfx).restype = None
        getattr(L, "orc_rho" + sfx).argtypes = [_I, _I, _D, _I64, _P, _P, _P, _P, _P]
        getattr(L, "orc_rho" + sfx).restype = None
    L.orc_tile_sort.argtypes = [_I, _I, _I, _I64, _P, _P, _P, _P, _P]
    L.orc_tile_sort.restype = None


def _sfx(dtype) -> str:
    dt = np.dtype(dtype)
    if dt == np.float64:
        return "_f64"
    if dt == np.float32:
        return "_f32"
    raise TypeError(f"oracle precision must be float64 or float32, not {dt}")


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------- primitives

def gather(E, B, ix, iy, x, y, open_x=False):
    """Fields at one particle (Fig. 3.1 staggering). E, B: (3, ny, nx); with
    open_x the fields are zero outside the box along x."""
    E = np.ascontiguousarray(E)
    B = np.ascontiguousarray(B, dtype=E.dtype)
    _, ny, nx = E.shape
    real = E.dtype.type
    Ep = np.zeros(3, E.dtype)
    Bp = np.zeros(3, E.dtype)
    getattr(lib(), "orc_gather" + _sfx(E.dtype))(nx, ny, int(bool(open_x)), _ptr(E), _ptr(B), int(ix), int(iy),
                                                  real(x), real(y), _ptr(Ep), _ptr(Bp))
    return Ep, Bp


def boris(u, Ep, Bp, tem):
    """One Boris push (Eqs. 6-10). Returns (u_new, gamma_minus)."""
    u = np.array(u, copy=True)
    Ep = np.ascontiguousarray(Ep, dtype=u.dtype)
    Bp = np.ascontiguousarray(Bp, dtype=u.dtype)
    g = getattr(lib(), "orc_boris" + _sfx(u.dtype))(_ptr(u), _ptr(Ep), _ptr(Bp), u.dtype.type(tem))
    return u, float(g)


def deposit_move(J, ix, iy, x0, y0, x1, y1, qjx, qjy, qvz, open_x=False):
    """Add the current of one straight move (cell frame of (ix, iy)) into J
    (with open_x, current falling outside the box along x is dropped)."""
    _, ny, nx = J.shape
    r = J.dtype.type
    getattr(lib(), "orc_deposit_move" + _sfx(J.dtype))(
        nx, ny, int(bool(open_x)), _ptr(J), int(ix), int(iy), r(x0), r(y0), r(x1), r(y1),
        r(qjx), r(qjy), r(qvz))


def advance(sp: "SpeciesState", E, B, J, dx, dy, dt, open_x=False, threads=1):
    """Particle loop of Listing 3.1 for one species; returns (status,
    sum(gamma-1)).  With open_x, particles that left the box along x are
    removed from ``sp`` afterwards.  threads > 1: the thesis's CPU scheme
    (blocks of tile-sorted particles over threads, private current arrays
    added afterwards), identical particles, J equal up to the order of the
    additions."""
    _, ny, nx = E.shape
    ke = C.c_double(0.0)
    gone = np.zeros(sp.n, np.uint8) if open_x else None
    args = (nx, ny, int(bool(open_x)), dx, dy, dt, sp.q_over_m, sp.qtilde, sp.n,
            _ptr(sp.ix), _ptr(sp.iy), _ptr(sp.x), _ptr(sp.y),
            _ptr(sp.ux), _ptr(sp.uy), _ptr(sp.uz), _ptr(E), _ptr(B), _ptr(J),
            None if gone is None else _ptr(gone), C.byref(ke))
    if threads > 1:
        st = getattr(lib(), "orc_advance_par" + _sfx(E.dtype))(*args, int(threads))
        if st < 0:
            raise MemoryError("oracle: private current arrays")
    else:
        st = getattr(lib(), "orc_advance" + _sfx(E.dtype))(*args)
    if open_x and gone.any():
        sp.keep(gone == 0)
    return st, ke.value


def binomial_filter(J, passes=1):
    """The current filter of the time loop (Listing 3.1, after the guard-cell
    reduction of J, before the field advance): the binomial stencil
    (1/4, 1/2, 1/4) along x and then along y on each component's own periodic
    lattice, `passes` times.  Each pass multiplies a Fourier mode (kx, ky) by
    cos^2(kx dx / 2) cos^2(ky dy / 2)."""
    J = np.array(J, dtype=np.float64, copy=True)
    for _ in range(passes):
        J = 0.25 * np.roll(J, 1, axis=2) + 0.5 * J + 0.25 * np.roll(J, -1, axis=2)
        J = 0.25 * np.roll(J, 1, axis=1) + 0.5 * J + 0.25 * np.roll(J, -1, axis=1)
    return J


def yee(E, B, J, dx, dy, dt, open_x=False):
    _, ny, nx = E.shape
    getattr(lib(), "orc_yee" + _sfx(E.dtype))(nx, ny, int(bool(open_x)), dx, dy, dt,
                                              _ptr(E), _ptr(B), _ptr(J))


def rho_nodes(nx, ny, species, dtype=np.float64, background=0.0):
    """Charge density on nodes (area weighting) plus a uniform background,
    accumulated in `dtype` (the offsets are taken in that precision)."""
    rho = np.zeros((ny, nx), dtype)
    for sp in species:
        if sp.x.dtype != np.dtype(dtype):
            sp = sp.astype(dtype)
        getattr(lib(), "orc_rho" + _sfx(dtype))(nx, ny, sp.qtilde, sp.n, _ptr(sp.ix), _ptr(sp.iy),
                                                _ptr(sp.x), _ptr(sp.y), _ptr(rho))
    return rho.astype(np.float64) + background


def tile_sort(nx, ny, T, ix, iy):
    """Stable counting sort by tile id; returns (perm, counts, offsets)."""
    ix = np.ascontiguousarray(ix, np.int32)
    iy = np.ascontiguousarray(iy, np.int32)
    n = ix.size
    nt = (nx // T) * (ny // T)
    perm = np.zeros(n, np.int64)
    counts = np.zeros(nt, np.int64)
    offsets = np.zeros(nt + 1, np.int64)
    lib().orc_tile_sort(nx, ny, T, n, _ptr(ix), _ptr(iy), _ptr(perm), _ptr(counts), _ptr(offsets))
    return perm, counts, offsets


def tile_order(nx, ny, T, window=False):
    """Tile ids (ty * ntx + tx, the order of ``tile_sort``) in the order in
    which the tile-sorted arrays hold the tiles: row by row in a periodic box;
    in the moving window's open box column by column from the right edge
    (tx = ntx - 1 first), each column from ty = 0 up.  §4.1 fixes only that a
    tile's particles are contiguous; the order of the tiles is free."""
    ntx, nty = nx // T, ny // T
    if not window:
        return np.arange(ntx * nty)
    return np.array([ty * ntx + tx for tx in range(ntx - 1, -1, -1) for ty in range(nty)],
                    np.int64)


def tile_offsets_in_order(nx, ny, T, ix, iy, window=False):
    """Bookmarks (ntiles + 1) of particles (ix, iy) with the tiles in
    ``tile_order``."""
    counts = tile_sort(nx, ny, T, ix, iy)[1]
    return np.concatenate([[0], np.cumsum(counts[tile_order(nx, ny, T, window)])]).astype(np.int64)


# ---------------------------------------------------------- grid diagnostics

def field_energy(F, dx, dy):
    """0.5 * sum(F^2) dx dy over the three components (FP64)."""
    F = np.asarray(F, np.float64)
    return 0.5 * float(np.sum(F * F)) * dx * dy


def div_e(E, dx, dy):
    """Discrete div E on nodes (Eq. 17 on the Yee grid), periodic, FP64."""
    E = np.asarray(E, np.float64)
    return ((E[0] - np.roll(E[0], 1, axis=1)) / dx
            + (E[1] - np.roll(E[1], 1, axis=0)) / dy)


def div_j(J, dx, dy):
    """Discrete div J on nodes (J co-located with E), periodic, FP64."""
    return div_e(J, dx, dy)


# ---------------------------------------------------------------- simulation

@dataclass
class SpeciesState:
    """One species: cell index (ix, iy), in-cell offset (x, y), momentum u."""
    q_over_m: float
    qtilde: float          # charge density carried by one particle: sign(q) n_s / ppc_s
    ix: np.ndarray
    iy: np.ndarray
    x: np.ndarray
    y: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    uz: np.ndarray
    pid: np.ndarray | None = None

    @property
    def n(self) -> int:
        return int(self.ix.size)

    def astype(self, dtype) -> "SpeciesState":
        # always copies: the oracle updates its arrays in place and must never
        # write into the caller's input arrays
        c = lambda a: np.array(a, dtype=dtype, copy=True, order="C")
        return SpeciesState(self.q_over_m, self.qtilde,
                            np.array(self.ix, dtype=np.int32, copy=True),
                            np.array(self.iy, dtype=np.int32, copy=True),
                            c(self.x), c(self.y), c(self.ux), c(self.uy), c(self.uz),
                            None if self.pid is None else self.pid.copy())

    def permute(self, perm):
        for name in ("ix", "iy", "x", "y", "ux", "uy", "uz"):
            setattr(self, name, np.ascontiguousarray(getattr(self, name)[perm]))
        if self.pid is not None:
            self.pid = np.ascontiguousarray(self.pid[perm])

    def keep(self, mask):
        """Drop the particles where mask is False."""
        self.permute(np.nonzero(mask)[0])

    def append(self, ix, iy, x, y, ux, uy, uz, pid=None):
        for name, v in (("ix", ix), ("iy", iy), ("x", x), ("y", y), ("ux", ux), ("uy", uy),
                        ("uz", uz)):
            a = getattr(self, name)
            setattr(self, name, np.ascontiguousarray(np.concatenate([a, np.asarray(v, a.dtype)])))
        if self.pid is not None:
            extra = np.full(len(ix), -1, self.pid.dtype) if pid is None else pid
            self.pid = np.concatenate([self.pid, extra])


@dataclass
class OracleSim:
    """Plain serial PIC following Listing 3.1.

    E, B, J are (3, ny, nx) arrays at the Yee locations of Fig. 3.1.  Each step:
    zero J; for each species push every particle and deposit its current; the
    optional binomial filter; Yee B/2, E, B/2; with the moving window (``window``
    set: the box is open along x) the window shift of ``oracle.window``; then
    re-sort each species by tile (stable counting sort, §4.3).  ``background``
    is the fixed neutralising ion density added to rho.  ``window`` is None or
    a list with one ``oracle.window.Inject`` (or None) per species.
    """
    nx: int
    ny: int
    dx: float
    dy: float
    dt: float
    tile: int
    species: list
    dtype: type = np.float64
    background: float = 0.0
    E: np.ndarray = None
    B: np.ndarray = None
    J: np.ndarray = None
    filter_passes: int = 0          # binomial current filter (0: off)
    window: list | None = None      # moving window: injection per species
    moves: int = 0                  # cells the window has moved
    threads: int = 1                # > 1: the threaded particle loop (same particles)
    step_count: int = 0
    status: int = 0
    ke_history: list = field(default_factory=list)

    def __post_init__(self):
        shape = (3, self.ny, self.nx)
        # copies: the Yee step updates E and B in place, never the caller's arrays
        self.E = (np.zeros(shape, self.dtype) if self.E is None
                  else np.array(self.E, dtype=self.dtype, copy=True, order="C"))
        self.B = (np.zeros(shape, self.dtype) if self.B is None
                  else np.array(self.B, dtype=self.dtype, copy=True, order="C"))
        self.J = np.zeros(shape, self.dtype)
        self.species = [s.astype(self.dtype) for s in self.species]

    def kinetic_energy_of(self, sp, gsum):
        # W_K = sum (gamma - 1) m_s n_s/ppc_s dx dy, with m_s n_s/ppc_s = qtilde / (q/m)
        return gsum * (sp.qtilde / sp.q_over_m) * self.dx * self.dy

    def step(self, nsteps: int = 1, sort: bool = True):
        open_x = self.window is not None
        for _ in range(nsteps):
            self.J[...] = 0
            ke = 0.0
            for sp in self.species:
                st, g = advance(sp, self.E, self.B, self.J, self.dx, self.dy, self.dt, open_x,
                                self.threads)
                self.status |= st
                ke += self.kinetic_energy_of(sp, g)
            self.ke_history.append(ke)
            if self.filter_passes:
                self.J[...] = binomial_filter(self.J, self.filter_passes)
            yee(self.E, self.B, self.J, self.dx, self.dy, self.dt, open_x)
            self.step_count += 1
            if open_x:
                from . import window as W
                if W.window_moves(self.step_count, self.dt, self.dx) > self.moves:
                    W.shift_window(self)
            if sort:
                self.sort()

    def sort(self):
        for sp in self.species:
            perm, _, _ = tile_sort(self.nx, self.ny, self.tile, sp.ix, sp.iy)
            sp.permute(perm)

    def tile_offsets(self, s: int = 0):
        sp = self.species[s]
        return tile_offsets_in_order(self.nx, self.ny, self.tile, sp.ix, sp.iy,
                                     window=self.window is not None)

    def rho(self):
        return rho_nodes(self.nx, self.ny, self.species, np.float64, self.background)

    def energies(self):
        return (field_energy(self.E, self.dx, self.dy),
                field_energy(self.B, self.dx, self.dy))
