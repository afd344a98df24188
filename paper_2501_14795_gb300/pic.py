"""Thin ctypes binding of the C ABI in include/pic.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does
nothing but convert arguments: all computation runs in libpic.so's CUDA
kernels.  Arrays may be numpy arrays (host memory) or torch tensors (host or
CUDA); ``on_device`` is inferred from the first array.  If libpic.so cannot be
loaded the binding raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpic.so")

PIC_MAX_SPECIES = 4
PIC_STRICT_FP = 1
PIC_TRACK_IDS = 2
PIC_TIMING = 4
PIC_NO_GRAPH = 8

STATUS = {0: "PIC_OK", 1: "PIC_EINVAL", 2: "PIC_ECFL", 3: "PIC_ENOMEM", 4: "PIC_ECUDA",
          5: "PIC_EOVERFLOW", 6: "PIC_EPARTICLE", 7: "PIC_ETIMEOUT"}
PIC_FP32_J = 16
FIELD_E, FIELD_B, FIELD_J, FIELD_RHO = 0, 1, 2, 3
(PIC_OK, PIC_EINVAL, PIC_ECFL, PIC_ENOMEM, PIC_ECUDA, PIC_EOVERFLOW, PIC_EPARTICLE,
 PIC_ETIMEOUT) = range(8)


class PicError(RuntimeError):
    def __init__(self, status: int, message: str = ""):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {message}")


class pic_species_cfg(C.Structure):
    _fields_ = [("q_over_m", C.c_double), ("density", C.c_double), ("ppc", C.c_double)]


class pic_config(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("dx", C.c_double), ("dy", C.c_double),
                ("dt", C.c_double), ("tile", C.c_int), ("threads", C.c_int),
                ("chunk", C.c_int), ("n_species", C.c_int), ("species", pic_species_cfg * PIC_MAX_SPECIES),
                ("background", C.c_double), ("flags", C.c_uint)]


class pic_diag(C.Structure):
    _fields_ = [("step", C.c_int64), ("time", C.c_double), ("w_e", C.c_double),
                ("w_b", C.c_double), ("w_k", C.c_double), ("gauss_max", C.c_double),
                ("continuity_max", C.c_double), ("charge_total", C.c_double),
                ("n_particles", C.c_int64 * PIC_MAX_SPECIES), ("leavers", C.c_int64),
                ("status_bits", C.c_uint32), ("window_moves", C.c_int64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "n_particles"}
        d["n_particles"] = list(self.n_particles)
        return d


class pic_inject(C.Structure):
    _fields_ = [("k", C.c_int), ("x_start", C.c_double), ("ux", C.c_float), ("uy", C.c_float),
                ("uz", C.c_float), ("capacity", C.c_int64)]


PIC_LASER_PLANE = 0
PIC_LASER_GAUSSIAN = 1


class pic_laser(C.Structure):
    _fields_ = [("type", C.c_int), ("start", C.c_double), ("fwhm", C.c_double),
                ("a0", C.c_double), ("omega0", C.c_double), ("polarization", C.c_double),
                ("W0", C.c_double), ("focus", C.c_double), ("axis", C.c_double)]


_lib = None
_P = C.c_void_p


def load_library() -> C.CDLL:
    """Load libpic.so (built by paper_2501_14795_gb300.build).  Raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        L.pic_init.argtypes = [C.POINTER(pic_config), _P, C.POINTER(_P)]
        L.pic_load_particles.argtypes = [_P, C.c_int, C.c_int64] + [_P] * 8 + [C.c_int]
        L.pic_set_fields.argtypes = [_P, _P, _P, C.c_int]
        L.pic_step.argtypes = [_P, C.c_int]
        L.pic_get_fields.argtypes = [_P, C.c_int, _P, C.c_int]
        L.pic_get_particles.argtypes = [_P, C.c_int] + [_P] * 9 + [C.c_int]
        L.pic_num_particles.argtypes = [_P, C.c_int]
        L.pic_num_particles.restype = C.c_int64
        L.pic_num_tiles.argtypes = [_P]
        L.pic_num_tiles.restype = C.c_int64
        L.pic_diagnostics.argtypes = [_P, C.POINTER(pic_diag)]
        L.pic_get_history.argtypes = [_P, C.c_int64, C.c_int64, _P, _P, _P]
        L.pic_sync.argtypes = [_P]
        L.pic_clear_status.argtypes = [_P]
        L.pic_timing.argtypes = [_P, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int]
        L.pic_timing_stages.argtypes = [_P, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int]
        L.pic_kernel_launches.argtypes = [_P]
        L.pic_kernel_launches.restype = C.c_int64
        L.pic_last_error.argtypes = [_P]
        L.pic_last_error.restype = C.c_char_p
        L.pic_destroy.argtypes = [_P]
        L.pic_destroy.restype = None
        L.pic_tile_sort_noalloc.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int64] + [_P] * 15 + [_P]
        L.pic_tile_sort_noalloc.restype = C.c_int
        L.pic_init_batch.argtypes = [C.POINTER(pic_config), C.c_int, _P, C.POINTER(_P)]
        L.pic_batch_create.argtypes = [C.POINTER(_P), C.c_int, _P, C.POINTER(_P)]
        L.pic_batch_step.argtypes = [_P, C.c_int]
        L.pic_batch_sync.argtypes = [_P, C.POINTER(C.c_int)]
        L.pic_batch_kernel_launches.argtypes = [_P, C.POINTER(C.c_int)]
        L.pic_batch_kernel_launches.restype = C.c_int64
        L.pic_batch_last_error.argtypes = [_P]
        L.pic_batch_last_error.restype = C.c_char_p
        L.pic_batch_destroy.argtypes = [_P]
        L.pic_batch_destroy.restype = None
        L.pic_batch_set_denoiser.argtypes = [_P, _P]
        L.pic_autotune.argtypes = [_P, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                   C.POINTER(C.c_double)]
        L.pic_set_tiling.argtypes = [_P, C.c_int, C.c_int]
        L.pic_denoiser_num_params.argtypes = []
        L.pic_denoiser_num_params.restype = C.c_int64
        L.pic_denoiser_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, _P, C.POINTER(_P)]
        L.pic_denoiser_set_params.argtypes = [_P, _P, C.c_int]
        L.pic_denoiser_get_params.argtypes = [_P, _P, C.c_int]
        L.pic_denoiser_forward.argtypes = [_P, _P, _P, C.c_int, C.c_int]
        L.pic_denoiser_grad.argtypes = [_P, _P, _P, C.c_int, C.POINTER(C.c_double), _P, C.c_int]
        L.pic_denoiser_train_step.argtypes = [_P, _P, _P, C.c_int, C.c_float,
                                              C.POINTER(C.c_double), C.c_int]
        L.pic_set_denoiser.argtypes = [_P, _P]
        L.pic_set_binomial_filter.argtypes = [_P, C.c_int]
        L.pic_set_moving_window.argtypes = [_P, _P]
        L.pic_add_laser.argtypes = [_P, C.POINTER(pic_laser)]
        L.pic_denoiser_last_error.argtypes = [_P]
        L.pic_denoiser_last_error.restype = C.c_char_p
        L.pic_denoiser_destroy.argtypes = [_P]
        L.pic_denoiser_destroy.restype = None
        L.pic_nn_conv3x3.argtypes = [_P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P,
                                     C.c_int, _P, _P, _P, _P]
        L.pic_nn_conv3x3_dgrad.argtypes = [_P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _P,
                                           _P, _P]
        L.pic_nn_conv3x3_wgrad.argtypes = [_P, _P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                           _P, _P]
        L.pic_probe_bounded_wait.argtypes = [C.c_int, C.c_int64, _P]
        L.pic_denoiser_set_low_k_restore.argtypes = [_P, C.c_int]
        L.pic_nn_low_k_restore.argtypes = [_P, _P, C.c_int, C.c_int, C.c_int, C.c_int, _P]
        for name in ("pic_init", "pic_load_particles", "pic_set_fields", "pic_step",
                     "pic_get_fields", "pic_get_particles", "pic_diagnostics",
                     "pic_get_history", "pic_sync", "pic_clear_status", "pic_timing",
                     "pic_timing_stages",
                     "pic_init_batch", "pic_batch_create", "pic_batch_step", "pic_batch_sync",
                     "pic_batch_set_denoiser",
                     "pic_autotune", "pic_set_tiling", "pic_denoiser_create",
                     "pic_denoiser_set_params", "pic_denoiser_get_params", "pic_denoiser_forward",
                     "pic_denoiser_grad", "pic_denoiser_train_step", "pic_set_denoiser",
                     "pic_nn_conv3x3", "pic_nn_conv3x3_dgrad", "pic_nn_conv3x3_wgrad",
                     "pic_set_binomial_filter", "pic_denoiser_set_low_k_restore",
                     "pic_nn_low_k_restore", "pic_probe_bounded_wait"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(h, status):
    if status != 0:
        msg = load_library().pic_last_error(h) if h else b""
        raise PicError(status, (msg or b"").decode())


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype):
    """(pointer, on_device) of a contiguous numpy array or torch tensor."""
    if a is None:
        return None, None
    if _is_torch(a):
        import torch
        want = {np.int32: torch.int32, np.float32: torch.float32,
                np.int64: torch.int64}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"tensor must be contiguous {want}")
        return a.data_ptr(), a.is_cuda
    if not isinstance(a, np.ndarray) or a.dtype != np.dtype(dtype) or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"array must be a C-contiguous numpy {np.dtype(dtype)} array")
    return a.ctypes.data, False


def _default_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


# ------------------------------------------------------------ C entry points

def pic_init(cfg: pic_config, stream=None):
    h = _P()
    if stream is None:
        stream = _default_stream()
    _check(None, load_library().pic_init(C.byref(cfg), stream, C.byref(h)))
    return h


def pic_load_particles(h, species, ix, iy, x, y, ux, uy, uz, id=None):
    arrs = [(ix, np.int32), (iy, np.int32), (x, np.float32), (y, np.float32),
            (ux, np.float32), (uy, np.float32), (uz, np.float32)]
    ptrs = [_ptr(a, d) for a, d in arrs]
    n = int(ix.shape[0]) if hasattr(ix, "shape") else len(ix)
    for a, _ in arrs:
        if int(a.shape[0]) != n:
            raise ValueError("particle arrays differ in length")
    dev = ptrs[0][1]
    if any(p[1] != dev for p in ptrs):
        raise ValueError("particle arrays must all be on the host or all on the device")
    pid = _ptr(id, np.int32)[0] if id is not None else None
    _check(h, load_library().pic_load_particles(h, species, n, *[p[0] for p in ptrs], pid,
                                                int(bool(dev))))


def pic_set_fields(h, E=None, B=None):
    pe, de = _ptr(E, np.float32)
    pb, db = _ptr(B, np.float32)
    dev = de if de is not None else db
    _check(h, load_library().pic_set_fields(h, pe, pb, int(bool(dev))))


def pic_step(h, nsteps=1):
    _check(h, load_library().pic_step(h, int(nsteps)))


def pic_get_fields(h, which, out):
    p, dev = _ptr(out, np.float32)
    _check(h, load_library().pic_get_fields(h, int(which), p, int(bool(dev))))
    return out


def pic_get_particles(h, species, ix=None, iy=None, x=None, y=None, ux=None, uy=None, uz=None,
                      id=None, tile_offset=None):
    ptrs = [_ptr(ix, np.int32), _ptr(iy, np.int32), _ptr(x, np.float32), _ptr(y, np.float32),
            _ptr(ux, np.float32), _ptr(uy, np.float32), _ptr(uz, np.float32),
            _ptr(id, np.int32), _ptr(tile_offset, np.int64)]
    devs = {p[1] for p in ptrs if p[1] is not None}
    if len(devs) > 1:
        raise ValueError("outputs must all be on the host or all on the device")
    dev = devs.pop() if devs else False
    _check(h, load_library().pic_get_particles(h, species, *[p[0] for p in ptrs], int(bool(dev))))


def pic_num_particles(h, species):
    return int(load_library().pic_num_particles(h, species))


def pic_num_tiles(h):
    return int(load_library().pic_num_tiles(h))


def pic_diagnostics(h) -> pic_diag:
    d = pic_diag()
    _check(h, load_library().pic_diagnostics(h, C.byref(d)))
    return d


def pic_get_history(h, first, count):
    we = np.empty(count, np.float64)
    wb = np.empty(count, np.float64)
    wk = np.empty(count, np.float64)
    _check(h, load_library().pic_get_history(h, int(first), int(count), we.ctypes.data,
                                             wb.ctypes.data, wk.ctypes.data))
    return we, wb, wk


def pic_sync(h):
    _check(h, load_library().pic_sync(h))


def pic_clear_status(h):
    _check(h, load_library().pic_clear_status(h))


def pic_timing(h, reset=False):
    ms = C.c_double()
    cnt = C.c_int64()
    _check(h, load_library().pic_timing(h, C.byref(ms), C.byref(cnt), int(reset)))
    return ms.value, cnt.value


def pic_timing_stages(h, reset=False):
    """(advance, re-sort, field) milliseconds summed over the timed steps, and
    the number of steps."""
    ms = (C.c_double * 3)()
    cnt = C.c_int64()
    _check(h, load_library().pic_timing_stages(h, ms, C.byref(cnt), int(reset)))
    return (ms[0], ms[1], ms[2]), cnt.value


def pic_kernel_launches(h):
    return int(load_library().pic_kernel_launches(h))


def pic_last_error(h):
    return (load_library().pic_last_error(h) or b"").decode()


def pic_destroy(h):
    load_library().pic_destroy(h)


def pic_init_batch(cfgs, stream=None):
    """n simulations on one stream; returns their handles."""
    n = len(cfgs)
    arr = (pic_config * n)(*cfgs)
    out = (_P * n)()
    if stream is None:
        stream = _default_stream()
    _check(None, load_library().pic_init_batch(arr, n, stream, out))
    return [_P(v) for v in out]


def _bcheck(b, status):
    if status != 0:
        msg = load_library().pic_batch_last_error(b) if b else b""
        raise PicError(status, (msg or b"").decode())


def pic_batch_create(members, stream=None):
    n = len(members)
    arr = (_P * n)(*[m.value if isinstance(m, _P) else m for m in members])
    b = _P()
    if stream is None:
        stream = _default_stream()
    st = load_library().pic_batch_create(arr, n, stream, C.byref(b))
    if st != 0:
        msg = ""
        for m in members:
            if m and pic_last_error(m):
                msg = pic_last_error(m)
                break
        raise PicError(st, msg or "pic_batch_create")
    return b


def pic_batch_step(b, nsteps=1):
    _bcheck(b, load_library().pic_batch_step(b, nsteps))


def pic_batch_sync(b):
    """Wait; raise the first failing member's status (PicError.member set)."""
    m = C.c_int(-1)
    st = load_library().pic_batch_sync(b, C.byref(m))
    if st != 0:
        e = PicError(st, (load_library().pic_batch_last_error(b) or b"").decode())
        e.member = m.value
        raise e


def pic_batch_kernel_launches(b):
    per = C.c_int(0)
    tot = load_library().pic_batch_kernel_launches(b, C.byref(per))
    return int(tot), per.value


def pic_batch_last_error(b):
    return (load_library().pic_batch_last_error(b) or b"").decode()


def pic_batch_set_denoiser(b, d):
    _bcheck(b, load_library().pic_batch_set_denoiser(b, d))


def pic_batch_destroy(b):
    load_library().pic_batch_destroy(b)


def pic_autotune(h, steps=5, force=False):
    """(tile, threads, step_ms) chosen for a loaded simulation (see pic.h)."""
    t, n, ms = C.c_int(), C.c_int(), C.c_double()
    _check(h, load_library().pic_autotune(h, steps, int(force), C.byref(t), C.byref(n),
                                          C.byref(ms)))
    return t.value, n.value, ms.value


def pic_set_tiling(h, tile, threads=0):
    _check(h, load_library().pic_set_tiling(h, tile, threads))


# ------------------------------------------------------------ denoiser

def _dcheck(d, status):
    if status != 0:
        msg = load_library().pic_denoiser_last_error(d) if d else b""
        raise PicError(status, (msg or b"").decode())


def pic_denoiser_num_params():
    return int(load_library().pic_denoiser_num_params())


def pic_denoiser_create(nx, ny, batch_max, scale, stream=None):
    d = _P()
    if stream is None:
        stream = _default_stream()
    st = load_library().pic_denoiser_create(nx, ny, batch_max, float(scale), stream, C.byref(d))
    if st != 0:
        raise PicError(st, "pic_denoiser_create")
    return d


def pic_denoiser_set_params(d, params):
    p, dev = _ptr(params, np.float32)
    _dcheck(d, load_library().pic_denoiser_set_params(d, p, int(dev)))


def pic_denoiser_get_params(d, out):
    p, dev = _ptr(out, np.float32)
    _dcheck(d, load_library().pic_denoiser_get_params(d, p, int(dev)))


def _same_place(*arrs):
    ptrs = [_ptr(a, np.float32) for a in arrs if a is not None]
    devs = {dv for _, dv in ptrs}
    if len(devs) != 1:
        raise ValueError("buffers must all be on the host or all on the device")
    return [p for p, _ in ptrs], devs.pop()


def pic_denoiser_forward(d, J_in, J_out, batch):
    (pi, po), dev = _same_place(J_in, J_out)
    _dcheck(d, load_library().pic_denoiser_forward(d, pi, po, batch, int(dev)))


def pic_denoiser_grad(d, J_in, J_target, batch, grads=None):
    ptrs, dev = _same_place(J_in, J_target, grads)
    loss = C.c_double()
    _dcheck(d, load_library().pic_denoiser_grad(d, ptrs[0], ptrs[1], batch, C.byref(loss),
                                                ptrs[2] if grads is not None else None, int(dev)))
    return loss.value


def pic_denoiser_train_step(d, J_in, J_target, batch, lr):
    (pi, pt), dev = _same_place(J_in, J_target)
    loss = C.c_double()
    _dcheck(d, load_library().pic_denoiser_train_step(d, pi, pt, batch, float(lr),
                                                      C.byref(loss), int(dev)))
    return loss.value


def pic_denoiser_set_low_k_restore(d, passes):
    _dcheck(d, load_library().pic_denoiser_set_low_k_restore(d, int(passes)))


def pic_set_denoiser(h, d):
    _check(h, load_library().pic_set_denoiser(h, d))


def pic_set_binomial_filter(h, passes):
    _check(h, load_library().pic_set_binomial_filter(h, int(passes)))


def pic_set_moving_window(h, injects=None):
    """injects: None or one dict per species with keys k, x_start, ux, uy, uz,
    capacity (None entries: no injection)."""
    L = load_library()
    if injects is None:
        _check(h, L.pic_set_moving_window(h, None))
        return
    arr = (pic_inject * len(injects))()
    for a, q in zip(arr, injects):
        q = q or {}
        a.k = int(q.get("k", 0))
        a.x_start = float(q.get("x_start", 0.0))
        a.ux, a.uy, a.uz = (float(q.get(c, 0.0)) for c in ("ux", "uy", "uz"))
        a.capacity = int(q.get("capacity", 0))
    _check(h, L.pic_set_moving_window(h, arr))


def pic_add_laser(h, kind="plane", start=0.0, fwhm=1.0, a0=1.0, omega0=10.0, polarization=0.0,
                  W0=1.0, focus=0.0, axis=0.0):
    l = pic_laser(PIC_LASER_GAUSSIAN if kind == "gaussian" else PIC_LASER_PLANE, start, fwhm, a0,
                  omega0, polarization, W0, focus, axis)
    if kind not in ("plane", "gaussian"):
        raise ValueError(kind)
    _check(h, load_library().pic_add_laser(h, C.byref(l)))


def pic_denoiser_destroy(d):
    load_library().pic_denoiser_destroy(d)


def _dptr(t):
    """device pointer of a contiguous torch CUDA tensor (any dtype)."""
    if t is None:
        return None
    if not (_is_torch(t) and t.is_cuda and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def pic_nn_conv3x3(x, w, bias, a_out, relu=True, skip=None, y_out=None, stream=None):
    """x, skip, a_out, y_out: bfloat16 NHWC CUDA tensors; w [3,3,cin,cout], bias FP32."""
    B, H, W, _ = x.shape
    cin, cout = int(w.shape[2]), int(w.shape[3])
    if stream is None:
        stream = _default_stream()
    st = load_library().pic_nn_conv3x3(_dptr(x), B, H, W, cin, cout, _dptr(w), _dptr(bias),
                                       int(relu), _dptr(skip), _dptr(a_out), _dptr(y_out), stream)
    if st != 0:
        raise PicError(st, "pic_nn_conv3x3")


def pic_nn_conv3x3_dgrad(dz, w, dx, stream=None):
    B, H, W, _ = dz.shape
    cin, cout = int(w.shape[2]), int(w.shape[3])
    if stream is None:
        stream = _default_stream()
    st = load_library().pic_nn_conv3x3_dgrad(_dptr(dz), B, H, W, cin, cout, _dptr(w), _dptr(dx),
                                             stream)
    if st != 0:
        raise PicError(st, "pic_nn_conv3x3_dgrad")


def pic_nn_conv3x3_wgrad(x, dz, dw, stream=None):
    B, H, W, _ = x.shape
    cin, cout = int(dw.shape[2]), int(dw.shape[3])
    if stream is None:
        stream = _default_stream()
    st = load_library().pic_nn_conv3x3_wgrad(_dptr(x), _dptr(dz), B, H, W, cin, cout, _dptr(dw),
                                             stream)
    if st != 0:
        raise PicError(st, "pic_nn_conv3x3_wgrad")


def pic_probe_bounded_wait(arrive, limit_cycles, stream=None):
    """Status code of the bounded-wait probe (0 = PIC_OK, PIC_ETIMEOUT)."""
    if stream is None:
        stream = _default_stream()
    return load_library().pic_probe_bounded_wait(int(arrive), int(limit_cycles), stream)


def pic_nn_low_k_restore(raw, out, passes, stream=None):
    """out <- out + L^passes (raw - out) on device FP32 currents [B, 3, H, W]."""
    B, three, H, W = out.shape
    if three != 3 or tuple(raw.shape) != tuple(out.shape):
        raise ValueError("raw and out must both be [B, 3, H, W]")
    if stream is None:
        stream = _default_stream()
    st = load_library().pic_nn_low_k_restore(_dptr(raw), _dptr(out), B, H, W, int(passes), stream)
    if st != 0:
        raise PicError(st, "pic_nn_low_k_restore")


def pic_tile_sort_noalloc(nx, ny, tile, ix, iy, x, y, ux, uy, uz, ix_out, iy_out, x_out,
                          y_out, ux_out, uy_out, uz_out, tile_offset, stream=None):
    """Allocation-free tile sort of device arrays into device arrays (see pic.h)."""
    ins = [_ptr(ix, np.int32), _ptr(iy, np.int32)] + [_ptr(a, np.float32) for a in (x, y, ux, uy, uz)]
    outs = [_ptr(ix_out, np.int32), _ptr(iy_out, np.int32)] + \
        [_ptr(a, np.float32) for a in (x_out, y_out, ux_out, uy_out, uz_out)]
    off = _ptr(tile_offset, np.int64)
    if not all(p[1] for p in ins + outs + [off]):
        raise ValueError("pic_tile_sort_noalloc takes device arrays only")
    n = int(ix.shape[0])
    if stream is None:
        stream = _default_stream()
    st = load_library().pic_tile_sort_noalloc(nx, ny, tile, n, *[p[0] for p in ins],
                                              *[p[0] for p in outs], off[0], stream)
    if st != 0:
        raise PicError(st, "pic_tile_sort_noalloc")


# ------------------------------------------------------------- conveniences

def make_config(nx, ny, dx, dy, dt, species, tile=16, threads=256, background=1.0, flags=0,
                chunk=0):
    """pic_config from (q_over_m, qtilde) pairs: qtilde = sign(q/m) n_s/ppc_s."""
    cfg = pic_config()
    cfg.nx, cfg.ny, cfg.dx, cfg.dy, cfg.dt = nx, ny, dx, dy, dt
    cfg.tile, cfg.threads, cfg.background, cfg.flags = tile, threads, background, flags
    cfg.chunk = chunk
    cfg.n_species = len(species)
    for k, (qm, qt) in enumerate(species):
        cfg.species[k].q_over_m = qm
        cfg.species[k].density = abs(qt)
        cfg.species[k].ppc = 1.0
    return cfg


def config_for(workload, tile=None, threads=256, flags=0, chunk=0):
    return make_config(workload.nx, workload.ny, workload.dx, workload.dy, workload.dt,
                       [(s.q_over_m, s.qtilde) for s in workload.species],
                       tile=tile or workload.tile, threads=threads,
                       background=workload.background, flags=flags, chunk=chunk)


class Simulation:
    """Owner of one pic_sim handle; methods forward to the entry points above."""

    def __init__(self, cfg: pic_config, stream=None):
        self.cfg = cfg
        self.window = False
        self.h = pic_init(cfg, stream)

    @classmethod
    def from_workload(cls, w, tile=None, threads=256, flags=0, stream=None, device=False,
                      chunk=0):
        sim = cls(config_for(w, tile, threads, flags, chunk), stream)
        if getattr(w, "window", None) is not None:
            sim.set_moving_window(w.window)
        for k, s in enumerate(w.species):
            arrs = s.arrays()
            if device:
                import torch
                arrs = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]
            pic_load_particles(sim.h, k, *arrs)
        if w.E0 is not None or w.B0 is not None:
            E = None if w.E0 is None else np.ascontiguousarray(w.E0, np.float32).reshape(-1)
            B = None if w.B0 is None else np.ascontiguousarray(w.B0, np.float32).reshape(-1)
            pic_set_fields(sim.h, E, B)
        for l in getattr(w, "lasers", None) or []:
            sim.add_laser(**l)
        return sim

    def set_moving_window(self, injects=None):
        pic_set_moving_window(self.h, injects)
        self.window = True

    def add_laser(self, **laser):
        pic_add_laser(self.h, **laser)

    @classmethod
    def init_batch(cls, cfgs, stream=None):
        """Simulations created together on one stream (pic_init_batch)."""
        out = []
        for cfg, h in zip(cfgs, pic_init_batch(cfgs, stream)):
            s = cls.__new__(cls)
            s.cfg, s.h = cfg, h
            out.append(s)
        return out

    def step(self, n=1):
        pic_step(self.h, n)

    def autotune(self, steps=5, force=False):
        t, n, ms = pic_autotune(self.h, steps, force)
        self.cfg.tile, self.cfg.threads = t, n
        return t, n, ms

    def set_tiling(self, tile, threads=0):
        pic_set_tiling(self.h, tile, threads)
        self.cfg.tile = tile
        if threads:
            self.cfg.threads = threads

    def num_tiles(self):
        return pic_num_tiles(self.h)

    def fields(self, which):
        n = 3 if which in (FIELD_E, FIELD_B, FIELD_J) else 1
        out = np.empty(n * self.cfg.nx * self.cfg.ny, np.float32)
        pic_get_fields(self.h, which, out)
        return out.reshape((n, self.cfg.ny, self.cfg.nx) if n == 3 else (self.cfg.ny, self.cfg.nx))

    def particles(self, species=0, ids=False):
        if self.window:
            pic_sync(self.h)     # synchronises and refreshes the changing counts
        n = pic_num_particles(self.h, species)
        out = dict(ix=np.empty(n, np.int32), iy=np.empty(n, np.int32), x=np.empty(n, np.float32),
                   y=np.empty(n, np.float32), ux=np.empty(n, np.float32),
                   uy=np.empty(n, np.float32), uz=np.empty(n, np.float32))
        if ids:
            out["id"] = np.empty(n, np.int32)
        out["tile_offset"] = np.empty(pic_num_tiles(self.h) + 1, np.int64)
        pic_get_particles(self.h, species, **out)
        return out

    def diagnostics(self):
        return pic_diagnostics(self.h).as_dict()

    def history(self, first, count):
        return pic_get_history(self.h, first, count)

    def close(self):
        if self.h:
            pic_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owner of a pic_batch over existing Simulation objects (kept alive here)."""

    def __init__(self, sims, stream=None):
        self.sims = list(sims)
        self.b = pic_batch_create([s.h for s in self.sims], stream)

    def step(self, n=1):
        pic_batch_step(self.b, n)

    def sync(self):
        pic_batch_sync(self.b)

    def kernel_launches(self):
        return pic_batch_kernel_launches(self.b)

    def set_denoiser(self, net):
        """Install a Denoiser (None: remove) in every member's current-filter
        slot, run over all members at once; the network is kept alive here."""
        pic_batch_set_denoiser(self.b, net.d if net is not None else None)
        self.net = net

    def close(self):
        if self.b:
            pic_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Denoiser:
    """Owner of a pic_denoiser handle."""

    def __init__(self, nx, ny, batch_max=1, scale=1.0, stream=None):
        self.nx, self.ny, self.batch_max, self.scale = nx, ny, batch_max, scale
        self.d = pic_denoiser_create(nx, ny, batch_max, scale, stream)

    @staticmethod
    def num_params():
        return pic_denoiser_num_params()

    def set_params(self, flat):
        pic_denoiser_set_params(self.d, flat)

    def params(self):
        out = np.empty(self.num_params(), np.float32)
        pic_denoiser_get_params(self.d, out)
        return out

    def forward(self, J_in, J_out=None):
        batch = J_in.shape[0] if J_in.ndim == 4 else 1
        if J_out is None:
            J_out = np.empty_like(J_in)
        pic_denoiser_forward(self.d, J_in, J_out, batch)
        return J_out

    def set_low_k_restore(self, passes):
        """Passes of the low-wavenumber restoration after the network (0: off);
        a simulation picks a change up when the denoiser is installed again."""
        pic_denoiser_set_low_k_restore(self.d, passes)

    def grad(self, J_in, J_target, grads=None):
        batch = J_in.shape[0] if J_in.ndim == 4 else 1
        return pic_denoiser_grad(self.d, J_in, J_target, batch, grads)

    def train_step(self, J_in, J_target, lr):
        batch = J_in.shape[0] if J_in.ndim == 4 else 1
        return pic_denoiser_train_step(self.d, J_in, J_target, batch, lr)

    def close(self):
        if self.d:
            pic_denoiser_destroy(self.d)
            self.d = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
