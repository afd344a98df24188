"""Host-side checks of the C ABI (no GPU): the library builds, loads, and
exports every entry point include/pic.h declares; the binding rejects bad
arguments before any device call."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "pic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2501_14795_gb300 import build
    path = build.build_library()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for want in ("pic_init", "pic_load_particles", "pic_step", "pic_get_fields",
                 "pic_diagnostics", "pic_destroy", "pic_set_fields", "pic_get_particles"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_entry_points() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_and_rejects_bad_arrays(lib):
    from paper_2501_14795_gb300 import pic
    L = pic.load_library()
    assert L.pic_num_tiles(None) == -1
    assert L.pic_last_error(None) == b"null handle"
    with pytest.raises(TypeError):
        pic._ptr(np.zeros(4, np.float64), np.float32)
    with pytest.raises(TypeError):
        pic._ptr(np.zeros((4, 4), np.float32)[:, 1], np.float32)


def test_init_validation_without_gpu(lib):
    """Argument checks run before any CUDA call: they answer on a CPU machine."""
    from paper_2501_14795_gb300 import pic
    L = pic.load_library()
    h = ctypes.c_void_p()

    def status(**kw):
        base = dict(nx=64, ny=64, dx=0.1, dy=0.1, dt=0.05, tile=16)
        base.update(kw)
        cfg = pic.make_config(base["nx"], base["ny"], base["dx"], base["dy"], base["dt"],
                              [(-1.0, -1.0 / 16)], tile=base["tile"])
        return L.pic_init(ctypes.byref(cfg), None, ctypes.byref(h))

    assert status(dt=0.08) == 2          # PIC_ECFL: dt >= (1/dx^2+1/dy^2)^-1/2 = 0.0707
    assert status(dt=0.0707107) == 2
    assert status(tile=12) == 1          # tile not in {8,16,32}
    assert status(nx=72) == 1            # nx not a multiple of the tile
    assert status(nx=4, tile=8) == 1
    assert status(dx=-0.1) == 1
    assert h.value is None
