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


def test_batch_and_tuner_entry_points_check_arguments_without_gpu(lib):
    """Null handles and bad counts answer before any CUDA call."""
    from paper_2501_14795_gb300 import pic
    L = pic.load_library()
    out = ctypes.c_void_p(1)
    assert L.pic_batch_create(None, 2, None, ctypes.byref(out)) == 1 and out.value is None
    members = (ctypes.c_void_p * 2)(None, None)
    assert L.pic_batch_create(members, 0, None, ctypes.byref(out)) == 1
    assert L.pic_batch_create(members, 2, None, ctypes.byref(out)) == 1 and out.value is None
    assert L.pic_batch_step(None, 1) == 1
    assert L.pic_batch_sync(None, None) == 1
    assert L.pic_batch_kernel_launches(None, None) == -1
    assert L.pic_batch_last_error(None) == b"null handle"
    L.pic_batch_destroy(None)
    assert L.pic_autotune(None, 3, 0, None, None, None) == 1
    assert L.pic_set_tiling(None, 16, 0) == 1
    # a batch of configurations fails on the first invalid one, all handles NULL
    good = pic.make_config(64, 64, 0.1, 0.1, 0.05, [(-1.0, -1.0 / 16)])
    bad = pic.make_config(64, 64, 0.1, 0.1, 0.08, [(-1.0, -1.0 / 16)])
    cfgs = (pic.pic_config * 1)(bad)
    hs = (ctypes.c_void_p * 1)(7)
    assert L.pic_init_batch(cfgs, 1, None, hs) == 2 and hs[0] is None
    assert L.pic_init_batch(None, 1, None, hs) == 1
    del good


def test_window_and_laser_entry_points_check_arguments_without_gpu(lib):
    """Null handles answer PIC_EINVAL before any CUDA call; the ABI structs of
    the binding have the sizes of the C declarations (field by field)."""
    from paper_2501_14795_gb300 import pic
    L = pic.load_library()
    assert L.pic_set_moving_window(None, None) == 1
    l = pic.pic_laser(pic.PIC_LASER_PLANE, 1.0, 1.0, 1.0, 10.0, 0.0, 1.0, 0.0, 0.0)
    assert L.pic_add_laser(None, ctypes.byref(l)) == 1
    assert L.pic_add_laser(None, None) == 1


def test_denoiser_restoration_entry_points_check_arguments_without_gpu(lib):
    """Null handles and buffers, and pass counts out of range, answer PIC_EINVAL
    before any CUDA call."""
    from paper_2501_14795_gb300 import pic
    L = pic.load_library()
    assert L.pic_denoiser_set_low_k_restore(None, 2) == 1
    assert L.pic_nn_low_k_restore(None, None, 1, 8, 8, 1, None) == 1
    fake = ctypes.c_void_p(16)      # never dereferenced: the arguments fail first
    assert L.pic_nn_low_k_restore(fake, fake, 1, 8, 8, -1, None) == 1
    assert L.pic_nn_low_k_restore(fake, fake, 1, 8, 8, 65, None) == 1
    assert L.pic_nn_low_k_restore(fake, fake, 0, 8, 8, 1, None) == 1


def test_bounded_wait_probe_checks_its_limit_without_gpu(lib):
    from paper_2501_14795_gb300 import pic
    L = pic.load_library()
    assert L.pic_probe_bounded_wait(0, 0, None) == 1
    assert L.pic_probe_bounded_wait(0, 4_000_000_001, None) == 1


def test_binding_structs_match_the_c_header(tmp_path):
    """sizeof and offsetof of every ABI struct as gcc lays them out from
    include/pic.h equal the ctypes mirrors of the binding."""
    import shutil
    import subprocess
    from paper_2501_14795_gb300 import pic
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    structs = {"pic_config": pic.pic_config, "pic_diag": pic.pic_diag,
               "pic_inject": pic.pic_inject, "pic_laser": pic.pic_laser,
               "pic_species_cfg": pic.pic_species_cfg}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pic.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "abi"
    inc = os.path.join(ROOT, "include")
    subprocess.run(["gcc", "-std=c11", f"-I{inc}", str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, (name, f)
