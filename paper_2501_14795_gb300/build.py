"""Build the sm_103a CUDA library (libpic.so) in-tree with nvcc.

The translation units compile in parallel; kernels_push.cu is compiled twice
(FMA-contracting "fast" build and the no-contraction "strict" build).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libpic.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpic.so")
    return p


def _units():
    common = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              f"-I{os.path.join(ROOT, 'include')}", f"-I{CSRC}"]
    return [
        # flush-to-zero: no subnormal handling around the fast reciprocal
        # square roots and divisions (every value on this path is far from
        # the subnormal range)
        ("push_fast.o", "kernels_push.cu", common + ["-DPIC_VARIANT=fast", "-ftz=true"]),
        ("push_strict.o", "kernels_push.cu",
         common + ["-DPIC_VARIANT=strict", "-DPIC_STRICT_BUILD", "-fmad=false"]),
        ("sort.o", "kernels_sort.cu", common),
        ("grid.o", "kernels_grid.cu", common),
        ("host.o", "pic_host.cu", common),
        ("batch.o", "pic_batch.cu", common),
        ("nn.o", "nn_kernels.cu", common),
        ("nn_tc.o", "nn_tc.cu", common),
        ("denoiser.o", "denoiser.cu", common),
        ("noalloc.o", "noalloc.cu", common),
    ]


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "pic.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build_library(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()

    def compile_one(u):
        obj, src, flags = u
        cmd = [cc, *flags, "-c", os.path.join(CSRC, src), "-o", os.path.join(BUILD, obj)]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        return obj, cmd, r

    with ThreadPoolExecutor(max_workers=min(10, os.cpu_count() or 1)) as ex:
        results = list(ex.map(compile_one, _units()))
    for obj, cmd, r in results:
        if verbose or ptxas_info:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {obj}:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *[os.path.join(BUILD, u[0]) for u in _units()]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build_library(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
