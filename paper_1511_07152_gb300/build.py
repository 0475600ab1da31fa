"""Build libsepw.so from csrc/*.cu with nvcc for sm_103a (GB300), in tree.

Each translation unit is compiled in parallel, then linked into
``paper_1511_07152_gb300/_build/libsepw.so`` (static CUDA runtime, dynamic
cuFFT).  Portable host flags only: the same sources build on x86-64 and on
aarch64 (Grace).  ``build(checked=True)`` builds the bounds-checked variant
``_build/libsepw_checked.so`` (-DSEPW_CHECKED=1: the scatter-form kernels
check work items and plan records before use and record SEPW_EBOUNDS instead
of accessing out of range); setting SEPW_CHECKED=1 in the environment makes
the binding load it.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libsepw.so")
LIB_CHECKED = os.path.join(OUT_DIR, "libsepw_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _cuda_lib_dir(nvcc: str) -> str:
    root = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    for sub in ("lib64", "lib", "targets/sbsa-linux/lib", "targets/x86_64-linux/lib"):
        d = os.path.join(root, sub)
        if os.path.exists(os.path.join(d, "libcufft.so")):
            return d
    return os.path.join(root, "lib64")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + \
        sorted(glob.glob(os.path.join(INCLUDE, "*.h")))


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    lib = LIB_CHECKED if checked else LIB
    if not force and up_to_date(lib):
        return lib
    nvcc = _nvcc()
    obj_dir = os.path.join(OUT_DIR, "checked") if checked else OUT_DIR
    os.makedirs(obj_dir, exist_ok=True)
    # host arithmetic that must match the FP64 oracle bit for bit (facet
    # centre n0) is not contracted into fused multiply-adds
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-ffp-contract=off",
                    "-Xcompiler", "-fPIC",
                    "-Xcompiler", "-fvisibility=hidden", f"-I{INCLUDE}"] + \
        (["-DSEPW_CHECKED=1"] if checked else [])
    objs = []

    def compile_one(src):
        obj = os.path.join(obj_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc] + flags + ["-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd))
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, _sources()))
    libdir = _cuda_lib_dir(nvcc)
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + \
        [f"-L{libdir}", "-lcufft", "-Xlinker", f"-rpath={libdir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
