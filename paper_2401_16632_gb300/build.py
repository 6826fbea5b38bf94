"""Build the sm_103a shared library ``libhfr.so`` in-tree with nvcc.

Translation units are compiled in parallel (one ``-gencode``, no cmake) and linked into
``paper_2401_16632_gb300/libhfr.so``.
"""

from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhfr.so")
LIB_CHECKED = os.path.join(HERE, "libhfr_checked.so")
UNITS = ["hfr_residual", "hfr_jacobian", "hfr_condense", "hfr_linalg", "hfr_krylov", "hfr_gmres_fused", "hfr_api", "hfr_noalloc", "hfr_layout", "hfr_peaks", "hfr_general", "hfr_hex"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhfr.so")
    return exe


def _sources_newer_than(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    for name in os.listdir(CSRC):
        if os.path.getmtime(os.path.join(CSRC, name)) > t:
            return True
    hdr = os.path.join(os.path.dirname(HERE), "include", "hfr.h")
    return os.path.getmtime(hdr) > t


def build(force: bool = False, verbose: bool = False, extra_flags=None, checked: bool = False) -> str:
    """Compile every CUDA translation unit for sm_103a and link libhfr.so (checked: the
    bounds-checked variant libhfr_checked.so, compiled with FR_CHECKED); returns its path."""
    lib = LIB_CHECKED if checked else LIB
    bdir = BUILD + "_checked" if checked else BUILD
    if not force and not _sources_newer_than(lib):
        return lib
    os.makedirs(bdir, exist_ok=True)
    exe = nvcc()
    extra = list(extra_flags or []) + (["-DFR_CHECKED"] if checked else [])

    def compile_unit(u):
        src = os.path.join(CSRC, u + ".cu")
        obj = os.path.join(bdir, u + ".o")
        cmd = [exe, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {u}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_unit, UNITS))
    tmp = lib + ".tmp"
    cmd = [exe, "-shared", *ARCH, *objs, "-ldl", "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
