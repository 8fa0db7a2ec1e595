"""Build the CUDA library in-tree for sm_103a.

``python -m paper_1604_01829_gb300.build`` compiles the translation units
under ``csrc/`` in parallel with nvcc and links ``_lib/liblbrasp.so``; the
Python binding loads that file. No torch types cross the library boundary,
so the library links only the CUDA runtime.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
OBJ_DIR = os.path.join(OUT_DIR, "obj")
LIB = os.path.join(OUT_DIR, "liblbrasp.so")
# checked build (-DLB_CHECKS): every kernel index tested against its array's
# extent, a failure reported as LB_ERR_STATE instead of an out-of-bounds access
LIB_CHECKED = os.path.join(OUT_DIR, "liblbrasp_checked.so")
OBJ_DIR_CHECKED = os.path.join(OUT_DIR, "obj_checked")
SOURCES = ["lb_fluid.cu", "lb_fluid_tma.cu", "lb_bodies.cu", "lb_api.cu", "lb_batch.cu", "lb_adjoint.cu", "lb_static.cu",
           "lb_traj.cu", "lb_shell.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return cand


def _deps():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [
        os.path.join(os.path.dirname(HERE), "include", "lb.h"), __file__]


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=(), checked: bool = False) -> str:
    """Compile the library (checked=True: the index-checked build, a separate
    file) unless it is newer than every source; returns its path."""
    lib = LIB_CHECKED if checked else LIB
    obj_dir = OBJ_DIR_CHECKED if checked else OBJ_DIR
    if checked:
        extra_flags = tuple(extra_flags) + ("-DLB_CHECKS",)
    if not force and up_to_date(lib):
        return lib
    os.makedirs(obj_dir, exist_ok=True)
    nv = nvcc()

    def compile_one(src):
        obj = os.path.join(obj_dir, src.replace(".cu", ".o"))
        cmd = [nv, *ARCH, *FLAGS, *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    # --no-undefined: a declaration without a matching definition fails here
    # rather than when the library is loaded
    cmd = [nv, *ARCH, "-shared", "-Xlinker", "--no-undefined", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    v = "-v" in sys.argv
    flags = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(force=True, verbose=v or bool(flags), extra_flags=flags, checked="--checked" in sys.argv))
