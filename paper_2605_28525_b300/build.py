"""Build the native library libmpm_b300.so in-tree with nvcc for sm_103a.

    python -m paper_2605_28525_b300.build        # incremental
    python -m paper_2605_28525_b300.build --force

Each .cu under csrc/ is compiled to an object (-gencode
arch=compute_103a,code=sm_103a, -O3, -lineinfo), then linked into one shared
library against the shared CUDA runtime, so that a process that already
loaded PyTorch's libcudart.so.13 uses that same runtime.
"""
from __future__ import annotations

import argparse
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmpm_b300.so")
# the checked build: every indirect index of the hot kernels tested against its
# buffer (MPM_CHECKED=1); same entry points, for validation runs
CHECKED_LIB = os.path.join(HERE, "libmpm_b300_checked.so")
CHECKED_OBJ = os.path.join(HERE, "_build_checked")
HEADERS = [os.path.join(ROOT, "include", "mpm.h"), os.path.join(CSRC, "mpm_internal.cuh")]
NVCC = "/usr/local/cuda/bin/nvcc"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
         "-Xptxas", "-warn-spills"]


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _newer(src_list, target):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in src_list)


def build(force: bool = False, verbose: bool = False, out: str = LIB, obj_dir: str = OBJ, defines=()) -> str:
    """Compile every csrc/*.cu and link `out`.  `defines` (e.g. ("MPM_JACOBI_SWEEPS=3",))
    and a separate `obj_dir` build variants side by side."""
    os.makedirs(obj_dir, exist_ok=True)
    extra = ["-D" + d for d in defines]
    objs = []
    for src in sources():
        obj = os.path.join(obj_dir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or _newer([src] + HEADERS, obj):
            cmd = [NVCC] + ARCH + FLAGS + extra + ["-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd), flush=True)
            subprocess.check_call(cmd)
    if force or _newer(objs, out):
        tmp = out + ".tmp%d" % os.getpid()
        cmd = [NVCC] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + \
              ["-Xlinker", "-rpath,/usr/local/cuda/lib64"]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.check_call(cmd)
        os.replace(tmp, out)
    return out


def build_checked(force: bool = False, verbose: bool = False) -> str:
    """The checked library (MPM_CHECKED=1) beside the normal one."""
    return build(force=force, verbose=verbose, out=CHECKED_LIB, obj_dir=CHECKED_OBJ, defines=("MPM_CHECKED=1",))


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--checked", action="store_true", help="also build the checked library")
    a = ap.parse_args()
    print(build(force=a.force, verbose=True))
    if a.checked:
        print(build_checked(force=a.force, verbose=True))
