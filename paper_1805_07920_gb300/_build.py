"""In-tree build of the native libraries of this package.

* ``_lib/libamh.so``      -- the CUDA library behind the C-ABI in ``include/amh.h``
                             (nvcc, sm_103a only, static cudart, no torch types).
* ``_lib/libscenegen.so`` -- the seeded synthetic-scene ray caster (gcc, OpenMP).

The CUDA sources compile one object each, side by side, then link; nothing
is installed outside the source tree.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
REPO_DIR = os.path.dirname(PKG_DIR)
LIB_DIR = os.path.join(PKG_DIR, "_lib")
OBJ_DIR = os.path.join(LIB_DIR, "obj")
CSRC = os.path.join(PKG_DIR, "csrc")
INCLUDE = os.path.join(REPO_DIR, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def amh_sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _run_all(cmds: list[list[str]], verbose: bool) -> None:
    """Run the commands side by side; raise with the log of the first failure."""
    procs = []
    for cmd in cmds:
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    failed = None
    for cmd, p in procs:
        log, _ = p.communicate()
        if p.returncode != 0 and failed is None:
            failed = f"build failed ({' '.join(cmd)}):\n{log}"
        elif verbose and log.strip():
            print(log, file=sys.stderr)
    if failed:
        raise RuntimeError(failed)


def build(verbose: bool = False, extra_nvcc: list[str] | None = None, bounds_checked: bool = False) -> list[str]:
    """Compile every native library of the package; raise on any failure.
    Each CUDA source compiles to its own object at the same time as the
    others (and the scene generator), then one link makes ``libamh.so``.
    ``bounds_checked`` builds ``libamh_checked.so`` instead: the same library
    with -DAMH_BOUNDS_CHECK (every index of the update checked, see
    amh_bounds_checked in include/amh.h)."""
    obj_dir = OBJ_DIR + ("_checked" if bounds_checked else "")
    os.makedirs(obj_dir, exist_ok=True)
    nvcc = _nvcc()
    flags = [*(extra_nvcc or []), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
             "-Xcompiler", "-fvisibility=hidden", "-I", INCLUDE]
    if bounds_checked:
        flags.append("-DAMH_BOUNDS_CHECK")
    objs, cmds = [], []
    for src in amh_sources():
        obj = os.path.join(obj_dir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmds.append([nvcc, *flags, "-c", "-o", obj, src])
    sg = os.path.join(PKG_DIR, "synth", "scenegen.c")
    scenegen = os.path.join(LIB_DIR, "libscenegen.so")
    cmds.append(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", scenegen, sg, "-lm"])
    _run_all(cmds, verbose)
    lib = os.path.join(LIB_DIR, "libamh_checked.so" if bounds_checked else "libamh.so")
    _run_all([[nvcc, *ARCH, "-shared", "-o", lib, *objs]], verbose)
    return [lib, scenegen]


if __name__ == "__main__":
    for o in build(verbose=True):
        print(o)
