"""In-tree build of the native libraries of this package.

* ``_lib/libamh.so``      -- the CUDA library behind the C-ABI in ``include/amh.h``
                             (nvcc, sm_103a only, static cudart, no torch types).
* ``_lib/libscenegen.so`` -- the seeded synthetic-scene ray caster (gcc, OpenMP).

Both compile in parallel in a few seconds; nothing is installed outside the
source tree.
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


def commands(extra_nvcc: list[str] | None = None) -> list[tuple[str, list[str]]]:
    os.makedirs(LIB_DIR, exist_ok=True)
    cmds = []
    srcs = amh_sources()
    if srcs:
        out = os.path.join(LIB_DIR, "libamh.so")
        cmd = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared",
               "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
               "-I", INCLUDE, "-o", out, *srcs]
        if extra_nvcc:
            cmd[1:1] = extra_nvcc
        cmds.append((out, cmd))
    sg = os.path.join(PKG_DIR, "synth", "scenegen.c")
    out = os.path.join(LIB_DIR, "libscenegen.so")
    cmds.append((out, ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                       "-o", out, sg, "-lm"]))
    return cmds


def build(verbose: bool = False, extra_nvcc: list[str] | None = None) -> list[str]:
    """Compile every native library of the package; raise on any failure."""
    procs = []
    for out, cmd in commands(extra_nvcc):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((out, cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                                 stderr=subprocess.STDOUT, text=True)))
    outs = []
    for out, cmd, p in procs:
        log, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(f"build failed ({' '.join(cmd)}):\n{log}")
        if verbose and log.strip():
            print(log, file=sys.stderr)
        outs.append(out)
    return outs


if __name__ == "__main__":
    for o in build(verbose=True):
        print(o)
