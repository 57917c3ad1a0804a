"""Builds libdw.so (the sm_103a CUDA library behind include/dw.h) in-tree.

Every csrc/*.cu file is compiled by nvcc in parallel for sm_103a only, then
linked into paper_2001_05218_gb300/libdw.so with the static CUDA runtime.
Objects go to paper_2001_05218_gb300/_build/; a file is recompiled when it or
any header in csrc/ or include/ is newer than its object.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libdw.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdw.so")


def _newest_header() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    return max(os.path.getmtime(h) for h in hs)


def build(verbose: bool = False, jobs: int | None = None, extra: list[str] | None = None) -> str:
    """extra (or the DW_EXTRA_NVCC environment variable) adds nvcc flags; a
    change of flags rebuilds every object."""
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    extra = list(extra or []) + os.environ.get("DW_EXTRA_NVCC", "").split()
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdr = _newest_header()
    stamp = os.path.join(BUILD, "flags.txt")
    flags_now = " ".join(ARCH + FLAGS + extra)
    if not os.path.exists(stamp) or open(stamp).read() != flags_now:
        for o in glob.glob(os.path.join(BUILD, "*.o")):
            os.remove(o)
        with open(stamp, "w") as f:
            f.write(flags_now)
    todo = []
    objs = []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hdr):
            todo.append((s, o))

    def comp(so):
        s, o = so
        cmd = [cc] + ARCH + FLAGS + extra + ["-c", s, "-o", o + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s%s" % (s, r.stdout, r.stderr))
        os.replace(o + ".tmp", o)
        if verbose:
            sys.stderr.write(r.stdout + r.stderr)
        return s

    if todo:
        n = jobs or max(1, min(len(todo), os.cpu_count() or 4))
        with ThreadPoolExecutor(n) as ex:
            for s in ex.map(comp, todo):
                if verbose:
                    print("compiled", os.path.basename(s))
    if todo or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
