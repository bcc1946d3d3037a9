"""Build the CUDA library libkftrack.so in-tree for GB300 (sm_103a).

Each translation unit compiles in parallel with nvcc, then one link step makes
the shared library next to this file. No fast-math: the association decisions
rely on IEEE-rounded division and square root.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libkftrack.so")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["kf_frontend.cu", "kf_icp.cu", "kf_api.cu", "kf_tsdf.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libkftrack.so")


def flags(verbose: bool = False) -> list[str]:
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _newer(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return False
    t = os.path.getmtime(target)
    return all(os.path.getmtime(d) <= t for d in deps)


def _stamp_ok(bdir: str, defines: list[str]) -> bool:
    """True when the objects in bdir were compiled with these defines."""
    path = os.path.join(bdir, "defines.txt")
    want = "\n".join(defines)
    have = open(path).read() if os.path.exists(path) else None
    if have == want:
        return True
    with open(path, "w") as f:
        f.write(want)
    return False


def build(force: bool = False, verbose: bool = False, defines=(), out: str | None = None,
          use_tuned: bool = True) -> str:
    """Compile the library (incrementally unless force). defines: extra -D
    macros, after those of tuned.json (the autotuner's choice of the kernels'
    shapes) unless use_tuned is False; out: library path (default: in-tree
    libkftrack.so)."""
    from .tune import TUNED, tuned_defines
    lib = out or LIB
    bdir = BUILD if out is None else os.path.join(os.path.dirname(out), "_build")
    os.makedirs(bdir, exist_ok=True)
    defs = (tuned_defines() if use_tuned else []) + list(defines)
    if not _stamp_ok(bdir, defs):
        force = True
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith(".cuh")]
    headers.append(os.path.join(INCLUDE, "kf_track.h"))
    if use_tuned and os.path.exists(TUNED):
        headers.append(TUNED)
    objs, jobs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(bdir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or verbose or not _newer(o, [s] + headers):
            jobs.append([nvcc()] + flags(verbose) + [f"-D{d}" for d in defs] + ["-c", s, "-o", o])
    with cf.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
    for cmd, r in zip(jobs, results):
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stderr + r.stdout)
    if force or jobs or not _newer(lib, objs):
        cmd = [nvcc()] + ARCH + ["-shared", "-o", lib] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + " ".join(cmd) + "\n" + r.stderr + r.stdout)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
