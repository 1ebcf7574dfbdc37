"""Build the CUDA library (sm_103a) and the host-only scheduler simulator.

  python -m paper_2603_17168_gb300.build

compiles every csrc/*.cu translation unit in parallel with
``nvcc -gencode arch=compute_103a,code=sm_103a -O3 -lineinfo`` into
``paper_2603_17168_gb300/libhkv.so`` (in-tree, git-ignored), and the
triple-group scheduler's simulation harness (plain g++, no CUDA) into
``libhkv_sched_sim.so``. nvcc cross-compiles, so this runs without a GPU.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libhkv.so")
SIM = os.path.join(PKG, "libhkv_sched_sim.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
              "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h", ".hpp"))]
    return hs + [os.path.join(ROOT, "include", "hkv.h")]


def _newer(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"command failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return r.stdout + r.stderr


def build_lib(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    hdrs = _headers()
    objs = [os.path.join(BUILD, os.path.basename(s)[:-3] + ".o") for s in srcs]
    jobs = []
    for s, o in zip(srcs, objs):
        if force or _newer(o, [s] + hdrs):
            jobs.append([nvcc(), *ARCH, *NVCC_FLAGS, *(extra or []), "-c", s, "-o", o])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for out in ex.map(_run, jobs):
                if verbose and out.strip():
                    print(out)
    if force or jobs or _newer(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        _run([nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs])
        os.replace(tmp, LIB)
    return LIB


def build_sim(force: bool = False) -> str:
    src = os.path.join(CSRC, "sched_sim.cpp")
    deps = [src, os.path.join(CSRC, "sched.hpp")]
    if force or _newer(SIM, deps):
        tmp = SIM + f".tmp{os.getpid()}"
        _run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", "-o", tmp, src])
        os.replace(tmp, SIM)
    return SIM


def build(force: bool = False, verbose: bool = False) -> None:
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        a = ex.submit(build_lib, force, verbose)
        b = ex.submit(build_sim, force)
        a.result()
        b.result()


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
