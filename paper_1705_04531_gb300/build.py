"""Build the CUDA library (libietidp.so) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into one
shared library next to this file.  Objects go to ``_build/`` (git-ignored).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libietidp.so")
SOURCES = ["setup_kernels.cu", "solver_kernels.cu", "dual_kernels.cu", "ietidp_host.cu", "ietidp_engine.cu",
           "ietidp_saddle.cu", "saddle_kernels.cu", "direct_kernels.cu",
           "ietidp_server.cu", "highorder_setup.cu",
           "solver_dispatch.cu"] + sorted(f for f in os.listdir(SRC) if f.startswith("solver_t_"))
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _flags():
    # IETIDP_DEBUG_BOUNDS=1 builds the self-checking variant of the local
    # solver (every computed index is checked against its buffer);
    # IETIDP_PHASE_TIMERS=1 adds per-phase clock counters
    f = list(FLAGS)
    if os.environ.get("IETIDP_DEBUG_BOUNDS") == "1":
        f.append("-DIETI_DEBUG_BOUNDS")
    if os.environ.get("IETIDP_PHASE_TIMERS") == "1":
        f.append("-DIETI_PHASE_TIMERS")
    return f


def _compile(src):
    obj = os.path.join(OUT, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, *_flags(), "-c", os.path.join(SRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
    return obj


def _stamp():
    return LIB + ".flags"


def stale():
    if not os.path.exists(LIB):
        return True
    # built with other compile flags (debug bounds, phase timers)
    try:
        with open(_stamp()) as fh:
            if fh.read() != " ".join(_flags()):
                return True
    except OSError:
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(SRC, f) for f in os.listdir(SRC)] + [os.path.join(HERE, "..", "include", "ietidp.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), max(2, os.cpu_count() or 2))) as ex:
        objs = list(ex.map(_compile, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(_stamp(), "w") as fh:
        fh.write(" ".join(_flags()))
    if verbose:
        print("built", LIB, file=sys.stderr)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
