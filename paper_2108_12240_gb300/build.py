"""Builds libbhac_gb300.so in-tree with nvcc for sm_103a (translation units
compiled in parallel, then linked as a shared library against the shared
CUDA runtime)."""
from __future__ import annotations

import glob
import os
import subprocess
import sys
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libbhac_gb300.so")
UNITS = ["api.cu", "aux.cu", "amr.cu", "stage_fp64.cu", "stage_mixed.cu", "flops.cu", "static_cfl.cu", "selfcheck.cu", "peaks.cu", "ct.cu", "imex.cu", "regrid.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE]
_lock = threading.Lock()


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _inputs():
    return ([os.path.join(CSRC, u) for u in UNITS] + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.h")))


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _inputs())


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    with _lock:
        if not force and not stale():
            return LIB
        os.makedirs(OUT_DIR, exist_ok=True)
        procs = []
        objs = []
        for u in UNITS:
            obj = os.path.join(OUT_DIR, u.replace(".cu", ".o"))
            objs.append(obj)
            cmd = [nvcc(), *FLAGS, *extra, "-c", os.path.join(CSRC, u), "-o", obj]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((u, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
        failed = []
        for u, p in procs:
            out, _ = p.communicate()
            if p.returncode != 0:
                failed.append((u, out))
            elif verbose and out:
                print(out, file=sys.stderr)
        if failed:
            raise RuntimeError("nvcc failed:\n" + "\n".join(f"--- {u}\n{o}" for u, o in failed))
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run([nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs], check=True)
        os.replace(tmp, LIB)
        return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
