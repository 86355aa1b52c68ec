"""Builds the CUDA library ``libvelo_gb300.so`` in-tree for sm_103a with nvcc.

Each translation unit compiles in its own process (in parallel), then nvcc
links the shared library.  The library exports the C ABI of
``include/velo.h``; it links no torch.
"""
from __future__ import annotations

import os
import subprocess
import sys
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libvelo_gb300.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]
SOURCES = ["velo_api.cu", "velo_cluster.cu", "velo_track.cu", "velo_track_ring.cu", "velo_emit.cu", "velo_static.cu", "velo_mlp.cu",
           "velo_serve.cu", "velo_pv.cu", "velo_sp.cu"]

_lock = threading.Lock()


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _deps() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    return files + [os.path.join(INCLUDE, "velo.h"), os.path.abspath(__file__)]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compiles the library if any source is newer than it; returns its path."""
    with _lock:
        if not force and up_to_date():
            return LIB
        os.makedirs(BUILD, exist_ok=True)
        nvcc = _nvcc()
        procs = []
        objs = []
        for src in SOURCES:
            obj = os.path.join(BUILD, src.replace(".cu", ".o"))
            cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
            if ptxas_info:
                cmd.insert(1, "-Xptxas=-v")
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
            objs.append(obj)
        errors = []
        for src, p in procs:
            out, _ = p.communicate()
            if p.returncode != 0 or verbose or ptxas_info:
                (errors if p.returncode else [None]).append(f"--- {src}\n{out}")
                if p.returncode == 0:
                    print(f"--- {src}\n{out}", file=sys.stderr)
        if errors:
            raise RuntimeError("nvcc failed:\n" + "\n".join(e for e in errors if e))
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
