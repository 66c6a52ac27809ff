"""Build libniorca.so from csrc/*.cu with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel into _build/, then linked into
a shared library next to this file. Nothing is rebuilt when the objects are
newer than every source and header.
"""
from __future__ import annotations

import glob
import os
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libniorca.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, *ARCH]

_lock = threading.Lock()


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps_mtime() -> float:
    files = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    return max((os.path.getmtime(f) for f in files), default=0.0)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every CUDA source and link libniorca.so; returns its path."""
    with _lock:
        os.makedirs(BUILD, exist_ok=True)
        nvcc = _nvcc()
        deps = _deps_mtime()
        procs, objs = [], []
        for src in sources():
            obj = os.path.join(BUILD, os.path.splitext(os.path.basename(src))[0] + ".o")
            objs.append(obj)
            fresh = os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), deps)
            if fresh and not force:
                continue
            cmd = [nvcc, *NVCC_FLAGS, "-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd))
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        errors = []
        for src, p in procs:
            out, _ = p.communicate()
            if p.returncode != 0:
                errors.append(f"{os.path.basename(src)}:\n{out.decode(errors='replace')}")
            elif verbose and out:
                print(out.decode(errors="replace"))
        if errors:
            raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
        newest = max(os.path.getmtime(o) for o in objs)
        if force or procs or not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
            tmp = LIB + f".tmp{os.getpid()}"
            subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
            os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
