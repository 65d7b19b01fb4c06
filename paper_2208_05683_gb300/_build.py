"""Build of the CUDA library ``libpsf.so`` (sm_103a) with nvcc, in-tree.

Every translation unit is compiled in parallel, then linked into one shared
library against the shared CUDA runtime.  Host code is compiled with
floating-point contraction off and device code with ``-fmad=false``: the only
fused multiply-adds are the explicit ones.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libpsf.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["psf_kernels.cu", "psf_api.cu", "psf_batch.cu", "psf_normest.cu", "psf_dense.cu", "psf_server.cpp",
           "psf_plan.cpp"]
_lock = threading.Lock()


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpsf.so")
    return cand


def _flags():
    return [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-fmad=false",
            "-Xcompiler", "-fPIC,-ffp-contract=off,-fno-fast-math,-fvisibility=hidden,-fvisibility-inlines-hidden", "-I", os.path.join(HERE, "..", "include")]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "psf.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    with _lock:
        if not force and not _stale():
            return LIB
        os.makedirs(OUT_DIR, exist_ok=True)
        cc = nvcc()
        objs, procs = [], []
        for src in SOURCES:
            obj = os.path.join(OUT_DIR, src.rsplit(".", 1)[0] + ".o")
            cmd = [cc, *_flags(), "-c", os.path.join(CSRC, src), "-o", obj]
            if src.endswith(".cpp"):
                cmd = [cc, "-x", "cu", *cmd[1:]]
            objs.append(obj)
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        for cmd, p in procs:
            out, _ = p.communicate()
            if verbose or p.returncode:
                print(out.decode(errors="replace"))
            if p.returncode:
                raise RuntimeError("nvcc failed: " + " ".join(cmd))
        tmp = LIB + f".{os.getpid()}.tmp"
        link = [cc, *ARCH, "-shared", "--cudart", "shared", "-o", tmp, *objs]
        r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if r.returncode:
            print(r.stdout.decode(errors="replace"))
            raise RuntimeError("link failed: " + " ".join(link))
        os.replace(tmp, LIB)
        return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
