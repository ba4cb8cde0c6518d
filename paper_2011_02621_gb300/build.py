"""In-tree build of libtn.so (the C ABI of include/tn.h) for sm_103a.

Compiles the host C++ with g++ and the CUDA translation units with nvcc
(``-gencode arch=compute_103a,code=sm_103a``) in parallel, then links one
shared library next to this file. Usage: ``python -m paper_2011_02621_gb300.build``.
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
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtn.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

CU = ["evolve.cu", "contract.cu", "tc_gemm.cu", "tc_tma.cu", "tc_tma_persist.cu", "tc_tma_persist_loadb.cu",
      "static_scratch.cu", "stream.cu"]
CPP = ["host.cpp", "server.cpp", "tune.cpp", "batch.cpp"]


def cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtn.so")


def _sources():
    out = []
    for f in CU + CPP:
        p = os.path.join(CSRC, f)
        if os.path.exists(p):
            out.append(p)
    return out


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = _sources() + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    deps.append(os.path.join(ROOT, "include", "tn.h"))
    deps.append(__file__)
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def _big_stack():
    """The compiler's optimiser recurses deeply on the large unrolled tensor-core kernels; on some
    hosts the default 8 MiB stack is too small for it, so the build raises its own soft stack
    limit to the hard one (the compiles inherit it)."""
    try:
        import resource
        soft, hard = resource.getrlimit(resource.RLIMIT_STACK)
        want = hard if hard == resource.RLIM_INFINITY else max(soft, hard)
        resource.setrlimit(resource.RLIMIT_STACK, (want, hard))
    except (ImportError, ValueError, OSError):
        pass


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libtn.so if any source is newer than it; returns its path."""
    if not force and not _stale():
        return LIB
    cuda = cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(BUILD, exist_ok=True)
    _big_stack()
    inc = ["-I" + CSRC, "-I" + os.path.join(ROOT, "include"), "-I" + os.path.join(cuda, "include")]
    jobs = []
    for f in _sources():
        obj = os.path.join(BUILD, os.path.basename(f) + ".o")
        if f.endswith(".cu"):
            cmd = [nvcc, "-std=c++17", "-O3", ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                   "-diag-suppress", "550"] + inc + ["-c", f, "-o", obj]
        else:
            cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-Wall", "-Wno-unused-function"] + inc + ["-c", f, "-o", obj]
        jobs.append((cmd, obj))
    with cf.ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        logs = list(ex.map(lambda j: _run(j[0]), jobs))
    if verbose:
        for l in logs:
            if l.strip():
                print(l)
    tmp = LIB + ".tmp"
    _run([nvcc, "-shared", ARCH, "-o", tmp] + [o for _, o in jobs] + ["-lpthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
