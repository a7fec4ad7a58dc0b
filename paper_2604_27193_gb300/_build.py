"""Build ``libaeb.so`` in-tree for sm_103a (GB300).

Every translation unit is compiled in parallel, then linked with nvcc.  The
rollout kernels are compiled with ``-fmad=false`` (no fused multiply-add is
formed unless the source writes ``fma``): the binary64 kernel so that it
mirrors the oracle's operation order, the binary32 kernel so that a replayed
window repeats the window's arithmetic exactly.  Host code is compiled with
``-ffp-contract=off``; nothing is built with fast-math.  Set ``AEB_PTXAS_VERBOSE=1`` to print ptxas resource
usage of the kernels.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libaeb.so")
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = {
    "rollout_fp64.cu": ["-fmad=false"],
    "rollout_fp32.cu": ["-fmad=false"],
    "reduce.cu": [],
    "reduce_noalloc.cu": [],
    "reduce_weighted.cu": [],
    "peaks.cu": ["-fmad=true"],
}
CPP_SOURCES = ["capi.cpp", "sampler.cpp", "batch.cpp", "serve.cpp", "sweep.cpp", "stats.cpp"]
HEADERS = ["aeb_internal.h", "rollout_common.cuh", "host_util.h"]


def _sources():
    return [os.path.join(CSRC, f) for f in list(CU_SOURCES) + CPP_SOURCES + HEADERS] + [
        os.path.join(HERE, "..", "include", "aeb.h")]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"build step failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    ptxas_v = os.environ.get("AEB_PTXAS_VERBOSE") == "1"
    jobs = []
    for src, extra in CU_SOURCES.items():
        obj = os.path.join(OUT_DIR, src + ".o")
        cmd = [NVCC, *ARCH, "-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC",
               "-Xcompiler", "-ffp-contract=off", *extra, "-c", os.path.join(CSRC, src),
               "-o", obj]
        if ptxas_v:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append((cmd, obj))
    for src in CPP_SOURCES:
        obj = os.path.join(OUT_DIR, src + ".o")
        cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-ffp-contract=off", "-fno-fast-math",
               "-pthread", f"-I{CUDA_HOME}/include", "-c", os.path.join(CSRC, src), "-o", obj]
        jobs.append((cmd, obj))
    with ThreadPoolExecutor(len(jobs)) as ex:
        logs = list(ex.map(lambda j: _run(j[0]), jobs))
    if verbose or ptxas_v:
        for log in logs:
            if log.strip():
                print(log, file=sys.stderr)
    tmp = LIB + f".tmp{os.getpid()}"
    _run([NVCC, *ARCH, "-shared", "-o", tmp, *[o for _, o in jobs], "-lpthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
