"""Build librbs.so in-tree (paper_2302_04180_gb300/_build) with nvcc for sm_103a.

The translation units compile in parallel; device code is built with
-fmad=false so that the compiler never contracts a*b+c (Sec. 3.3): every fused
multiply-add in the library is an explicit fma().
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "librbs.so")
SOURCES = ["kernels_dot.cu", "kernels_exdot_w1.cu", "kernels_exdot_w2.cu", "kernels_spmv.cu", "kernels_solver.cu",
           "kernels_step.cu", "kernels_batch.cu", "capi.cu", "server.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-fmad=false", "-std=c++17", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-fno-fast-math", "-Xcompiler", "-ffp-contract=off",
              f"-I{INC}", f"-I{CSRC}"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librbs.so")
    return p


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INC, "rbs.h"))
    files.append(os.path.abspath(__file__))
    return files


def _stale(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(f) > t for f in _deps())


def _compile(src: str, obj: str, verbose: bool) -> str:
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if stale) and return the path of librbs.so."""
    if not force and not verbose and not _stale(LIB):
        return LIB
    os.makedirs(OUT, exist_ok=True)
    objs = [os.path.join(OUT, s.replace(".cu", f".{os.getpid()}.o")) for s in SOURCES]
    logs = {}
    tmp = LIB + f".tmp{os.getpid()}"
    try:
        with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
            futs = {ex.submit(_compile, s, o, verbose): s for s, o in zip(SOURCES, objs)}
            for f in cf.as_completed(futs):
                logs[futs[f]] = f.result()
        r = subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs], capture_output=True,
                           text=True)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        for s in SOURCES:
            print(f"== {s}\n{logs[s]}")
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
