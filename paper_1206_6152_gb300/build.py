"""Builds the CUDA library libvp.so in-tree for sm_103a.

Each .cu file under csrc/ is compiled by nvcc in parallel
(-gencode arch=compute_103a,code=sm_103a, -O3, -lineinfo, -ftz=true) and the objects are
linked into paper_1206_6152_gb300/libvp.so with the CUDA runtime linked
statically.  Object files go to paper_1206_6152_gb300/_build/.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libvp.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["vp_api.cu", "vp_sweep.cu", "vp_sweep_fast.cu", "vp_kick_big.cu", "vp_field.cu",
           "vp_adjoint.cu", "vp_adjoint_fast.cu", "vp_noalloc.cu", "vp_shard.cu", "vp_sweep_f64.cu"]


def nvcc() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libvp.so")


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


FLAGS_STAMP = os.path.join(BUILD, "flags.txt")
FLAGS = "-O3 -lineinfo -std=c++17 -ftz=true"


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    # FP32 denormals are flushed to zero: the positivity argument of the
    # saturating-multiply corrector relies on relative rounding, which
    # denormals do not have
    if not os.path.exists(FLAGS_STAMP) or open(FLAGS_STAMP).read() != FLAGS:
        force = True
        with open(FLAGS_STAMP, "w") as fh:
            fh.write(FLAGS)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith(".cuh")]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "vp.h"))
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    jobs = []
    for s in srcs:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, s.replace(".cu", ".o"))
        if force or _stale(obj, [src] + headers):
            cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-ftz=true", "-Xcompiler",
                   "-fPIC", "-c", src, "-o", obj]
            jobs.append((cmd, obj))
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            futs = [ex.submit(subprocess.run, cmd, capture_output=True, text=True)
                    for cmd, _ in jobs]
            for (cmd, obj), fu in zip(jobs, futs):
                r = fu.result()
                if r.returncode != 0:
                    raise RuntimeError(f"nvcc failed for {obj}:\n{r.stderr}")
                if verbose and r.stderr:
                    print(r.stderr, file=sys.stderr)
    objs = [os.path.join(BUILD, s.replace(".cu", ".o")) for s in srcs]
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
