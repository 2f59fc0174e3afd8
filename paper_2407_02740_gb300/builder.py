"""Builds the CUDA library libvecchia_gb300.so in-tree with nvcc for sm_103a.

Translation units are compiled in parallel, then linked into one shared library whose
C ABI is declared in include/vecchia.h.  Only one -gencode is used
(compute_103a -> sm_103a).
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
LIB = os.path.join(HERE, "libvecchia_gb300.so")
SOURCES = ["vg_kernels.cu", "vg_pass_f64.cu", "vg_pass_f32.cu", "vg_capi.cu", "vg_noalloc.cu",
           "vg_fit.cu", "vg_features.cu", "vg_mlp.cu", "vg_nn.cu", "vg_predict.cu", "vg_peaks.cu",
           "vg_pass_group.cu", "vg_maxmin.cu"]
HEADERS = ["vg_common.cuh", "vg_matern.cuh", "vg_pass.cuh", "vg_internal.h", "vg_fit.h"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden", "-Xptxas", "-v",
           "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str) -> tuple[str, str]:
    obj = os.path.join(BUILD, src.replace(".cu", ".o"))
    log = os.path.join(BUILD, src.replace(".cu", ".ptxas.txt"))
    deps = [os.path.join(CSRC, src)] + [os.path.join(CSRC, h) for h in HEADERS] + [
        os.path.join(HERE, "..", "include", "vecchia.h")]
    if _stale(obj, deps):
        cmd = [nvcc()] + ARCH + NVFLAGS + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        with open(log, "w") as f:
            f.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s" % (src, r.stderr[-6000:]))
    return src, obj


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if force:
        for f in os.listdir(BUILD):
            os.remove(os.path.join(BUILD, f))
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = [o for _, o in ex.map(_compile, SOURCES)]
    if _stale(LIB, objs) or force:
        tmp = LIB + ".%d.tmp" % os.getpid()
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s" % r.stderr[-4000:])
        os.replace(tmp, LIB)
    if verbose:
        for src in SOURCES:
            with open(os.path.join(BUILD, src.replace(".cu", ".ptxas.txt"))) as f:
                sys.stdout.write(f.read())
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
