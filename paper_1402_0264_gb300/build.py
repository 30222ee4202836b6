"""Builds libpolymul.so in-tree: nvcc for sm_103a, one object per .cu, compiled in parallel.

    python -m paper_1402_0264_gb300.build [--force] [--ptxas-info] [--checked]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libpolymul.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["api.cu", "plain.cu", "plain_ell.cu", "ntt.cu", "tensor.cu", "div.cu", "gcd.cu", "probe.cu", "tune.cu",
           "hostio.cu"]
DEPS = {"plain_ell.cu": ["plain.cu"]}  # sources that include another source


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpolymul")


def _flags(ptxas_info: bool) -> list[str]:
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
                "--expt-relaxed-constexpr"]
    if ptxas_info:
        f += ["-Xptxas", "-v"]
    return f


def _headers_mtime() -> float:
    hs = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".cuh", ".h"))]
    hs.append(os.path.join(INCLUDE, "polymul.h"))
    return max(os.path.getmtime(h) for h in hs)


def build(force: bool = False, ptxas_info: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Builds libpolymul.so; with checked=True the range-checked variant (-DPOLYMUL_CHECKED: guarded
    indices that set PM_ERR_INTERNAL, inputs >= p that set PM_ERR_RANGE) into _build/checked/."""
    bdir = os.path.join(BUILD, "checked") if checked else BUILD
    lib = os.path.join(bdir, "libpolymul.so")
    extra = ["-DPOLYMUL_CHECKED"] if checked else []
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    hdr = _headers_mtime()
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(bdir, src.replace(".cu", ".o"))
        newest = max([os.path.getmtime(s), hdr] + [os.path.getmtime(os.path.join(CSRC, d)) for d in DEPS.get(src, [])])
        if force or ptxas_info or not os.path.exists(o) or os.path.getmtime(o) < newest:
            jobs.append((s, o))

    def compile_one(job):
        s, o = job
        cmd = [nvcc] + _flags(ptxas_info) + extra + ["-c", s, "-o", o + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(s)}:\n{r.stderr}")
        os.replace(o + ".tmp", o)
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for out in ex.map(compile_one, jobs):
            if (verbose or ptxas_info) and out:
                print(out)
    objs = [os.path.join(bdir, s.replace(".cu", ".o")) for s in SOURCES]
    if jobs or not os.path.exists(lib) or any(os.path.getmtime(o) > os.path.getmtime(lib) for o in objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--ptxas-info", action="store_true")
    ap.add_argument("--checked", action="store_true", help="the range-checked variant (-DPOLYMUL_CHECKED)")
    args = ap.parse_args()
    print(build(force=args.force, ptxas_info=args.ptxas_info, verbose=True, checked=args.checked))
