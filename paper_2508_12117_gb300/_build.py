"""Builds libspider.so (sm_103a) in-tree: one nvcc/g++ process per translation
unit, in parallel, then one link.  Used by `__graft_entry__.build()`."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libspider.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["api.cu", "k_step.cu", "k_whiten.cu", "k_units.cu", "k_tt.cu", "k_mlp_tc.cu", "tt_noalloc.cu", "k_outlier.cu",
              "k_uq.cu"]
CPP_SOURCES = ["prep.cpp", "pieces.cpp"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def build(verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    jobs = []
    for s in CU_SOURCES:
        o = os.path.join(OUT_DIR, s + ".o")
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3",
               *inc, "-c", os.path.join(CSRC, s), "-o", o]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append((cmd, o))
    gxx = shutil.which("g++") or "g++"
    for s in CPP_SOURCES:
        o = os.path.join(OUT_DIR, s + ".o")
        cmd = [gxx, "-O3", "-fPIC", "-std=c++17", "-pthread", "-ffp-contract=off",
               "-I", "/usr/local/cuda/include", *inc, "-c", os.path.join(CSRC, s), "-o", o]
        jobs.append((cmd, o))
    logs = []
    with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        for out in ex.map(lambda j: _run(j[0]), jobs):
            logs.append(out)
    objs = [o for _, o in jobs]
    tmp = LIB + ".tmp"
    _run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-pthread"])
    os.replace(tmp, LIB)
    text = "\n".join(l for l in logs if l.strip())
    if verbose and text:
        print(text, file=sys.stderr)
    return text


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="-v" in sys.argv))
