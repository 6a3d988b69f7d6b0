"""Build librecon.so (hand-written sm_103a CUDA behind the C ABI of
include/recon.h) in-tree, into paper_1709_06350_gb300/_build/.

Each translation unit is compiled by its own nvcc process (in parallel),
then linked with ``nvcc -shared``.  The CUDA runtime is linked statically, so
the library needs nothing but the driver at run time.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "librecon.so")
SOURCES = ["recon_mg.cu", "recon_sweep.cu", "recon_cic.cu", "recon_adjoint.cu", "recon_batch.cu",
           "recon_api.cu", "recon_noalloc.cu", "recon_gauss.cu", "recon_smooth.cu",
           "recon_measure.cu", "recon_slab.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: librecon cannot be built")
    return exe


def _flags(verbose_ptxas: bool):
    f = ["-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC",
         "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    deps = [src] + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith(".cuh")]
    deps += [os.path.join(ROOT, "include", h) for h in os.listdir(os.path.join(ROOT, "include"))]
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    """Compile (if stale) and return the path of librecon.so."""
    os.makedirs(OUT, exist_ok=True)
    exe = nvcc()
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT, src.replace(".cu", ".o"))
        objs.append(o)
        if force or verbose_ptxas or _stale(o, s):
            jobs.append([exe, *_flags(verbose_ptxas), "-c", s, "-o", o])

    def run(cmd):
        p = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, p

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            for cmd, p in ex.map(run, jobs):
                if p.returncode != 0:
                    sys.stderr.write(p.stdout + p.stderr)
                    raise RuntimeError(f"nvcc failed: {' '.join(cmd)}")
                if verbose_ptxas:
                    sys.stderr.write(p.stderr)
    if jobs or not os.path.exists(LIB):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [exe, "-shared", *ARCH, "-o", tmp, *objs]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            sys.stderr.write(p.stdout + p.stderr)
            raise RuntimeError("link of librecon.so failed")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
