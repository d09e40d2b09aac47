"""Build libspiir.so in-tree with nvcc for sm_103a (no cmake).

Each .cu under csrc/ compiles in parallel to an object file; the objects link
into paper_1702_02256_gb300/_build/libspiir.so with the CUDA runtime linked
statically. The result is loaded by paper_1702_02256_gb300.spiir.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libspiir.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


# Reduction ablations of the recursion kernel (compile-time switch
# SPIIR_REDUCE_ABLATION in csrc/spiir_plain.cu): name -> value.
ABLATIONS = {"adopted": 0, "shuffle": 1, "smem": 2, "atomics": 3}


def build_ablation(name: str, verbose: bool = False) -> str:
    """libspiir.so with the recursion kernel's reduction switched to `name`
    (see ABLATIONS), in _build/ablation_<name>/; only spiir_plain.cu is
    recompiled, the other objects are the default build's."""
    k = ABLATIONS[name]
    build(verbose=verbose)
    if k == 0:
        return LIB
    out = os.path.join(BUILD, f"ablation_{name}")
    os.makedirs(out, exist_ok=True)
    src = os.path.join(CSRC, "spiir_plain.cu")
    obj = os.path.join(out, "spiir_plain.o")
    lib = os.path.join(out, "libspiir.so")
    headers = sorted(glob.glob(os.path.join(CSRC, "*.h"))) + [os.path.join(ROOT, "include", "spiir.h")]
    if _stale(obj, [src] + headers):
        r = subprocess.run([nvcc()] + ARCH + FLAGS + [f"-DSPIIR_REDUCE_ABLATION={k}", "-c", src, "-o", obj],
                           capture_output=True, text=True)
        if verbose or r.returncode:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode:
            raise RuntimeError(f"nvcc failed for the {name} ablation")
    others = [os.path.join(BUILD, os.path.basename(f)[:-3] + ".o")
              for f in sorted(glob.glob(os.path.join(CSRC, "*.cu"))) if not f.endswith("spiir_plain.cu")]
    if _stale(lib, [obj] + others):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc()] + ARCH + ["-shared", "-o", tmp, obj] + others)
        os.replace(tmp, lib)
    return lib


def build_ablations(names, verbose: bool = False) -> dict:
    """build_ablation for several names, compiled in parallel."""
    build(verbose=verbose)
    with cf.ThreadPoolExecutor(max_workers=max(1, len(names))) as ex:
        return dict(zip(names, ex.map(lambda n: build_ablation(n, verbose), names)))


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    headers = sorted(glob.glob(os.path.join(CSRC, "*.h"))) + [os.path.join(ROOT, "include", "spiir.h")]
    jobs = []
    for src in sources:
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        if force or _stale(obj, [src] + headers):
            cmd = [nvcc()] + ARCH + FLAGS + (["-Xptxas", "-v"] if ptxas_info else []) + ["-c", src, "-o", obj]
            jobs.append((src, cmd))
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        futs = {ex.submit(subprocess.run, cmd, capture_output=True, text=True): src for src, cmd in jobs}
        for f in cf.as_completed(futs):
            r = f.result()
            if verbose or ptxas_info or r.returncode:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode:
                raise RuntimeError(f"nvcc failed for {futs[f]}")
    objs = [os.path.join(BUILD, os.path.basename(s)[:-3] + ".o") for s in sources]
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
