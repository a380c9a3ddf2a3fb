"""Builds the sm_103a shared library libnnqs_gb300.so in-tree with nvcc.

Every translation unit under csrc/ is compiled in parallel for
arch=compute_103a,code=sm_103a and linked into one shared object exporting the
C ABI of include/nnqs.h.  The mixed-batch kernel and its per-shape bodies
(k_batch.cu, k_mixed_*.cu) are relocatable device code, joined by a device
link step before the final link.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libnnqs_gb300.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", os.path.join(HERE, "..", "include")]


def _is_rdc(src: str) -> bool:
    b = os.path.basename(src)
    return b == "k_batch.cu" or b.startswith("k_mixed_")


RDC = ["-rdc=true", "-maxrregcount=128"]


def _stale(obj: str, deps: list[str]) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, extra: list[str] | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    headers = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(HERE, "..", "include", "*.h"))
    extra = list(extra or [])

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        if _stale(obj, [src] + headers) or extra:
            cmd = [NVCC, *ARCH, *FLAGS, *(RDC if _is_rdc(src) else []), *extra, "-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd))
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
            if verbose and r.stderr:
                print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, srcs))
    rdc_objs = [o for o, s in zip(objs, srcs) if _is_rdc(s)]
    if rdc_objs:
        dlink = os.path.join(BUILD, "device_link.o")
        if _stale(dlink, rdc_objs):
            cmd = [NVCC, *ARCH, "-Xcompiler", "-fPIC", "-dlink", *rdc_objs, "-o", dlink]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"device link failed:\n{r.stdout}\n{r.stderr}")
        objs = objs + [dlink]
    if _stale(LIB, objs):
        tmp = LIB + ".tmp"
        cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(verbose="-v" in sys.argv))
