"""Build liblbs.so (sm_103a) in-tree with nvcc.

Compiles the translation units under csrc/ in parallel and links them into
``paper_2502_00920_gb300/liblbs.so``.  Used by ``__graft_entry__.build()``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "liblbs.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# --fmad=false: no implicit contraction of products and sums into fused
# multiply-adds; the kernels write the fused ones they want (fmr), so a node's
# rounding is fixed by the source in every kernel that computes it
FLAGS = ["-O3", "--fmad=false", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xcompiler", "-Wall", "-Xcompiler", "-ffp-contract=off"]
UNITS = ["lbs_api.cu", "lbs_autotune.cu", "lbs_serve.cu", "lbs_fields_static.cu", "lbs_selftest.cu", "kernels_fp64.cu",
         "kernels_fp32.cu", "kernels_fp16.cu"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    inc = os.path.join(HERE, "..", "include")
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))] + [
        os.path.join(inc, f) for f in os.listdir(inc) if f.endswith(".h")]


STEP_KERNEL_SOURCES = ["lbs_device.cuh", "lbs_tiles.h", "lbs_internal.h", "kernels_fp64.cu", "kernels_fp32.cu", "kernels_fp16.cu"]


def source_hash() -> str:
    """Hash of the sources of the step kernels (identifies the kernels a
    profile was taken on)."""
    import hashlib
    h = hashlib.sha256()
    for path in [os.path.join(CSRC, f) for f in STEP_KERNEL_SOURCES]:
        if os.path.exists(path):
            h.update(os.path.basename(path).encode())
            h.update(open(path, "rb").read())
    return h.hexdigest()[:16]


def up_to_date() -> bool:
    if not os.path.exists(OUT):
        return False
    t = os.path.getmtime(OUT)
    return all(os.path.getmtime(s) <= t for s in _sources() if os.path.exists(s))


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and up_to_date():
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()

    def compile_one(unit):
        obj = os.path.join(BUILD, unit.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, unit), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {unit}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = OUT + f".{os.getpid()}.tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
