"""Builds libezo.so in-tree for sm_103a with nvcc (one process per translation
unit, then one shared link). Usage: python -m paper_2504_10783_gb300.build"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libezo.so")
SOURCES = ["ezo_capi.cu", "ezo_api.cu", "ezo_k_flat.cu", "ezo_k_round_a.cu", "ezo_k_round_b.cu", "ezo_noalloc.cu", "ezo_tune.cu",
           "ezo_mlp.cu", "ezo_mlp_tc.cu", "ezo_mlp_gemm_tc.cu", "ezo_k_recover.cu"]
# the collision kernels for scenes with box geometries: the same sources built
# a second time with EZO_BOX_TU=1, in parallel with the rest
BOX_SOURCES = ["ezo_k_flat.cu", "ezo_k_round_a.cu", "ezo_k_round_b.cu", "ezo_k_recover.cu"]
UNITS = [(src, src.replace(".cu", ".o"), []) for src in SOURCES] + \
        [(src, src.replace(".cu", "_box.o"), ["-DEZO_BOX_TU=1"]) for src in BOX_SOURCES]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "-Xcompiler", "-ffp-contract=off"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _deps() -> list[str]:
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh"))]
    out.append(os.path.join(os.path.dirname(HERE), "include", "ezo.h"))
    return out


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()

    def compile_one(unit):
        src, obj_name, extra = unit
        obj = os.path.join(BUILD, obj_name)
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = LIB + ".tmp"
    cmd = [cc, "-shared", *ARCH, "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
