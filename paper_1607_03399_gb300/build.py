"""Build the dgwedge shared library in-tree for sm_103a with nvcc.

Translation units are compiled in parallel (one nvcc/g++ process each) and
linked into paper_1607_03399_gb300/libdgwedge.so.  Objects go to
paper_1607_03399_gb300/_build/.  A unit is rebuilt when its source or any
header is newer than its object.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdgwedge.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_UNITS = [f"k_{p}_n{n}.cu" for p in ("f32", "f64") for n in (1, 2, 3, 4, 5)] + ["energy_static.cu", "peak.cu"]
CPP_UNITS = ["capi.cpp", "refel.cpp"]
HEADERS = ["dg_internal.hpp", "kernels.cuh", "adjoint_kernels.cuh", "stage_split.cuh", "refel.hpp"]


def _newer(src_list, target):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in src_list)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "dgwedge.h")]
    jobs = []
    objs = []
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
    for u in CU_UNITS + CPP_UNITS:
        src = os.path.join(CSRC, u)
        obj = os.path.join(BUILD, u + ".o")
        objs.append(obj)
        if force or _newer([src] + hdrs, obj):
            cmd = [NVCC] + ARCH + common + ["-lineinfo", "-c", src, "-o", obj]
            if u.endswith(".cu"):
                cmd += ["-Xptxas", "-v"] if verbose else []
            jobs.append((u, cmd))
    procs = [(u, cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
             for u, cmd in jobs]
    failed = []
    for u, cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((u, out))
        elif verbose and out:
            sys.stdout.write(out)
    if failed:
        msg = "\n".join(f"--- {u} ---\n{o}" for u, o in failed)
        raise RuntimeError(f"dgwedge build failed:\n{msg}")
    if force or jobs or _newer(objs, LIB):
        cmd = [NVCC] + ARCH + ["-shared", "-o", LIB] + objs
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"dgwedge link failed:\n{r.stdout}")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
