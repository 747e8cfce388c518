"""Builds libbnb.so (the C-ABI library, include/bnb.h) and libbnb_diag.so (its
diagnostics, include/bnb_diag.h) in-tree for sm_103a with nvcc.

    python -m paper_2602_04551_b300.build [--verbose]

The libraries have no torch dependency; they link only the CUDA runtime, and the
diagnostics library links libbnb.so for the operand helpers it shares.
"""
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libbnb.so")
DIAG_LIB = os.path.join(HERE, "libbnb_diag.so")
DIAG_SOURCES = ("diag.cu",)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))


def headers():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cuh")) +
                  glob.glob(os.path.join(ROOT, "include", "*.h")))


def up_to_date():
    if not (os.path.exists(LIB) and os.path.exists(DIAG_LIB)):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(DIAG_LIB))
    return all(os.path.getmtime(f) <= t for f in sources() + headers())


def build(verbose=False, force=False):
    if not force and up_to_date():
        return LIB
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                    "-I", os.path.join(ROOT, "include")]
    if verbose:
        flags += ["-Xptxas", "-v"]
    objs = []
    procs = []
    for src in sources():
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmd = [nvcc, "-c", src, "-o", obj] + flags
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, pr in procs:
        out, _ = pr.communicate()
        if verbose or pr.returncode:
            sys.stdout.write(out.decode())
        if pr.returncode:
            raise RuntimeError("nvcc failed: " + " ".join(cmd))
    main = [o for o, src in zip(objs, sources()) if os.path.basename(src) not in DIAG_SOURCES]
    diag = [o for o, src in zip(objs, sources()) if os.path.basename(src) in DIAG_SOURCES]
    subprocess.check_call([nvcc] + ARCH + ["-shared", "-o", LIB] + main + ["-lcudart"])
    subprocess.check_call([nvcc] + ARCH + ["-shared", "-o", DIAG_LIB] + diag +
                          ["-L", HERE, "-lbnb", "-Xlinker", "-rpath=$ORIGIN", "-lcudart"])
    return LIB


if __name__ == "__main__":
    build(verbose="--verbose" in sys.argv, force=True)
    print(LIB)
