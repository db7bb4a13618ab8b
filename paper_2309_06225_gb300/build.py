"""Builds libgrf.so (the C-ABI CUDA library) in-tree for sm_103a with nvcc.

Translation units are compiled in parallel and linked into paper_2309_06225_gb300/libgrf.so.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgrf.so")
SOURCES = ["grf_api.cu", "grf_stage.cu", "grf_stage_dec.cu", "grf_stage_fold.cu", "grf_stage_lop.cu", "grf_stage_gen.cu",
           "grf_stage6.cu", "grf_stage6l.cu", "grf_rhs.cu", "grf_rhs6.cu", "grf_boundary.cu", "grf_extract.cu",
           "grf_batch.cu", "grf_batch_persistent.cu", "grf_patches.cu", "grf_noalloc.cu", "grf_tlm.cu", "grf_adjoint.cu"]
NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INC, "-I" + CSRC]
# Per-source ptxas flags. The dual-number (tangent) kernels are very large functions on which
# ptxas -O2/-O3 settles for 32 registers and an 87 KB stack; -O1 keeps 255 registers and a
# 36 KB stack. The reverse-mode stage (about 4,300 recording calls) takes ptxas 10 minutes at
# -O3 and under 2 at -O1, with the same 255 registers and 7 KB stack.
SOURCE_FLAGS = {"grf_tlm.cu": ["-Xptxas", "-O1"], "grf_adjoint.cu": ["-Xptxas", "-O1"]}


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INC, "grf.h")]
    return max(os.path.getmtime(f) for f in files)


FLOPS_SRC = os.path.join(CSRC, "grf_flops.cpp")
FLOPS_LIB = os.path.join(HERE, "libgrf_flops.so")


def build_flops(force=False, verbose=False):
    """Host build of the pointwise RHS source: operation counts and a double-precision
    instance used by CPU checks (no GPU code)."""
    if not force and os.path.exists(FLOPS_LIB) and os.path.getmtime(FLOPS_LIB) >= _deps():
        return FLOPS_LIB
    cmd = [os.environ.get("CXX", "g++"), "-std=c++17", "-O2", "-ffp-contract=off", "-shared", "-fPIC", "-I" + INC,
           "-I" + CSRC, FLOPS_SRC, "-o", FLOPS_LIB + ".tmp"]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.check_call(cmd)
    os.replace(FLOPS_LIB + ".tmp", FLOPS_LIB)
    return FLOPS_LIB


def build(force=False, verbose=False, ptxas_verbose=False):
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    extra = ["-Xptxas", "-v"] if ptxas_verbose else []

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [NVCC] + ARCH + FLAGS + SOURCE_FLAGS.get(src, []) + extra + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
        if ptxas_verbose:
            print(res.stdout + res.stderr)
        return obj

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    cmd = [NVCC] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs + ["-lcudart"]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_verbose="-v" in sys.argv)
    build_flops(force="--force" in sys.argv, verbose=True)
