"""Builds the CPU oracle shared libraries (test infrastructure; see grf_oracle.cpp header):
liborc.so (the plain double oracle) and liborc_tlm.so (the same core on dual numbers and on
complex-step numbers: the tangent-linear model)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "grf_oracle.cpp")
TLM_SRC = os.path.join(HERE, "grf_oracle_tlm.cpp")
DEPS = [os.path.join(HERE, f) for f in ("orc_types.h", "orc_core.inc")]
LIB = os.path.join(HERE, "liborc.so")
TLM_LIB = os.path.join(HERE, "liborc_tlm.so")
FLAGS = ["-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC"]


def _stale(lib, src):
    if not os.path.exists(lib):
        return True
    return os.path.getmtime(lib) < max(os.path.getmtime(f) for f in [src] + DEPS)


def _compile(src, lib, verbose):
    cmd = ["g++"] + FLAGS + [src, "-o", lib + ".tmp"]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(lib + ".tmp", lib)


def build(force=False, verbose=False):
    if force or _stale(LIB, SRC):
        _compile(SRC, LIB, verbose)
    return LIB


def build_tlm(force=False, verbose=False):
    if force or _stale(TLM_LIB, TLM_SRC):
        _compile(TLM_SRC, TLM_LIB, verbose)
    return TLM_LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    build_tlm(force="--force" in sys.argv, verbose=True)
