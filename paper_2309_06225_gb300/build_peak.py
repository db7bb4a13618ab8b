"""Builds libgrf_peak.so (FP64 FMA throughput microbenchmark, a measurement tool)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc", "peak_fp64.cu")
INC = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libgrf_peak.so")


def build(force=False, verbose=False):
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = [os.environ.get("NVCC", "nvcc"), "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo",
           "-Xcompiler", "-fPIC", "-shared", "-I" + INC, SRC, "-o", LIB + ".tmp"]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


def measure(threads=256, iters=20000):
    """Measured FP64 FMA throughput in TFLOP/s on the current CUDA device: best over a small
    sweep of resident blocks per SM."""
    import ctypes as C

    import torch
    L = C.CDLL(build())
    L.grf_peak_fp64.argtypes = [C.c_int, C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_float), C.c_void_p]
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    out = torch.empty(nsm * 16 * threads, dtype=torch.float64, device="cuda")
    ms = C.c_float()
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    best = 0.0
    for per_sm in (2, 4, 8, 16):
        blocks = nsm * per_sm
        for _ in range(3):
            rc = L.grf_peak_fp64(blocks, threads, iters, C.c_void_p(out.data_ptr()), C.byref(ms), st)
            assert rc == 0
            best = max(best, 16.0 * iters * blocks * threads / (ms.value * 1e-3) / 1e12)
    return best


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
