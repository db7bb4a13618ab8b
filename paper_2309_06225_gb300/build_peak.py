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


KINDS = {0: "dfma", 1: "dadd", 2: "dmul", 3: "mix 1:1:2", 4: "dfma, per-chain operands", 5: "dfma + integer"}


def measure(target_ms=150.0, repeats=10, sample_clocks=True):
    """Measured FP64 throughput on the current CUDA device.

    Sweeps the instruction kind (DFMA, DADD, DMUL, the DADD:DMUL:DFMA = 1:1:2 mix, DFMA with
    per-chain operands, DFMA beside integer work), the
    chains per thread (4, 8, 16) and the resident blocks per SM (2, 4, 8 of 256 threads). Each
    configuration is sized to about `target_ms` of back-to-back launches, timed `repeats` times;
    its best time counts. nvidia-smi samples the SM clock meanwhile. Returns a dict with the best
    FP64 instruction rate (instructions/s) and flop rate (an FMA counts 2) over the sweep, the
    configuration that reached each, and the clocks seen."""
    import ctypes as C
    import statistics
    import subprocess

    import torch
    L = C.CDLL(build())
    L.grf_peak_fp64.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                C.POINTER(C.c_float), C.c_void_p]
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    threads = 256
    out = torch.empty(nsm * 8 * threads, dtype=torch.float64, device="cuda")
    ms = C.c_float()
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    smi = None
    if sample_clocks:
        try:
            smi = subprocess.Popen(["nvidia-smi", "--query-gpu=clocks.sm,clocks.max.sm,power.draw,"
                                    "clocks_event_reasons.active", "--format=csv,noheader,nounits", "-lms", "100",
                                    "-i", str(torch.cuda.current_device())],
                                   stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            smi = None
    results = []
    for kind in (0, 1, 2, 3, 4, 5):
        for chains in (4, 8, 16):
            for per_sm in (2, 4, 8):
                blocks = nsm * per_sm
                iters = 2000
                rc = L.grf_peak_fp64(kind, chains, blocks, threads, iters, 1, C.c_void_p(out.data_ptr()), C.byref(ms), st)
                assert rc == 0, rc
                launches = max(1, int(target_ms / max(ms.value, 1e-3)))
                best = float("inf")
                for _ in range(repeats):
                    rc = L.grf_peak_fp64(kind, chains, blocks, threads, iters, launches, C.c_void_p(out.data_ptr()),
                                         C.byref(ms), st)
                    assert rc == 0, rc
                    best = min(best, ms.value)
                instr = float(launches) * blocks * threads * chains * iters
                flops_per_instr = {0: 2.0, 1: 1.0, 2: 1.0, 3: 1.5, 4: 2.0, 5: 2.0}[kind]
                results.append({"kind": KINDS[kind], "chains": chains, "blocks_per_sm": per_sm, "threads": threads,
                                "launches": launches, "ms": best, "instr_per_s": instr / (best * 1e-3),
                                "flops_per_s": flops_per_instr * instr / (best * 1e-3)})
    clocks = None
    if smi is not None:
        smi.terminate()
        try:
            text, _ = smi.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            smi.kill()
            text = ""
        rows = [r.split(",") for r in text.strip().splitlines() if r.strip()]
        try:
            sm = [float(r[0]) for r in rows]
            clocks = {"samples": len(sm), "sm_mhz_median": statistics.median(sm), "sm_mhz_min": min(sm),
                      "sm_max_mhz": float(rows[0][1]), "power_w_max": max(float(r[2]) for r in rows),
                      "reasons": sorted({r[3].strip() for r in rows})}
        except (ValueError, IndexError):
            clocks = None
    best_i = max(results, key=lambda r: r["instr_per_s"])
    best_f = max(results, key=lambda r: r["flops_per_s"])
    return {"instr_per_s": best_i["instr_per_s"], "instr_config": best_i, "tflops": best_f["flops_per_s"] / 1e12,
            "tflops_config": best_f, "clocks": clocks, "sweep": results}


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    if "--measure" in sys.argv:
        import json
        print(json.dumps(measure(), indent=1))
