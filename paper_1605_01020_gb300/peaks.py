"""Measured peak rates of the arithmetic units on the current GPU (the denominators
of the roofline fractions the benchmark reports).

    python -m paper_1605_01020_gb300.peaks [--out FILE]

runs each probe of libiedg_probes.so (FP64 FMA, FP32 FMA, FP64 mma.sync, tcgen05 MMA
with TF32 and with BF16 operands) a few times on the current device, keeps the best
run, samples the SM clock while they run, and prints one JSON object (also written to
FILE when given).  A few seconds on one GPU."""
import argparse
import ctypes
import json
import os
import subprocess
import time

HERE = os.path.dirname(os.path.abspath(__file__))
KINDS = {0: "dfma_tflops", 1: "ffma_tflops", 2: "dmma_tflops", 3: "tf32_tcgen05_tflops", 4: "bf16_tcgen05_tflops"}
REPS = {0: 20, 1: 4, 2: 10, 3: 40, 4: 40}


def measure(tries=3):
    import torch
    from paper_1605_01020_gb300 import build
    build.build_probes()
    lib = ctypes.CDLL(build.PROBE_LIB)
    lib.iedg_peak_probe.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    lib.iedg_peak_probe.restype = ctypes.c_int
    torch.cuda.init()
    dev = torch.cuda.current_device()
    out = {"gpu": torch.cuda.get_device_name(dev), "sms": torch.cuda.get_device_properties(dev).multi_processor_count}
    smi = None
    try:
        smi = subprocess.Popen(["nvidia-smi", f"--id={dev}", "--query-gpu=clocks.sm,clocks.max.sm",
                                "--format=csv,noheader,nounits", "-lms", "100"], stdout=subprocess.PIPE,
                               stderr=subprocess.DEVNULL, text=True)
    except OSError:
        smi = None
    for kind, key in KINDS.items():
        best = 0.0
        for _ in range(tries):
            v = ctypes.c_double()
            rc = lib.iedg_peak_probe(kind, REPS[kind], ctypes.byref(v))
            if rc != 0:
                raise RuntimeError(f"probe {key} failed ({rc})")
            best = max(best, v.value)
        out[key] = round(best, 2)
    if smi is not None:
        time.sleep(0.2)
        smi.terminate()
        lines = smi.communicate(timeout=5)[0].split("\n")
        mhz = [float(l.split(",")[0]) for l in lines if l.strip() and l.split(",")[0].strip().isdigit()]
        mx = [float(l.split(",")[1]) for l in lines if l.strip() and len(l.split(",")) > 1
              and l.split(",")[1].strip().isdigit()]
        if mhz:
            out["sm_mhz_median"] = sorted(mhz)[len(mhz) // 2]
            out["sm_max_mhz"] = max(mx) if mx else None
    out["how"] = ("best of 3 runs per probe, CUDA events around one launch over all SMs: DFMA / FFMA 8 "
                  "independent FMA chains per thread; DMMA mma.sync m8n8k4 f64, 8 chains per warp; tcgen05.mma "
                  "cta_group::1 M=128 N=256 (K=8 TF32, K=16 BF16) back to back from one thread per SM into one "
                  "TMEM accumulator")
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    res = measure()
    line = json.dumps(res)
    print(line)
    if a.out:
        with open(a.out, "w") as f:
            f.write(line + "\n")


if __name__ == "__main__":
    main()
