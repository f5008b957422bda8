"""Measure the arithmetic rates that bound the integration kernels (the
denominators of bench.py's ALU roofline) on the current GPU and print them
as a markdown table:

    python bench_peaks.py

Compiles bench_peaks.cu (register-resident chains, 8 blocks of 256 threads
per SM, one warm-up and one timed launch of roughly 0.1 s each) for sm_103a
into a temporary directory, runs every probe, and reports the SM clock
nvidia-smi gives after them. The probes are a measurement program, not part
of the library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))

PROBES = [  # (label, kind, active lanes, iterations)
    ("FP64 FMA, all 32 lanes", 0, 32, 24_000),
    ("FP64 FMA, 16 of 32 lanes active", 0, 16, 24_000),
    ("FP64 FMA, 8 of 32 lanes active", 0, 8, 24_000),
    ("FP64 FMA, 1 of 32 lanes active", 0, 1, 24_000),
    ("FP32 FMA, all lanes", 1, 32, 1_000_000),
    ("FP64 mma.sync m8n8k4 (DMMA)", 2, 32, 5_000),
    ("exp(double)", 3, 32, 1_000),
    ("1.0/x (double)", 4, 32, 3_000),
]


def build(out_dir: str) -> str:
    lib = os.path.join(out_dir, "libbench_peaks.so")
    nvcc = "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc"
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared",
                           "-Xcompiler", "-fPIC", "-o", lib, os.path.join(HERE, "bench_peaks.cu")])
    return lib


def main() -> None:
    with tempfile.TemporaryDirectory(prefix="bench_peaks_") as d:
        lib = ctypes.CDLL(build(d))
        lib.peak_probe.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_longlong, ctypes.POINTER(ctypes.c_double)]
        rows = []
        for label, kind, active, iters in PROBES:
            r = ctypes.c_double()
            code = lib.peak_probe(kind, active, iters, ctypes.byref(r))
            if code != 0:
                raise SystemExit(f"probe {label!r} failed with CUDA error {code}")
            rows.append((label, r.value))
    try:
        clk = subprocess.run(["nvidia-smi", "--query-gpu=clocks.sm,clocks.max.sm", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=30).stdout.strip()
    except (OSError, subprocess.SubprocessError):
        clk = "unknown"
    print("| probe | rate |\n|---|---|")
    for label, v in rows:
        unit = "/s" if "exp" in label or "1.0/x" in label else " FLOP/s"
        print(f"| {label} | {v:.3e}{unit} |")
    print(f"\nSM clock after the probes (current, max): {clk}")


if __name__ == "__main__":
    main()
