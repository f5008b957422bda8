"""Measure the arithmetic rates that bound the integration kernels (the
denominators of bench.py's ALU roofline) on cuda:0 and print them as a
markdown table:

    python -m paper_2510_10005_gb300.peaks

Runs the library's throughput probes (cgx_rate_probe: register-resident
chains, 8 blocks of 256 threads per SM, one warm-up and one timed launch of
roughly 0.1 s each) and the SM clock nvidia-smi reports after them.
"""
from __future__ import annotations

import subprocess

from . import chemgb

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


def main() -> None:
    chemgb.load(build_if_missing=True)
    rows = [(label, chemgb.cgx_rate_probe(kind, iters, active)) for label, kind, active, iters in PROBES]
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
