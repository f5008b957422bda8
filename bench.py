"""Benchmark: cells integrated per second over dt on the GPU.

Workload (N = 1): the 53-species / 325-reaction synthetic methane-shaped
mechanism, 1,048,576 cells of the 1-D flame-like field (60% unburnt,
10% front, 30% burnt; p 1-10 atm), constant pressure, SDIRK-4 with error
control (rtol 1e-6, atol 1e-12) over dt = 1e-6 s, FP64. One step = one
cg_integrate call over all cells (after a device-to-device restore of the
initial state, which is part of the step). The per-cell state is
1,048,576 x 55 doubles = 461 MB, larger than the 129 MB L2, so no L2 flush
is needed between steps.

Prints one JSON line (see the keys below). --impl reference times the FP64
CPU oracle on the host cores instead.

Multi-GPU (torchrun): every rank integrates its own 1,048,576 cells (the
cells of a field are independent; no collective on the data path);
value = all cells / max-over-ranks time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CELLS = 1 << 20
OPTS = dict(method=2, reactor=1, adaptive=1, dt=1e-6, rtol=1e-6, atol=1e-12, newton_tol=0.03,
            max_newton=7, max_steps=100000, max_halvings=10, err_filter=1, neg_tol=1e-6)
METRIC = "cells integrated/s over dt"
WORKLOAD = ("53-species/325-reaction synthetic methane-shaped mechanism, 1,048,576-cell 1-D "
            "flame-like field, constant pressure, adaptive SDIRK-4 rtol 1e-6 atol 1e-12, dt 1e-6 s")


def algorithmic_flops_per_newton(n_species: int, n_reactions: int, j_terms: int) -> float:
    """FP64 flops of one Newton iteration of one cell:
    LU 2n^3/3, two triangular solves 2n^2, Newton matrix 2n^2, temperature
    row and constant-pressure correction 4n^2, Jacobian terms 2 per term,
    rates 30 per reaction, thermo 40 per species. Transcendentals excluded."""
    n = n_species + 1
    return 2.0 * n**3 / 3 + 8.0 * n * n + 2.0 * j_terms + 30.0 * n_reactions + 40.0 * n_species


def j_term_count(mech) -> int:
    """Number of sparse Jacobian terms the assembly schedule adds (same rule
    as the library: for every species with nonzero net coefficient in a
    reaction, one temperature term, one per used slot, one per efficiency)."""
    total = 0
    for j in range(mech.nr):
        nu = {}
        for s in range(3):
            if mech.rf_idx[j, s] >= 0:
                nu[mech.rf_idx[j, s]] = nu.get(mech.rf_idx[j, s], 0) - mech.rf_nu[j, s]
            if mech.rr_idx[j, s] >= 0:
                nu[mech.rr_idx[j, s]] = nu.get(mech.rr_idx[j, s], 0) + mech.rr_nu[j, s]
        slots = int((mech.rf_idx[j] >= 0).sum() + (mech.rr_idx[j] >= 0).sum())
        effs = int(mech.eff_ptr[j + 1] - mech.eff_ptr[j]) if mech.rtype[j] != 0 else 0
        total += sum(1 for v in nu.values() if v != 0) * (1 + slots + effs)
    return total


def fp64_peak(sm_count: int, sm_max_mhz: float) -> float:
    """FP64 FMA pipe: 2 lanes per clock per SM on GB300 (measured: a
    register-resident DFMA loop reaches 1.195e12 FLOP/s at 1987 MHz on 152
    SMs = 3.96 FLOP/clk/SM), taken at the maximum SM clock."""
    return 4.0 * sm_count * sm_max_mhz * 1e6


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.idx = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def make_workload(seed: int = 0, cells: int = CELLS):
    from paper_2510_10005_gb300 import inputs
    mech = inputs.gen_mechanism("ch4")
    T, Y, p = inputs.field_flames(mech, cells, seed=seed)
    return mech, T, Y, p


def cpu_oracle_sample(mech, T, Y, p, n_sample: int, threads: int):
    """Time the oracle on a stratified sample; returns (cells/s, seconds)."""
    import oracle
    r = oracle.RefMech(mech)
    idx = np.linspace(0, len(T) - 1, n_sample).astype(np.int64)
    t0 = time.perf_counter()
    r.integrate(T[idx], Y[idx], p[idx], OPTS, nthreads=threads)
    el = time.perf_counter() - t0
    return n_sample / el, el


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    mech, T, Y, p = make_workload()
    threads = os.cpu_count() or 1
    n_sample = args.ref_sample
    for _ in range(args.warmup):
        cpu_oracle_sample(mech, T, Y, p, max(16, n_sample // 8), threads)
    times = []
    for _ in range(args.steps):
        v, el = cpu_oracle_sample(mech, T, Y, p, n_sample, threads)
        times.append(el)
    value = n_sample * args.steps / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD},
        "cpu_baseline": {"value": value, "unit": "cells/s", "cores": threads, "kind": "oracle",
                         "sample": f"{n_sample} cells evenly spaced through the field, per step"},
        "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import torch
    from paper_2510_10005_gb300 import chemgb

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device(f"cuda:{local}")
    chemgb.load(build_if_missing=(rank == 0 and ws == 1))

    mech, T, Y, p = make_workload(seed=rank, cells=args.cells)
    h = chemgb.cg_mech_create(mech)
    if args.team:
        chemgb.cg_mech_set_launch(h, args.team, args.tpb)
    opts = chemgb.make_opts(**OPTS, precision=args.precision)
    N = len(T)
    T0 = torch.tensor(T, dtype=torch.float64, device=dev)
    Y0 = torch.tensor(np.ascontiguousarray(Y.T), dtype=torch.float64, device=dev)
    P0 = torch.tensor(p, dtype=torch.float64, device=dev)
    Tw, Yw = torch.empty_like(T0), torch.empty_like(Y0)
    st = torch.empty(N, dtype=torch.int32, device=dev)
    stats = torch.empty((4, N), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        Tw.copy_(T0)
        Yw.copy_(Y0)
        chemgb.cg_integrate(h, opts, Tw, Yw, P0, st, stats, stream=stream.cuda_stream)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    barrier()
    ms = ev0.elapsed_time(ev1)
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = ws * N * args.steps / (ms * 1e-3)

    st_h = st.cpu().numpy()
    stats_h = stats.cpu().numpy()
    newton = int(stats_h[2].astype(np.int64).sum())
    jt = j_term_count(mech)
    fpu = algorithmic_flops_per_newton(mech.ns, mech.nr, jt)
    launch_ms = ms / args.steps
    achieved = fpu * newton / (launch_ms * 1e-3)
    props = torch.cuda.get_device_properties(dev)
    clocks = clk.summary()
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    peak = fp64_peak(props.multi_processor_count, sm_max)

    # end to end: host arrays through cg_integrate_host (copies inside the timed region)
    e2e_steps = min(args.steps, args.e2e_steps)
    Th0 = np.ascontiguousarray(T)
    Yh0 = np.ascontiguousarray(Y.T)
    ph = np.ascontiguousarray(p)
    sh = np.zeros(N, np.int32)
    sth = np.zeros((4, N), np.int32)
    e2e_t = 0.0
    for k in range(e2e_steps + 1):
        Th, Yh = Th0.copy(), Yh0.copy()
        barrier()
        t0 = time.perf_counter()
        chemgb.cg_integrate_host(h, opts, Th, Yh, ph, sh, sth)
        el = time.perf_counter() - t0
        if k > 0:   # first call allocates the library's workspace: untimed
            e2e_t += el
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([e2e_t], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_t = float(t.item())
    e2e_value = ws * N * e2e_steps / e2e_t
    h2d = N * (1 + mech.ns + 1) * 8
    d2h = N * (1 + mech.ns) * 8 + N * 4 + 4 * N * 4

    if rank != 0:
        return
    cpu = None
    if ws == 1 and not args.no_cpu:
        threads = os.cpu_count() or 1
        v, el = cpu_oracle_sample(mech, T, Y, p, args.cpu_sample, threads)
        cpu = {"value": v, "unit": "cells/s", "cores": threads, "kind": "oracle",
               "sample": f"{args.cpu_sample} cells evenly spaced through the field ({el:.1f} s)"}
    line = {
        "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": launch_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells_per_gpu": N, "state_bytes": int(N * 55 * 8),
                   "l2": "state (461 MB) larger than L2; no flush"},
        "e2e": {"value": e2e_value, "unit": "cells/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "peak_source": "derived: 4 FP64 FLOP/clk/SM (measured DFMA rate) x SMs x max SM clock",
                     "kernel": "integrate_kernel", "newton_per_launch": newton,
                     "flops_per_newton": fpu},
        "cpu_baseline": cpu,
        "clocks": clocks,
        "gpu_launches": args.steps,
        "cells_failed": int((st_h != 0).sum()),
        "stats_mean": {"steps": float(stats_h[0].mean()), "rejects": float(stats_h[1].mean()),
                       "newton": float(stats_h[2].mean())},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--cpu-sample", type=int, default=2048)
    ap.add_argument("--ref-sample", type=int, default=1024)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cells", type=int, default=CELLS, help="cells per GPU (default: the workload's)")
    ap.add_argument("--team", type=int, default=0, help="threads per cell (default: the library's choice)")
    ap.add_argument("--tpb", type=int, default=1, help="cells per block with --team 32")
    ap.add_argument("--precision", type=int, default=0, help="0: FP64 Newton matrix, 1: FP32 LU")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
