"""Benchmark: cells integrated per second over dt on the GPU.

Default workload (--config 2, N = 1): the 53-species / 325-reaction
synthetic methane-shaped mechanism, 1,048,576 cells of the 1-D flame-like
field (60% unburnt, 10% front, 30% burnt; p 1-10 atm), constant pressure,
SDIRK-4 with error control (rtol 1e-6, atol 1e-12) over dt = 1e-6 s, FP64.
One step = one cg_integrate call over all cells after a device-to-device
restore of the initial state (part of the step). The per-cell state is
1,048,576 x 55 doubles = 461 MB, larger than the 129 MB L2, so no L2 flush is
needed between steps.

Other workloads (reported beside the default line):
  --config 1  9 species, one backward-Euler step of 1e-5 s, 4096 cells
  --config 3  53 + 9 species in ONE persistent work-stealing launch,
              1,048,576 heavy-tailed cells each (90% frozen, 5% burnt,
              5% reacting, randomly interleaved), FP32 Newton matrix,
              autotuned launch shape for the 53 species (the 9 species run
              one warp per cell inside it), replayed from a captured CUDA graph
  --config 4  discrete adjoint: 53 species, 65,536 cells, T0 in U[1100, 1400] K,
              1 atm, phi in U[0.5, 2], adaptive SDIRK-4 over dt = 1e-4 s with
              checkpoints, then the backward sweep for
              L = sum (T_end - T_target)^2 (target from ln A + N(0, 0.1^2));
              gradients w.r.t. (ln A, b, Ea) of all reactions and (T0, Y0)
  --config 5  160 species / 900 reactions, T in U[700, 1600] K,
              p in U[20, 40] atm, adaptive SDIRK-4 (use --cells for a subset);
              with --adjoint: config 4's forward with checkpoints plus the
              discrete adjoint on 8,192 cells of this field

Prints one JSON line. --impl reference times the FP64 CPU oracle on the
host cores instead (a bounded sample of the same workload). The oracle runs
only in that arm and in the cpu_baseline leg; parity at these sizes is
checked by the GPU tests (tests/test_gpu_zfull_size.py).

Multi-GPU (torchrun): every rank integrates its own cells (cells are
independent; no collective on the data path); value = all cells /
max-over-ranks time ("scaling": "weak").
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

METRIC = "cells integrated/s over dt"
METRIC_ADJ = "cells differentiated/s over dt (forward with checkpoints + adjoint)"
SDIRK4 = dict(method=2, reactor=1, adaptive=1, dt=1e-6, rtol=1e-6, atol=1e-12, newton_tol=0.03,
              max_newton=7, max_steps=100000, max_halvings=10, err_filter=1, neg_tol=1e-6)
BE = dict(method=0, reactor=1, adaptive=0, dt=1e-5, rtol=1e-10, atol=1e-16, newton_tol=1.0,
          max_newton=20, max_halvings=10, neg_tol=1e-6)

CONFIGS = {
    1: dict(cells=4096, opts=BE, precision=0,
            workload="9-species/21-reaction synthetic H2/O2 mechanism, 4096 cells, T0 U[1000,1500] K, "
                     "1 atm, phi U[0.5,2], constant pressure, one backward-Euler step of 1e-5 s (+halvings)"),
    2: dict(cells=1 << 20, opts=SDIRK4, precision=0,
            workload="53-species/325-reaction synthetic methane-shaped mechanism, 1,048,576-cell 1-D "
                     "flame-like field, constant pressure, adaptive SDIRK-4 rtol 1e-6 atol 1e-12, dt 1e-6 s"),
    3: dict(cells=1 << 20, opts=SDIRK4, precision=1,
            workload="53-species + 9-species mechanisms in one persistent work-stealing launch, "
                     "2 x 1,048,576 heavy-tailed cells (90% frozen, 5% burnt, 5% reacting, interleaved), "
                     "FP32 Newton matrix, autotuned, CUDA graph, adaptive SDIRK-4 rtol 1e-6, dt 1e-6 s"),
    4: dict(cells=1 << 16, opts=dict(SDIRK4, dt=1e-4), precision=0,
            workload="53-species/325-reaction synthetic methane-shaped mechanism, 65,536 cells, T0 U[1100,1400] K, "
                     "1 atm, phi U[0.5,2], constant pressure, adaptive SDIRK-4 rtol 1e-6 over dt 1e-4 s with "
                     "checkpoints + discrete adjoint of L = sum (T_end - T_target)^2, T_target from "
                     "ln A + N(0, 0.1^2); gradients w.r.t. 975 Arrhenius parameters and (T0, Y0)"),
    5: dict(cells=1 << 18, opts=SDIRK4, precision=0,
            workload="160-species/900-reaction synthetic n-heptane-shaped mechanism, T U[700,1600] K, "
                     "p U[20,40] atm, phi U[0.5,1.5], constant pressure, adaptive SDIRK-4 rtol 1e-6, dt 1e-6 s"),
}


# DRAM bytes per cell of integrate_kernel from one ncu capture (65,536 cells of
# the flame field, dram__bytes_read.sum + dram__bytes_write.sum), valid only
# for the kernel sources it was taken on (sha256 of the files below,
# concatenated); scaled to a launch by its cell count.
TRAFFIC_SOURCES = ("integrate.cuh", "chem_device.cuh", "stepper.cuh", "chem_internal.h", "instances.cu")
TRAFFIC = {2: dict(bytes_per_cell=(43841536 + 873657344) / 65536,
                   sha256="d035387d5285847fed9ee9c75cfb26615ff4ba202cfb42518f5fb591f01359f8")}


def measured_traffic(config: int, cells: int):
    import hashlib
    t = TRAFFIC.get(config)
    if t is None:
        return None
    csrc = os.path.join(ROOT, "paper_2510_10005_gb300", "csrc")
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return t["bytes_per_cell"] * cells if h.hexdigest() == t["sha256"] else None


def algorithmic_flops_per_newton(n_species: int, n_reactions: int, j_terms: int, fp32_lu: bool) -> float:
    """FP64 flops of one Newton iteration of one cell: LU 2n^3/3 (FP64 mode
    only), two triangular solves 2n^2, Newton matrix 2n^2, temperature row
    and constant-pressure correction 4n^2, Jacobian terms 2 per term, rates
    30 per reaction, thermo 40 per species. Transcendentals excluded."""
    n = n_species + 1
    lu = 0.0 if fp32_lu else 2.0 * n**3 / 3
    return lu + 8.0 * n * n + 2.0 * j_terms + 30.0 * n_reactions + 40.0 * n_species


def j_term_count(mech) -> int:
    """Sparse Jacobian terms of the assembly schedule: for every species with
    a nonzero net coefficient in a reaction, one temperature term, one per
    used slot and one per efficiency."""
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


FP32_PEAK = 7.679e13  # FLOP/s, FP32 FMA rate measured by bench_peaks.py on this GB300 (2070 MHz)


def fp64_peak(sm_count: int, sm_max_mhz: float) -> float:
    """FP64 FMA pipe: one unit per SM sub-partition retiring half a lane per
    clock, 2 lanes (4 FLOP) per clock per SM (measured: 1.195e12 FLOP/s at
    1987 MHz on 152 SMs), at the maximum SM clock."""
    return 4.0 * sm_count * sm_max_mhz * 1e6


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
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
        rows = [[p.strip() for p in line.split(",")] for line in open(self.path)]
        rows = [r for r in rows if len(r) >= 9]
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        num = lambda v: v.replace(".", "").isdigit()
        sm = [float(r[1]) for r in rows if num(r[1])]
        mx = [float(r[2]) for r in rows if num(r[2])]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# workloads: list of (mechanism, T, Y, p)


def make_workload(config: int, cells: int, seed: int = 0):
    from paper_2510_10005_gb300 import inputs
    if config == 1:
        m = inputs.gen_mechanism("h2")
        T, Y, p = inputs.field_reactor(m, cells, (1000, 1500), (1, 1), (0.5, 2), "H2", seed=seed)
        return [(m, T, Y, p)]
    if config == 2:
        m = inputs.gen_mechanism("ch4")
        T, Y, p = inputs.field_flames(m, cells, seed=seed)
        return [(m, T, Y, p)]
    if config == 3:
        m53, m9 = inputs.gen_mechanism("ch4"), inputs.gen_mechanism("h2")
        T, Y, p, _ = inputs.field_mixed(m53, cells, "CH4", seed=seed, argon=0.0093)
        T9, Y9, p9, _ = inputs.field_mixed(m9, cells, "H2", seed=seed + 1000)
        return [(m53, T, Y, p), (m9, T9, Y9, p9)]
    if config == 4:
        m = inputs.gen_mechanism("ch4")
        T, Y, p = inputs.field_reactor(m, cells, (1100, 1400), (1, 1), (0.5, 2), "CH4", seed=seed)
        return [(m, T, Y, p)]
    if config == 5:
        m = inputs.gen_mechanism("c7")
        T, Y, p = inputs.field_reactor(m, cells, (700, 1600), (20, 40), (0.5, 1.5), "C7H16", seed=seed)
        return [(m, T, Y, p)]
    raise ValueError(config)


# --method: the integrator of the workload (default: the workload's own)
METHODS = {
    "be": dict(method=0, adaptive=0),
    "sdirk2": dict(method=1),
    "sdirk4": dict(method=2),
    "ros2": dict(method=3),                       # Appendix A.3, one factorisation per step
    "yass": dict(method=4, adaptive=0, rtol=1e-3, atol=1e-6, newton_tol=1.0, max_halvings=12),
}


# --linear: the Newton systems' solver (Section 3.4); GMRES with
# Gauss-Seidel preconditioning, restart 30, tolerance 1e-10 unless overridden
LINEAR = {"lu": dict(linear_solver=0),
          "gmres": dict(linear_solver=1, preconditioner=2, gmres_restart=30, gmres_maxit=200, gmres_tol=1e-10)}
PRECS = {"none": 0, "jacobi": 1, "gs": 2}


def opts_dict(config: int, precision: int, method: str | None = None, linear: str | None = None,
              prec: str | None = None):
    o = dict(CONFIGS[config]["opts"])
    if method:
        o.update(METHODS[method])
    if linear:
        o.update(LINEAR[linear])
        if prec:
            o["preconditioner"] = PRECS[prec]
    o["precision"] = precision
    if config == 3:
        o["persistent"] = 1
    return o


def workload_name(config: int, method: str | None, linear: str | None = None, prec: str | None = None) -> str:
    w = CONFIGS[config]["workload"]
    if method:
        extra = {"yass": "YASS (alpha 1, WRMS weights 1e-6 + 1e-3|y|, up to 12 halvings)",
                 "ros2": "Rosenbrock-2", "be": "backward Euler", "sdirk2": "SDIRK-2", "sdirk4": "SDIRK-4"}[method]
        w += "; integrator replaced by " + extra
    if linear == "gmres":
        w += "; Newton systems by GMRES(30), tol 1e-10, preconditioner " + {
            "none": "none", "jacobi": "Jacobi", "gs": "Gauss-Seidel", None: "Gauss-Seidel"}[prec]
    return w


def workload_variant(parts, args):
    """The workload's mechanisms with SRI falloff and PLOG reactions
    (--sri-plog) and/or refitted thermodynamics (--thermo-degree)."""
    from paper_2510_10005_gb300 import inputs
    if args.sri_plog:
        parts = [(inputs.with_sri_plog(m, n_sri=max(1, m.nr // 40), n_plog=max(1, m.nr // 16), seed=3), T, Y, p)
                 for m, T, Y, p in parts]
    if args.thermo_degree is not None:
        parts = [(inputs.with_thermo_degree(m, args.thermo_degree), T, Y, p) for m, T, Y, p in parts]
    return parts


def flow_state(m, T, Y, p):
    """Conserved variables of a compressible flow solver for the split
    surface (input construction): rho from the ideal gas, u = sum Y_i u_i(T)
    from the mechanism's c_p polynomials (NASA-7 or another degree), rho Y."""
    R = 8314.46261815324
    rho = p / (R * T * (Y / m.W).sum(axis=1))
    a = m.thermo_coef
    P = a.shape[1] - 3
    Tc = T[:, None]
    h_RT = a[:, P] / (P + 1)
    for k in range(P - 1, -1, -1):
        h_RT = a[:, k] / (k + 1) + Tc * h_RT
    h_RT = h_RT + a[:, P + 1] / Tc
    u = (Y * (R / m.W) * Tc * (h_RT - 1.0)).sum(axis=1)
    return rho, u, rho[:, None] * Y


def oracle_opts(o: dict) -> dict:
    return {k: v for k, v in o.items() if k not in ("precision", "persistent")}


# cells of the adjoint workloads (--config 4, --config 5 --adjoint: a subset
# of the 262,144-cell field, since a 160-species cell takes about 1.5 ms of
# the GPU forward and backward)
ADJOINT_CELLS = {4: 1 << 16, 5: 8192}
# the oracle's forward + adjoint timing samples (several seconds per cell at 160 species)
CPU_SAMPLE_ADJ = {4: 256, 5: 16}
ONE_CORE_SAMPLE_ADJ = {4: 16, 5: 1}


def adjoint_workload(config: int, n_cells: int) -> str:
    if config == 4:
        return CONFIGS[4]["workload"]
    return (CONFIGS[config]["workload"] + f", {n_cells:,} cells of the field recipe, with checkpoints + discrete "
            "adjoint of L = sum (T_end - T_target)^2, T_target from ln A + N(0, 0.1^2); gradients w.r.t. "
            "2700 Arrhenius parameters and (T0, Y0)")


# The oracle's timing sample of each workload: cells evenly spaced through
# every mechanism's field (so in proportion from the regions of the
# contiguous flame field, and a uniform sample of the interleaved ones)
CPU_SAMPLE = {1: 4096, 2: 4096, 3: 4096, 4: 256, 5: 256}
# and of the one-core timing beside it (160 species: about 1 s per cell)
ONE_CORE_SAMPLE = {1: 256, 2: 256, 3: 256, 4: 16, 5: 16}


def sample_indices(n_cells: int, k: int) -> np.ndarray:
    return np.linspace(0, n_cells - 1, min(k, n_cells)).astype(np.int64)


def cpu_oracle_sample(parts, opts, n_sample: int, threads: int, split: bool = False):
    """Time the oracle on an evenly spaced sample of every mechanism's cells
    (shares in proportion to the cells); returns (cells/s, seconds, cells).
    split: the operator-split step (T from the conserved variables, then the
    constant-volume integration) instead of the integration alone."""
    import oracle
    total = sum(len(T) for _, T, _, _ in parts)
    t, done = 0.0, 0
    for m, T, Y, p in parts:
        k = max(1, int(round(n_sample * len(T) / total)))
        idx = sample_indices(len(T), k)
        k = len(idx)
        r = oracle.RefMech(m)
        if split:
            rho, u, rhoY = flow_state(m, T[idx], Y[idx], p[idx])
            t0 = time.perf_counter()
            r.react_split(rho, u, rhoY, T[idx], oracle_opts(opts), nthreads=threads)
        else:
            t0 = time.perf_counter()
            r.integrate(T[idx], Y[idx], p[idx], oracle_opts(opts), nthreads=threads)
        t += time.perf_counter() - t0
        done += k
    return done / t, t, done


def median_timing(run, cells: int, repeats: int):
    """Times the oracle `repeats` times on the same sample of `cells` cells;
    run(k) returns (seconds, cells run). Returns (cells run, median seconds,
    all timings)."""
    times, done = [], 0
    for _ in range(max(1, repeats)):
        el, done = run(cells)
        times.append(el)
    return done, statistics.median(times), times


def full_workload_name(args) -> str:
    """The workload as both arms state it, with every option that changes it."""
    return (workload_name(args.config, args.method, args.linear, args.prec)
            + ("; operator-split surface: (rho, u, rho Y) in, T recovered (5 Newton iterations), "
               "constant volume, T and R out" if args.surface == "split" else "")
            + ("; mechanism with nr/40 Troe reactions made SRI and nr/16 elementary reactions made "
               "PLOG (3-6 levels, 0.1-100 atm)" if args.sri_plog else "")
            + (f"; thermodynamics refitted with a c_p polynomial of degree {args.thermo_degree}"
               if getattr(args, "thermo_degree", None) is not None else ""))


def dist_env():
    from paper_2510_10005_gb300 import multirank
    return multirank.env()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    cfg = CONFIGS[args.config]
    parts = workload_variant(make_workload(args.config, args.cells or cfg["cells"]), args)
    opts = opts_dict(args.config, 0, args.method, args.linear, args.prec)
    split = args.surface == "split"
    if split:
        if len(parts) != 1:
            raise SystemExit("--surface split takes one mechanism")
        opts["reactor"] = 0   # the split step is at constant volume
    threads = os.cpu_count() or 1
    n_sample = args.cpu_sample or CPU_SAMPLE[args.config]
    for _ in range(args.warmup):
        cpu_oracle_sample(parts, opts, n_sample, threads, split)
    times, k = [], 0
    for _ in range(args.steps):
        _, el, k = cpu_oracle_sample(parts, opts, n_sample, threads, split)
        times.append(el)
    value = k / statistics.median(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": full_workload_name(args), "config": args.config},
        "cpu_baseline": {"value": value, "unit": "cells/s", "cores": threads, "kind": "oracle",
                         "sample": f"the same {k} cells evenly spaced through the field every step; "
                                   f"value = cells / median step time"},
        "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import torch
    from paper_2510_10005_gb300 import chemgb, multirank

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    chemgb.load(build_if_missing=(ws == 1))
    cfg = CONFIGS[args.config]
    precision = cfg["precision"] if args.precision is None else args.precision
    parts = workload_variant(make_workload(args.config, args.cells or cfg["cells"], seed=rank), args)
    opts_d = opts_dict(args.config, precision, args.method, args.linear, args.prec)
    split = args.surface == "split"
    if split:
        if len(parts) != 1:
            raise SystemExit("--surface split takes one mechanism")
        opts_d["reactor"] = 0   # the split step is at constant volume
    opts = chemgb.make_opts(**opts_d)
    stream = torch.cuda.Stream(dev)   # a side stream (graph capture needs one); all work goes there
    torch.cuda.set_stream(stream)

    handles, bufs = [], []
    for m, T, Y, p in parts:
        h = chemgb.cg_mech_create(m)
        if args.smem_limit:
            chemgb.cg_mech_set_smem_limit(h, args.smem_limit)
        if args.team:
            chemgb.cg_mech_set_launch(h, args.team, args.tpb)
        if args.lu_panel is not None:
            chemgb.cg_mech_set_lu_panel(h, args.lu_panel)
        N = len(T)
        b = dict(T0=torch.tensor(T, dtype=torch.float64, device=dev),
                 Y0=torch.tensor(np.ascontiguousarray(Y.T), dtype=torch.float64, device=dev),
                 P=torch.tensor(p, dtype=torch.float64, device=dev),
                 st=torch.empty(N, dtype=torch.int32, device=dev),
                 stats=torch.empty((4, N), dtype=torch.int32, device=dev))
        b["T"], b["Y"] = torch.empty_like(b["T0"]), torch.empty_like(b["Y0"])
        if split:
            rho, u, rhoY = flow_state(m, T, Y, p)
            b.update(RHO=torch.tensor(rho, dtype=torch.float64, device=dev),
                     E=torch.tensor(u, dtype=torch.float64, device=dev),
                     RHOY=torch.tensor(np.ascontiguousarray(rhoY.T), dtype=torch.float64, device=dev),
                     R=torch.empty_like(b["Y0"]))
        handles.append(h)
        bufs.append(b)
    N_total = sum(len(b["T0"]) for b in bufs)

    tuned = None
    if (args.config == 3 or args.autotune) and not args.team:
        # autotune the launch shape on the dominant mechanism; the others keep
        # their own team size (a one-warp mechanism in a wider launch runs
        # split: each warp of a team integrates its own cells)
        k = min(16384, len(bufs[0]["T0"]))
        sel = torch.linspace(0, len(bufs[0]["T0"]) - 1, k, device=dev).long()
        cache = os.path.join(tempfile.mkdtemp(prefix="chemgb_tune_"), "shape.json")   # new: always tunes
        ms = chemgb.cg_autotune(handles[0], opts, bufs[0]["T0"][sel].contiguous(),
                                bufs[0]["Y0"][:, sel].contiguous(), bufs[0]["P"][sel].contiguous(), cache)
        team, tpb = chemgb.cg_mech_get_launch(handles[0])
        for h in handles[1:]:
            t_own, _ = chemgb.cg_mech_get_launch(h)
            if t_own != 32 and t_own != team:   # only one-warp mechanisms can run split
                chemgb.cg_mech_set_launch(h, team, tpb if team == 32 else 1)
        tuned = {"team": team, "teams_per_block": tpb, "sample_ms": ms}
        try:   # the shared-memory limit per cell and the LU panel width the tuner chose
            with open(cache) as f:
                c = json.load(f)
            tuned["smem_limit"], tuned["lu_panel"] = c["smem_limit"], c["lu_panel"]
        except (OSError, ValueError, KeyError):
            pass

    def integrate():
        for b in bufs:
            b["T"].copy_(b["T0"])
            if not split:
                b["Y"].copy_(b["Y0"])
        if split:   # conserved variables in; T (guess: the flow solver's last one) and R out
            b = bufs[0]
            chemgb.cg_react_split(handles[0], opts, b["RHO"], b["E"], b["RHOY"], b["T"], b["R"], 5, b["st"],
                                  b["stats"], stream=stream.cuda_stream)
        elif len(handles) == 1:
            b = bufs[0]
            chemgb.cg_integrate(handles[0], opts, b["T"], b["Y"], b["P"], b["st"], b["stats"],
                                stream=stream.cuda_stream)
        else:
            chemgb.cg_integrate_batch(handles, opts, [b["T"] for b in bufs], [b["Y"] for b in bufs],
                                      [b["P"] for b in bufs], [b["st"] for b in bufs],
                                      [b["stats"] for b in bufs], stream=stream.cuda_stream)

    step = integrate
    graph = None
    if args.config == 3 and not args.no_graph:
        integrate()                      # first call outside capture (kernel attributes, pools)
        torch.cuda.synchronize(dev)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            integrate()
        step = graph.replay

    barrier = multirank.barrier

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
    ms = multirank.max_over_ranks(ev0.elapsed_time(ev1), dev)
    value = multirank.job_throughput(N_total, ws, args.steps, ms * 1e-3)
    launch_ms = ms / args.steps

    newton, flops, flops32, failed, stat_means = 0, 0.0, 0.0, 0, []
    for (m, *_), b in zip(parts, bufs):
        sh = b["stats"].cpu().numpy()
        nwt = int(sh[2].astype(np.int64).sum())
        newton += nwt
        n1 = m.ns + 1
        gm = opts_d.get("linear_solver", 0) == 1
        per = algorithmic_flops_per_newton(m.ns, m.nr, j_term_count(m), precision == 1 or gm)
        if opts_d["method"] == 3:   # Rosenbrock-2: plus a second rate evaluation and solve per step
            per += 30.0 * m.nr + 40.0 * m.ns + 2.0 * n1 ** 2
        flops += nwt * per
        if precision == 1 and not gm:   # the FP32 factorisations (stats row 3), 2n^3/3 each
            flops32 += float(sh[3].astype(np.int64).sum()) * 2.0 * n1 ** 3 / 3
        if gm:   # GMRES iterations (stats row 3): matvec 2n^2, preconditioner, Gram-Schmidt and norms ~10n
            pc = {0: 0.0, 1: n1, 2: n1 * n1}[opts_d.get("preconditioner", 2)]
            flops += float(sh[3].astype(np.int64).sum()) * (2.0 * n1 * n1 + pc + 10.0 * n1) - nwt * 2.0 * n1 * n1
        failed += int((b["st"].cpu().numpy() != 0).sum())
        stat_means.append({"species": m.ns, "steps": float(sh[0].mean()), "rejects": float(sh[1].mean()),
                           "newton": float(sh[2].mean())})
    props = torch.cuda.get_device_properties(dev)
    clocks = clk.summary()
    peak = fp64_peak(props.multi_processor_count, clocks.get("sm_max_mhz") or 2070.0)
    achieved = flops / (launch_ms * 1e-3)

    # end to end through the host entry point (copies inside the timed region)
    e2e = None
    if len(handles) > 1 and args.e2e_steps > 0:
        # the batch call with the inputs copied from pinned host memory and the
        # results copied back inside the timed region, every call
        host = [dict(T=torch.tensor(T, dtype=torch.float64).pin_memory(),
                     Y=torch.tensor(np.ascontiguousarray(Y.T), dtype=torch.float64).pin_memory(),
                     P=torch.tensor(p, dtype=torch.float64).pin_memory(),
                     To=torch.empty(len(T), dtype=torch.float64).pin_memory(),
                     Yo=torch.empty((m.ns, len(T)), dtype=torch.float64).pin_memory(),
                     So=torch.empty(len(T), dtype=torch.int32).pin_memory()) for m, T, Y, p in parts]
        calls = []
        for _ in range(args.e2e_steps):
            barrier()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            for hb, b in zip(host, bufs):
                b["T"].copy_(hb["T"], non_blocking=True)
                b["Y"].copy_(hb["Y"], non_blocking=True)
                b["P"].copy_(hb["P"], non_blocking=True)
            chemgb.cg_integrate_batch(handles, opts, [b["T"] for b in bufs], [b["Y"] for b in bufs],
                                      [b["P"] for b in bufs], [b["st"] for b in bufs], [b["stats"] for b in bufs],
                                      stream=stream.cuda_stream)
            for hb, b in zip(host, bufs):
                hb["To"].copy_(b["T"], non_blocking=True)
                hb["Yo"].copy_(b["Y"], non_blocking=True)
                hb["So"].copy_(b["st"], non_blocking=True)
            torch.cuda.synchronize(dev)
            calls.append(multirank.max_over_ranks(time.perf_counter() - t0, dev))
        e2e = {"value": multirank.job_throughput(N_total, ws, 1, statistics.median(calls)), "unit": "cells/s",
               "h2d_bytes_per_step": sum(len(T) * (m.ns + 2) * 8 for m, T, _, _ in parts),
               "d2h_bytes_per_step": sum(len(T) * ((m.ns + 1) * 8 + 4) for m, T, _, _ in parts),
               "steps": args.e2e_steps, "call_s": calls,
               "how": "median of timed cg_integrate_batch calls with the inputs copied from pinned host memory "
                      "and T, Y, status copied back inside the timed region (no graph)"}
    if len(handles) == 1 and args.e2e_steps > 0 and not split:
        m, T, Y, p = parts[0]
        N = len(T)
        Th0, Yh0, ph = np.ascontiguousarray(T), np.ascontiguousarray(Y.T), np.ascontiguousarray(p)
        sh_, sth = np.zeros(N, np.int32), np.zeros((4, N), np.int32)
        calls = []
        for k in range(args.e2e_steps):
            Th, Yh = Th0.copy(), Yh0.copy()
            barrier()
            t0 = time.perf_counter()
            chemgb.cg_integrate_host(handles[0], opts, Th, Yh, ph, sh_, sth)
            calls.append(multirank.max_over_ranks(time.perf_counter() - t0, dev))
        e2e_t = statistics.median(calls)
        e2e = {"value": multirank.job_throughput(N, ws, 1, e2e_t), "unit": "cells/s",
               "h2d_bytes_per_step": N * (m.ns + 2) * 8, "d2h_bytes_per_step": N * (m.ns + 1) * 8 + 20 * N,
               "steps": args.e2e_steps, "call_s": calls,
               "how": "median of the timed cg_integrate_host calls (host arrays in and out, copies inside; "
                      "the first call also grows the library's device workspace once)"}

    if rank != 0:
        return
    cpu = None
    if ws == 1 and not args.no_cpu:
        threads = os.cpu_count() or 1
        n_sample = args.cpu_sample or CPU_SAMPLE[args.config]
        k, el, times = median_timing(lambda n: cpu_oracle_sample(parts, opts_d, n, threads, split)[1:], n_sample,
                                     args.cpu_repeats)
        cpu = {"value": k / el, "unit": "cells/s", "cores": threads, "kind": "oracle",
               "sample": f"{k} cells evenly spaced through the field, median of {len(times)} timings "
                         f"({', '.join(f'{t:.2f}' for t in times)} s)"}
        one = ONE_CORE_SAMPLE[args.config] if args.cpu_1core_cells is None else args.cpu_1core_cells
        if one > 0:   # the same oracle on one host core
            k1, el1, t1 = median_timing(lambda n: cpu_oracle_sample(parts, opts_d, n, 1, split)[1:], one, 1)
            cpu["one_core"] = {"value": k1 / el1, "unit": "cells/s", "cores": 1,
                               "sample": f"{k1} cells evenly spaced through the field ({el1:.1f} s)"}
    state_bytes = sum(len(T) * (m.ns + 2) * 8 for m, T, _, _ in parts)
    line = {
        "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": launch_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": full_workload_name(args),
                   "config": args.config,
                   "cells_per_gpu": N_total,
                   "newton_matrix": "fp32" if precision == 1 else "fp64", "state_bytes": state_bytes,
                   "l2": "state larger than L2 (129 MB); no flush" if state_bytes > 129e6
                   else "state smaller than L2; each step restores it from a second copy"},
        "e2e": e2e,
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": measured_traffic(args.config, N_total),
                     "peak_source": "derived: 4 FP64 FLOP/clk/SM (measured DFMA rate) x SMs x max SM clock",
                     "kernel": "integrate_kernel", "newton_per_launch": newton},
        **({"roofline_fp32": {"bound": "alu", "achieved": flops32 / (launch_ms * 1e-3) / 1e12, "peak": FP32_PEAK / 1e12,
                              "unit": "TFLOP/s", "frac": flops32 / (launch_ms * 1e-3) / FP32_PEAK,
                              "what": "FP32 LU factorisations of the mixed-precision Newton (2n^3/3 each)",
                              "peak_source": "measured FP32 FMA rate (bench_peaks.py)",
                              "time_weighted_frac": (flops / peak + flops32 / FP32_PEAK) / (launch_ms * 1e-3)}}
           if flops32 > 0 else {}),
        "cpu_baseline": cpu,
        "clocks": clocks,
        "gpu_launches": args.steps,
        "cells_failed": failed,
        "stats_mean": stat_means,
    }
    line["launch"] = [dict(zip(("team", "teams_per_block"), chemgb.cg_mech_get_launch(h)),
                           lu_panel=chemgb.cg_mech_get_lu_panel(h)) for h in handles]
    if tuned:
        line["autotune"] = tuned
    if graph is not None:
        line["cuda_graph"] = True
    print(json.dumps(line), flush=True)


def adjoint_flops(m, stats, s_stages: int) -> float:
    """Algorithmic FP64 flops of the backward sweep of cells with the given
    forward counters: the recomputed stages (every forward Newton iteration
    of the accepted steps, taken as the forward's iterations), and per stage
    one Jacobian and LU of G_p (one Newton iteration's work), the transposed
    solve 2 n^2, the stage coupling 2 s n, and the parameter gradient
    (2 per slot of every reaction, 6 per reaction)."""
    fpn = algorithmic_flops_per_newton(m.ns, m.nr, j_term_count(m), False)
    n = m.ns + 1
    per_stage = fpn + 2.0 * n * n + 2.0 * s_stages * n + 18.0 * m.nr
    steps = float(stats[0].astype(np.int64).sum())
    return float(stats[2].astype(np.int64).sum()) * fpn + steps * s_stages * per_stage


def run_adjoint(args):
    """--config 4 (and --config 5 --adjoint): forward with checkpoints plus
    the discrete adjoint."""
    import torch
    from paper_2510_10005_gb300 import autograd, chemgb, multirank

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    chemgb.load(build_if_missing=(ws == 1))
    cid = args.config
    (m, T, Y, p), = make_workload(cid, args.cells or ADJOINT_CELLS[cid], seed=rank)
    N = len(T)
    opts_d = opts_dict(cid, 0)
    opts = chemgb.make_opts(**opts_d)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    h = chemgb.cg_mech_create(m)
    f64 = dict(dtype=torch.float64, device=dev)
    T0 = torch.tensor(T, **f64)
    Y0 = torch.tensor(np.ascontiguousarray(Y.T), **f64)
    P = torch.tensor(p, **f64)
    Tb, Yb = torch.empty_like(T0), torch.empty_like(Y0)
    st = torch.empty(N, dtype=torch.int32, device=dev)
    stats = torch.empty((4, N), dtype=torch.int32, device=dev)

    # the target: the same cells integrated with ln A + N(0, 0.1^2) (seed 1)
    arr_t = m.arr.copy()
    arr_t[:, 0] += np.random.default_rng(1).normal(0.0, 0.1, m.nr)
    chemgb.cg_mech_set_arrhenius(h, arr_t)
    Tb.copy_(T0); Yb.copy_(Y0)
    chemgb.cg_integrate(h, opts, Tb, Yb, P, st, stats)
    T_target = Tb.clone()
    chemgb.cg_mech_set_arrhenius(h, m.arr)
    # checkpoint slots: the largest accepted-step count of the forward pass, with margin
    Tb.copy_(T0); Yb.copy_(Y0)
    chemgb.cg_integrate(h, opts, Tb, Yb, P, st, stats)
    torch.cuda.synchronize(dev)
    cap = int(stats[0].max().item()) * 2 + 8
    ckpt = torch.empty((N, cap, m.ns + 2), **f64)
    ckpt_n = torch.empty(N, dtype=torch.int32, device=dev)
    gY = torch.zeros((m.ns, N), **f64)
    dT0, dY0 = torch.empty(N, **f64), torch.empty((m.ns, N), **f64)
    dth = torch.empty((m.nr, 3), **f64)
    dcells = torch.empty((m.nr, 3, N), **f64)
    ast = torch.empty(N, dtype=torch.int32, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

    def step(split=False):
        Tb.copy_(T0)
        Yb.copy_(Y0)
        if split:
            ev[0].record(stream)
        chemgb.cg_integrate_ckpt(h, opts, Tb, Yb, P, ckpt, ckpt_n, st, stats, stream=stream.cuda_stream)
        if split:
            ev[1].record(stream)
        gT = 2.0 * (Tb - T_target)
        chemgb.cg_integrate_adjoint(h, opts, ckpt, ckpt_n, gT, gY, dT0, dY0, dth, dcells, ast,
                                    stream=stream.cuda_stream)
        if split:
            ev[2].record(stream)

    barrier = multirank.barrier

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    step(split=True)                      # per-kernel durations (forward, adjoint)
    torch.cuda.synchronize(dev)
    fwd_ms, adj_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
    barrier()
    ms = multirank.max_over_ranks(e0.elapsed_time(e1), dev)
    multirank.sum_over_ranks_(dth)        # the parameter gradient of the whole job
    value = multirank.job_throughput(N, ws, args.steps, ms * 1e-3)
    sh = stats.cpu().numpy()
    s_stages = 5
    a_flops = adjoint_flops(m, sh, s_stages)
    f_flops = float(sh[2].astype(np.int64).sum()) * algorithmic_flops_per_newton(m.ns, m.nr, j_term_count(m),
                                                                                  False)
    props = torch.cuda.get_device_properties(dev)
    clocks = clk.summary()
    peak = fp64_peak(props.multi_processor_count, clocks.get("sm_max_mhz") or 2070.0)
    adj_status = ast.cpu().numpy()
    loss = float(((Tb - T_target) ** 2).sum().item())

    # end to end through the torch.autograd entry point: pinned host inputs
    # in, gradients out, every step
    e2e = None
    if args.e2e_steps > 0:
        Th = torch.tensor(T, dtype=torch.float64).pin_memory()
        Yh = torch.tensor(np.ascontiguousarray(Y.T), dtype=torch.float64).pin_memory()
        ph = torch.tensor(p, dtype=torch.float64).pin_memory()
        theta = torch.tensor(m.arr, dtype=torch.float64, requires_grad=True)
        out = [torch.empty(N, dtype=torch.float64).pin_memory(),
               torch.empty((m.ns, N), dtype=torch.float64).pin_memory()]
        e2e_t = 0.0
        for k in range(args.e2e_steps + 1):
            barrier()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            Td = Th.to(dev, non_blocking=True).requires_grad_()
            Yd = Yh.to(dev, non_blocking=True).requires_grad_()
            Te, _, _ = autograd.integrate(h, opts, Td, Yd, ph.to(dev, non_blocking=True), theta, cap=cap)
            L = ((Te - T_target) ** 2).sum()
            theta.grad = None
            L.backward()
            out[0].copy_(Td.grad, non_blocking=True)
            out[1].copy_(Yd.grad, non_blocking=True)
            torch.cuda.synchronize(dev)
            if k > 0:
                e2e_t += time.perf_counter() - t0
        e2e_t = multirank.max_over_ranks(e2e_t, dev)
        e2e = {"value": multirank.job_throughput(N, ws, args.e2e_steps, e2e_t), "unit": "cells/s",
               "h2d_bytes_per_step": N * (m.ns + 2) * 8,
               "d2h_bytes_per_step": N * (m.ns + 1) * 8 + m.nr * 3 * 8, "steps": args.e2e_steps,
               "api": "paper_2510_10005_gb300.autograd.integrate + loss.backward()"}

    if rank != 0:
        return
    cpu = None
    if ws == 1 and not args.no_cpu:
        import oracle
        threads = os.cpu_count() or 1
        r = oracle.RefMech(m)

        def run(k, nthreads=threads):
            idx = sample_indices(N, k)
            t0 = time.perf_counter()
            r.adjoint_TY(T[idx], Y[idx], p[idx], np.ones(len(idx)), np.zeros((len(idx), m.ns)), oracle_opts(opts_d),
                         nthreads=nthreads)
            return time.perf_counter() - t0, len(idx)
        k, el, times = median_timing(run, args.cpu_sample or CPU_SAMPLE_ADJ[cid], args.cpu_repeats)
        cpu = {"value": k / el, "unit": "cells/s", "cores": threads, "kind": "oracle",
               "sample": f"{k} cells evenly spaced, forward + adjoint, median of {len(times)} timings "
                         f"({', '.join(f'{t:.2f}' for t in times)} s)"}
        one = ONE_CORE_SAMPLE_ADJ[cid] if args.cpu_1core_cells is None else args.cpu_1core_cells
        if one > 0:   # the same oracle on one host core
            k1, el1, _ = median_timing(lambda n: run(n, 1), one, 1)
            cpu["one_core"] = {"value": k1 / el1, "unit": "cells/s", "cores": 1,
                               "sample": f"{k1} cells evenly spaced, forward + adjoint ({el1:.1f} s)"}
    line = {
        "metric": METRIC_ADJ, "value": value, "unit": "cells/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": adjoint_workload(cid, N), "config": cid, "cells_per_gpu": N, "ckpt_cap": cap,
                   "ckpt_bytes": int(ckpt.numel() * 8),
                   "l2": "checkpoints larger than L2 (129 MB); no flush" if ckpt.numel() * 8 > 129e6
                   else "state smaller than L2"},
        "e2e": e2e,
        "roofline": {"bound": "alu", "achieved": a_flops / (adj_ms * 1e-3) / 1e12, "peak": peak / 1e12,
                     "unit": "TFLOP/s", "frac": a_flops / (adj_ms * 1e-3) / peak, "traffic": None,
                     "peak_source": "derived: 4 FP64 FLOP/clk/SM (measured DFMA rate) x SMs x max SM clock",
                     "kernel": "adjoint_kernel (+ sum_rows_kernel)", "kernel_ms": adj_ms,
                     "forward_kernel_ms": fwd_ms,
                     "forward_frac": f_flops / (fwd_ms * 1e-3) / peak},
        "cpu_baseline": cpu,
        "clocks": clocks,
        "gpu_launches": 3 * args.steps,
        "cells_failed": int((adj_status != 0).sum()),
        "stats_mean": {"steps": float(sh[0].mean()), "max_steps": int(sh[0].max()), "newton": float(sh[2].mean())},
        "loss": loss,
    }
    print(json.dumps(line), flush=True)


def run_reference_adjoint(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    cid = args.config
    (m, T, Y, p), = make_workload(cid, args.cells or ADJOINT_CELLS[cid])
    o = oracle_opts(opts_dict(cid, 0))
    r = oracle.RefMech(m)
    threads = os.cpu_count() or 1
    idx = sample_indices(len(T), args.cpu_sample or CPU_SAMPLE_ADJ[cid])
    k = len(idx)

    def sample():
        t0 = time.perf_counter()
        r.adjoint_TY(T[idx], Y[idx], p[idx], np.ones(k), np.zeros((k, m.ns)), o, nthreads=threads)
        return time.perf_counter() - t0

    for _ in range(args.warmup):
        sample()
    times = [sample() for _ in range(args.steps)]
    value = k / statistics.median(times)
    print(json.dumps({
        "impl": "reference", "metric": METRIC_ADJ, "value": value, "unit": "cells/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": adjoint_workload(cid, len(T)), "config": cid},
        "cpu_baseline": {"value": value, "unit": "cells/s", "cores": threads, "kind": "oracle",
                         "sample": f"the same {k} cells evenly spaced every step, forward + adjoint; "
                                   f"value = cells / median step time"},
        "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--config", type=int, default=2, choices=sorted(CONFIGS))
    ap.add_argument("--cells", type=int, default=0, help="cells per mechanism (default: the workload's)")
    ap.add_argument("--e2e-steps", type=int, default=3, help="timed host-array calls; e2e is their median")
    ap.add_argument("--cpu-sample", type=int, default=0,
                    help="cells of the oracle's timing sample, in the cpu_baseline leg and the reference arm "
                         "(0: the workload's, " + ", ".join(f"config {c}: {k}" for c, k in CPU_SAMPLE.items()) + ")")
    ap.add_argument("--cpu-repeats", type=int, default=5, help="timings of the cpu_baseline sample (median)")
    ap.add_argument("--cpu-1core-cells", type=int, default=None,
                    help="cells of the one-core oracle timing reported beside cpu_baseline (0: skip; default "
                         + ", ".join(f"config {c}: {k}" for c, k in ONE_CORE_SAMPLE.items()) + ")")
    ap.add_argument("--lu-panel", type=int, default=None,
                    help="panel width of the blocked LU (0: unblocked; default: the library's choice)")
    ap.add_argument("--smem-limit", type=int, default=0,
                    help="shared memory per cell in bytes before arrays go to global scratch (default: 227 KB)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--team", type=int, default=0, help="threads per cell (default: the library's choice)")
    ap.add_argument("--autotune", action="store_true",
                    help="pick the launch shape and shared-memory limit with cg_autotune (always on for config 3)")
    ap.add_argument("--tpb", type=int, default=1, help="cells per block with --team 32")
    ap.add_argument("--precision", type=int, default=None, help="0: FP64 Newton matrix, 1: FP32 LU")
    ap.add_argument("--method", choices=sorted(METHODS), default=None,
                    help="replace the workload's integrator (configs 1, 2, 3, 5)")
    ap.add_argument("--linear", choices=sorted(LINEAR), default=None, help="Newton systems: dense LU or GMRES")
    ap.add_argument("--prec", choices=sorted(PRECS), default=None, help="GMRES preconditioner (default gs)")
    ap.add_argument("--sri-plog", action="store_true",
                    help="give the workload's mechanisms SRI falloff and PLOG reactions")
    ap.add_argument("--thermo-degree", type=int, default=None,
                    help="refit the mechanisms' c_p polynomials to this degree (0-15; NASA-7 is 4)")
    ap.add_argument("--adjoint", action="store_true",
                    help="config 5: forward with checkpoints plus the discrete adjoint (config 4's loss), "
                         f"{ADJOINT_CELLS[5]:,} cells unless --cells")
    ap.add_argument("--surface", choices=["integrate", "split"], default="integrate",
                    help="split: the operator-split call of a compressible solver (rho, u, rho Y in; T, R out), "
                         "constant volume")
    args = ap.parse_args()
    if args.adjoint and args.config != 5:
        ap.error("--adjoint applies to --config 5 (config 4 is the adjoint workload)")
    if args.config == 4 or args.adjoint:
        (run_reference_adjoint if args.impl == "reference" else run_adjoint)(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
