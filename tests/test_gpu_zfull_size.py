"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times, on sampled outputs the oracle computes cell by cell:

* the 53-species flame field, 1,048,576 cells, adaptive SDIRK-4 in FP64
  (the default bench line): 1024 cells evenly spaced through the field (so
  in proportion from its unburnt, front and burnt regions), T and every Y_k
  within the integrator's own element-wise weight (tests/parity.py),
  statuses identical;
* the heavy-tailed batch of 53 + 9 species, 2 x 1,048,576 cells, one
  persistent launch with the FP32 Newton matrix: 1024 cells per mechanism,
  the same element-wise bound against the FP64 oracle;
* the adjoint workload, 65,536 cells over 1e-4 s: 64 sampled cells,
  dL/dT0, dL/dY0 and the per-cell dL/dtheta element-wise within 1e-6 plus
  1e-9 of the largest entry of each kind, on the cells whose accepted step
  count equals the oracle's.

Slow: a 1,048,576-cell launch takes about 45 s, the batch about 30 s plus
the autotuning, the adjoint about 15 s. Collected after the other GPU
tests."""
import os

import numpy as np
import pytest

import bench
import oracle
from paper_2510_10005_gb300 import chemgb
from parity import check_adaptive, check_elementwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
THREADS = min(16, os.cpu_count() or 1)
F64 = torch.float64


def _dev(a, dtype=F64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def test_full_size_flame_field():
    chemgb.load(build_if_missing=True)
    (m, T, Y, p), = bench.make_workload(2, 1 << 20)
    o = bench.opts_dict(2, 0)
    h = chemgb.cg_mech_create(m)
    Tt, Yt, pt = _dev(T), _dev(Y.T), _dev(p)
    st = torch.empty(len(T), dtype=torch.int32, device=DEV)
    chemgb.cg_integrate(h, chemgb.make_opts(**o), Tt, Yt, pt, st)
    torch.cuda.synchronize()
    idx = np.linspace(0, len(T) - 1, 1024).astype(np.int64)
    To, Yo, so, _ = oracle.RefMech(m).integrate(T[idx], Y[idx], p[idx], bench.oracle_opts(o), nthreads=THREADS)
    sel = torch.as_tensor(idx, device=DEV)
    Tg = Tt.index_select(0, sel).cpu().numpy()
    Yg = Yt.index_select(1, sel).cpu().numpy().T
    assert np.array_equal(st.index_select(0, sel).cpu().numpy(), so) and np.all(so == 0)
    assert int((st != 0).sum()) == 0
    check_adaptive("full_size_flame_field_1M", m, Tg, Yg, To, Yo, p[idx], o["reactor"], o["rtol"], o["atol"])


def test_full_size_mixed_batch_fp32():
    chemgb.load(build_if_missing=True)
    parts = bench.make_workload(3, 1 << 20)
    o = bench.opts_dict(3, 1)
    og = chemgb.make_opts(**o)
    handles = [chemgb.cg_mech_create(m) for m, *_ in parts]
    Ts, Ys, ps, sts = [], [], [], []
    for m, T, Y, p in parts:
        Ts.append(_dev(T))
        Ys.append(_dev(Y.T))
        ps.append(_dev(p))
        sts.append(torch.empty(len(T), dtype=torch.int32, device=DEV))
    # the benchmark's launch shape: autotuned on 16,384 cells of the dominant
    # mechanism; the 9-species one keeps one warp per cell (split in a wider launch)
    sel = torch.linspace(0, len(Ts[0]) - 1, 16384, device=DEV).long()
    chemgb.cg_autotune(handles[0], og, Ts[0][sel].contiguous(), Ys[0][:, sel].contiguous(), ps[0][sel].contiguous())
    assert chemgb.cg_mech_get_launch(handles[1])[0] == 32
    chemgb.cg_integrate_batch(handles, og, Ts, Ys, ps, sts)
    torch.cuda.synchronize()
    for (m, T, Y, p), Tt, Yt, st in zip(parts, Ts, Ys, sts):
        idx = np.linspace(0, len(T) - 1, 1024).astype(np.int64)
        To, Yo, so, _ = oracle.RefMech(m).integrate(T[idx], Y[idx], p[idx], bench.oracle_opts(o), nthreads=THREADS)
        sel = torch.as_tensor(idx, device=DEV)
        assert np.array_equal(st.index_select(0, sel).cpu().numpy(), so)
        check_adaptive(f"full_size_fp32_batch_{m.ns}sp", m, Tt.index_select(0, sel).cpu().numpy(),
                       Yt.index_select(1, sel).cpu().numpy().T, To, Yo, p[idx], o["reactor"], o["rtol"], o["atol"])


def test_full_size_adjoint():
    chemgb.load(build_if_missing=True)
    (m, T, Y, p), = bench.make_workload(4, 1 << 16)
    o = bench.opts_dict(4, 0)
    og = chemgb.make_opts(**o)
    h = chemgb.cg_mech_create(m)
    N = len(T)
    Tt, Yt, pt = _dev(T), _dev(Y.T), _dev(p)
    stats = torch.empty((4, N), dtype=torch.int32, device=DEV)
    chemgb.cg_integrate(h, og, Tt.clone(), Yt.clone(), pt, None, stats)
    torch.cuda.synchronize()
    cap = int(stats[0].max().item()) * 2 + 8
    ckpt = torch.empty((N, cap, m.ns + 2), dtype=F64, device=DEV)
    ckpt_n = torch.empty(N, dtype=torch.int32, device=DEV)
    st = torch.empty(N, dtype=torch.int32, device=DEV)
    chemgb.cg_integrate_ckpt(h, og, Tt, Yt, pt, ckpt, ckpt_n, st)
    rng = np.random.default_rng(4)
    gT = rng.normal(size=N)
    dT0, dY0 = torch.empty(N, dtype=F64, device=DEV), torch.empty((m.ns, N), dtype=F64, device=DEV)
    dth = torch.empty((m.nr, 3), dtype=F64, device=DEV)
    dcell = torch.empty((m.nr, 3, N), dtype=F64, device=DEV)
    ast = torch.empty(N, dtype=torch.int32, device=DEV)
    chemgb.cg_integrate_adjoint(h, og, ckpt, ckpt_n, _dev(gT), torch.zeros((m.ns, N), dtype=F64, device=DEV),
                                dT0, dY0, dth, dcell, ast)
    torch.cuda.synchronize()
    assert int((st != 0).sum()) == 0 and int((ast != 0).sum()) == 0
    idx = np.linspace(0, N - 1, 64).astype(np.int64)
    r = oracle.RefMech(m)
    oo = bench.oracle_opts(o)
    oT, oY, og_, ost = r.adjoint_TY(T[idx], Y[idx], p[idx], gT[idx], np.zeros((len(idx), m.ns)), oo,
                                    nthreads=THREADS)
    assert np.all(ost == 0)
    # both sides differentiate their own accepted steps: compare the cells
    # whose step counts agree (an accept/reject flip at the threshold gives
    # another, equally valid, step sequence)
    C0 = r.concentrations(T[idx], Y[idx], p[idx], o["reactor"])
    _, _, _, hn = r.integrate_hist(np.concatenate([T[idx, None], C0], axis=1), oo, cap=cap, nthreads=THREADS)
    sel = torch.as_tensor(idx, device=DEV)
    same = ckpt_n.index_select(0, sel).cpu().numpy() == hn
    assert same.mean() >= 0.9, (same.mean(), ckpt_n.index_select(0, sel).cpu().numpy(), hn)
    check_elementwise("full_size_adjoint_dT0", dT0.index_select(0, sel).cpu().numpy()[same], oT[same], 1e-6, 1e-9)
    check_elementwise("full_size_adjoint_dY0", dY0.index_select(1, sel).cpu().numpy().T[same], oY[same], 1e-6, 1e-9)
    gc = np.moveaxis(dcell.index_select(2, sel).cpu().numpy(), 2, 0)
    for k, name in enumerate(("lnA", "b", "Ea")):
        check_elementwise(f"full_size_adjoint_dtheta_{name}", gc[same][:, :, k], og_[same][:, :, k], 1e-6, 1e-9)
