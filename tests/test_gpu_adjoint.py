"""GPU parity of the discrete adjoint (cg_integrate_ckpt + cg_integrate_adjoint)
against the oracle's adjoint in flow variables (RefMech.adjoint_TY, itself
pinned against central differences and the forward sensitivity).

Both sides differentiate the same frozen step sequence; a cell whose GPU
step count differs from the oracle's (an accept/reject decision flipped by
rounding) is left out of the element-wise comparison, and at least 90% of
the cells must match. Tolerance: the two sides agree on the stage states to
rounding (Newton iterated with the same matrices), so gradients agree to
1e-7 relative, with an absolute floor of 1e-9 of the largest entry of the
same kind (tiny entries are sums of cancelling terms).
"""
import numpy as np
import pytest

import oracle
from paper_2510_10005_gb300 import chemgb, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
F64 = torch.float64


@pytest.fixture(scope="module")
def handles(mechs):
    chemgb.load(build_if_missing=True)
    return {k: chemgb.cg_mech_create(m) for k, m in mechs.items()}


def d(a, dtype=F64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def both_opts(**kw):
    """The same options for the oracle (dict) and the library (struct)."""
    o = dict(method=chemgb.CG_SDIRK4, reactor=chemgb.CG_CONP, adaptive=1, nsub=1, max_newton=20,
             max_steps=100000, max_halvings=10, err_filter=1, dt=1e-6, rtol=1e-8, atol=1e-14,
             newton_tol=1e-6, h0=0.0, hmin=1e-20, neg_tol=1e-6)
    o.update(kw)
    g = chemgb.make_opts(**{k: v for k, v in o.items() if k != "precision"})
    g.precision = kw.get("precision", chemgb.CG_FP64)
    o.pop("precision", None)
    return o, g


def gpu_adjoint(h, og, T, Y, p, dT_end, dY_end, cap=1024):
    N = len(T)
    Tt, Yt, pt = d(T), d(Y.T), d(p)
    ckpt = torch.empty((N, cap, h.n + 1), dtype=F64, device=DEV)
    ckpt_n = torch.empty(N, dtype=torch.int32, device=DEV)
    st = torch.empty(N, dtype=torch.int32, device=DEV)
    chemgb.cg_integrate_ckpt(h, og, Tt, Yt, pt, ckpt, ckpt_n, st)
    dT0 = torch.empty(N, dtype=F64, device=DEV)
    dY0 = torch.empty((h.ns, N), dtype=F64, device=DEV)
    dth = torch.empty((h.nr, 3), dtype=F64, device=DEV)
    dcell = torch.empty((h.nr, 3, N), dtype=F64, device=DEV)
    ast = torch.empty(N, dtype=torch.int32, device=DEV)
    chemgb.cg_integrate_adjoint(h, og, ckpt, ckpt_n, d(dT_end), d(np.asarray(dY_end).T), dT0, dY0, dth, dcell,
                                ast)
    torch.cuda.synchronize()
    return dict(T=Tt.cpu().numpy(), Y=Yt.cpu().numpy().T, status=st.cpu().numpy(),
                steps=ckpt_n.cpu().numpy(), dT0=dT0.cpu().numpy(), dY0=dY0.cpu().numpy().T,
                dtheta=dth.cpu().numpy(), cells=np.moveaxis(dcell.cpu().numpy(), 2, 0), astatus=ast.cpu().numpy())


def close(a, b, rtol=1e-7, floor=1e-9):
    scale = max(np.abs(b).max(), 1e-300)
    np.testing.assert_allclose(a, b, rtol=rtol, atol=floor * scale)


def compare(m, r, h, o, og, T, Y, p, seed=7, rtol=1e-7):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=len(T))
    b = rng.normal(size=Y.shape)
    g = gpu_adjoint(h, og, T, Y, p, a, b)
    assert np.all(g["status"] == 0), g["status"]
    assert np.all(g["astatus"] == 0), g["astatus"]
    dT0, dY0, grad, st = r.adjoint_TY(T, Y, p, a, b, o, nthreads=8)
    assert np.all(st == 0)
    C0 = r.concentrations(T, Y, p, o["reactor"])
    _, _, _, hn = r.integrate_hist(np.concatenate([T[:, None], C0], axis=1), o, nthreads=8)
    same = g["steps"] == hn
    assert same.mean() >= 0.9, (g["steps"], hn)
    close(g["dT0"][same], dT0[same], rtol)
    close(g["dY0"][same], dY0[same], rtol)
    for k in range(3):
        close(g["cells"][same][:, :, k], grad[same][:, :, k], rtol)
    # the fixed-order cell sum equals the sum of the per-cell gradients
    np.testing.assert_allclose(g["dtheta"], g["cells"].sum(axis=0), rtol=1e-12,
                               atol=1e-14 * np.abs(g["cells"]).sum(axis=0).max())
    if same.all():
        for k in range(3):
            close(g["dtheta"][:, k], grad.sum(axis=0)[:, k], rtol)
    return g


CASES = {
    "h2-be-conp": ("h2", dict(method=chemgb.CG_BE, adaptive=0, nsub=3, dt=1e-6, newton_tol=1e-3)),
    "h2-sdirk2-conv": ("h2", dict(method=chemgb.CG_SDIRK2, adaptive=0, nsub=4, dt=2e-6,
                                  reactor=chemgb.CG_CONV)),
    "h2-sdirk4-adaptive": ("h2", dict(dt=5e-6, rtol=1e-7, atol=1e-13)),   # 96-681 steps, heat release
    "h2-be-literal": ("h2", dict(method=chemgb.CG_BE, adaptive=0, nsub=2, dt=1e-6, newton_tol=1e-3,
                                 reactor=chemgb.CG_CONP_LITERAL)),
    "ch4-sdirk4-adaptive": ("ch4", dict(dt=2e-6, rtol=1e-7, atol=1e-13)),
}


@pytest.mark.parametrize("case", list(CASES))
def test_adjoint_parity(mechs, ref, handles, case):
    kind, kw = CASES[case]
    m, r, h = mechs[kind], ref[kind], handles[kind]
    o, og = both_opts(**kw)
    fuel = "H2" if kind == "h2" else "CH4"
    T, Y, p = inputs.field_reactor(m, 37, (1150, 1400), (1, 3), (0.5, 2.0), fuel, seed=11)   # a ragged warp count
    if o["reactor"] == chemgb.CG_CONV:
        p = p / (inputs.R_UNIV * T * (Y / m.W).sum(axis=1))
    compare(m, r, h, o, og, T, Y, p)


def test_adjoint_parity_flame_cells(mechs, ref, handles):
    """Cells of the 1-D flame field (unburnt, front and burnt), 53 species."""
    m, r, h = mechs["ch4"], ref["ch4"], handles["ch4"]
    T, Y, p = inputs.field_flames(m, 4096, seed=3)
    idx = np.linspace(0, 4095, 40).astype(int)
    o, og = both_opts(dt=1e-6, rtol=1e-6, atol=1e-12, newton_tol=0.03, max_newton=7)
    compare(m, r, h, o, og, T[idx], Y[idx], p[idx], rtol=1e-6)


def test_adjoint_mixed_precision_forward(mechs, ref, handles):
    """FP32 Newton matrices in the forward pass (and in the recomputed
    stages), FP64 transposed solves: the adjoint of the converged stage
    equations, so it agrees with the FP64 oracle to the Newton tolerance."""
    m, r, h = mechs["ch4"], ref["ch4"], handles["ch4"]
    T, Y, p = inputs.field_reactor(m, 24, (1150, 1350), (1, 1), (0.7, 1.3), "CH4", seed=12)
    o, og = both_opts(dt=1e-6, newton_tol=1e-4, precision=chemgb.CG_FP32LU)
    compare(m, r, h, o, og, T, Y, p, rtol=1e-5)


@pytest.mark.parametrize("cap", [2, 5, 40])
def test_adjoint_recomputes_steps_that_did_not_fit(mechs, handles, cap):
    """Adaptive SDIRK-4 cells of 53 species over 5e-6 s (1 to about 50 steps
    each; the front cells the most), their records cut to `cap` slots: the
    adjoint replays the forward integration from the initial state in
    segments of 32 steps and sweeps each backwards; gradients and statuses
    are identical to the last bit to those from a record that holds every
    step."""
    m, h = mechs["ch4"], handles["ch4"]
    T, Y, p = inputs.field_flames(m, 4096, seed=3)
    idx = np.concatenate([np.linspace(0, 4095, 12).astype(int), np.arange(2500, 2900, 100)])   # + front cells
    T, Y, p = T[idx], Y[idx], p[idx]
    _, og = both_opts(dt=5e-6, rtol=1e-6, atol=1e-12, newton_tol=0.03, max_newton=7)
    rng = np.random.default_rng(3)
    a, b = rng.normal(size=len(T)), rng.normal(size=Y.shape)
    full = gpu_adjoint(h, og, T, Y, p, a, b, cap=2048)
    S = full["steps"]
    assert np.all(S >= 0) and S.max() > 40          # some cells need more than one segment
    cut = gpu_adjoint(h, og, T, Y, p, a, b, cap=cap)
    np.testing.assert_array_equal(cut["steps"], np.where(S < cap, S, -(S + 2)))
    assert np.all(cut["astatus"] == 0)
    for k in ("dT0", "dY0", "dtheta", "cells"):
        assert np.array_equal(cut[k], full[k]), k


def test_adjoint_deterministic_and_shape_independent(mechs, handles):
    m, h = mechs["ch4"], handles["ch4"]
    T, Y, p = inputs.field_reactor(m, 300, (1150, 1400), (1, 3), (0.5, 2.0), "CH4", seed=13)
    _, og = both_opts(dt=1e-6, rtol=1e-6, atol=1e-12)
    rng = np.random.default_rng(1)
    a, b = rng.normal(size=len(T)), rng.normal(size=Y.shape)
    g1 = gpu_adjoint(h, og, T, Y, p, a, b)
    g2 = gpu_adjoint(h, og, T, Y, p, a, b)
    for k in ("dT0", "dY0", "dtheta", "cells"):
        assert np.array_equal(g1[k], g2[k]), k        # bit for bit, whatever the work-stealing order
    team0, tpb0 = chemgb.cg_mech_get_launch(h)
    try:
        chemgb.cg_mech_set_launch(h, 32, 2)
        g3 = gpu_adjoint(h, og, T, Y, p, a, b)
    finally:
        chemgb.cg_mech_set_launch(h, team0, tpb0)
    assert np.array_equal(g3["steps"], g1["steps"])
    for k in ("dT0", "dY0", "dtheta"):
        close(g3[k], g1[k], rtol=1e-9, floor=1e-12)


def test_adjoint_finite_differences_on_gpu(mechs, handles):
    """The GPU's own forward pass, differenced: fixed SDIRK-4 steps (no step
    decisions to freeze), Newton to a tight tolerance; central differences
    in ln A, b, Ea of the reactions with the largest gradients (through
    cg_mech_set_arrhenius) and in T0."""
    m, h = mechs["ch4"], handles["ch4"]
    T, Y, p = inputs.field_reactor(m, 64, (1250, 1400), (1, 1), (0.5, 2.0), "CH4", seed=14)
    _, og = both_opts(adaptive=0, nsub=3, dt=3e-7, newton_tol=1e-4, max_newton=40, max_halvings=0)
    ones = np.ones(len(T))
    g = gpu_adjoint(h, og, T, Y, p, ones, np.zeros_like(Y))   # L = sum_c T_end
    arr0 = h.arr.copy()

    def loss(arr=None, T_=T):
        if arr is not None:
            chemgb.cg_mech_set_arrhenius(h, arr)
        Tt, Yt = d(T_), d(Y.T)
        st = torch.empty(len(T), dtype=torch.int32, device=DEV)
        chemgb.cg_integrate(h, og, Tt, Yt, d(p), st)
        assert int(st.abs().sum()) == 0
        return Tt.cpu().numpy()

    try:
        steps = {0: 1e-3, 1: 1e-3, 2: 1e4}   # ln k moves by ~1e-3: above the rounding of sum T_end
        for k, dv in steps.items():
            gk = np.abs(g["dtheta"][:, k])
            top = [j for j in np.argsort(-gk)[:4] if gk[j] >= 1e-2 * gk.max()]   # above the rounding of L
            assert top
            for j in top:
                ap, am = arr0.copy(), arr0.copy()
                ap[j, k] += dv
                am[j, k] -= dv
                fd = (loss(ap).sum() - loss(am).sum()) / (2 * dv)
                assert fd == pytest.approx(g["dtheta"][j, k], rel=2e-5)
    finally:
        chemgb.cg_mech_set_arrhenius(h, arr0)
    fd = (loss(None, T + 1e-3) - loss(None, T - 1e-3)) / 2e-3
    np.testing.assert_allclose(fd, g["dT0"], rtol=1e-5)


def test_adjoint_edge_cases(mechs, handles):
    m, h = mechs["h2"], handles["h2"]
    T, Y, p = inputs.field_reactor(m, 40, (1150, 1400), (1, 1), (0.5, 2.0), "H2", seed=15)
    T[5] = np.nan                                   # non-finite input: no record
    _, og = both_opts(method=chemgb.CG_BE, adaptive=0, nsub=3, dt=1e-6)
    rng = np.random.default_rng(2)
    a, b = rng.normal(size=len(T)), rng.normal(size=Y.shape)
    g = gpu_adjoint(h, og, T, Y, p, a, b)
    assert g["status"][5] == chemgb.CG_CELL_NONFINITE and g["steps"][5] == -1
    assert g["astatus"][5] == chemgb.CG_CELL_NO_RECORD
    assert g["dT0"][5] == 0.0 and not g["dY0"][5].any() and not g["cells"][5].any()
    ok = np.arange(len(T)) != 5
    assert np.all(g["astatus"][ok] == 0) and np.all(g["steps"][ok] == 3)
    # 3 steps need 4 records; with fewer the adjoint recomputes the steps
    # from the initial state (two-level checkpointing): the same bits
    g3 = gpu_adjoint(h, og, T, Y, p, a, b, cap=4)
    assert np.array_equal(g3["dtheta"], g["dtheta"])
    for cap in (3, 2):
        g2 = gpu_adjoint(h, og, T, Y, p, a, b, cap=cap)
        assert np.all(g2["steps"][ok] == -(3 + 2)) and g2["steps"][5] == -1
        assert np.all(g2["astatus"][ok] == 0) and g2["astatus"][5] == chemgb.CG_CELL_NO_RECORD
        for k in ("dT0", "dY0", "dtheta", "cells"):
            assert np.array_equal(g2[k], g[k]), (cap, k)
    # no cells: the parameter gradient is zero
    dth = torch.full((h.nr, 3), 7.0, dtype=F64, device=DEV)
    e = torch.empty(0, dtype=F64, device=DEV)
    chemgb.cg_integrate_adjoint(h, og, torch.empty((0, 4, h.n + 1), dtype=F64, device=DEV),
                                torch.empty(0, dtype=torch.int32, device=DEV), e,
                                torch.empty((h.ns, 0), dtype=F64, device=DEV), e.clone(),
                                torch.empty((h.ns, 0), dtype=F64, device=DEV), dth)
    torch.cuda.synchronize()
    assert not dth.cpu().numpy().any()
    with pytest.raises(chemgb.ChemgbError):
        gpu_adjoint(h, og, T, Y, p, a, b, cap=1)


def test_autograd_function(mechs, ref, handles):
    """L = sum (T_end - T_target)^2 + w . Y_end through torch.autograd, the
    target from a perturbed ln A (the loss of a parameter fit)."""
    from paper_2510_10005_gb300 import autograd
    m, r, h = mechs["h2"], ref["h2"], handles["h2"]
    T, Y, p = inputs.field_reactor(m, 50, (1100, 1400), (1, 1), (0.5, 2.0), "H2", seed=1)
    o, og = both_opts(dt=5e-6, rtol=1e-7, atol=1e-13)
    mt = m.copy()
    mt.arr[:, 0] += np.random.default_rng(1).normal(0.0, 0.1, m.nr)
    T_target, _, st, _ = oracle.RefMech(mt).integrate(T, Y, p, o)
    assert np.all(st == 0)
    w = np.random.default_rng(3).normal(size=m.ns)
    T0 = d(T).requires_grad_()
    Y0 = d(Y.T).requires_grad_()
    theta = torch.tensor(m.arr, dtype=F64, requires_grad=True)
    Tend, Yend, status = autograd.integrate(h, og, T0, Y0, d(p), theta)
    L = ((Tend - d(T_target)) ** 2).sum() + (d(w)[:, None] * Yend).sum()
    L.backward()
    assert int(status.abs().sum()) == 0
    Tend_np = Tend.detach().cpu().numpy()
    dT0, dY0, grad, st = r.adjoint_TY(T, Y, p, 2 * (Tend_np - T_target), np.tile(w, (len(T), 1)), o,
                                      nthreads=8)
    assert np.all(st == 0)
    close(T0.grad.cpu().numpy(), dT0, 1e-6)
    close(Y0.grad.cpu().numpy().T, dY0, 1e-6)
    for k in range(3):
        close(theta.grad.numpy()[:, k], grad.sum(axis=0)[:, k], 1e-6)


def test_adjoint_parity_sri_plog():
    """The adjoint with SRI falloff and PLOG reactions present (their rate
    derivatives enter through the Jacobian and, for SRI, the parameter
    factor Pr/(1+Pr) - dlog10F/dlog10Pr; PLOG rates take no (ln A, b, Ea))."""
    m = inputs.with_sri_plog(inputs.gen_mechanism("ch4"), n_sri=8, n_plog=20, seed=3)
    r, h = oracle.RefMech(m), chemgb.cg_mech_create(m)
    T, Y, p = inputs.field_reactor(m, 29, (1250, 1450), (0.5, 40), (0.5, 2.0), "CH4", seed=17)
    o, og = both_opts(dt=2e-6, rtol=1e-7, atol=1e-13)
    g = compare(m, r, h, o, og, T, Y, p)
    plog = np.flatnonzero(m.rtype == inputs.RXN_PLOG)
    assert not g["dtheta"][plog].any()
