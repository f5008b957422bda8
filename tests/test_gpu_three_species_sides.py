"""GPU parity on reactions with three species on one side (the third
stoichiometric slot of the reactants or of the products): the 9-species
set plus H + OH + H2 <=> H2O + H2 and HO2 + N2 <=> H + O2 + N2
(inputs.with_three_species_sides). The generated mechanisms never fill that
slot, and the library compiles its rate code without it when no reaction
uses it; this mechanism takes the other branch. Rates, the Jacobian,
fixed-step backward Euler and the discrete adjoint against the oracle, with
the tolerances of the other parity tests."""
import numpy as np
import pytest

import oracle
from paper_2510_10005_gb300 import chemgb, inputs
from parity import check_fixed

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def d(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


@pytest.fixture(scope="module")
def tri():
    chemgb.load(build_if_missing=True)
    m = inputs.with_three_species_sides(inputs.gen_mechanism("h2"))
    assert (m.rf_idx[:, 2] >= 0).any() and (m.rr_idx[:, 2] >= 0).any()
    return m, oracle.RefMech(m), chemgb.cg_mech_create(m)


@pytest.mark.parametrize("reactor", [chemgb.CG_CONV, chemgb.CG_CONP])
def test_rates_and_jacobian(tri, reactor):
    m, r, h = tri
    T, C, _ = inputs.random_states(m, 70, seed=31)   # two warps of 32 and a ragged tail
    S = torch.empty((h.n, len(T)), dtype=torch.float64, device=DEV)
    chemgb.cg_eval_rates(h, reactor, d(T), d(C.T), S)
    J = torch.empty((len(T), h.n, h.n), dtype=torch.float64, device=DEV)
    chemgb.cg_eval_jacobian(h, reactor, d(T), d(C.T), J)
    torch.cuda.synchronize()
    Sg, So = S.cpu().numpy().T, r.source(T, C, reactor)
    # the bounds of the rate parity test: 1e-12 of sum_j |nu_ij q_j| (plus the
    # dilution terms at constant pressure) and of the same sum weighted by
    # |W e| / (rho c) for omega_T
    from test_gpu_parity import nu_matrix
    nu = np.abs(nu_matrix(m))
    for c in range(len(T)):
        q = np.abs(r.rates(T[c], C[c])[2])
        scale = nu @ q
        if reactor == chemgb.CG_CONP:
            scale = scale + C[c] * (np.abs(So[c, 0]) / T[c] + scale.sum() / C[c].sum())
        th = r.thermo(T[c])
        e = th["u"] if reactor == chemgb.CG_CONV else th["h"]
        cv = th["cv"] if reactor == chemgb.CG_CONV else th["cp"]
        tscale = np.sum(np.abs(m.W * e) * (nu @ q)) / np.sum(m.W * C[c] * cv)
        assert abs(Sg[c, 0] - So[c, 0]) <= 1e-12 * tscale + 1e-12 * abs(So[c, 0])
        np.testing.assert_array_less(np.abs(Sg[c, 1:] - So[c, 1:]), 1e-12 * scale + 1e-300)
    Jg, Jo = J.cpu().numpy(), r.jacobian(T, C, reactor)
    rowmax = np.abs(Jo).max(axis=2, keepdims=True)
    assert np.all(np.abs(Jg - Jo) <= 1e-10 * np.abs(Jo) + 1e-12 * rowmax)


@pytest.mark.parametrize("team", [32, 64])
def test_backward_euler(tri, team):
    """One backward-Euler step of 1e-5 s (halvings where Newton fails) on
    64 cells of the 9-species reactor recipe, Newton to 1e-10 of the state,
    one warp per cell and two: relative 1e-10 on T and Y, statuses and step
    counts identical."""
    m, r, _ = tri
    h = chemgb.cg_mech_create(m)
    chemgb.cg_mech_set_launch(h, team, 1)
    T, Y, p = inputs.field_reactor(m, 64, (1000, 1500), (1, 1), (0.5, 2), "H2", seed=9)
    o = dict(method=oracle.BE, adaptive=0, dt=1e-5, rtol=1e-10, atol=1e-16, newton_tol=1.0, max_newton=20,
             max_halvings=10, reactor=oracle.CONP)
    To, Yo, so, sto = r.integrate(T, Y, p, o, nthreads=8)
    Tt, Yt = d(T), d(Y.T)
    st = torch.empty(len(T), dtype=torch.int32, device=DEV)
    stats = torch.empty((4, len(T)), dtype=torch.int32, device=DEV)
    chemgb.cg_integrate(h, chemgb.make_opts(**o), Tt, Yt, d(p), st, stats)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(st.cpu().numpy(), so)
    np.testing.assert_array_equal(stats.cpu().numpy().T[:, :2], sto[:, :2])
    ok = so == 0
    assert ok.mean() > 0.9
    check_fixed(f"three_species_sides_be_team{team}", Tt.cpu().numpy()[ok], Yt.cpu().numpy().T[ok], To[ok], Yo[ok],
                1e-10, 1e-22)


def test_adjoint(tri):
    """The discrete adjoint (three fixed backward-Euler substeps of a 1e-8 s
    interval) on cells of the random-state recipe, where every species is
    present and the added reactions run: against the oracle's adjoint
    element-wise at 1e-7 with the floor of the other adjoint tests, and the
    added reactions' parameter gradients (which run over the third slots)
    also against their own largest entry."""
    from test_gpu_adjoint import both_opts, close, compare
    m, r, h = tri
    o, og = both_opts(method=chemgb.CG_BE, adaptive=0, nsub=3, dt=1e-8, newton_tol=1e-3)
    T, C, _ = inputs.random_states(m, 37, seed=17)
    Y = C * m.W / (C * m.W).sum(axis=1, keepdims=True)
    p = inputs.R_UNIV * T * C.sum(axis=1)
    g = compare(m, r, h, o, og, T, Y, p)
    rng = np.random.default_rng(7)   # the loss gradients compare() drew
    a, b = rng.normal(size=len(T)), rng.normal(size=Y.shape)
    _, _, grad, st = r.adjoint_TY(T, Y, p, a, b, o, nthreads=8)
    assert np.all(st == 0)
    tail = grad[:, -2:, :]
    assert np.abs(tail).max() > 1e-6 * np.abs(grad).max()
    for k in range(3):
        close(g["cells"][:, -2:, k], tail[:, :, k])
