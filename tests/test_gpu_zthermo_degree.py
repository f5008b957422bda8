"""GPU parity of the thermodynamics of other polynomial degrees (Section 2.1,
eq. specific_heat_polynomial; Appendix C.1 refits to n_p = 7 and 15)
against the oracle: the source term, the Jacobian, temperature recovery,
integration and the split step, for mechanisms refitted by
`inputs.with_thermo_degree`.

The library evaluates every polynomial by Horner's rule and the oracle by
a sum of powers. At n_p = 15 the fitted coefficients make terms some 5e3
times the value, so the two orders differ by up to ~2e-13 in c_p and ~6e-13
in g/RT (measured over 300-3000 K on the 53-species refit). The tolerances
below are 1e-10 relative (1e-8 for J). A table row in the wrong place
misses by O(1)."""
import numpy as np
import pytest

import oracle
from paper_2510_10005_gb300 import chemgb, inputs
from parity import check_adaptive, check_fixed

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def d(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


@pytest.fixture(scope="module")
def refits(mechs):
    chemgb.load(build_if_missing=True)
    out = {}
    for n_p in (2, 4, 7, 15):
        m = inputs.with_thermo_degree(mechs["ch4"], n_p)
        out[n_p] = (m, oracle.RefMech(m), chemgb.cg_mech_create(m))
    return out


def gpu_rates(h, T, C, reactor):
    S = torch.empty((h.n, len(T)), dtype=torch.float64, device=DEV)
    chemgb.cg_eval_rates(h, reactor, d(T), d(C.T), S)
    torch.cuda.synchronize()
    return S.cpu().numpy().T


@pytest.mark.parametrize("n_p", [2, 7, 15])
@pytest.mark.parametrize("reactor", [chemgb.CG_CONV, chemgb.CG_CONP])
def test_rates_any_degree(refits, n_p, reactor):
    m, r, h = refits[n_p]
    T, C, _ = inputs.random_states(m, 96, seed=31)
    Sg = gpu_rates(h, T, C, reactor)
    So = r.source(T, C, reactor)
    scale = np.abs(So).max(axis=0, keepdims=True)
    assert np.all(np.abs(Sg - So) <= 1e-10 * (np.abs(So) + scale))


@pytest.mark.parametrize("n_p", [7, 15])
def test_jacobian_any_degree(refits, n_p):
    m, r, h = refits[n_p]
    T, C, _ = inputs.random_states(m, 33, seed=32)
    for reactor in (chemgb.CG_CONV, chemgb.CG_CONP):
        J = torch.empty((33, h.n, h.n), dtype=torch.float64, device=DEV)
        chemgb.cg_eval_jacobian(h, reactor, d(T), d(C.T), J)
        torch.cuda.synchronize()
        Jg, Jo = J.cpu().numpy(), r.jacobian(T, C, reactor)
        rowmax = np.abs(Jo).max(axis=2, keepdims=True)
        assert np.all(np.abs(Jg - Jo) <= 1e-8 * np.abs(Jo) + 1e-10 * rowmax)


def test_degree_four_table_equals_nasa7(mechs, refits):
    """Setting the NASA-7 rows again through the degree entry leaves every
    result bit for bit as created."""
    m4, _, h4 = refits[4]
    h = chemgb.cg_mech_create(mechs["ch4"])
    T, C, _ = inputs.random_states(m4, 64, seed=33)
    np.testing.assert_array_equal(gpu_rates(h4, T, C, chemgb.CG_CONP), gpu_rates(h, T, C, chemgb.CG_CONP))
    chemgb.cg_mech_set_thermo(h, mechs["ch4"].nasa7)
    np.testing.assert_array_equal(gpu_rates(h4, T, C, chemgb.CG_CONV), gpu_rates(h, T, C, chemgb.CG_CONV))


@pytest.mark.parametrize("n_p", [7, 15])
def test_temperature_recovery_any_degree(refits, n_p):
    m, r, h = refits[n_p]
    T, Y, p = inputs.field_flames(m, 200, seed=5)
    for reactor, key in ((oracle.CONP, "h"), (oracle.CONV, "u")):
        e = np.array([Y[c] @ r.thermo(T[c])[key] for c in range(200)])
        T0 = T + 250.0
        To = r.temperature(e, Y, T0, iters=5, reactor=reactor)
        Tg = d(T0)
        chemgb.cg_temperature_from_energy(h, reactor, d(e), d(Y.T), Tg, 5)
        torch.cuda.synchronize()
        np.testing.assert_allclose(Tg.cpu().numpy(), To, rtol=1e-10)


def run(h, o, T, Y, p):
    N = len(T)
    Tt, Yt = d(T), d(Y.T)
    st = torch.empty(N, dtype=torch.int32, device=DEV)
    chemgb.cg_integrate(h, chemgb.make_opts(**o), Tt, Yt, d(p), st)
    torch.cuda.synchronize()
    return Tt.cpu().numpy(), Yt.cpu().numpy().T, st.cpu().numpy()


def test_backward_euler_any_degree(refits):
    """Fixed steps with Newton to 1e-10 of the state: the same root."""
    m, r, h = refits[15]
    T, Y, p = inputs.field_reactor(m, 70, (1100, 1500), (1, 1), (0.5, 2), "CH4", seed=9)
    o = dict(method=oracle.BE, adaptive=0, dt=1e-6, rtol=1e-10, atol=1e-16, newton_tol=1.0, max_newton=20,
             max_halvings=10, reactor=oracle.CONP)
    To, Yo, so, _ = r.integrate(T, Y, p, o, nthreads=8)
    Tg, Yg, sg = run(h, o, T, Y, p)
    np.testing.assert_array_equal(sg, so)
    check_fixed("be_thermo_degree_15", Tg, Yg, To, Yo, 1e-9, 1e-20)


def test_adaptive_flame_any_degree(refits):
    m, r, h = refits[7]
    T, Y, p = inputs.field_flames(m, 4096, seed=0)
    idx = np.arange(0, 4096, 64)
    o = dict(method=oracle.SDIRK4, adaptive=1, dt=1e-6, rtol=1e-6, atol=1e-12, newton_tol=0.03, max_newton=7,
             reactor=oracle.CONP)
    To, Yo, so, _ = r.integrate(T[idx], Y[idx], p[idx], o, nthreads=8)
    Tg, Yg, sg = run(h, o, T[idx], Y[idx], p[idx])
    np.testing.assert_array_equal(sg, so)
    check_adaptive("adaptive_flame_thermo_degree_7", m, Tg, Yg, To, Yo, p[idx], o["reactor"], o["rtol"], o["atol"])


def test_split_step_any_degree(refits):
    """The split step's temperature recovery and constant-volume step with
    n_p = 7 thermodynamics."""
    m, r, h = refits[7]
    T, Y, p = inputs.field_reactor(m, 64, (1100, 1400), (1, 1), (0.5, 2), "CH4", seed=4)
    rho = p / (inputs.R_UNIV * T * (Y / m.W).sum(1))
    u = np.array([Y[c] @ r.thermo(T[c])["u"] for c in range(64)])
    rhoY = rho[:, None] * Y
    o = dict(method=oracle.BE, adaptive=0, dt=1e-6, rtol=1e-10, atol=1e-16, newton_tol=1.0, max_newton=20,
             max_halvings=10, reactor=oracle.CONV)
    To, Ro, so, _ = r.react_split(rho, u, rhoY, T + 30.0, o, nthreads=8)
    Tt, R = d(T + 30.0), torch.empty((m.ns, 64), dtype=torch.float64, device=DEV)
    st = torch.empty(64, dtype=torch.int32, device=DEV)
    chemgb.cg_react_split(h, chemgb.make_opts(**o), d(rho), d(u), d(rhoY.T), Tt, R, 5, st)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(st.cpu().numpy(), so)
    np.testing.assert_allclose(Tt.cpu().numpy(), To, rtol=1e-10)
    Rg = R.cpu().numpy().T
    assert np.all(np.abs(Rg - Ro) <= 1e-9 * (np.abs(Ro) + rhoY / o["dt"]))
