"""Pins of the oracle's thermodynamics for a c_p polynomial of any degree n_p
(Section 2.1, eq. specific_heat_polynomial and Table 1; Appendix C.1 refits
to n_p = 7 and 15).

The generator fits each species' drawn c_p curve with a polynomial of degree
n_p and anchors h and s at 298.15 K (eq. enthalpy-adjustment). These tests
pin the oracle's Table 1 sets for every degree to things other than
themselves: the drawn anchor values, the textbook constant-c_p gas (n_p = 0),
derivative identities by Richardson-extrapolated finite differences, the
complex-step Jacobian, the conservation laws of the two reactors, and the
fall of the fit error with the degree that Appendix C.1 reports."""
import numpy as np
import pytest

import oracle
from paper_2510_10005_gb300 import inputs

R = inputs.R_UNIV
T0 = inputs.T_ANCHOR


@pytest.fixture(scope="module")
def ch4():
    return inputs.gen_mechanism("ch4")


def refm(m, n_p):
    mm = inputs.with_thermo_degree(m, n_p)
    return mm, oracle.RefMech(mm)


def test_degree_four_refit_is_nasa7(ch4):
    """n_p = 4 reproduces the NASA-7 rows, and the oracle's source through the
    degree-n_p entry equals the one through the NASA-7 entry bit for bit."""
    mm = inputs.with_thermo_degree(ch4, 4)
    np.testing.assert_array_equal(mm.thermo, ch4.nasa7)
    T, C, _ = inputs.random_states(ch4, 4, seed=5)
    for reactor in (oracle.CONV, oracle.CONP):
        np.testing.assert_array_equal(oracle.RefMech(mm).source(T, C, reactor),
                                      oracle.RefMech(ch4).source(T, C, reactor))


@pytest.mark.parametrize("T", [300.0, 1000.0, 2800.0])
def test_constant_cp_closed_form(ch4, T):
    """n_p = 0: the ideal gas of constant c_p, h = h_f + c_p (T - T0),
    s = s_298 + c_p ln(T/T0), u = h - R T, per kmol."""
    mm, r = refm(ch4, 0)
    th = r.thermo(T)
    cp = mm.thermo[:, 0] * R                      # J/(kmol K), constant
    hf, s298 = mm.cp_src[:, 3], mm.cp_src[:, 4]
    W = ch4.W
    np.testing.assert_allclose(th["cp"] * W, cp, rtol=1e-14)
    np.testing.assert_allclose(th["h"] * W, hf + cp * (T - T0), rtol=1e-12, atol=1e-9 * np.abs(cp * T).max())
    np.testing.assert_allclose(th["s"] * W, s298 + cp * np.log(T / T0), rtol=1e-12)
    np.testing.assert_allclose(th["u"] * W, hf + cp * (T - T0) - R * T, rtol=1e-12,
                               atol=1e-9 * np.abs(cp * T).max())


@pytest.mark.parametrize("n_p", [2, 7, 15])
def test_anchors_at_298(ch4, n_p):
    """h and s equal the drawn h_f and s_298 at 298.15 K for every degree
    (eq. enthalpy-adjustment and its entropy analogue)."""
    mm, r = refm(ch4, n_p)
    th = r.thermo(T0)
    hf, s298 = mm.cp_src[:, 3], mm.cp_src[:, 4]
    np.testing.assert_allclose(th["h"] * ch4.W, hf, rtol=1e-12, atol=1e-12 * np.abs(hf).max())
    np.testing.assert_allclose(th["s"] * ch4.W, s298, rtol=1e-12)


def _richardson(f, x, h):
    d1 = (f(x + h) - f(x - h)) / (2 * h)
    d2 = (f(x + h / 2) - f(x - h / 2)) / h
    return (4 * d2 - d1) / 3


@pytest.mark.parametrize("n_p", [7, 15])
@pytest.mark.parametrize("T", [400.0, 1200.0, 2500.0])
def test_derivative_identities_any_degree(ch4, n_p, T):
    _, r = refm(ch4, n_p)
    th = r.thermo(T)
    np.testing.assert_allclose(_richardson(lambda x: r.thermo(x)["h"], T, 1.0), th["cp"], rtol=1e-8)
    np.testing.assert_allclose(_richardson(lambda x: r.thermo(x)["u"], T, 1.0), th["cv"], rtol=1e-8)
    np.testing.assert_allclose(_richardson(lambda x: r.thermo(x)["s"], T, 1.0), th["cp"] / T, rtol=1e-8)
    np.testing.assert_allclose(th["cp"] - th["cv"], R / ch4.W, rtol=1e-12)
    np.testing.assert_allclose(th["g"], th["h"] - T * th["s"], rtol=1e-12,
                               atol=1e-12 * np.abs(T * th["s"]).max())


def test_fit_error_falls_with_degree(ch4):
    """Appendix C.1: each step 4 -> 7 -> 15 of the degree cuts the error by
    at least an order of magnitude; here the relative error of c_p against
    the drawn curve over 300-3000 K."""
    Tg = np.linspace(300.0, 3000.0, 541)
    c_lo, c_hi, theta = ch4.cp_src[:, 0], ch4.cp_src[:, 1], ch4.cp_src[:, 2]
    err = {}
    for n_p in (4, 7, 15):
        _, r = refm(ch4, n_p)
        e = 0.0
        for T in Tg:
            src = c_lo + (c_hi - c_lo) * (1.0 - np.exp(-T / theta))
            e = max(e, float(np.max(np.abs(r.thermo(T)["cp"] * ch4.W / R - src) / src)))
        err[n_p] = e
    assert err[4] < 0.05
    assert err[7] < err[4] / 10
    assert err[15] < err[7] / 10


def complex_step_jacobian(r, y, reactor):
    n = len(y)
    J = np.zeros((n, n))
    for k in range(n):
        h = 1e-30 * max(abs(y[k]), 1e-12)
        yy = y.astype(complex)
        yy[k] += 1j * h
        J[:, k] = r.source_complex(yy, reactor).imag / h
    return J


@pytest.mark.parametrize("n_p", [7, 15])
@pytest.mark.parametrize("reactor", [oracle.CONV, oracle.CONP])
def test_jacobian_any_degree_matches_complex_step(ch4, n_p, reactor):
    """The omega_T row takes d c_p/dT of the degree-n_p polynomial."""
    _, r = refm(ch4, n_p)
    T, C, _ = inputs.random_states(ch4, 2, seed=23)
    for c in range(2):
        y = np.concatenate([[T[c]], C[c]])
        Ja = r.jacobian(T[c], C[c], reactor)[0]
        Jc = complex_step_jacobian(r, y, reactor)
        scale = np.maximum(np.abs(Jc), 1e-13 * np.abs(Jc).max(axis=1, keepdims=True) + 1e-300)
        assert np.max(np.abs(Ja - Jc) / scale) < 1e-10


@pytest.mark.parametrize("reactor,key", [(oracle.CONP, "h"), (oracle.CONV, "u")])
def test_energy_conserved_any_degree(reactor, key):
    """Constant pressure keeps the mixture enthalpy, constant volume its
    internal energy, through ignition with n_p = 7 thermodynamics."""
    m = inputs.gen_mechanism("h2")
    mm, r = refm(m, 7)
    T, Y, p = inputs.field_reactor(mm, 3, (1250, 1350), (1, 1), (0.7, 1.5), "H2", seed=8)
    rho = p / (R * T * (Y / m.W).sum(1))
    opts = dict(method=oracle.SDIRK4, dt=5e-5, reactor=reactor, rtol=1e-9, atol=1e-16)
    T1, Y1, st, _ = r.integrate(T, Y, p if reactor == oracle.CONP else rho, opts)
    assert np.all(st == 0) and np.all(T1 > T + 300)
    e0 = np.array([Y[c] @ r.thermo(T[c])[key] for c in range(3)])
    e1 = np.array([Y1[c] @ r.thermo(T1[c])[key] for c in range(3)])
    np.testing.assert_allclose(e1, e0, rtol=1e-6, atol=1e-6 * np.abs(e0).max())


def test_refit_arguments():
    m = inputs.gen_mechanism("h2")
    with pytest.raises(ValueError):
        inputs.with_thermo_degree(m, 16)
    bare = inputs.isomer_mechanism(1e3, True)
    with pytest.raises(ValueError):
        inputs.with_thermo_degree(bare, 7)
