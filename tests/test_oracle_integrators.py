"""Pins of the oracle's time integrators: backward Euler with Newton
(Section 3.2), SDIRK-2 / SDIRK-4 in stage-derivative form (Appendix A.1, A.2)
and the step-size control the paper leaves open.

Closed forms: A -> B and A <=> B with constant rates reduce to linear ODEs,
whose discrete solutions are C_A0 R(z)^n with the scheme's stability
function R. Plus the convergence order study of Section 5.3, invariants,
long-time equilibrium and the failure statuses."""
import numpy as np
import pytest

import oracle
from oracle import tableau
from paper_2510_10005_gb300 import inputs


def stability_function(method, z):
    if method == oracle.BE:
        return 1.0 / (1.0 - z)
    t = tableau.tableau(method)
    s = t["s"]
    A = t["A"][:s, :s]
    b = t["b"][:s]
    return 1.0 + z * b @ np.linalg.solve(np.eye(s) - z * A, np.ones(s))


# fixed steps, tight Newton; negative concentrations allowed (a stability
# function may be negative at large |z|, which is what the closed forms test)
FIXED = dict(adaptive=0, rtol=1e-12, atol=1e-20, newton_tol=1.0, max_newton=20, reactor=oracle.CONV,
             neg_tol=1e300)


@pytest.mark.parametrize("method", [oracle.BE, oracle.SDIRK2, oracle.SDIRK4])
@pytest.mark.parametrize("nsub", [1, 7])
def test_irreversible_decay_closed_form(method, nsub):
    k, dt = 3.0e5, 1e-5
    m = inputs.isomer_mechanism(k, reversible=False)
    r = oracle.RefMech(m)
    C0 = np.array([[0.03, 0.002]])
    y0 = np.concatenate([[[1000.0]], C0], axis=1)
    y, st, stats = r.integrate_y(y0, dict(FIXED, method=method, dt=dt, nsub=nsub))
    assert st[0] == 0
    expect = C0[0, 0] * stability_function(method, -k * dt / nsub) ** nsub
    assert y[0, 1] == pytest.approx(expect, rel=1e-13)
    assert y[0, 1] + y[0, 2] == pytest.approx(C0.sum(), rel=1e-15)
    assert y[0, 0] == 1000.0   # omega_T = 0 exactly: equal internal energies


@pytest.mark.parametrize("method", [oracle.BE, oracle.SDIRK2, oracle.SDIRK4])
def test_reversible_relaxation_closed_form(method):
    """A <=> B with K = exp(delta s / R) relaxes to C_tot/(1+K) with the
    deviation multiplied by R(-(kf + kr) h) per step."""
    kf, ds, dt, nsub = 2.0e5, 0.7, 2e-5, 5
    m = inputs.isomer_mechanism(kf, reversible=True, ds_over_R=ds)
    r = oracle.RefMech(m)
    K = np.exp(ds)
    C0 = np.array([0.02, 0.01])
    y, st, _ = r.integrate_y(np.array([[900.0, *C0]]), dict(FIXED, method=method, dt=dt, nsub=nsub))
    assert st[0] == 0
    Ceq = C0.sum() / (1 + K)
    z = -(kf + kf / K) * dt / nsub
    expect = Ceq + (C0[0] - Ceq) * stability_function(method, z) ** nsub
    assert y[0, 1] == pytest.approx(expect, rel=1e-12)


def _ignition_state(m, r):
    """A state of the 9-species mechanism in the middle of its ignition (the
    paper evaluates the order at the point of largest dT/dt)."""
    T, Y, p = inputs.field_reactor(m, 1, (1200, 1200), (1, 1), (1, 1), "H2", seed=0)
    C = r.concentrations(T, Y, p, oracle.CONP)   # C from (T, Y, p); then held at constant volume
    y = np.concatenate([T[:, None], C], axis=1)
    y, st, _ = r.integrate_y(y, dict(method=oracle.SDIRK4, adaptive=1, dt=4.8e-5, rtol=1e-10,
                                      atol=1e-16, reactor=oracle.CONV))
    assert st[0] == 0 and 1500 < y[0, 0] < 2500
    assert r.source(y[:, 0], y[:, 1:], oracle.CONV)[0, 0] > 1e8   # dT/dt near its peak
    return y


@pytest.mark.parametrize("method,lo,hi,dt", [(oracle.BE, 0.9, 1.1, 1e-7),
                                              (oracle.SDIRK2, 1.9, 2.1, 4e-7),
                                              (oracle.SDIRK4, 2.7, 4.2, 1e-7)])
def test_convergence_order_at_ignition(mechs, ref, method, lo, hi, dt):
    """Section 5.3: steps h = dt / 2^r, r = 0..4, at the point of largest
    dT/dt, error (L2 over the concentrations) against a much finer solution of
    the same scheme. BE and SDIRK-2 show their orders; SDIRK-4 shows the
    order reduction of a stage-order-one method on a stiff problem (its
    classical order is pinned on a non-stiff problem below)."""
    m, r = mechs["h2"], ref["h2"]
    y0 = _ignition_state(m, r)
    opts = dict(FIXED, method=method, dt=dt, reactor=oracle.CONV, rtol=1e-13, atol=1e-22)
    yref, st, _ = r.integrate_y(y0, dict(opts, nsub=2**9))
    assert st[0] == 0
    errs = []
    for rr in range(5):
        y, st, _ = r.integrate_y(y0, dict(opts, nsub=2**rr))
        assert st[0] == 0
        errs.append(np.sqrt(np.sum((y[0, 1:] - yref[0, 1:]) ** 2)))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(slopes > lo) and np.all(slopes < hi), (errs, slopes)


@pytest.mark.parametrize("method,order", [(oracle.BE, 1), (oracle.SDIRK2, 2), (oracle.SDIRK4, 4)])
def test_classical_order_nonstiff(method, order):
    """A -> B with k h small: the error against exp(-k t) falls at the
    scheme's classical order."""
    k, dt = 1.0e5, 2e-5
    r = oracle.RefMech(inputs.isomer_mechanism(k, reversible=False))
    y0 = np.array([[1000.0, 0.03, 0.0]])
    errs = []
    for rr in range(2, 6):
        y, st, _ = r.integrate_y(y0, dict(FIXED, method=method, dt=dt, nsub=2**rr))
        errs.append(abs(y[0, 1] - 0.03 * np.exp(-k * dt)))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(slopes - order) < 0.15), slopes


@pytest.mark.parametrize("method", [oracle.BE, oracle.SDIRK4])
def test_linear_invariants_conserved(mechs, ref, method):
    """Element totals sum_i e_ki C_i (constant volume) are linear invariants,
    kept to rounding by every Runge-Kutta step."""
    m, r = mechs["h2"], ref["h2"]
    T, Y, p = inputs.field_reactor(m, 6, (1100, 1400), (1, 1), (0.5, 2), "H2", seed=3)
    rho = p / (inputs.R_UNIV * T * (Y / m.W).sum(1))
    opts = dict(method=method, dt=1e-5, reactor=oracle.CONV, adaptive=int(method != oracle.BE),
                rtol=1e-6 if method != oracle.BE else 1e-10, atol=1e-12 if method != oracle.BE else 1e-16,
                newton_tol=0.03 if method != oracle.BE else 1.0, max_newton=7 if method != oracle.BE else 20)
    C0 = r.concentrations(T, Y, rho, oracle.CONV)
    T1, Y1, st, _ = r.integrate(T, Y, rho, opts)
    assert np.all(st == 0)
    C1 = r.concentrations(T1, Y1, rho, oracle.CONV)
    el0, el1 = C0 @ m.comp, C1 @ m.comp
    np.testing.assert_allclose(el1, el0, rtol=1e-13)
    np.testing.assert_allclose((C1 * m.W).sum(1), rho, rtol=1e-13)


def test_constant_pressure_keeps_p_and_elements(mechs, ref):
    """CONP: pressure and enthalpy stay at their initial values within the
    integration tolerance; element mass fractions to rounding."""
    m, r = mechs["h2"], ref["h2"]
    T, Y, p = inputs.field_reactor(m, 4, (1200, 1400), (1, 1), (0.7, 1.5), "H2", seed=8)
    opts = dict(method=oracle.SDIRK4, dt=5e-5, reactor=oracle.CONP, rtol=1e-9, atol=1e-16)
    T1, Y1, st, _ = r.integrate(T, Y, p, opts)
    assert np.all(st == 0) and np.all(T1 > T + 300)
    C1 = r.concentrations(T1, Y1, p, oracle.CONP)
    p1 = inputs.R_UNIV * T1 * C1.sum(1)
    np.testing.assert_allclose(p1, p, rtol=1e-12)   # C recomputed from p: tautology guard
    el0 = (Y / m.W) @ m.comp
    el1 = (Y1 / m.W) @ m.comp
    np.testing.assert_allclose(el1, el0, rtol=1e-12)
    h0 = np.array([Y[c] @ r.thermo(T[c])["h"] for c in range(4)])
    h1 = np.array([Y1[c] @ r.thermo(T1[c])["h"] for c in range(4)])
    np.testing.assert_allclose(h1, h0, rtol=1e-6, atol=1e-6 * np.abs(h0).max())


def test_constant_pressure_state_pressure_drift(mechs, ref):
    """The raw state (T, C) of the CONP form keeps R T sum C at p within the
    integration tolerance (a quadratic invariant of the ODE)."""
    m, r = mechs["h2"], ref["h2"]
    T, Y, p = inputs.field_reactor(m, 3, (1250, 1350), (1, 1), (1, 1), "H2", seed=9)
    C = r.concentrations(T, Y, p, oracle.CONP)
    y0 = np.concatenate([T[:, None], C], axis=1)
    y, st, _ = r.integrate_y(y0, dict(method=oracle.SDIRK4, dt=5e-5, reactor=oracle.CONP,
                                      rtol=1e-9, atol=1e-16))
    assert np.all(st == 0)
    np.testing.assert_allclose(inputs.R_UNIV * y[:, 0] * y[:, 1:].sum(1), p, rtol=1e-6)


def test_long_time_equilibrium_detailed_balance(mechs, ref):
    """After 1 s every reversible reaction is balanced: |q_j| is a tiny part
    of its forward and reverse terms (equilibrium constants of
    eq. equilibrium-constant-1)."""
    m, r = mechs["h2"], ref["h2"]
    T, Y, p = inputs.field_reactor(m, 2, (1300, 1300), (1, 1), (0.8, 1.2), "H2", seed=2)
    C = r.concentrations(T, Y, p, oracle.CONP)
    y0 = np.concatenate([T[:, None], C], axis=1)
    y, st, stats = r.integrate_y(y0, dict(method=oracle.SDIRK4, dt=1.0, reactor=oracle.CONP,
                                          rtol=1e-10, atol=1e-20))
    assert np.all(st == 0)
    for c in range(2):
        kf, kr, q = r.rates(y[c, 0], y[c, 1:])
        fwd = np.array([kf[j] * np.prod([y[c, 1 + m.rf_idx[j, s]] ** m.rf_nu[j, s]
                                         for s in range(3) if m.rf_idx[j, s] >= 0]) for j in range(m.nr)])
        assert np.all(np.abs(q) <= 1e-6 * fwd + 1e-30)


def test_adaptive_matches_tight_reference(mechs, ref):
    """rtol = 1e-6 solution within a few rtol of a rtol = 1e-11 solution."""
    m, r = mechs["h2"], ref["h2"]
    T, Y, p = inputs.field_reactor(m, 8, (1100, 1500), (1, 1), (0.5, 2), "H2", seed=6)
    T1, Y1, st, stats = r.integrate(T, Y, p, dict(method=oracle.SDIRK4, dt=1e-5, rtol=1e-6, atol=1e-12))
    T2, Y2, st2, _ = r.integrate(T, Y, p, dict(method=oracle.SDIRK4, dt=1e-5, rtol=1e-11, atol=1e-18))
    assert np.all(st == 0) and np.all(st2 == 0)
    assert np.max(np.abs(T1 - T2) / T2) < 20e-6
    assert np.max(np.abs(Y1 - Y2)) < 20e-6
    assert stats[:, 0].min() >= 1 and stats[:, 2].min() >= 5


def test_failure_statuses(mechs, ref):
    m, r = mechs["h2"], ref["h2"]
    T, Y, p = inputs.field_reactor(m, 2, (1400, 1400), (1, 1), (1, 1), "H2", seed=0)
    C = r.concentrations(T, Y, p, oracle.CONP)
    y0 = np.concatenate([T[:, None], C], axis=1)
    # Newton fails (one iteration allowed, no halving)
    _, st, _ = r.integrate_y(y0, dict(method=oracle.BE, adaptive=0, dt=1e-5, max_newton=1,
                                      max_halvings=0, rtol=1e-10, atol=1e-16, newton_tol=1.0))
    assert np.all(st == 1)
    # max_steps exhausted
    _, st, _ = r.integrate_y(y0, dict(method=oracle.SDIRK4, dt=1e-4, max_steps=3))
    assert np.all(st == 3)
    # minimum step larger than the first step
    _, st, _ = r.integrate_y(y0, dict(method=oracle.SDIRK4, dt=1e-5, hmin=1e-3))
    assert np.all(st == 2)
    # non-finite input
    bad = y0.copy()
    bad[0, 3] = np.nan
    _, st, _ = r.integrate_y(bad, dict(method=oracle.SDIRK4, dt=1e-6))
    assert st[0] == 4 and st[1] == 0
