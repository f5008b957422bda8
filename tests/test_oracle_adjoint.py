"""Pins of the oracle's discrete adjoint (gradients of the integrated state
with respect to ln A, b, Ea of every reaction and to the initial state, with
the accepted steps frozen) and of its forward sensitivity.

Three independent checks: closed forms for A -> B, agreement of the adjoint
with the forward (tangent) sensitivity, and central differences of the map
y_0 -> y_end with the recorded step sizes replayed."""
import numpy as np
import pytest

import oracle
from oracle import tableau
from paper_2510_10005_gb300 import inputs

FIX = dict(adaptive=0, rtol=1e-12, atol=1e-20, newton_tol=1.0, max_newton=20, reactor=oracle.CONV,
           neg_tol=1e300)


@pytest.mark.parametrize("nsub", [1, 5])
def test_backward_euler_decay_closed_form(nsub):
    """C_A^n = C_A0 (1+kh)^-n: dC_A^n/d ln k = -n kh C_A0 (1+kh)^(-n-1),
    dC_A^n/dC_A0 = (1+kh)^-n, and d/db = ln T d/d ln k."""
    k, dt = 3e5, 1e-5
    r = oracle.RefMech(inputs.isomer_mechanism(k, reversible=False))
    y0 = np.array([[1000.0, 0.03, 0.002]])
    lam = np.array([[0.0, 1.0, 0.0]])
    dy0, g, st = r.adjoint(y0, lam, dict(FIX, method=oracle.BE, dt=dt, nsub=nsub))
    kh = k * dt / nsub
    assert st[0] == 0
    assert g[0, 0, 0] == pytest.approx(-nsub * kh * 0.03 * (1 + kh) ** (-nsub - 1), rel=1e-12)
    assert g[0, 0, 1] == pytest.approx(np.log(1000.0) * g[0, 0, 0], rel=1e-12)
    assert g[0, 0, 2] == pytest.approx(-g[0, 0, 0] / (inputs.R_UNIV * 1000.0), rel=1e-12)
    assert dy0[0, 1] == pytest.approx((1 + kh) ** -nsub, rel=1e-12)
    assert dy0[0, 2] == 0.0


@pytest.mark.parametrize("method", [oracle.SDIRK2, oracle.SDIRK4])
def test_sdirk_decay_closed_form(method):
    """C_A^n = C_A0 R(z)^n with z = -kh: d/d ln k = n R^(n-1) R'(z) z."""
    k, dt, nsub = 2e5, 1e-5, 3
    r = oracle.RefMech(inputs.isomer_mechanism(k, reversible=False))
    y0 = np.array([[1000.0, 0.03, 0.0]])
    dy0, g, st = r.adjoint(y0, np.array([[0.0, 1.0, 0.0]]), dict(FIX, method=method, dt=dt, nsub=nsub))
    t = tableau.tableau(method)
    s = t["s"]
    R = lambda z: 1.0 + z * t["b"][:s] @ np.linalg.solve(np.eye(s) - z * t["A"][:s, :s], np.ones(s))
    z = -k * dt / nsub
    dR = R(z + 1e-30j).imag / 1e-30     # complex step: R'(z) to rounding
    expect = 0.03 * nsub * R(z).real ** (nsub - 1) * dR * z
    assert st[0] == 0
    assert g[0, 0, 0] == pytest.approx(expect, rel=1e-10)
    assert dy0[0, 1] == pytest.approx(R(z) ** nsub, rel=1e-12)


@pytest.fixture(scope="module")
def h2_case(mechs):
    m = mechs["h2"]
    r = oracle.RefMech(m)
    T, Y, p = inputs.field_reactor(m, 3, (1200, 1400), (1, 1), (0.8, 1.2), "H2", seed=2)
    C = r.concentrations(T, Y, p, oracle.CONP)
    y0 = np.concatenate([T[:, None], C], axis=1)
    o = dict(method=oracle.SDIRK4, adaptive=1, dt=1e-5, rtol=1e-8, atol=1e-14, reactor=oracle.CONP,
             newton_tol=1e-6, max_newton=20)
    lam = np.zeros_like(y0)
    lam[:, 0] = 1.0                     # L = T_end
    dy0, g, st = r.adjoint(y0, lam, o)
    assert np.all(st == 0)
    return m, r, y0, o, lam, dy0, g


def test_adjoint_equals_forward_sensitivity(h2_case):
    m, r, y0, o, lam, dy0, g = h2_case
    for pj in range(0, m.nr, 4):
        for pk in range(3):
            dyend, st = r.tangent(y0, np.zeros_like(y0), o, pj, pk)
            assert np.all(st == 0)
            np.testing.assert_allclose(g[:, pj, pk], dyend[:, 0], rtol=1e-9,
                                       atol=1e-12 * np.abs(g[:, :, pk]).max())
    for k in (0, 1, 4):
        e = np.zeros_like(y0)
        e[:, k] = 1.0
        dyend, _ = r.tangent(y0, e, o)
        np.testing.assert_allclose(dy0[:, k], dyend[:, 0], rtol=1e-9)


def test_adjoint_against_finite_differences(h2_case):
    """Central differences of T_end with the accepted steps replayed (the
    adjoint differentiates the map with the step sizes frozen); relative
    1e-5 on every gradient entry above 1e-3 of the largest of its kind."""
    m, r, y0, o, lam, dy0, g = h2_case
    yend, st, hs, hn = r.integrate_hist(y0, o)
    assert np.all(hn > 0)
    steps = {0: 1e-4, 1: 1e-4, 2: 1e3}
    checked = 0
    for pj in range(m.nr):
        for pk, dv in steps.items():
            big = np.abs(g[:, pj, pk]) > 1e-3 * np.abs(g[:, :, pk]).max()
            if not big.any():
                continue
            out = []
            for s in (+1, -1):
                mm = m.copy()
                mm.arr[pj, pk] += s * dv
                ye, st2 = oracle.RefMech(mm).replay(y0, o, hs, hn)
                assert np.all(st2 == 0)
                out.append(ye[:, 0])
            fd = (out[0] - out[1]) / (2 * dv)
            np.testing.assert_allclose(fd[big], g[big, pj, pk], rtol=1e-5)
            checked += 1
    assert checked >= 10
    # initial temperature
    out = []
    for s in (+1, -1):
        yy = y0.copy()
        yy[:, 0] += s * 1e-3
        out.append(r.replay(yy, o, hs, hn)[0][:, 0])
    np.testing.assert_allclose((out[0] - out[1]) / 2e-3, dy0[:, 0], rtol=1e-6)


@pytest.mark.parametrize("reactor", [oracle.CONP, oracle.CONV])
def test_adjoint_in_flow_variables_against_finite_differences(mechs, reactor):
    """adjoint_TY (the state adjoint chained through Y = W C / rho at the end
    and C = rho Y / W at the start) against central differences of
    L = sum_c a_c T_end + b_c . Y_end over (T0, Y0), steps replayed."""
    m = mechs["h2"]
    r = oracle.RefMech(m)
    T, Y, p = inputs.field_reactor(m, 3, (1200, 1350), (1, 1.5), (0.8, 1.2), "H2", seed=4)
    if reactor == oracle.CONV:
        p = p / (inputs.R_UNIV * T * (Y / m.W).sum(axis=1))   # the density of the same state
    o = dict(method=oracle.SDIRK4, adaptive=1, dt=1e-5, rtol=1e-8, atol=1e-14, reactor=reactor,
             newton_tol=1e-6, max_newton=20)
    rng = np.random.default_rng(5)
    a = rng.normal(size=len(T))
    b = rng.normal(size=Y.shape)
    dT0, dY0, g, st = r.adjoint_TY(T, Y, p, a, b, o)
    assert np.all(st == 0)
    y0 = np.concatenate([T[:, None], r.concentrations(T, Y, p, reactor)], axis=1)
    _, st, hs, hn = r.integrate_hist(y0, o)
    assert np.all(st == 0) and np.all(hn > 0)

    def loss(T_, Y_):
        y = np.concatenate([T_[:, None], r.concentrations(T_, Y_, p, reactor)], axis=1)
        ye, s2 = r.replay(y, o, hs, hn)
        assert np.all(s2 == 0)
        return a * ye[:, 0] + (b * r.mass_fractions(ye[:, 1:])).sum(axis=1)

    dT = 1e-3
    fd = (loss(T + dT, Y) - loss(T - dT, Y)) / (2 * dT)
    np.testing.assert_allclose(fd, dT0, rtol=1e-6)
    scale = np.abs(dY0).max()
    L0 = loss(T, Y)
    for k in range(m.ns):
        dY = np.zeros_like(Y)
        dY[:, k] = 1e-7
        if np.all(Y[:, k] > 1e-5):
            fd = (loss(T, Y + dY) - loss(T, Y - dY)) / 2e-7
        else:   # absent species: one-sided second-order difference (no negative mass fraction)
            fd = (-3 * L0 + 4 * loss(T, Y + dY) - loss(T, Y + 2 * dY)) / 2e-7
        np.testing.assert_allclose(fd, dY0[:, k], rtol=1e-5, atol=1e-6 * scale)
