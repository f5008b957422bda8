"""Pins of the oracle's SRI falloff (Section 2.2.3) and pressure-dependent
Arrhenius "PLOG" reactions (Section 2.2.4, eqs. plog_p1_p2, plog_rate).

Independent checks: the analytical Jacobian against complex-step
derivatives of S(y) on a mechanism with both kinds; PLOG's defining
properties (the level's summed Arrhenius rate at a level pressure, the
geometric mean halfway in ln p, constant outside the pressure range,
continuity across levels); SRI's falloff limits (k_inf d T^e at high
pressure, k_0 [M] d T^e at low pressure, where X -> 0); and the adjoint
against the forward sensitivity with SRI and PLOG reactions present."""
import numpy as np
import pytest

import oracle
from paper_2510_10005_gb300 import inputs

R = inputs.R_UNIV


@pytest.fixture(scope="module")
def xmech():
    return inputs.with_sri_plog(inputs.gen_mechanism("ch4"), n_sri=8, n_plog=20, seed=3)


def complex_step_jacobian(r, y, reactor):
    n = len(y)
    J = np.zeros((n, n))
    for k in range(n):
        h = 1e-30 * max(abs(y[k]), 1e-12)
        yy = y.astype(complex)
        yy[k] += 1j * h
        J[:, k] = r.source_complex(yy, reactor).imag / h
    return J


@pytest.mark.parametrize("reactor", [oracle.CONV, oracle.CONP])
def test_jacobian_matches_complex_step(xmech, reactor):
    r = oracle.RefMech(xmech)
    T, C, p = inputs.random_states(xmech, 3, seed=22)
    for c in range(3):
        y = np.concatenate([[T[c]], C[c]])
        Ja = r.jacobian(T[c], C[c], reactor)[0]
        Jc = complex_step_jacobian(r, y, reactor)
        scale = np.maximum(np.abs(Jc), 1e-13 * np.abs(Jc).max(axis=1, keepdims=True) + 1e-300)
        assert np.max(np.abs(Ja - Jc) / scale) < 1e-10


def _arrhenius(rows, T):
    return np.sum(np.exp(rows[:, 1] + rows[:, 2] * np.log(T) - rows[:, 3] / (R * T)))


def _state_at(m, T, p):
    """Concentrations with R T sum C = p (equal shares)."""
    C = np.full(m.ns, p / (R * T) / m.ns)
    return C


def test_plog_definition(xmech):
    m = xmech
    r = oracle.RefMech(m)
    js = [j for j in range(m.nr) if m.rtype[j] == inputs.RXN_PLOG]
    T = 1234.0
    for j in js:
        rows = m.plog[m.plog_ptr[j]:m.plog_ptr[j + 1]]
        ps = np.unique(rows[:, 0])
        level = [_arrhenius(rows[rows[:, 0] == p], T) for p in ps]
        for p, k in zip(ps, level):                              # at a level: its summed rate
            assert r.rates(T, _state_at(m, T, p))[0][j] == pytest.approx(k, rel=1e-12)
        for a in range(len(ps) - 1):                             # halfway in ln p: geometric mean
            pm = np.sqrt(ps[a] * ps[a + 1])
            assert r.rates(T, _state_at(m, T, pm))[0][j] == pytest.approx(np.sqrt(level[a] * level[a + 1]),
                                                                           rel=1e-12)
        lo = r.rates(T, _state_at(m, T, ps[0] / 7))[0][j]         # outside: the nearest level
        hi = r.rates(T, _state_at(m, T, ps[-1] * 7))[0][j]
        assert lo == pytest.approx(level[0], rel=1e-12) and hi == pytest.approx(level[-1], rel=1e-12)
    assert any(len(np.unique(m.plog[m.plog_ptr[j]:m.plog_ptr[j + 1], 0])) <
               m.plog_ptr[j + 1] - m.plog_ptr[j] for j in js)   # a repeated pressure is exercised


def test_sri_falloff_limits(xmech):
    m = xmech
    r = oracle.RefMech(m)
    js = [j for j in range(m.nr) if m.rtype[j] == inputs.RXN_SRI]
    assert js
    T = 1500.0
    for j in js:
        lnA, b, Ea = m.arr[j]
        lnA0, b0, Ea0 = m.arr0[j]
        kinf = np.exp(lnA + b * np.log(T) - Ea / (R * T))
        k0 = np.exp(lnA0 + b0 * np.log(T) - Ea0 / (R * T))
        d, e = m.sri[j, 3], m.sri[j, 4]
        # [M] = sum C (+ efficiencies): scale a state up and down by many decades
        for scale, expect in ((1e25, lambda M: kinf * d * T ** e), (1e-25, lambda M: k0 * M * d * T ** e)):
            C = np.full(m.ns, 1e-3 * scale)
            M = C.sum() + sum((m.eff_val[k] - 1.0) * C[m.eff_idx[k]] for k in range(m.eff_ptr[j], m.eff_ptr[j + 1]))
            kf = r.rates(T, C)[0][j]
            assert kf == pytest.approx(expect(M), rel=2e-2)      # X = 1/(1 + log10^2 Pr) ~ 1/600


def test_adjoint_equals_forward_sensitivity_with_sri_plog(xmech):
    m = xmech
    r = oracle.RefMech(m)
    T, Y, p = inputs.field_reactor(m, 2, (1300, 1500), (2, 30), (0.8, 1.2), "CH4", seed=4)
    y0 = np.concatenate([T[:, None], r.concentrations(T, Y, p, oracle.CONP)], axis=1)
    o = dict(method=oracle.SDIRK4, adaptive=1, dt=2e-6, rtol=1e-8, atol=1e-14, reactor=oracle.CONP,
             newton_tol=1e-6, max_newton=20)
    lam = np.zeros_like(y0)
    lam[:, 0] = 1.0
    dy0, g, st = r.adjoint(y0, lam, o)
    assert np.all(st == 0)
    sri = [j for j in range(m.nr) if m.rtype[j] == inputs.RXN_SRI]
    plog = [j for j in range(m.nr) if m.rtype[j] == inputs.RXN_PLOG]
    for pj in sri[:3] + plog[:2]:
        for pk in range(3):
            dyend, st = r.tangent(y0, np.zeros_like(y0), o, pj, pk)
            assert np.all(st == 0)
            np.testing.assert_allclose(g[:, pj, pk], dyend[:, 0], rtol=1e-9,
                                       atol=1e-12 * np.abs(g[:, :, pk]).max())
    assert not g[:, plog, :].any()          # PLOG rates are not set by (ln A, b, Ea)
    for k in (0, 3):
        e = np.zeros_like(y0)
        e[:, k] = 1.0
        dyend, _ = r.tangent(y0, e, o)
        np.testing.assert_allclose(dy0[:, k], dyend[:, 0], rtol=1e-9)


def _golden_plog():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "plog_section_2_2_4.txt")
    rows = np.array([[float(v) for v in line.split()] for line in open(path)
                     if line.strip() and not line.startswith("#")])
    # SI-kmol: p in Pa, A of a bimolecular reaction in m^3/(kmol s), Ea in J/kmol
    return np.stack([rows[:, 0] * inputs.P_ATM, np.log(rows[:, 1] * 1e-3), rows[:, 2], rows[:, 3] * 4184.0],
                    axis=1)


def test_plog_printed_example():
    """The rate table printed in Section 2.2.4: seven pressure intervals (six
    levels); the level's own rate at each printed pressure, log-linear in
    between, the end levels' rates at and beyond 0.1 and 100 atm."""
    table = _golden_plog()
    c = np.array([3.5, 1e-4, -2e-8, 1e-12, -1e-16, -1000.0, 5.0])
    m = inputs.Mechanism(
        names=["A", "B", "C", "D"], elements=["X", "Y"], comp=np.array([[1, 0], [0, 1], [1, 0], [0, 1]]),
        W=np.array([14.0, 18.0, 14.0, 18.0]), nasa7=np.stack([c] * 4),
        rtype=np.array([inputs.RXN_PLOG], dtype=np.int32), reversible=np.array([1], dtype=np.int32),
        rf_idx=np.array([[0, 1, -1]], dtype=np.int32), rf_nu=np.array([[1, 1, 0]], dtype=np.int32),
        rr_idx=np.array([[2, 3, -1]], dtype=np.int32), rr_nu=np.array([[1, 1, 0]], dtype=np.int32),
        arr=np.zeros((1, 3)), arr0=np.zeros((1, 3)), troe=np.zeros((1, 4)),
        eff_ptr=np.zeros(2, dtype=np.int32), eff_idx=np.zeros(0, dtype=np.int32), eff_val=np.zeros(0),
        plog_ptr=np.array([0, len(table)], dtype=np.int32), plog=table)
    m.validate()
    r = oracle.RefMech(m)
    assert len(np.unique(table[:, 0])) + 1 == 7            # the seven interval tests the section counts
    for T in (800.0, 1500.0, 2400.0):
        ks = np.exp(table[:, 1] + table[:, 2] * np.log(T) - table[:, 3] / (R * T))
        kf = lambda p: r.rates(T, _state_at(m, T, p))[0][0]
        for p, k in zip(table[:, 0], ks):
            assert kf(p) == pytest.approx(k, rel=1e-12)
        for a in range(len(ks) - 1):
            for w in (0.25, 0.5, 0.9):
                p = np.exp((1 - w) * np.log(table[a, 0]) + w * np.log(table[a + 1, 0]))
                assert kf(p) == pytest.approx(ks[a] ** (1 - w) * ks[a + 1] ** w, rel=1e-11)
        assert kf(0.01 * inputs.P_ATM) == pytest.approx(ks[0], rel=1e-12)
        assert kf(1000.0 * inputs.P_ATM) == pytest.approx(ks[-1], rel=1e-12)
