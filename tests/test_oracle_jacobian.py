"""Pins of the oracle's analytical Jacobian (Section 3.2) and of its dense
direct solver (Section 3.4).

J is compared with complex-step derivatives of the oracle's S(y) (exact to
rounding, independent of the hand derivation), with the paper's
second-order finite-difference study (Section 5.2) and with the error
metrics of Appendix C.2 (E_rel, E_norm)."""
import numpy as np
import pytest

import oracle
from paper_2510_10005_gb300 import inputs


def complex_step_jacobian(r, y, reactor):
    n = len(y)
    J = np.zeros((n, n))
    for k in range(n):
        h = 1e-30 * max(abs(y[k]), 1e-12)
        yy = y.astype(complex)
        yy[k] += 1j * h
        J[:, k] = r.source_complex(yy, reactor).imag / h
    return J


@pytest.mark.parametrize("kind", ["h2", "ch4"])
@pytest.mark.parametrize("reactor", [oracle.CONV, oracle.CONP, oracle.CONP_LITERAL])
def test_jacobian_matches_complex_step(mechs, ref, kind, reactor):
    m, r = mechs[kind], ref[kind]
    T, C, p = inputs.random_states(m, 3, seed=21)
    for c in range(3):
        y = np.concatenate([[T[c]], C[c]])
        Ja = r.jacobian(T[c], C[c], reactor)[0]
        Jc = complex_step_jacobian(r, y, reactor)
        # entry-wise relative error, with a floor at 1e-13 of the row scale
        scale = np.maximum(np.abs(Jc), 1e-13 * np.abs(Jc).max(axis=1, keepdims=True) + 1e-300)
        assert np.max(np.abs(Ja - Jc) / scale) < 1e-10


@pytest.mark.parametrize("reactor", [oracle.CONV, oracle.CONP])
def test_jacobian_matches_complex_step_160_species(reactor):
    """The same pin on the 160-species / 900-reaction mechanism (falloff and
    third-body reactions with 3-6 efficiencies each), two random states."""
    m = inputs.gen_mechanism("c7")
    r = oracle.RefMech(m)
    T, C, p = inputs.random_states(m, 2, seed=23)
    for c in range(2):
        y = np.concatenate([[T[c]], C[c]])
        Ja = r.jacobian(T[c], C[c], reactor)[0]
        Jc = complex_step_jacobian(r, y, reactor)
        scale = np.maximum(np.abs(Jc), 1e-13 * np.abs(Jc).max(axis=1, keepdims=True) + 1e-300)
        assert np.max(np.abs(Ja - Jc) / scale) < 1e-10


def test_jacobian_with_zero_concentrations(mechs, ref):
    """Exact at C_i = 0 (products of concentrations differentiated exactly)."""
    m, r = mechs["h2"], ref["h2"]
    T, Y, p = inputs.field_reactor(m, 2, (1100, 1400), (1, 1), (0.5, 2), "H2", seed=4)
    C = r.concentrations(T, Y, p, oracle.CONP)
    assert (C == 0).any()
    for c in range(2):
        y = np.concatenate([[T[c]], C[c]])
        Ja = r.jacobian(T[c], C[c], oracle.CONP)[0]
        Jc = complex_step_jacobian(r, y, oracle.CONP)
        scale = np.maximum(np.abs(Jc), 1e-13 * np.abs(Jc).max(axis=1, keepdims=True) + 1e-300)
        assert np.max(np.abs(Ja - Jc) / scale) < 1e-10


def _fd_jacobian(r, T, C, dT, dC, reactor):
    """Second-order central differences of Section 5.2
    (eq. finite_difference_Tevolve)."""
    n = len(C) + 1
    J = np.zeros((n, n))
    J[:, 0] = (r.source(T + dT, C, reactor)[0] - r.source(T - dT, C, reactor)[0]) / (2 * dT)
    for j in range(len(C)):
        Cp, Cm = C.copy(), C.copy()
        Cp[j] += dC
        Cm[j] -= dC
        J[:, 1 + j] = (r.source(T, Cp, reactor)[0] - r.source(T, Cm, reactor)[0]) / (2 * dC)
    return J


def test_fd_second_order_convergence(mechs, ref):
    """Paper's refinement study: dT0 = 100 K, dC0 = min C / 4, halved four
    times; the L2 error of the FD Jacobian falls at second order."""
    m, r = mechs["h2"], ref["h2"]
    T, C, p = inputs.random_states(m, 1, seed=31)
    T, C = T[0], C[0]
    Ja = r.jacobian(T, C, oracle.CONV)[0]
    dT, dC = 100.0, C[C > 0].min() / 4
    errs = []
    for k in range(5):
        Jf = _fd_jacobian(r, T, C, dT / 2**k, dC / 2**k, oracle.CONV)
        errs.append(np.sqrt(np.sum((Ja - Jf) ** 2)))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(slopes > 1.7) and np.all(slopes < 2.3), slopes


@pytest.mark.parametrize("kind", ["h2", "ch4"])
def test_niemeyer_error_metrics_within_paper_bounds(mechs, ref, kind):
    """E_norm (Appendix C.2) with dC = 1e-6 kmol/m3, dT = 1e-3 K over elements
    with |J| > ||J_fd||_F / 1e20 stays below the largest value the paper
    reports (3.35e-5). E_rel is taken over the elements the differences can
    resolve (|J_fd| above 1e-6 of its row maximum; below that the quotient of
    two rounded source terms carries no digits) and stays below 3e-3."""
    m, r = mechs[kind], ref[kind]
    T, C, p = inputs.random_states(m, 8 if kind == "h2" else 3, seed=41)
    for c in range(len(T)):
        Ja = r.jacobian(T[c], C[c], oracle.CONV)[0]
        Jf = _fd_jacobian(r, T[c], C[c], 1e-3, 1e-6, oracle.CONV)
        fro = np.sqrt(np.sum(Jf**2))
        mask = np.abs(Ja) > fro / 1e20
        e_norm = np.sqrt(np.sum((Ja - Jf)[mask] ** 2)) / fro
        assert e_norm < 3.35e-5
        resolved = mask & (np.abs(Jf) > 1e-6 * np.abs(Jf).max(axis=1, keepdims=True))
        e_rel = np.sqrt(np.sum(((Ja - Jf)[resolved] / Jf[resolved]) ** 2))
        assert e_rel < 3e-3


def test_lu_solve_against_numpy():
    rng = np.random.default_rng(0)
    for n in (1, 2, 5, 10, 54):
        A = rng.standard_normal((n, n))
        b = rng.standard_normal(n)
        x = oracle.lu_solve(A, b)
        np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)


def test_lu_needs_pivoting():
    """A zero leading entry forces a row swap: [[0, 1], [2, 3]] x = [1, 8]."""
    x = oracle.lu_solve(np.array([[0.0, 1.0], [2.0, 3.0]]), np.array([1.0, 8.0]))
    np.testing.assert_array_equal(x, [2.5, 1.0])
    with pytest.raises(np.linalg.LinAlgError):
        oracle.lu_solve(np.array([[1.0, 2.0], [2.0, 4.0]]), np.array([1.0, 1.0]))


def test_lu_on_newton_matrices(mechs, ref):
    """The solver on actual Newton matrices I - gamma h J of the 53-species
    mechanism, against numpy within its condition number."""
    m, r = mechs["ch4"], ref["ch4"]
    T, C, p = inputs.random_states(m, 2, seed=51)
    rng = np.random.default_rng(1)
    for c in range(2):
        J = r.jacobian(T[c], C[c], oracle.CONP)[0]
        for h in (1e-9, 1e-7):
            G = np.eye(m.ns + 1) - (4.0 / 15.0) * h * J
            b = rng.standard_normal(m.ns + 1)
            x = oracle.lu_solve(G, b)
            kappa = np.linalg.cond(G)
            np.testing.assert_allclose(G @ x, b, atol=1e-14 * kappa * np.abs(b).max())
