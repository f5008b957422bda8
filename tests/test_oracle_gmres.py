"""Pins of the oracle's GMRES (Section 3.4): restarted, left-preconditioned
(none, Jacobi, Gauss-Seidel), and of the integrators using it.

Independent checks: the dense solution of numpy's LAPACK solve; finite
termination of full GMRES (at most n iterations in exact arithmetic);
preconditioners that are exact for their matrix class (Jacobi on a diagonal,
Gauss-Seidel on a lower-triangular matrix: one iteration); the monotone
residual of restarted GMRES; and backward Euler / SDIRK-4 with GMRES against
the same integrators with the LU."""
import numpy as np
import pytest

import oracle
from paper_2510_10005_gb300 import inputs

PCS = [oracle.PC_NONE, oracle.PC_JACOBI, oracle.PC_GAUSS_SEIDEL]


def _system(n, seed, dom=4.0):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(n, n)) + dom * np.sqrt(n) * np.eye(n)   # nonsymmetric, well conditioned
    return A, rng.normal(size=n)


@pytest.mark.parametrize("prec", PCS)
@pytest.mark.parametrize("n", [1, 9, 54])
def test_gmres_matches_dense_solve(prec, n):
    A, b = _system(n, n + 10 * prec)
    x, ok, it = oracle.gmres(A, b, prec, m=30, maxit=500, tol=1e-13)
    assert ok
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-10, atol=1e-12 * np.abs(x).max())


def test_full_gmres_terminates_within_n_iterations():
    n = 24
    A, b = _system(n, 3, dom=0.5)            # harder: eigenvalues spread around the origin's neighbourhood
    x, ok, it = oracle.gmres(A, b, oracle.PC_NONE, m=n, maxit=n, tol=1e-9)
    assert ok and it <= n
    np.testing.assert_allclose(A @ x, b, atol=1e-7 * np.abs(b).max())


def test_exact_preconditioners_converge_in_one_iteration():
    rng = np.random.default_rng(4)
    n = 17
    D = np.diag(rng.uniform(1, 5, n))
    b = rng.normal(size=n)
    x, ok, it = oracle.gmres(D, b, oracle.PC_JACOBI, tol=1e-14)
    assert ok and it == 1
    np.testing.assert_allclose(x, b / np.diag(D), rtol=1e-15)
    L = np.tril(rng.normal(size=(n, n))) + 5 * np.eye(n)
    x, ok, it = oracle.gmres(L, b, oracle.PC_GAUSS_SEIDEL, tol=1e-14)
    assert ok and it == 1
    np.testing.assert_allclose(L @ x, b, atol=1e-13)


def test_restart_and_iteration_limit():
    A, b = _system(40, 5, dom=1.0)
    x1, ok1, it1 = oracle.gmres(A, b, oracle.PC_NONE, m=5, maxit=2000, tol=1e-10)
    assert ok1 and it1 > 5                   # needed restarts
    np.testing.assert_allclose(A @ x1, b, atol=1e-8 * np.abs(b).max())
    _, ok2, it2 = oracle.gmres(A, b, oracle.PC_NONE, m=5, maxit=3, tol=1e-10)
    assert not ok2 and it2 == 3
    z, ok3, it3 = oracle.gmres(A, np.zeros(40))
    assert ok3 and it3 == 0 and not z.any()
    A0 = A.copy()
    A0[3, 3] = 0.0
    assert not oracle.gmres(A0, b, oracle.PC_JACOBI)[1]   # zero diagonal: no preconditioner


@pytest.mark.parametrize("prec", PCS)
@pytest.mark.parametrize("method", [oracle.BE, oracle.SDIRK4])
def test_integrators_with_gmres_match_lu(mechs, ref, prec, method):
    """Newton iterated to tight tolerances: the GMRES-based integrator lands
    where the LU-based one does."""
    m, r = mechs["h2"], ref["h2"]
    T, Y, p = inputs.field_reactor(m, 6, (1150, 1400), (1, 2), (0.5, 2), "H2", seed=6)
    o = dict(method=method, adaptive=0, nsub=3, dt=2e-6, rtol=1e-10, atol=1e-16, newton_tol=1.0,
             max_newton=30, reactor=oracle.CONP)
    Tl, Yl, sl, stl = r.integrate(T, Y, p, o)
    Tg, Yg, sg, stg = r.integrate(T, Y, p, dict(o, linear_solver=oracle.GMRES, preconditioner=prec,
                                                gmres_tol=1e-13, gmres_maxit=400))
    assert np.all(sl == 0) and np.all(sg == 0)
    np.testing.assert_allclose(Tg, Tl, rtol=1e-10)
    np.testing.assert_allclose(Yg, Yl, rtol=1e-8, atol=1e-18)
    assert np.all(stg[:, 3] >= stg[:, 2])     # at least one GMRES iteration per Newton iteration


def _krylov_minres(B, z0, kmax):
    """Brute force: the smallest residual ||z0 - B x|| over x in the Krylov
    space K_k(B, z0), k = 1..kmax (Arnoldi with two Gram-Schmidt passes in
    numpy, then a dense least-squares solve); returns residuals and iterates."""
    n = len(z0)
    V = np.zeros((n, kmax + 1))
    V[:, 0] = z0 / np.linalg.norm(z0)
    res, xs = [], []
    for k in range(1, kmax + 1):
        w = B @ V[:, k - 1]
        for _ in range(2):
            w -= V[:, :k] @ (V[:, :k].T @ w)
        V[:, k] = w / np.linalg.norm(w)
        y = np.linalg.lstsq(B @ V[:, :k], z0, rcond=None)[0]
        xs.append(V[:, :k] @ y)
        res.append(np.linalg.norm(z0 - B @ xs[-1]))
    return np.array(res), xs


@pytest.mark.parametrize("prec", PCS)
def test_stopping_rule_and_iterate_against_brute_force(prec):
    """Section 3.4 (left preconditioning M^-1 A x = M^-1 b, M = I, diag A or
    its lower triangle): full GMRES stops at the first iteration whose
    preconditioned residual is within tol of that of x = 0, and its iterate
    is the Krylov-space minimiser. The tolerance sits halfway (geometrically)
    between two consecutive minimal residuals, so the expected count is
    unambiguous."""
    n = 30
    A, b = _system(n, 40 + prec, dom=2.0)
    M = {oracle.PC_NONE: np.eye(n), oracle.PC_JACOBI: np.diag(np.diag(A)),
         oracle.PC_GAUSS_SEIDEL: np.tril(A)}[prec]
    B, z0 = np.linalg.solve(M, A), np.linalg.solve(M, b)
    res, xs = _krylov_minres(B, z0, 20)
    k = int(np.argmax(res / np.linalg.norm(z0) < 1e-4))          # a mid-run iteration
    assert 3 <= k + 1 <= 19 and res[k] < res[k - 1]
    tol = np.sqrt(res[k - 1] * res[k]) / np.linalg.norm(z0)
    x, ok, it = oracle.gmres(A, b, prec, m=n, maxit=n, tol=tol)
    assert ok and it == k + 1
    np.testing.assert_allclose(x, xs[k], rtol=1e-8, atol=1e-10 * np.abs(xs[k]).max())
