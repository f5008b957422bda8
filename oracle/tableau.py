"""ORACLE -- test infrastructure only.

Butcher tableaux of the implicit schemes, Appendix A of the paper.

SDIRK-2 (Appendix A.1): gamma = 1 - sqrt(2)/2, a21 = 1 - gamma,
b = (1 - gamma, gamma). Embedded first-order solution: b_hat = (1, 0).

SDIRK-4 (Appendix A.2): five stages, a_ii = 4/15, coefficients printed to
seven digits, with a_52 missing from the list. Reading taken here:
  * the scheme is stiffly accurate (row 5 of A equals b), so a_52 = b_2;
  * the printed row sums give c2 = 23/30 and c3 = 17/30 (a31 + a32 = 3/10);
  * full-precision coefficients are the root, nearest the printed values, of
    the eight order-4 conditions for (a31, a32, a41, a42, a43, a51..a54) with
    a21 = 1/2 and a31 + a32 = 3/10 held fixed (nine equations, nine unknowns).
Embedded third-order solution (not given by the paper): b_hat with
b_hat_5 = 0 from the four order-<=3 conditions.
"""
from __future__ import annotations

import numpy as np

GAMMA4 = 4.0 / 15.0

# Appendix A.2, as printed
PRINTED_SDIRK4 = {
    "a21": 0.5, "a31": 3.541539e-1, "a32": -5.415395e-2, "a41": 8.515494e-2,
    "a42": -6.484332e-2, "a43": 7.915325e-2, "a51": 2.100115, "a53": 2.399816,
    "a54": -2.998818, "b1": 2.100115, "b2": -7.677800e-1, "b3": 2.399816,
    "b4": -2.998818, "b5": 0.2666666666666667,
}


def _sdirk4_matrix(x, one=1.0):
    a31, a32, a41, a42, a43, a51, a52, a53, a54 = x
    g = one * 4 / 15
    z = one * 0
    return [[g, z, z, z, z],
            [one / 2, g, z, z, z],
            [a31, a32, g, z, z],
            [a41, a42, a43, g, z],
            [a51, a52, a53, a54, g]]


def order_conditions(A, b, order):
    """Residuals of the Runge-Kutta order conditions up to the given order
    (all trees of order <= 4), with c = row sums of A. Works on floats or
    decimal.Decimal entries (plain Python lists or numpy arrays)."""
    s = len(b)
    A = [[A[i][j] for j in range(s)] for i in range(s)]
    b = [b[i] for i in range(s)]
    c = [sum(A[i]) for i in range(s)]
    Ac = [sum(A[i][j] * c[j] for j in range(s)) for i in range(s)]
    Ac2 = [sum(A[i][j] * c[j] ** 2 for j in range(s)) for i in range(s)]
    AAc = [sum(A[i][j] * Ac[j] for j in range(s)) for i in range(s)]
    one = b[0] * 0 + 1
    dot = lambda u, v: sum(u[i] * v[i] for i in range(s))
    res = [sum(b) - one]
    if order >= 2:
        res.append(dot(b, c) - one / 2)
    if order >= 3:
        res += [dot(b, [x ** 2 for x in c]) - one / 3, dot(b, Ac) - one / 6]
    if order >= 4:
        res += [dot(b, [x ** 3 for x in c]) - one / 4,
                dot(b, [c[i] * Ac[i] for i in range(s)]) - one / 8,
                dot(b, Ac2) - one / 12, dot(b, AAc) - one / 24]
    return res


def _residual(x, one):
    A = _sdirk4_matrix(x, one)
    r = order_conditions(A, A[4], 4)
    return r + [x[0] + x[1] - one * 3 / 10]


def _solve(M, r):
    """Gaussian elimination with partial pivoting on lists (Decimal entries)."""
    n = len(r)
    M = [row[:] + [r[i]] for i, row in enumerate(M)]
    for k in range(n):
        p = max(range(k, n), key=lambda i: abs(M[i][k]))
        M[k], M[p] = M[p], M[k]
        for i in range(k + 1, n):
            f = M[i][k] / M[k][k]
            for j in range(k, n + 1):
                M[i][j] -= f * M[k][j]
    x = [0] * n
    for i in range(n - 1, -1, -1):
        x[i] = (M[i][n] - sum(M[i][j] * x[j] for j in range(i + 1, n))) / M[i][i]
    return x


def sdirk4_full_precision():
    """Newton iteration in 50-digit decimal arithmetic from the printed values;
    returns the 5x5 matrix A (numpy, rounded to double) with residual of the
    order conditions below 1e-40 before rounding."""
    import decimal
    ctx = decimal.Context(prec=50)
    D = lambda v: ctx.create_decimal(v if isinstance(v, str) else repr(v))
    one = D(1)
    p = PRINTED_SDIRK4
    x = [D(p[k]) for k in ("a31", "a32", "a41", "a42", "a43", "a51", "b2", "a53", "a54")]
    with decimal.localcontext(ctx):
        eps = D("1e-22")
        for _ in range(30):
            r = _residual(x, one)
            cols = []
            for k in range(9):
                xp = list(x); xp[k] += eps
                xm = list(x); xm[k] -= eps
                rp, rm = _residual(xp, one), _residual(xm, one)
                cols.append([(rp[i] - rm[i]) / (2 * eps) for i in range(9)])
            Jm = [[cols[k][i] for k in range(9)] for i in range(9)]
            step = _solve(Jm, [-v for v in r])
            x = [x[i] + step[i] for i in range(9)]
            if max(abs(v) for v in _residual(x, one)) < D("1e-40"):
                break
        assert max(abs(v) for v in _residual(x, one)) < D("1e-40")
    A = _sdirk4_matrix(x, one)
    return np.array([[float(v) for v in row] for row in A])


def embedded_weights(A, order, s_used):
    """Weights b_hat over the first s_used stages satisfying the order
    conditions up to `order` (one linear system, as many conditions as stages)."""
    A = np.asarray(A, dtype=float)
    c = A.sum(axis=1)
    rows, rhs = [np.ones(s_used)], [1.0]
    if order >= 2:
        rows.append(c[:s_used]); rhs.append(0.5)
    if order >= 3:
        rows.append(c[:s_used] ** 2); rhs.append(1.0 / 3)
        rows.append((A @ c)[:s_used]); rhs.append(1.0 / 6)
    M = np.array(rows)
    bh = np.zeros(A.shape[0])
    bh[:s_used] = np.linalg.solve(M, np.array(rhs))
    return bh


def tableau(method: int):
    """Return dict(s, A[5x5], b[5], bhat[5], err_order) for
    method 0 = backward Euler, 1 = SDIRK-2, 2 = SDIRK-4; 3 = Rosenbrock-2
    and 4 = YASS carry only their stage count and embedded order here (the
    oracle evaluates their coefficients itself)."""
    A = np.zeros((5, 5)); b = np.zeros(5); bh = np.zeros(5)
    if method == 0:
        A[0, 0] = 1.0; b[0] = 1.0
        return dict(s=1, A=A, b=b, bhat=bh, err_order=0)
    if method == 1:
        g = 1.0 - np.sqrt(2.0) / 2.0
        A[0, 0] = g; A[1, 0] = 1.0 - g; A[1, 1] = g
        b[:2] = (1.0 - g, g)
        bh[:2] = (1.0, 0.0)
        return dict(s=2, A=A, b=b, bhat=bh, err_order=1)
    if method == 2:
        A = sdirk4_full_precision()
        b = A[4].copy()
        bh = embedded_weights(A, 3, 4)
        return dict(s=5, A=A, b=b, bhat=bh, err_order=3)
    if method == 3:
        return dict(s=2, A=A, b=b, bhat=bh, err_order=1)
    if method == 4:
        return dict(s=1, A=A, b=b, bhat=bh, err_order=0)
    raise ValueError(method)


def pack(t) -> np.ndarray:
    """Flatten a tableau into the oracle's 37-double layout."""
    out = np.zeros(37)
    out[0] = t["s"]; out[1] = t["err_order"]
    out[2:27] = np.asarray(t["A"]).reshape(25)
    out[27:32] = t["b"]; out[32:37] = t["bhat"]
    return out
