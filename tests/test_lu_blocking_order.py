"""The blocked LU's order of operations (CPU, no GPU).

The library's blocked factorisation (right-looking, panels of nb columns,
partial pivoting with whole rows swapped, U12 by forward substitution, the
trailing block updated from RA x CB register tiles whose reads clamp at
the ragged edge and whose writes are masked) is claimed to give every
entry of the matrix the same multiply-adds, in the same order, as the
column-by-column factorisation, so that both produce the same bits. This
test replays both orders in IEEE doubles (numpy scalars, one rounding per
operation on both sides) on matrices whose entries span many orders of
magnitude (so that pivoting swaps rows inside panels), for panel widths
that divide n, that do not, and that exceed it: pivots and factors must be
identical to the last bit, and P A = L U must hold."""
import numpy as np
import pytest


def _pivot(G, k, piv):
    """Column k: the largest |G_ik|, i >= k (the lowest row on ties), whole
    rows swapped, the column below the pivot scaled by its reciprocal."""
    bi = k + int(np.argmax(np.abs(G[k:, k])))
    piv[k] = bi
    if bi != k:
        G[[k, bi], :] = G[[bi, k], :]
    r = 1.0 / G[k, k]
    G[k + 1:, k] = G[k + 1:, k] * r


def lu_by_columns(A):
    G, n = A.copy(), A.shape[0]
    piv = np.zeros(n, dtype=int)
    for k in range(n):
        _pivot(G, k, piv)
        for i in range(k + 1, n):
            for c in range(k + 1, n):
                G[i, c] = G[i, c] + (-G[i, k]) * G[k, c]
    return G, piv


def lu_by_panels(A, nb, RA=4, CB=4):
    G, n = A.copy(), A.shape[0]
    piv = np.zeros(n, dtype=int)
    for k0 in range(0, n, nb):
        kend = min(k0 + nb, n)
        for k in range(k0, kend):            # the panel: its own columns only
            _pivot(G, k, piv)
            for i in range(k + 1, n):
                for c in range(k + 1, kend):
                    G[i, c] = G[i, c] + (-G[i, k]) * G[k, c]
        m = n - kend
        if m <= 0:
            break
        for c in range(kend, n):               # U12 = L11^-1 A12, one column at a time
            for i in range(k0 + 1, kend):
                a = G[i, c]
                for j in range(k0, i):
                    a = a + (-G[i, j]) * G[j, c]
                G[i, c] = a
        # trailing block: tile t covers rows tr + a*TR and columns tc + b*TC
        TR, TC = -(-m // RA), -(-m // CB)
        for t in range(TR * TC):
            tr, tc = divmod(t, TC)
            rows = [tr + a * TR for a in range(RA)]
            cols = [tc + b * TC for b in range(CB)]
            rr = [min(r, m - 1) for r in rows]   # clamped reads at the ragged edge
            cc = [min(c, m - 1) for c in cols]
            acc = [[G[kend + rr[a], kend + cc[b]] for b in range(CB)] for a in range(RA)]
            for j in range(kend - k0):
                lv = [G[kend + rr[a], k0 + j] for a in range(RA)]
                uv = [G[k0 + j, kend + cc[b]] for b in range(CB)]
                for a in range(RA):
                    for b in range(CB):
                        acc[a][b] = acc[a][b] + (-lv[a]) * uv[b]
            for a in range(RA):
                for b in range(CB):
                    if rows[a] < m and cols[b] < m:   # masked writes
                        G[kend + rows[a], kend + cols[b]] = acc[a][b]
    return G, piv


@pytest.mark.parametrize("n", [10, 17, 54])
def test_panels_give_the_column_order_bit_for_bit(n):
    rng = np.random.default_rng(n)
    for _ in range(2):
        A = rng.normal(size=(n, n)) * np.exp(3.0 * rng.normal(size=(n, n)))
        Gc, pc = lu_by_columns(A)
        assert (pc != np.arange(n)).any()      # rows were swapped
        for nb in (1, 3, 5, 8, 16, 64):
            Gp, pp = lu_by_panels(A, nb)
            np.testing.assert_array_equal(pp, pc)
            assert np.array_equal(Gp.view(np.int64), Gc.view(np.int64)), (nb, np.abs(Gp - Gc).max())
        L, U = np.tril(Gc, -1) + np.eye(n), np.triu(Gc)
        PA = A.copy()
        for k in range(n):
            PA[[k, pc[k]]] = PA[[pc[k], k]]
        np.testing.assert_allclose(L @ U, PA, rtol=1e-10, atol=1e-10 * np.abs(A).max())


def test_a_wrong_order_is_detected():
    """Updating the panel rows' right part column by column inside the panel
    (before later pivots of the same panel) is the order the first blocked
    version had: a later swap then moves a row that missed updates, and the
    bits differ. The replay above must be able to see such a mistake."""
    n, nb = 17, 8
    rng = np.random.default_rng(3)
    A = rng.normal(size=(n, n)) * np.exp(3.0 * rng.normal(size=(n, n)))
    Gc, pc = lu_by_columns(A)
    G = A.copy()
    piv = np.zeros(n, dtype=int)
    for k0 in range(0, n, nb):
        kend = min(k0 + nb, n)
        for k in range(k0, kend):
            _pivot(G, k, piv)
            for i in range(k + 1, n):
                for c in range(k + 1, kend):
                    G[i, c] = G[i, c] + (-G[i, k]) * G[k, c]
            for c in range(kend, n):           # the panel row's right part, too early
                G[k + 1:kend, c] = G[k + 1:kend, c] + (-G[k + 1:kend, k]) * G[k, c]
        for i in range(kend, n):
            for c in range(kend, n):
                for j in range(k0, kend):
                    G[i, c] = G[i, c] + (-G[i, j]) * G[j, c]
    assert not np.array_equal(G.view(np.int64), Gc.view(np.int64))
