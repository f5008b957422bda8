"""Tolerance checks of the GPU parity tests, and a record of the largest
error each check measured.

Adaptive integration (error control with rtol, atol on the state y = (T, C),
weights w_i = atol + rtol |y_i|): the CUDA path and the oracle run the same
algorithm, so they agree to rounding while they take the same steps; where an
accept/reject decision sits at the threshold, each side's result is a valid
integration within the tolerance of the other. Element-wise bound, on every
species of every cell:

    |T_gpu - T_ref|     <= c (rtol T_ref + atol)
    |Y_k,gpu - Y_k,ref| <= c (rtol |Y_k,ref| + atol W_k / rho)

with rho the end-state density (atol is a concentration, kmol/m^3, so its
weight in mass-fraction units is atol W_k / rho) and c = 1: the integrator's
own per-component weight. (Flipping accept/reject decisions of the oracle
against itself, by a relative change of 1e-3 of rtol, moves no component by
more than 1e-3 of this bound.)

Fixed steps (Newton iterated until its change is below 1e-10 of the state):
relative `rel` on T and on every Y_k, with an absolute floor below which a
mass fraction carries no more digits than the Newton tolerance leaves it.

Every check stores its largest error under the test's name in REPORT; with
CHEMGB_PARITY_REPORT set to a file name, tests/conftest.py writes REPORT
there as JSON at the end of the session.
"""
import numpy as np

R_UNIV = 8314.46261815324
CONV = 0
REPORT = {}


def record(name, **values):
    entry = REPORT.setdefault(name, {})
    for k, v in values.items():
        v = float(v) if np.ndim(v) == 0 else v
        entry[k] = max(entry.get(k, v), v) if isinstance(v, float) else v


def end_density(m, T, Y, p_or_rho, reactor):
    """rho of the end state: the given density at constant volume, the ideal
    gas p / (R T sum Y/W) otherwise."""
    if reactor == CONV:
        return np.asarray(p_or_rho, dtype=float)
    return p_or_rho / (R_UNIV * T * (Y / m.W).sum(axis=1))


def check_adaptive(name, m, Tg, Yg, To, Yo, p_or_rho, reactor, rtol, atol, c=1.0):
    """Element-wise bound of the module docstring; returns the largest ratio
    error / bound over T and Y."""
    Tg, Yg, To, Yo = (np.asarray(a, dtype=float) for a in (Tg, Yg, To, Yo))
    rho = end_density(m, To, Yo, p_or_rho, reactor)
    bT = c * (rtol * np.abs(To) + atol)
    bY = c * (rtol * np.abs(Yo) + atol * m.W[None, :] / rho[:, None])
    rT = np.abs(Tg - To) / bT
    rY = np.abs(Yg - Yo) / bY
    record(name, cells=len(To), T_rel=np.max(np.abs(Tg - To) / np.abs(To)), Y_abs=np.max(np.abs(Yg - Yo)),
           T_over_bound=rT.max(), Y_over_bound=rY.max())
    assert rT.max() <= 1.0, ("T", int(np.argmax(rT)), rT.max())
    bad = np.argwhere(rY > 1.0)
    assert len(bad) == 0, ("Y (cell, species)", bad[:5], rY[rY > 1.0][:5])
    return max(rT.max(), rY.max())


def check_fixed(name, Tg, Yg, To, Yo, rel, floor):
    """|dT| <= rel T and |dY_k| <= rel |Y_k| + floor."""
    Tg, Yg, To, Yo = (np.asarray(a, dtype=float) for a in (Tg, Yg, To, Yo))
    eT = np.abs(Tg - To) / np.abs(To)
    eY = np.abs(Yg - Yo)
    big = np.abs(Yo) > floor / rel
    record(name, cells=len(To), T_rel=eT.max() if eT.size else 0.0,
           Y_rel=np.max(eY[big] / np.abs(Yo[big])) if big.any() else 0.0, Y_abs=eY.max() if eY.size else 0.0)
    np.testing.assert_allclose(Tg, To, rtol=rel, atol=0)
    bad = eY > rel * np.abs(Yo) + floor
    assert not bad.any(), (np.argwhere(bad)[:5], eY[bad][:5], Yo[bad][:5])


def check_elementwise(name, a, b, rtol, floor):
    """|a - b| <= rtol |b| + floor max|b| (gradients: tiny entries are sums of
    cancelling terms, resolved only to the scale of the largest)."""
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    scale = max(np.abs(b).max(), 1e-300)
    err = np.abs(a - b)
    big = np.abs(b) > floor * scale / rtol
    record(name, rel=np.max(err[big] / np.abs(b[big])) if big.any() else 0.0, abs_over_max=err.max() / scale)
    bad = err > rtol * np.abs(b) + floor * scale
    assert not bad.any(), (np.argwhere(bad)[:5], err[bad][:5], b[bad][:5])
