"""Pins of the oracle's operator-split reaction step (Section 5.5): the
source R_i = W_i (C_i^{n+1} - C_i^n)/dt of the species equations conserves
mass and elements, the internal energy the flow solver holds is unchanged
by the chemistry at constant volume (so it gives back the new temperature),
and the step is the constant-volume integration of the same state."""
import numpy as np
import pytest

import oracle
from paper_2510_10005_gb300 import inputs


def _flow_state(m, r, n, seed):
    T, Y, p = inputs.field_reactor(m, n, (1100, 1500), (1, 3), (0.5, 2.0), "H2", seed=seed)
    rho = p / (inputs.R_UNIV * T * (Y / m.W).sum(axis=1))
    u = np.array([Y[c] @ r.thermo(T[c])["u"] for c in range(n)])
    return T, Y, rho, u


@pytest.mark.parametrize("method", [oracle.BE, oracle.SDIRK4])
def test_split_step_conserves_and_matches_integration(mechs, ref, method):
    m, r = mechs["h2"], ref["h2"]
    T, Y, rho, u = _flow_state(m, r, 12, seed=8)
    o = dict(method=method, adaptive=int(method != oracle.BE), dt=1e-5, rtol=1e-10, atol=1e-16,  # tight
             newton_tol=1.0 if method == oracle.BE else 1e-3, max_newton=20, reactor=oracle.CONV)
    rhoY = rho[:, None] * Y
    guess = T * 1.07                                     # the flow solver's stale temperature
    T1, R, st, _ = r.react_split(rho, u, rhoY, guess, o)
    assert np.all(st == 0)
    # R is a difference of states over dt: its rounding is that of rhoY / dt
    floor = 1e-14 * rhoY.sum(axis=1) / o["dt"]
    assert np.all(np.abs(R.sum(axis=1)) <= 1e-12 * np.abs(R).sum(axis=1) + floor)          # mass
    el = (R / m.W) @ m.comp                                                                # kmol / m^3 / s
    el_floor = 1e-14 * ((rhoY / m.W) @ m.comp) / o["dt"]
    assert np.all(np.abs(el) <= 1e-11 * (np.abs(R / m.W) @ m.comp) + el_floor)             # elements
    # the energy is that of the new state: recovering T from it gives T1 (to
    # the integrator's truncation error: backward Euler does not conserve the
    # nonlinear u(T) over a large step, SDIRK-4 at rtol 1e-10 does to rounding)
    Y1 = (rhoY + R * o["dt"]) / rho[:, None]
    Tr = r.temperature(u, Y1, T1 * 0.97, 8, oracle.CONV)
    np.testing.assert_allclose(Tr, T1, rtol=1e-12 if method == oracle.SDIRK4 else 1e-2)
    # and the step is the constant-volume integration of (T, Y, rho)
    Ti, Yi, st2, _ = r.integrate(T, Y, rho, o)
    assert np.all(st2 == 0)
    np.testing.assert_allclose(T1, Ti, rtol=1e-9)
    np.testing.assert_allclose(Y1, Yi, rtol=1e-7, atol=1e-16)
    assert np.abs(R).max() > 0
