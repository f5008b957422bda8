"""Pins of the oracle's second-order Rosenbrock (Appendix A.3) and YASS
(Appendix A.4) integrators.

Rosenbrock-2: on y' = lambda y a two-stage Rosenbrock method of order 2
with diagonal gamma has the stability function
R(z) = (1 + (1 - 2 gamma) z + (gamma^2 - 2 gamma + 1/2) z^2) / (1 - gamma z)^2
(the order conditions of two-stage Rosenbrock methods; with
gamma = 1 + sqrt(2)/2 the z^2 term vanishes and R(-inf) = 0, L-stability);
classical order 2 on a non-stiff problem and at the ignition point. The
scheme printed with an extra -S(y_n) in its second stage fails all three.
YASS: one backward-Euler Newton step from y_n, exact backward Euler on a
linear problem; first order; halving when the decrement's norm exceeds
alpha."""
import numpy as np
import pytest

import oracle
from paper_2510_10005_gb300 import inputs

GAMMA = 1.0 + np.sqrt(2.0) / 2.0
FIXED = dict(adaptive=0, rtol=1e-12, atol=1e-20, newton_tol=1e300, max_newton=20, reactor=oracle.CONV,
             neg_tol=1e300)


def r_ros2(z):
    g = GAMMA
    return (1 + (1 - 2 * g) * z + (g * g - 2 * g + 0.5) * z * z) / (1 - g * z) ** 2


@pytest.mark.parametrize("nsub", [1, 4])
@pytest.mark.parametrize("kdt", [0.01, 3.0, 300.0])
def test_ros2_stability_function(nsub, kdt):
    k = 1e5
    dt = kdt / k
    r = oracle.RefMech(inputs.isomer_mechanism(k, reversible=False))
    y, st, stats = r.integrate_y(np.array([[1000.0, 0.03, 0.002]]), dict(FIXED, method=oracle.ROS2, dt=dt,
                                                                            nsub=nsub))
    assert st[0] == 0
    assert y[0, 1] == pytest.approx(0.03 * r_ros2(-kdt / nsub) ** nsub, rel=1e-12)
    assert y[0, 1] + y[0, 2] == pytest.approx(0.032, rel=1e-15)
    assert stats[0, 2] == nsub and stats[0, 3] == nsub     # one factorisation per step


def test_ros2_l_stable():
    assert abs(GAMMA * GAMMA - 2 * GAMMA + 0.5) < 1e-15
    z = -np.logspace(-3, 8, 50)
    assert np.all(np.abs(r_ros2(z)) <= 1.0) and abs(r_ros2(-1e12)) < 1e-11


@pytest.mark.parametrize("method,order", [(oracle.ROS2, 2), (oracle.YASS, 1)])
def test_classical_order_nonstiff(method, order):
    k, dt = 1.0e5, 2e-5
    r = oracle.RefMech(inputs.isomer_mechanism(k, reversible=False))
    y0 = np.array([[1000.0, 0.03, 0.0]])
    errs = []
    for rr in range(5, 10):   # k h from 0.06 down to 0.004: the asymptotic regime
        y, st, _ = r.integrate_y(y0, dict(FIXED, method=method, dt=dt, nsub=2**rr))
        assert st[0] == 0
        errs.append(abs(y[0, 1] - 0.03 * np.exp(-k * dt)))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(slopes - order) < 0.15), slopes


def test_ros2_order_at_ignition(mechs, ref):
    """Section 5.3's study for the Rosenbrock scheme: second order at the
    point of largest dT/dt (exact Jacobian, so no order reduction to one)."""
    m, r = mechs["h2"], ref["h2"]
    T, Y, p = inputs.field_reactor(m, 1, (1200, 1200), (1, 1), (1, 1), "H2", seed=0)
    y0 = np.concatenate([T[:, None], r.concentrations(T, Y, p, oracle.CONP)], axis=1)
    y0, st, _ = r.integrate_y(y0, dict(method=oracle.SDIRK4, adaptive=1, dt=4.8e-5, rtol=1e-10, atol=1e-16,
                                       reactor=oracle.CONV))
    assert st[0] == 0
    opts = dict(FIXED, method=oracle.ROS2, dt=1e-7)
    yref, st, _ = r.integrate_y(y0, dict(opts, nsub=2**10))
    errs = []
    for rr in range(1, 6):
        y, st, _ = r.integrate_y(y0, dict(opts, nsub=2**rr))
        assert st[0] == 0
        errs.append(np.sqrt(np.sum((y[0, 1:] - yref[0, 1:]) ** 2)))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(slopes > 1.8) and np.all(slopes < 2.3), (errs, slopes)


def test_ros2_adaptive_matches_tight_reference(mechs, ref):
    m, r = mechs["h2"], ref["h2"]
    T, Y, p = inputs.field_reactor(m, 8, (1100, 1400), (1, 1), (0.5, 2), "H2", seed=5)
    base = dict(dt=5e-6, reactor=oracle.CONP, adaptive=1, atol=1e-14)
    Ta, Ya, st, stats = r.integrate(T, Y, p, dict(base, method=oracle.ROS2, rtol=1e-7))
    Tr, Yr, st2, _ = r.integrate(T, Y, p, dict(base, method=oracle.SDIRK4, rtol=1e-11, atol=1e-18))
    assert np.all(st == 0) and np.all(st2 == 0)
    assert np.all(stats[:, 0] > 3)           # several accepted steps
    np.testing.assert_allclose(Ta, Tr, rtol=2e-5)
    np.testing.assert_allclose(Ya, Yr, atol=2e-6)


@pytest.mark.parametrize("nsub", [1, 3])
def test_yass_is_one_backward_euler_newton_step(nsub):
    """On a linear problem one Newton step is the backward-Euler solution:
    C_A0 (1 - z)^-n."""
    k, dt = 3e5, 1e-5
    r = oracle.RefMech(inputs.isomer_mechanism(k, reversible=False))
    y, st, stats = r.integrate_y(np.array([[1000.0, 0.03, 0.002]]), dict(FIXED, method=oracle.YASS, dt=dt,
                                                                            nsub=nsub))
    assert st[0] == 0 and stats[0, 2] == nsub
    assert y[0, 1] == pytest.approx(0.03 * (1 + k * dt / nsub) ** -nsub, rel=1e-13)


def test_yass_halves_when_the_decrement_is_large():
    """A -> B: the full step's decrement is z C_A/(1 - z) in A and B; with
    alpha between the WRMS norms of the full and the half step, YASS halves
    once and takes two half steps."""
    k, dt, C0 = 1e5, 1e-5, 0.03
    r = oracle.RefMech(inputs.isomer_mechanism(k, reversible=False))
    rtol, atol = 1e-3, 1e-12

    def norm(h, CA):
        d = k * h * CA / (1 + k * h)             # |decrement| of A and of B
        wA = atol + rtol * CA                    # max(|y_n|, |y_n+1|) = C_A for A ...
        wB = atol + rtol * d                     # ... and the new B for B (B starts at 0)
        return np.sqrt(((d / wA) ** 2 + (d / wB) ** 2) / 3)

    full, half = norm(dt, C0), norm(dt / 2, C0)
    alpha = np.sqrt(full * half)
    assert half < alpha < full
    y, st, stats = r.integrate_y(np.array([[1000.0, C0, 0.0]]),
                                 dict(FIXED, method=oracle.YASS, dt=dt, rtol=rtol, atol=atol, newton_tol=alpha))
    assert st[0] == 0
    assert stats[0, 0] == 2 and stats[0, 1] == 1            # two accepted half steps, one rejection
    assert y[0, 1] == pytest.approx(C0 * (1 + k * dt / 2) ** -2, rel=1e-13)
    # alpha = 0: every step fails down to max_halvings
    _, st, _ = r.integrate_y(np.array([[1000.0, C0, 0.0]]),
                             dict(FIXED, method=oracle.YASS, dt=dt, newton_tol=0.0, max_halvings=3))
    assert st[0] == 1
