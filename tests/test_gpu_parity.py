"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.

Tolerances (derived from the arithmetic):
  * omega: both sides sum the same terms nu_ij q_j in different orders, so
    the difference is bounded by a few ulp of sum_j |nu_ij q_j|; the test
    allows 1e-12 of that scale (the exps of rates and equilibrium constants
    are evaluated differently and differ by ~1e-15 relative).
  * J: 1e-10 of the entry plus 1e-12 of its row's largest entry.
  * Fixed-step integration (backward Euler, Newton iterated to 1e-10 of the
    state): relative 1e-10 on T and on every Y_k above 1e-12, absolute 1e-20
    below (the fixed-step parity bar, with the floor where a mass fraction
    carries no more digits than the Newton tolerance leaves it).
  * Adaptive integration: element-wise within the integrator's own weight,
    |dY_k| <= rtol |Y_k| + atol W_k / rho and |dT| <= rtol T + atol
    (tests/parity.py).
"""
import numpy as np
import pytest

import oracle
from paper_2510_10005_gb300 import chemgb, inputs
from parity import check_adaptive, check_fixed

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def handles(mechs):
    chemgb.load(build_if_missing=True)
    return {k: chemgb.cg_mech_create(m) for k, m in mechs.items()}


def d(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def gpu_rates(h, T, C, reactor):
    Tt, Ct = d(T), d(C.T)                      # SoA [ns][N]
    S = torch.empty((h.n, len(T)), dtype=torch.float64, device=DEV)
    chemgb.cg_eval_rates(h, reactor, Tt, Ct, S)
    torch.cuda.synchronize()
    return S.cpu().numpy().T                   # [N][n]


def nu_matrix(m):
    nu = np.zeros((m.ns, m.nr))
    for j in range(m.nr):
        for s in range(3):
            if m.rf_idx[j, s] >= 0:
                nu[m.rf_idx[j, s], j] -= m.rf_nu[j, s]
            if m.rr_idx[j, s] >= 0:
                nu[m.rr_idx[j, s], j] += m.rr_nu[j, s]
    return nu


@pytest.mark.parametrize("kind", ["h2", "ch4"])
@pytest.mark.parametrize("reactor", [chemgb.CG_CONV, chemgb.CG_CONP, chemgb.CG_CONP_LITERAL])
def test_rates_parity(mechs, ref, handles, kind, reactor):
    m, r, h = mechs[kind], ref[kind], handles[kind]
    T, C, p = inputs.random_states(m, 200, seed=101)   # Section 5.1 recipe; 200 = 6 warps of 32 + tail
    Sg = gpu_rates(h, T, C, reactor)
    So = r.source(T, C, reactor)
    nu = np.abs(nu_matrix(m))
    for c in range(len(T)):
        q = np.abs(r.rates(T[c], C[c])[2])
        scale = nu @ q
        if reactor == chemgb.CG_CONP:
            scale = scale + C[c] * (np.abs(So[c, 0]) / T[c] + scale.sum() / C[c].sum())
        th = r.thermo(T[c])
        e = th["u"] if reactor == chemgb.CG_CONV else th["h"]
        cv = th["cv"] if reactor == chemgb.CG_CONV else th["cp"]
        tscale = np.sum(np.abs(m.W * e) * (nu @ q)) / np.sum(m.W * C[c] * cv)
        assert abs(Sg[c, 0] - So[c, 0]) <= 1e-12 * tscale + 1e-12 * abs(So[c, 0])
        np.testing.assert_array_less(np.abs(Sg[c, 1:] - So[c, 1:]), 1e-12 * scale + 1e-300)


@pytest.mark.parametrize("kind", ["h2", "ch4"])
@pytest.mark.parametrize("reactor", [chemgb.CG_CONV, chemgb.CG_CONP])
def test_jacobian_parity(mechs, ref, handles, kind, reactor):
    m, r, h = mechs[kind], ref[kind], handles[kind]
    N = 37   # a ragged count
    T, C, p = inputs.random_states(m, N, seed=202)
    J = torch.empty((N, h.n, h.n), dtype=torch.float64, device=DEV)
    chemgb.cg_eval_jacobian(h, reactor, d(T), d(C.T), J)
    torch.cuda.synchronize()
    Jg = J.cpu().numpy()
    Jo = r.jacobian(T, C, reactor)
    rowmax = np.abs(Jo).max(axis=2, keepdims=True)
    err = np.abs(Jg - Jo)
    assert np.all(err <= 1e-10 * np.abs(Jo) + 1e-12 * rowmax)


def test_temperature_recovery_parity(mechs, ref, handles):
    m, r, h = mechs["ch4"], ref["ch4"], handles["ch4"]
    T, Y, p = inputs.field_flames(m, 300, seed=5)
    e = np.array([Y[c] @ r.thermo(T[c])["h"] for c in range(300)])
    T0 = T + 250.0
    To = r.temperature(e, Y, T0, iters=5, reactor=oracle.CONP)
    Tg = d(T0)
    chemgb.cg_temperature_from_energy(h, chemgb.CG_CONP, d(e), d(Y.T), Tg, 5)
    torch.cuda.synchronize()
    np.testing.assert_allclose(Tg.cpu().numpy(), To, rtol=1e-12)
    np.testing.assert_allclose(Tg.cpu().numpy(), T, rtol=1e-8)


def run_gpu(h, opts, T, Y, p):
    N = len(T)
    Tt, Yt, pt = d(T), d(Y.T), d(p)
    st = torch.empty(N, dtype=torch.int32, device=DEV)
    stats = torch.empty((4, N), dtype=torch.int32, device=DEV)
    chemgb.cg_integrate(h, opts, Tt, Yt, pt, st, stats)
    torch.cuda.synchronize()
    return Tt.cpu().numpy(), Yt.cpu().numpy().T, st.cpu().numpy(), stats.cpu().numpy().T


BE_OPTS = dict(method=oracle.BE, adaptive=0, dt=1e-5, rtol=1e-10, atol=1e-16, newton_tol=1.0,
               max_newton=20, max_halvings=10, reactor=oracle.CONP)


def assert_state_close(Tg, Yg, To, Yo, rel, floor, name=None):
    import inspect
    check_fixed(name or inspect.stack()[1].function, Tg, Yg, To, Yo, rel, floor)


def test_backward_euler_parity_full_config(mechs, ref, handles):
    """9-species mechanism, constant pressure, one backward-Euler step of
    1e-5 s (plus halvings) on 4096 cells: T0 in U[1000, 1500] K, 1 atm,
    phi in U[0.5, 2]."""
    m, r, h = mechs["h2"], ref["h2"], handles["h2"]
    T, Y, p = inputs.field_reactor(m, 4096, (1000, 1500), (1, 1), (0.5, 2), "H2", seed=0)
    To, Yo, so, sto = r.integrate(T, Y, p, BE_OPTS, nthreads=8)
    Tg, Yg, sg, stg = run_gpu(h, chemgb.make_opts(**BE_OPTS), T, Y, p)
    assert np.all(so == 0)
    np.testing.assert_array_equal(sg, so)
    assert np.mean(np.all(stg == sto, axis=1)) > 0.99
    assert_state_close(Tg, Yg, To, Yo, 1e-10, 1e-22)


@pytest.mark.parametrize("method", [chemgb.CG_SDIRK2, chemgb.CG_SDIRK4])
def test_fixed_step_sdirk_parity(mechs, ref, handles, method):
    m, r, h = mechs["h2"], ref["h2"], handles["h2"]
    T, Y, p = inputs.field_reactor(m, 67, (1100, 1400), (1, 1), (0.5, 2), "H2", seed=3)
    o = dict(BE_OPTS, method=method, dt=2e-6, nsub=4)
    To, Yo, so, _ = r.integrate(T, Y, p, o, nthreads=8)
    Tg, Yg, sg, _ = run_gpu(h, chemgb.make_opts(**o), T, Y, p)
    np.testing.assert_array_equal(sg, so)
    assert_state_close(Tg, Yg, To, Yo, 1e-10, 1e-22)


ADAPT = dict(method=oracle.SDIRK4, adaptive=1, dt=1e-6, rtol=1e-6, atol=1e-12, newton_tol=0.03,
             max_newton=7, reactor=oracle.CONP)


def test_adaptive_sdirk4_parity_flame_field(mechs, ref, handles):
    """53-species mechanism, 1-D flame-like field (unburnt, front, burnt),
    SDIRK-4 with error control, rtol 1e-6: a stratified 128-cell sample."""
    m, r, h = mechs["ch4"], ref["ch4"], handles["ch4"]
    T, Y, p = inputs.field_flames(m, 4096, seed=0)
    idx = np.arange(0, 4096, 32)
    To, Yo, so, sto = r.integrate(T[idx], Y[idx], p[idx], ADAPT, nthreads=8)
    Tg, Yg, sg, stg = run_gpu(h, chemgb.make_opts(**ADAPT), T[idx], Y[idx], p[idx])
    np.testing.assert_array_equal(sg, so)
    assert np.all(so == 0)
    check_adaptive("adaptive_sdirk4_flame_128", m, Tg, Yg, To, Yo, p[idx], ADAPT["reactor"], ADAPT["rtol"],
                   ADAPT["atol"])
    # both sides take the same steps except where err sits at the threshold
    assert np.mean(np.all(stg == sto, axis=1)) > 0.9


def test_adaptive_sdirk4_parity_h2(mechs, ref, handles):
    m, r, h = mechs["h2"], ref["h2"], handles["h2"]
    T, Y, p = inputs.field_reactor(m, 100, (1000, 1500), (1, 1), (0.5, 2), "H2", seed=7)
    o = dict(ADAPT, dt=1e-5)
    To, Yo, so, _ = r.integrate(T, Y, p, o, nthreads=8)
    Tg, Yg, sg, _ = run_gpu(h, chemgb.make_opts(**o), T, Y, p)
    np.testing.assert_array_equal(sg, so)
    check_adaptive("adaptive_sdirk4_h2", m, Tg, Yg, To, Yo, p, o["reactor"], o["rtol"], o["atol"])


def test_edge_cases(mechs, ref, handles):
    m, h = mechs["h2"], handles["h2"]
    o = chemgb.make_opts(**BE_OPTS)
    # N = 0 is a no-op
    e = torch.empty(0, dtype=torch.float64, device=DEV)
    chemgb.cg_integrate(h, o, e, torch.empty((m.ns, 0), dtype=torch.float64, device=DEV), e)
    # one cell, and a non-finite cell next to a good one
    T, Y, p = inputs.field_reactor(m, 2, (1200, 1200), (1, 1), (1, 1), "H2", seed=1)
    T[0] = np.nan
    Tg, Yg, sg, stg = run_gpu(h, o, T, Y, p)
    assert sg[0] == chemgb.CG_CELL_NONFINITE and sg[1] == chemgb.CG_CELL_OK
    assert np.isnan(Tg[0]) and np.all(stg[0] == 0)
    Tg1, Yg1, sg1, _ = run_gpu(h, o, T[1:], Y[1:], p[1:])
    assert Tg1[0] == Tg[1] and np.array_equal(Yg1[0], Yg[1])   # cells are independent
    # failure statuses, as the oracle's
    r = ref["h2"]
    T, Y, p = inputs.field_reactor(m, 3, (1400, 1400), (1, 1), (1, 1), "H2", seed=0)
    for kw, want in ((dict(BE_OPTS, max_newton=1, max_halvings=0), 1),
                     (dict(ADAPT, dt=1e-4, max_steps=3), 3),
                     (dict(ADAPT, dt=1e-5, hmin=1e-3), 2)):
        _, _, sg, _ = run_gpu(h, chemgb.make_opts(**kw), T, Y, p)
        _, _, so, _ = r.integrate(T, Y, p, kw)
        assert np.all(sg == want) and np.all(so == want)


@pytest.mark.parametrize("kind,shapes", [("h2", [(32, 1), (32, 4), (64, 1)]),
                                         ("ch4", [(64, 1), (32, 1), (128, 1), (256, 1)])])
def test_launch_shapes_agree(mechs, kind, shapes):
    """Every team size / cells-per-block gives the same integration up to the
    summation order of team-wide reductions."""
    m = mechs[kind]
    h = chemgb.cg_mech_create(m)
    if kind == "h2":
        T, Y, p = inputs.field_reactor(m, 77, (1000, 1500), (1, 1), (0.5, 2), "H2", seed=12)
        o = chemgb.make_opts(**BE_OPTS)
    else:
        T, Y, p = inputs.field_flames(m, 4096, seed=2)
        idx = np.arange(2400, 2400 + 67)   # front cells: many steps
        T, Y, p = T[idx], Y[idx], p[idx]
        o = chemgb.make_opts(**ADAPT)
    res = []
    for team, tpb in shapes:
        chemgb.cg_mech_set_launch(h, team, tpb)
        assert chemgb.cg_mech_get_launch(h) == (team, tpb)
        res.append(run_gpu(h, o, T, Y, p))
    for Tg, Yg, sg, _ in res[1:]:
        np.testing.assert_array_equal(sg, res[0][2])
        np.testing.assert_allclose(Tg, res[0][0], rtol=1e-9)
        assert np.max(np.abs(Yg - res[0][1])) < 1e-9


def test_host_entry_point_matches_device(mechs, handles):
    m, h = mechs["h2"], handles["h2"]
    T, Y, p = inputs.field_reactor(m, 513, (1000, 1500), (1, 1), (0.5, 2), "H2", seed=9)
    o = chemgb.make_opts(**BE_OPTS)
    Tg, Yg, sg, stg = run_gpu(h, o, T, Y, p)
    Th, Yh, ph = T.copy(), np.ascontiguousarray(Y.T), p.copy()
    sh = np.zeros(513, np.int32)
    sth = np.zeros((4, 513), np.int32)
    chemgb.cg_integrate_host(h, o, Th, Yh, ph, sh, sth)
    np.testing.assert_array_equal(Th, Tg)
    np.testing.assert_array_equal(Yh.T, Yg)
    np.testing.assert_array_equal(sh, sg)
    np.testing.assert_array_equal(sth.T, stg)


# ---------------------------------------------------------------------------
# mixed precision: FP32 Newton matrix and LU, FP64 residual/rates/updates


def test_mixed_precision_backward_euler(mechs, ref, handles):
    """The inexact Newton with an FP32 LU converges to the FP64 root: with the
    Newton change required below 1e-10 of the state, T and Y agree with the
    FP64 oracle to 1e-8 relative. Steps of 1e-6 s: at 1e-5 s across ignition
    the backward-Euler equations have several admissible roots, and which one
    a Newton iteration reaches depends on its first iterates (both the exact
    and the inexact iteration are correct there)."""
    m, r, h = mechs["h2"], ref["h2"], handles["h2"]
    T, Y, p = inputs.field_reactor(m, 1024, (1000, 1500), (1, 1), (0.5, 2), "H2", seed=0)
    o = dict(BE_OPTS, dt=1e-6)
    To, Yo, so, sto = r.integrate(T, Y, p, o, nthreads=8)
    Tg, Yg, sg, stg = run_gpu(h, chemgb.make_opts(**o, precision=chemgb.CG_FP32LU), T, Y, p)
    assert np.all(sg == 0) and np.all(so == 0)
    same = np.all(stg[:, :2] == sto[:, :2], axis=1)
    assert same.mean() > 0.99
    assert_state_close(Tg[same], Yg[same], To[same], Yo[same], 1e-8, 1e-18)


def test_mixed_precision_fixed_sdirk4(mechs, ref, handles):
    m, r, h = mechs["h2"], ref["h2"], handles["h2"]
    T, Y, p = inputs.field_reactor(m, 67, (1100, 1400), (1, 1), (0.5, 2), "H2", seed=3)
    o = dict(BE_OPTS, method=chemgb.CG_SDIRK4, dt=2e-6, nsub=4)
    To, Yo, so, _ = r.integrate(T, Y, p, o, nthreads=8)
    Tg, Yg, sg, _ = run_gpu(h, chemgb.make_opts(**o, precision=chemgb.CG_FP32LU), T, Y, p)
    np.testing.assert_array_equal(sg, so)
    assert_state_close(Tg, Yg, To, Yo, 1e-8, 1e-18)


def test_mixed_precision_adaptive_flame(mechs, ref, handles):
    m, r, h = mechs["ch4"], ref["ch4"], handles["ch4"]
    T, Y, p = inputs.field_flames(m, 4096, seed=0)
    idx = np.arange(0, 4096, 32)
    To, Yo, so, _ = r.integrate(T[idx], Y[idx], p[idx], ADAPT, nthreads=8)
    Tg, Yg, sg, stg = run_gpu(h, chemgb.make_opts(**ADAPT, precision=chemgb.CG_FP32LU),
                              T[idx], Y[idx], p[idx])
    np.testing.assert_array_equal(sg, so)
    check_adaptive("fp32lu_adaptive_sdirk4_flame", m, Tg, Yg, To, Yo, p[idx], ADAPT["reactor"], ADAPT["rtol"],
                   ADAPT["atol"])


def test_table_exp_within_two_ulp_of_cuda_exp(handles):
    """exp_tab (Tang's table-driven method, used for every exponential of
    the rates) against CUDA's exp over the whole double range, the
    reduction boundaries and special values."""
    h = handles["h2"]
    rng = np.random.default_rng(3)
    xs = [rng.uniform(-745.0, 710.0, 200000), rng.uniform(-50.0, 50.0, 200000),
          rng.uniform(-1e-3, 1e-3, 20000),
          np.arange(-4096, 4096) * (np.log(2.0) / 128.0),          # midpoints of the reduction intervals
          np.array([0.0, -0.0, 1e-300, -1e-300, 706.9, -706.9, 707.0, -707.0, 708.0, 709.78, 710.0,
                    -745.1, -800.0, 1e308, -1e308, np.inf, -np.inf, np.nan])]
    x = np.concatenate(xs)
    xt = d(x)
    yt, yl = torch.empty_like(xt), torch.empty_like(xt)
    chemgb.cgx_exp_check(h, xt, yt, yl)
    torch.cuda.synchronize()
    a, b = yt.cpu().numpy(), yl.cpu().numpy()
    nan = np.isnan(b)
    assert np.array_equal(np.isnan(a), nan)
    ia = a[~nan].view(np.int64)
    ib = b[~nan].view(np.int64)
    assert np.max(np.abs(ia - ib)) <= 2          # positive doubles order like their bit patterns


def test_pivot_reciprocal_within_one_ulp():
    """rcp_nr (the LU's pivot reciprocal: two Newton-Raphson steps from the
    single-precision approximation) against the correctly rounded 1/x (IEEE
    division on the host): every binary exponent of the double range, both
    signs, the edges of its single-precision window (exponents +-125, where
    it switches to division), powers of two and subnormals."""
    rng = np.random.default_rng(5)
    e = np.arange(-1022, 1024)
    mant = rng.uniform(1.0, 2.0, (len(e), 16))
    x = (mant * np.ldexp(1.0, e)[:, None]).ravel()
    edges = np.concatenate([rng.uniform(1.0, 2.0, 64) * 2.0 ** k for k in (-127, -126, -125, -124, 124, 125, 126)])
    x = np.concatenate([x, -x, edges, -edges, np.ldexp(1.0, np.arange(-1022, 1023)),
                        np.nextafter(np.ldexp(1.0, np.arange(-200, 200)), 0.0), [5e-324, 1e-310, -3e-320]])
    xt = d(x)
    yt = torch.empty_like(xt)
    chemgb.cgx_rcp_check(xt, yt)
    torch.cuda.synchronize()
    y = yt.cpu().numpy()
    with np.errstate(over="ignore", divide="ignore"):
        ref = 1.0 / x
    fin = np.isfinite(ref)
    assert np.array_equal(y[~fin], ref[~fin])
    ulp = np.abs(y[fin].view(np.int64) - ref[fin].view(np.int64))   # same sign: bit patterns order like |y|
    assert ulp.max() <= 1, (x[fin][ulp > 1][:5], ulp.max())


# --- Rosenbrock-2 (Appendix A.3) and YASS (Appendix A.4) --------------------

@pytest.mark.parametrize("kind", ["h2", "ch4"])
@pytest.mark.parametrize("reactor", [chemgb.CG_CONV, chemgb.CG_CONP])
def test_rosenbrock_fixed_parity(mechs, ref, handles, kind, reactor):
    """No Newton iteration: both sides evaluate the same two linear solves,
    so the states agree to rounding (1e-10)."""
    m, r, h = mechs[kind], ref[kind], handles[kind]
    fuel = "H2" if kind == "h2" else "CH4"
    T, Y, p = inputs.field_reactor(m, 77, (1100, 1500), (1, 3), (0.5, 2), fuel, seed=31)
    if reactor == chemgb.CG_CONV:
        p = p / (inputs.R_UNIV * T * (Y / m.W).sum(axis=1))
    o = dict(method=oracle.ROS2, adaptive=0, nsub=4, dt=2e-6, rtol=1e-8, atol=1e-14, reactor=reactor)
    To, Yo, so, sto = r.integrate(T, Y, p, o, nthreads=8)
    Tg, Yg, sg, stg = run_gpu(h, chemgb.make_opts(**o), T, Y, p)
    np.testing.assert_array_equal(sg, so)
    assert np.all(so == 0)
    np.testing.assert_array_equal(stg, sto)
    assert_state_close(Tg, Yg, To, Yo, 1e-10, 1e-20)


def test_rosenbrock_adaptive_parity_flame_field(mechs, ref, handles):
    m, r, h = mechs["ch4"], ref["ch4"], handles["ch4"]
    T, Y, p = inputs.field_flames(m, 4096, seed=0)
    idx = np.arange(5, 4096, 32)
    o = dict(ADAPT, method=oracle.ROS2)
    To, Yo, so, sto = r.integrate(T[idx], Y[idx], p[idx], o, nthreads=8)
    Tg, Yg, sg, stg = run_gpu(h, chemgb.make_opts(**o), T[idx], Y[idx], p[idx])
    np.testing.assert_array_equal(sg, so)
    assert np.all(so == 0)
    check_adaptive("adaptive_ros2_flame", m, Tg, Yg, To, Yo, p[idx], o["reactor"], o["rtol"], o["atol"])
    assert np.mean(np.all(stg == sto, axis=1)) > 0.9


def test_yass_parity_with_halving(mechs, ref, handles):
    """9 species, 4096 cells, YASS over 1e-5 s with alpha = 1 (WRMS weights
    1e-6 + 1e-3 |y|): every cell halves, up to a few hundred sub-steps (both
    sides take the same decisions, up to cells whose norm sits at alpha)."""
    m, r, h = mechs["h2"], ref["h2"], handles["h2"]
    T, Y, p = inputs.field_reactor(m, 4096, (1000, 1500), (1, 1), (0.5, 2), "H2", seed=0)
    o = dict(method=oracle.YASS, adaptive=0, dt=1e-5, rtol=1e-3, atol=1e-6, newton_tol=1.0,
             max_halvings=12, reactor=oracle.CONP)
    To, Yo, so, sto = r.integrate(T, Y, p, o, nthreads=8)
    Tg, Yg, sg, stg = run_gpu(h, chemgb.make_opts(**o), T, Y, p)
    np.testing.assert_array_equal(sg, so)
    assert np.all(so == 0)
    same = np.all(stg == sto, axis=1)
    assert same.mean() > 0.99 and np.mean(sto[:, 1] > 0) > 0.05   # halving happens
    assert_state_close(Tg[same], Yg[same], To[same], Yo[same], 1e-10, 1e-20)
    assert np.all(stg[:, 2] == stg[:, 0] + stg[:, 1])             # one linear solve per attempt


def test_rosenbrock_and_yass_refusals(mechs, handles):
    h = handles["h2"]
    T, Y, p = inputs.field_reactor(mechs["h2"], 4, (1200, 1200), (1, 1), (1, 1), "H2", seed=0)
    for method in (chemgb.CG_ROS2, chemgb.CG_YASS):
        with pytest.raises(chemgb.ChemgbError) as e:
            run_gpu(h, chemgb.make_opts(method=method, precision=chemgb.CG_FP32LU), T, Y, p)
        assert e.value.code == chemgb.CG_EUNSUPPORTED
        o = chemgb.make_opts(method=method, adaptive=0)
        ck = torch.empty((4, 8, h.n + 1), dtype=torch.float64, device=DEV)
        ckn = torch.zeros(4, dtype=torch.int32, device=DEV)
        z = torch.zeros(4, dtype=torch.float64, device=DEV)
        zy = torch.zeros((h.ns, 4), dtype=torch.float64, device=DEV)
        with pytest.raises(chemgb.ChemgbError) as e:
            chemgb.cg_integrate_adjoint(h, o, ck, ckn, z, zy, z.clone(), zy.clone())
        assert e.value.code == chemgb.CG_EUNSUPPORTED


# --- GMRES (Section 3.4) -----------------------------------------------------

GM = dict(linear_solver=oracle.GMRES, preconditioner=oracle.PC_GAUSS_SEIDEL, gmres_restart=30,
          gmres_maxit=400, gmres_tol=1e-13)


def merged(*ds, **kw):
    out = {}
    for d_ in ds:
        out.update(d_)
    out.update(kw)
    return out


@pytest.mark.parametrize("prec", [oracle.PC_NONE, oracle.PC_JACOBI, oracle.PC_GAUSS_SEIDEL])
def test_gmres_backward_euler_parity(mechs, ref, handles, prec):
    """Backward Euler with GMRES, Newton and GMRES iterated to tight
    tolerances, one step of 1e-6 s: the same states as the oracle's GMRES to
    1e-10, the same statuses and Newton counts (GMRES iteration counts may
    differ by rounding of the orthogonalisation: modified Gram-Schmidt
    there, classical twice here). At 1e-5 s steps across ignition the
    backward-Euler equations have several admissible roots and Newton paths
    that differ in rounding end on different ones (the oracle's own LU and
    GMRES runs do), so the step is kept where the root is unique."""
    m, r, h = mechs["h2"], ref["h2"], handles["h2"]
    T, Y, p = inputs.field_reactor(m, 1000, (1000, 1500), (1, 1), (0.5, 2), "H2", seed=0)
    o = merged(BE_OPTS, GM, preconditioner=prec, dt=1e-6)
    To, Yo, so, sto = r.integrate(T, Y, p, o, nthreads=8)
    Tg, Yg, sg, stg = run_gpu(h, chemgb.make_opts(**o), T, Y, p)
    np.testing.assert_array_equal(sg, so)
    assert np.all(so == 0)
    # a GMRES solve that stops at gmres_maxit on one side only fails that
    # Newton step there: the step is halved and the cell takes another (as
    # valid) path; compare the cells whose accepted, rejected and Newton
    # counts agree
    same = np.all(stg[:, :3] == sto[:, :3], axis=1)
    assert same.mean() > 0.98
    assert_state_close(Tg[same], Yg[same], To[same], Yo[same], 1e-10, 1e-22)


@pytest.mark.parametrize("method", [oracle.SDIRK4, oracle.ROS2])
def test_gmres_flame_field_parity(mechs, ref, handles, method):
    m, r, h = mechs["ch4"], ref["ch4"], handles["ch4"]
    T, Y, p = inputs.field_flames(m, 4096, seed=0)
    idx = np.arange(9, 4096, 40)
    o = merged(ADAPT, GM, method=method, gmres_tol=1e-10)
    To, Yo, so, _ = r.integrate(T[idx], Y[idx], p[idx], o, nthreads=8)
    Tg, Yg, sg, stg = run_gpu(h, chemgb.make_opts(**o), T[idx], Y[idx], p[idx])
    np.testing.assert_array_equal(sg, so)
    assert np.all(so == 0)
    check_adaptive(f"gmres_adaptive_flame_{method}", m, Tg, Yg, To, Yo, p[idx], o["reactor"], o["rtol"], o["atol"])
    assert np.all(stg[:, 3] >= stg[:, 2])          # at least one GMRES iteration per linear system


def test_gmres_fp32_matrix_flame_field(mechs, ref, handles):
    """GMRES on the FP32 Newton matrix (inexact Newton) lands on the FP64
    oracle's LU solution within the integrator's element-wise tolerance."""
    m, r, h = mechs["ch4"], ref["ch4"], handles["ch4"]
    T, Y, p = inputs.field_flames(m, 4096, seed=0)
    idx = np.arange(13, 4096, 64)
    o = merged(ADAPT, GM, gmres_tol=1e-8)
    To, Yo, so, _ = r.integrate(T[idx], Y[idx], p[idx], dict(ADAPT), nthreads=8)
    Tg, Yg, sg, _ = run_gpu(h, chemgb.make_opts(**merged(o, precision=chemgb.CG_FP32LU)), T[idx], Y[idx], p[idx])
    assert np.all(sg == 0) and np.all(so == 0)
    check_adaptive("gmres_fp32_adaptive_flame", m, Tg, Yg, To, Yo, p[idx], ADAPT["reactor"], ADAPT["rtol"],
                   ADAPT["atol"])


def test_gmres_limits_and_arguments(mechs, ref, handles):
    m, r, h = mechs["h2"], ref["h2"], handles["h2"]
    T, Y, p = inputs.field_reactor(m, 40, (1300, 1400), (1, 1), (0.5, 2), "H2", seed=2)
    o = merged(BE_OPTS, GM, gmres_maxit=1, preconditioner=oracle.PC_NONE, max_halvings=2)
    _, _, so, _ = r.integrate(T, Y, p, o, nthreads=8)
    _, _, sg, _ = run_gpu(h, chemgb.make_opts(**o), T, Y, p)
    np.testing.assert_array_equal(sg, so)
    assert np.any(sg == chemgb.CG_CELL_NEWTON_FAIL)     # one iteration does not solve the system
    for bad in (dict(gmres_restart=0), dict(gmres_restart=65), dict(gmres_maxit=0), dict(gmres_tol=0.0),
                dict(preconditioner=3), dict(linear_solver=2)):
        with pytest.raises(chemgb.ChemgbError) as e:
            run_gpu(h, chemgb.make_opts(**merged(BE_OPTS, GM, bad)), T, Y, p)
        assert e.value.code == chemgb.CG_EINVAL


# --- operator-split surface of a flow solver (Section 5.5) -------------------

def _flow_state(m, r, T, Y, p):
    rho = p / (inputs.R_UNIV * T * (Y / m.W).sum(axis=1))
    u = np.array([Y[c] @ r.thermo(T[c])["u"] for c in range(len(T))])
    return rho, u, rho[:, None] * Y


def run_split(h, opts, rho, u, rhoY, Tguess, iters=5):
    N = len(rho)
    Tt = d(Tguess)
    R = torch.empty((h.ns, N), dtype=torch.float64, device=DEV)
    st = torch.empty(N, dtype=torch.int32, device=DEV)
    chemgb.cg_react_split(h, opts, d(rho), d(u), d(rhoY.T), Tt, R, iters, st)
    torch.cuda.synchronize()
    return Tt.cpu().numpy(), R.cpu().numpy().T, st.cpu().numpy()


def test_split_step_parity_backward_euler(mechs, ref, handles):
    """(rho, u, rho Y) in, T and R out: one backward-Euler step of 1e-6 s
    from a stale temperature guess; T to 1e-10, R to 1e-9 of the scale
    rho Y / dt of the difference it is."""
    m, r, h = mechs["h2"], ref["h2"], handles["h2"]
    T, Y, p = inputs.field_reactor(m, 500, (1000, 1500), (1, 3), (0.5, 2), "H2", seed=41)
    rho, u, rhoY = _flow_state(m, r, T, Y, p)
    o = dict(BE_OPTS, reactor=oracle.CONV, dt=1e-6)
    To, Ro, so, _ = r.react_split(rho, u, rhoY, T * 1.05, o, nthreads=8)
    Tg, Rg, sg = run_split(h, chemgb.make_opts(**o), rho, u, rhoY, T * 1.05)
    np.testing.assert_array_equal(sg, so)
    assert np.all(so == 0)
    np.testing.assert_allclose(Tg, To, rtol=1e-10)
    scale = rhoY / o["dt"] + np.abs(Ro)
    assert np.all(np.abs(Rg - Ro) <= 1e-9 * scale)
    assert np.all(np.abs(Rg.sum(axis=1)) <= 1e-12 * np.abs(Rg).sum(axis=1) + 1e-13 * rhoY.sum(axis=1) / o["dt"])


def test_split_step_parity_flame_cells(mechs, ref, handles):
    m, r, h = mechs["ch4"], ref["ch4"], handles["ch4"]
    T, Y, p = inputs.field_flames(m, 4096, seed=0)
    idx = np.arange(3, 4096, 48)
    rho, u, rhoY = _flow_state(m, r, T[idx], Y[idx], p[idx])
    o = dict(ADAPT, reactor=oracle.CONV)
    To, Ro, so, _ = r.react_split(rho, u, rhoY, T[idx], o, nthreads=8)
    Tg, Rg, sg = run_split(h, chemgb.make_opts(**o), rho, u, rhoY, T[idx])
    np.testing.assert_array_equal(sg, so)
    assert np.all(so == 0)
    # R_i = W_i dC_i / dt: the end state's element-wise weight, over dt
    Yo_end = (rhoY + Ro * o["dt"]) / rho[:, None]
    Yg_end = (rhoY + Rg * o["dt"]) / rho[:, None]
    check_adaptive("split_adaptive_flame", m, Tg, Yg_end, To, Yo_end, rho, oracle.CONV, o["rtol"], o["atol"])


def test_split_step_edge_cases(mechs, ref, handles):
    m, r, h = mechs["h2"], ref["h2"], handles["h2"]
    T, Y, p = inputs.field_reactor(m, 3, (1200, 1200), (1, 1), (1, 1), "H2", seed=1)
    rho, u, rhoY = _flow_state(m, r, T, Y, p)
    u[1] = np.nan
    o = dict(BE_OPTS, reactor=oracle.CONV, dt=1e-6)
    Tg, Rg, sg = run_split(h, chemgb.make_opts(**o), rho, u, rhoY, T)
    assert sg[1] == chemgb.CG_CELL_NONFINITE and Tg[1] == T[1] and not Rg[1].any()
    assert sg[0] == 0 and sg[2] == 0
    with pytest.raises(chemgb.ChemgbError) as e:
        run_split(h, chemgb.make_opts(**BE_OPTS), rho, u, rhoY, T)     # constant pressure: refused
    assert e.value.code == chemgb.CG_EINVAL


# --- SRI falloff and PLOG reactions (Section 2.2.3, 2.2.4) ------------------

@pytest.fixture(scope="module")
def xset():
    m = inputs.with_sri_plog(inputs.gen_mechanism("ch4"), n_sri=8, n_plog=20, seed=3)
    return m, oracle.RefMech(m), chemgb.cg_mech_create(m)


@pytest.mark.parametrize("reactor", [chemgb.CG_CONV, chemgb.CG_CONP])
def test_sri_plog_rates_and_jacobian_parity(xset, reactor):
    """Random states of Section 5.1 (pressures 0.1-10 atm, so PLOG cells
    fall below, inside and between the 0.1-100 atm levels)."""
    m, r, h = xset
    N = 45
    T, C, p = inputs.random_states(m, N, seed=303)
    Sg = gpu_rates(h, T, C, reactor)
    So = r.source(T, C, reactor)
    nu = np.abs(nu_matrix(m))
    for c in range(N):
        scale = nu @ np.abs(r.rates(T[c], C[c])[2])
        if reactor == chemgb.CG_CONP:
            scale = scale + C[c] * (np.abs(So[c, 0]) / T[c] + scale.sum() / C[c].sum())
        np.testing.assert_array_less(np.abs(Sg[c, 1:] - So[c, 1:]), 1e-12 * scale + 1e-300)
        assert abs(Sg[c, 0] - So[c, 0]) <= 1e-11 * abs(So[c, 0]) + 1e-300 or abs(So[c, 0]) < 1e-300
    J = torch.empty((N, h.n, h.n), dtype=torch.float64, device=DEV)
    chemgb.cg_eval_jacobian(h, reactor, d(T), d(C.T), J)
    torch.cuda.synchronize()
    Jg, Jo = J.cpu().numpy(), r.jacobian(T, C, reactor)
    rowmax = np.abs(Jo).max(axis=2, keepdims=True)
    assert np.all(np.abs(Jg - Jo) <= 1e-10 * np.abs(Jo) + 1e-12 * rowmax)


def test_sri_plog_integration_parity(xset):
    m, r, h = xset
    T, Y, p = inputs.field_reactor(m, 70, (1200, 1500), (0.5, 40), (0.5, 2.0), "CH4", seed=7)
    o = dict(BE_OPTS, dt=1e-6, nsub=2)
    To, Yo, so, sto = r.integrate(T, Y, p, o, nthreads=8)
    Tg, Yg, sg, stg = run_gpu(h, chemgb.make_opts(**o), T, Y, p)
    np.testing.assert_array_equal(sg, so)
    assert np.all(so == 0)
    same = np.all(stg[:, :3] == sto[:, :3], axis=1)
    assert same.mean() > 0.98
    assert_state_close(Tg[same], Yg[same], To[same], Yo[same], 1e-10, 1e-22)
    o = dict(ADAPT, dt=2e-6)
    To, Yo, so, _ = r.integrate(T, Y, p, o, nthreads=8)
    Tg, Yg, sg, _ = run_gpu(h, chemgb.make_opts(**o), T, Y, p)
    np.testing.assert_array_equal(sg, so)
    check_adaptive("sri_plog_adaptive", m, Tg, Yg, To, Yo, p, o["reactor"], o["rtol"], o["atol"])
