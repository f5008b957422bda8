"""GPU: work distribution, global-scratch placement, batched launches of
several mechanisms, and the 160-species mechanism whose Newton matrix
fills shared memory (its other arrays live in global scratch).

Where the arithmetic of a cell is unchanged (persistent vs one slot per
cell, shared vs global placement, batched vs separate launches) the results
must be bit-identical."""
import numpy as np
import pytest

import oracle
from paper_2510_10005_gb300 import chemgb, inputs
from parity import check_adaptive, check_elementwise, check_fixed

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"

BE = dict(method=chemgb.CG_BE, adaptive=0, dt=1e-5, rtol=1e-10, atol=1e-16, newton_tol=1.0,
          max_newton=20, max_halvings=10, reactor=chemgb.CG_CONP)
ADAPT = dict(method=chemgb.CG_SDIRK4, adaptive=1, dt=1e-6, rtol=1e-6, atol=1e-12, newton_tol=0.03,
             max_newton=7, reactor=chemgb.CG_CONP)


def d(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def run(h, o, T, Y, p):
    N = len(T)
    Tt, Yt, pt = d(T), d(Y.T), d(p)
    st = torch.empty(N, dtype=torch.int32, device=DEV)
    stats = torch.empty((4, N), dtype=torch.int32, device=DEV)
    chemgb.cg_integrate(h, o, Tt, Yt, pt, st, stats)
    torch.cuda.synchronize()
    return Tt.cpu().numpy(), Yt.cpu().numpy().T, st.cpu().numpy(), stats.cpu().numpy().T


def same(a, b):
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


@pytest.fixture(scope="module")
def flame_cells(mechs):
    m = mechs["ch4"]
    T, Y, p = inputs.field_flames(m, 4096, seed=4)
    idx = np.concatenate([np.arange(0, 4096, 64), np.arange(2420, 2460)])   # all regions + front
    return T[idx], Y[idx], p[idx]


def test_persistent_queue_is_bit_identical(mechs, flame_cells):
    h = chemgb.cg_mech_create(mechs["ch4"])
    T, Y, p = flame_cells
    a = run(h, chemgb.make_opts(**ADAPT, persistent=0), T, Y, p)
    b = run(h, chemgb.make_opts(**ADAPT, persistent=1), T, Y, p)
    same(a, b)


@pytest.mark.parametrize("limit", [40 * 1024, 16 * 1024, 4 * 1024])
def test_global_scratch_placement_is_bit_identical(mechs, flame_cells, limit):
    """Arrays moved to the global scratch slot compute the same numbers."""
    h = chemgb.cg_mech_create(mechs["ch4"])
    T, Y, p = flame_cells
    o = chemgb.make_opts(**ADAPT)
    a = run(h, o, T, Y, p)
    chemgb.cg_mech_set_smem_limit(h, limit)
    b = run(h, o, T, Y, p)
    same(a, b)
    o32 = chemgb.make_opts(**ADAPT, precision=chemgb.CG_FP32LU)
    c = run(h, o32, T, Y, p)
    chemgb.cg_mech_set_smem_limit(h, 227 * 1024)
    same(c, run(h, o32, T, Y, p))


def test_batch_of_two_mechanisms_matches_separate_launches(mechs, flame_cells):
    h9 = chemgb.cg_mech_create(mechs["h2"])
    h53 = chemgb.cg_mech_create(mechs["ch4"])
    chemgb.cg_mech_set_launch(h9, 64, 1)        # one team size for the batch
    T9, Y9, p9 = inputs.field_reactor(mechs["h2"], 300, (1000, 1500), (1, 1), (0.5, 2), "H2", seed=5)
    T53, Y53, p53 = flame_cells
    o = chemgb.make_opts(**ADAPT)
    a9 = run(h9, o, T9, Y9, p9)
    a53 = run(h53, o, T53, Y53, p53)
    Ts = [d(T9), d(T53)]
    Ys = [d(Y9.T), d(Y53.T)]
    ps = [d(p9), d(p53)]
    sts = [torch.empty(len(T9), dtype=torch.int32, device=DEV), torch.empty(len(T53), dtype=torch.int32, device=DEV)]
    sas = [torch.empty((4, len(T9)), dtype=torch.int32, device=DEV),
           torch.empty((4, len(T53)), dtype=torch.int32, device=DEV)]
    chemgb.cg_integrate_batch([h9, h53], o, Ts, Ys, ps, sts, sas)
    torch.cuda.synchronize()
    same(a9, (Ts[0].cpu().numpy(), Ys[0].cpu().numpy().T, sts[0].cpu().numpy(), sas[0].cpu().numpy().T))
    same(a53, (Ts[1].cpu().numpy(), Ys[1].cpu().numpy().T, sts[1].cpu().numpy(), sas[1].cpu().numpy().T))


@pytest.mark.parametrize("team53", [64, 128, 256])
def test_split_batch_matches_separate_launches(mechs, flame_cells, team53):
    """A one-warp mechanism (9 species) in a launch of wider teams (53
    species with 64-256 threads per cell) runs split, each warp of a team
    integrating its own cells: the same bits as its own one-warp launch,
    for either mechanism, with FP64 and FP32 Newton matrices, and with the
    split cells alone (no cells of the wider mechanism)."""
    h9 = chemgb.cg_mech_create(mechs["h2"])
    h53 = chemgb.cg_mech_create(mechs["ch4"])
    chemgb.cg_mech_set_launch(h53, team53, 1)
    assert chemgb.cg_mech_get_launch(h9)[0] == 32
    T9, Y9, p9, _ = inputs.field_mixed(mechs["h2"], 700, "H2", seed=8)
    T53, Y53, p53 = flame_cells
    for prec in (chemgb.CG_FP64, chemgb.CG_FP32LU):
        o = chemgb.make_opts(**ADAPT, precision=prec)
        a9 = run(h9, o, T9, Y9, p9)
        a53 = run(h53, o, T53, Y53, p53)
        for with53 in (True, False):
            n53 = len(T53) if with53 else 0
            Ts = [d(T9), d(T53[:n53])]
            Ys = [d(Y9.T), d(Y53[:n53].T)]
            ps = [d(p9), d(p53[:n53])]
            sts = [torch.empty(len(T9), dtype=torch.int32, device=DEV), torch.empty(n53, dtype=torch.int32, device=DEV)]
            sas = [torch.empty((4, len(T9)), dtype=torch.int32, device=DEV),
                   torch.empty((4, n53), dtype=torch.int32, device=DEV)]
            chemgb.cg_integrate_batch([h9, h53], o, Ts, Ys, ps, sts, sas)
            torch.cuda.synchronize()
            same(a9, (Ts[0].cpu().numpy(), Ys[0].cpu().numpy().T, sts[0].cpu().numpy(), sas[0].cpu().numpy().T))
            if with53:
                same(a53, (Ts[1].cpu().numpy(), Ys[1].cpu().numpy().T, sts[1].cpu().numpy(),
                           sas[1].cpu().numpy().T))
    if team53 != 64:                                  # two wider team sizes cannot share a launch
        h9b = chemgb.cg_mech_create(mechs["h2"])
        chemgb.cg_mech_set_launch(h9b, 64, 1)
        with pytest.raises(chemgb.ChemgbError) as e:
            chemgb.cg_integrate_batch([h9b, h53], chemgb.make_opts(**ADAPT), [d(T9), d(T53)], [d(Y9.T), d(Y53.T)],
                                      [d(p9), d(p53)])
        assert e.value.code == chemgb.CG_EINVAL


def test_autotune_picks_a_shape_and_keeps_results(mechs, tmp_path):
    m = mechs["ch4"]
    h = chemgb.cg_mech_create(m)
    T, Y, p, _ = inputs.field_mixed(m, 2048, "CH4", seed=3, argon=0.0093)
    o = chemgb.make_opts(**ADAPT, precision=chemgb.CG_FP32LU)
    before = run(h, o, T, Y, p)
    cache = str(tmp_path / "tune.json")
    Tt, Yt, pt = d(T), d(Y.T), d(p)
    ms = chemgb.cg_autotune(h, o, Tt, Yt, pt, cache)
    assert ms > 0
    np.testing.assert_array_equal(Tt.cpu().numpy(), T)       # the sample is not modified
    team, tpb = chemgb.cg_mech_get_launch(h)
    assert team in (32, 64, 128, 256) and tpb in (1, 2, 4)
    after = run(h, o, T, Y, p)
    np.testing.assert_array_equal(after[2], before[2])
    np.testing.assert_allclose(after[0], before[0], rtol=1e-9)
    h2 = chemgb.cg_mech_create(m)                              # the cache file is applied
    assert chemgb.cg_autotune(h2, o, Tt, Yt, pt, cache) == pytest.approx(ms)
    assert chemgb.cg_mech_get_launch(h2) == (team, tpb)


def test_batch_replays_from_a_cuda_graph(mechs, flame_cells):
    """The batched launch (stream-ordered scratch, counter reset, kernel)
    captured in a CUDA graph and replayed gives the direct call's results."""
    h53 = chemgb.cg_mech_create(mechs["ch4"])
    T, Y, p = flame_cells
    o = chemgb.make_opts(**ADAPT, persistent=1)
    ref = run(h53, o, T, Y, p)
    T0, Y0, P0 = d(T), d(Y.T), d(p)
    Tw, Yw = torch.empty_like(T0), torch.empty_like(Y0)
    st = torch.empty(len(T), dtype=torch.int32, device=DEV)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        Tw.copy_(T0); Yw.copy_(Y0)
        chemgb.cg_integrate_batch([h53], o, [Tw], [Yw], [P0], [st], stream=stream.cuda_stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        Tw.copy_(T0); Yw.copy_(Y0)
        chemgb.cg_integrate_batch([h53], o, [Tw], [Yw], [P0], [st], stream=stream.cuda_stream)
    for _ in range(2):
        Tw.fill_(0.0)
        g.replay()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(Tw.cpu().numpy(), ref[0])
        np.testing.assert_array_equal(Yw.cpu().numpy().T, ref[1])


# ---------------------------------------------------------------------------
# 160 species, 900 reactions


@pytest.fixture(scope="module")
def big():
    m = inputs.gen_mechanism("c7")
    return m, oracle.RefMech(m), chemgb.cg_mech_create(m)


def test_big_mechanism_rates_and_jacobian(big):
    m, r, h = big
    T, C, p = inputs.random_states(m, 9, seed=31)
    S = torch.empty((m.ns + 1, 9), dtype=torch.float64, device=DEV)
    chemgb.cg_eval_rates(h, chemgb.CG_CONP, d(T), d(C.T), S)
    J = torch.empty((9, m.ns + 1, m.ns + 1), dtype=torch.float64, device=DEV)
    chemgb.cg_eval_jacobian(h, chemgb.CG_CONP, d(T), d(C.T), J)
    torch.cuda.synchronize()
    So = r.source(T, C, oracle.CONP)
    Jo = r.jacobian(T, C, oracle.CONP)
    Sg = S.cpu().numpy().T
    Jg = J.cpu().numpy()
    rowmax = np.abs(Jo).max(axis=2, keepdims=True)
    assert np.all(np.abs(Jg - Jo) <= 1e-10 * np.abs(Jo) + 1e-12 * rowmax)
    scale = np.abs(So).max(axis=1, keepdims=True)
    assert np.all(np.abs(Sg - So) <= 1e-10 * np.abs(So) + 1e-12 * scale)


@pytest.fixture(scope="module")
def big_cells(big):
    """64 cells of the large-mechanism field recipe: T in U[700, 1600] K,
    p in U[20, 40] atm, phi in U[0.5, 1.5] (n-heptane in air)."""
    m = big[0]
    return inputs.field_reactor(m, 64, (700, 1600), (20, 40), (0.5, 1.5), "C7H16", seed=0)


@pytest.mark.parametrize("precision", [chemgb.CG_FP64, chemgb.CG_FP32LU])
def test_big_mechanism_backward_euler(big, big_cells, precision):
    """Fixed-step backward Euler, Newton iterated until its change is below
    1e-10 of the state (at most 20 iterations): the FP64 Newton matrix lands
    on the oracle's root to 1e-10; the FP32 one (an inexact Newton whose
    residual stays FP64, its preconditioner applied in FP32) to 1e-8, with
    1e-7 s steps. On the worst conditioned cells the FP32 preconditioner may
    not contract at the full step, and the integrator's fallback halves it:
    such a cell (at most 5 %) must show exactly one failed attempt and two
    half steps, and must agree to 1e-8 with the oracle taking those two half
    steps."""
    m, r, h = big
    T, Y, p = big_cells
    o = dict(BE, dt=1e-6 if precision == chemgb.CG_FP64 else 1e-7)
    To, Yo, so, sto = r.integrate(T, Y, p, o, nthreads=8)
    Tg, Yg, sg, stg = run(h, chemgb.make_opts(**o, precision=precision), T, Y, p)
    np.testing.assert_array_equal(sg, so)      # a cell that exhausts its halvings fails on both sides
    ok = so == 0
    assert ok.mean() > 0.9
    same = ok & np.all(stg[:, :2] == sto[:, :2], axis=1)
    if precision == chemgb.CG_FP64:
        np.testing.assert_array_equal(same, ok)                  # the same halving path everywhere
        check_fixed("big_160sp_be_fp64", Tg[ok], Yg[ok], To[ok], Yo[ok], 1e-10, 1e-22)
        return
    check_fixed("big_160sp_be_fp32lu", Tg[same], Yg[same], To[same], Yo[same], 1e-8, 1e-18)
    other = ok & ~same
    assert other.mean() <= 0.05
    if other.any():
        np.testing.assert_array_equal(stg[other, :2], np.tile([2, 1], (int(other.sum()), 1)))
        To2, Yo2, so2, sto2 = r.integrate(T[other], Y[other], p[other], dict(o, nsub=2), nthreads=8)
        assert np.all(so2 == 0) and np.all(sto2[:, :2] == [2, 0])
        check_fixed("big_160sp_be_fp32lu_halved", Tg[other], Yg[other], To2, Yo2, 1e-8, 1e-18)


@pytest.mark.parametrize("kind,team,panels", [("c7", 256, (16, 5, 64)), ("c7", 64, (16,)), ("ch4", 64, (8, 16)),
                                              ("ch4", 32, (7,))])
@pytest.mark.parametrize("precision", [chemgb.CG_FP64, chemgb.CG_FP32LU])
def test_blocked_lu_is_bit_identical(mechs, big, big_cells, kind, team, panels, precision):
    """The blocked LU (panels of nb columns, register-tiled trailing update)
    applies the same fused multiply-adds in the same order as the column-by-
    column factorisation: every panel width, including ones that do not
    divide n and one wider than the matrix's first panel, gives the same
    bits in T, Y and the counters, for the FP64 and the FP32 Newton matrix."""
    if kind == "c7":
        m, _, _ = big
        T, Y, p = big_cells
        T, Y, p = T[:24], Y[:24], p[:24]
        o = chemgb.make_opts(**dict(BE, dt=1e-7), precision=precision)
    else:
        m = mechs["ch4"]
        T, Y, p = inputs.field_flames(m, 4096, seed=6)
        idx = np.concatenate([np.arange(0, 4096, 128), np.arange(2430, 2450)])
        T, Y, p = T[idx], Y[idx], p[idx]
        o = chemgb.make_opts(**ADAPT, precision=precision)
    h = chemgb.cg_mech_create(m)
    chemgb.cg_mech_set_launch(h, team, 1)
    chemgb.cg_mech_set_lu_panel(h, 0)
    ref = run(h, o, T, Y, p)
    for nb in panels:
        chemgb.cg_mech_set_lu_panel(h, nb)
        assert chemgb.cg_mech_get_lu_panel(h) == nb
        same(run(h, o, T, Y, p), ref)


@pytest.mark.parametrize("precision", [chemgb.CG_FP64, chemgb.CG_FP32LU])
def test_big_mechanism_adaptive(big, big_cells, precision):
    """Adaptive SDIRK-4 (rtol 1e-6, atol 1e-12) over 1e-6 s on the 64 cells,
    against the FP64 oracle element-wise within the integrator's weight."""
    m, r, h = big
    T, Y, p = big_cells
    To, Yo, so, _ = r.integrate(T, Y, p, ADAPT, nthreads=8)
    Tg, Yg, sg, _ = run(h, chemgb.make_opts(**ADAPT, precision=precision), T, Y, p)
    np.testing.assert_array_equal(sg, so)
    assert np.all(so == 0)
    check_adaptive("big_160sp_sdirk4_" + ("fp64" if precision == chemgb.CG_FP64 else "fp32lu"), m, Tg, Yg, To, Yo,
                   p, ADAPT["reactor"], ADAPT["rtol"], ADAPT["atol"])


def test_big_mechanism_adjoint(big, big_cells):
    """The discrete adjoint at 160 species (team of four warps, Newton
    matrices in global scratch, blocked LU and its transposed solves): 32 of
    the cells, adaptive SDIRK-4 over 1e-6 s with checkpoints, then the
    backward sweep for random dL/dT_end and dL/dY_end. dL/dT0, dL/dY0 and
    the per-cell dL/dtheta must match the oracle's adjoint element-wise
    within 1e-6 plus 1e-9 of the largest entry of each kind, on the cells
    whose accepted step count equals the oracle's (at least 90 %)."""
    m, r, h = big
    T, Y, p = (a[::2] for a in big_cells)
    N = len(T)
    og = chemgb.make_opts(**ADAPT)
    Tt, Yt, pt = d(T), d(Y.T), d(p)
    cap = 128
    ckpt = torch.empty((N, cap, m.ns + 2), dtype=torch.float64, device=DEV)
    ckpt_n = torch.empty(N, dtype=torch.int32, device=DEV)
    st = torch.empty(N, dtype=torch.int32, device=DEV)
    chemgb.cg_integrate_ckpt(h, og, Tt, Yt, pt, ckpt, ckpt_n, st)
    rng = np.random.default_rng(8)
    gT, gY = rng.normal(size=N), rng.normal(size=(N, m.ns))
    dT0, dY0 = torch.empty(N, dtype=torch.float64, device=DEV), torch.empty((m.ns, N), dtype=torch.float64, device=DEV)
    dth = torch.empty((m.nr, 3), dtype=torch.float64, device=DEV)
    dcell = torch.empty((m.nr, 3, N), dtype=torch.float64, device=DEV)
    ast = torch.empty(N, dtype=torch.int32, device=DEV)
    chemgb.cg_integrate_adjoint(h, og, ckpt, ckpt_n, d(gT), d(gY.T), dT0, dY0, dth, dcell, ast)
    torch.cuda.synchronize()
    assert int((st != 0).sum()) == 0 and int((ast != 0).sum()) == 0
    kn = ckpt_n.cpu().numpy()
    assert np.all((kn > 0) & (kn < cap))
    oo = {k: v for k, v in ADAPT.items()}
    oT, oY, og_, ost = r.adjoint_TY(T, Y, p, gT, gY, oo, nthreads=8)
    assert np.all(ost == 0)
    C0 = r.concentrations(T, Y, p, ADAPT["reactor"])
    _, _, _, hn = r.integrate_hist(np.concatenate([T[:, None], C0], axis=1), oo, cap=cap, nthreads=8)
    same = kn == hn
    assert same.mean() >= 0.9, (kn, hn)
    check_elementwise("big_160sp_adjoint_dT0", dT0.cpu().numpy()[same], oT[same], 1e-6, 1e-9)
    check_elementwise("big_160sp_adjoint_dY0", dY0.cpu().numpy().T[same], oY[same], 1e-6, 1e-9)
    gc = np.moveaxis(dcell.cpu().numpy(), 2, 0)
    for k, name in enumerate(("lnA", "b", "Ea")):
        check_elementwise(f"big_160sp_adjoint_dtheta_{name}", gc[same][:, :, k], og_[same][:, :, k], 1e-6, 1e-9)
    np.testing.assert_allclose(dth.cpu().numpy(), gc.sum(axis=0), rtol=1e-12, atol=1e-12 * np.abs(gc).max())
