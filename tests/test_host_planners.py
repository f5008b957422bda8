"""The CUDA library's host-side planners, on the CPU (no GPU needed): the
thread-owned assembly schedules of the sparse sums (the production rates
of Section 2.2 and the Jacobian entries of Section 3.2), the reaction
chunks of the rate loop, and the placement of a cell's working set in
shared memory and global scratch.

Each plan is checked for the properties the kernels rely on: a schedule
walked as the kernels walk it (each lane in slot order, groups of four
terms whose loads precede their stores) gives the same sums, in the same
order, as a direct accumulation; no destination is shared by two lanes;
chunks cover every reaction once with one branch kind per warp; arrays
never overlap and stay 16-byte aligned within their budget."""
import numpy as np
import pytest

from paper_2510_10005_gb300 import build, chemgb, inputs

FIRST, LAST = 1, 2


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return chemgb.load()


def walk(sched, out0, x, lanes):
    """Replay of the kernels' walk: per lane, groups of four slots whose
    loads (source and, on a first term, the destination's value) all
    precede the group's accumulations and stores."""
    n, dst, flags, src, fac = sched
    out = out0.copy()
    for l in range(lanes):
        acc = 0.0
        t = 0
        while t < n:
            g = range(t, min(t + 4, n))
            loads = [(x[src[k, l]], out[dst[k, l]] if flags[k, l] & FIRST else 0.0) for k in g]
            for k, (xv, ov) in zip(g, loads):
                if flags[k, l] & FIRST:
                    acc = ov
                acc = fac[k, l] * xv + acc
                if flags[k, l] & LAST:
                    out[dst[k, l]] = acc
            t += 4
    return out


def direct(terms, out0, x):
    dst, src, fac, order = terms
    out = out0.copy()
    for i in np.lexsort((order, dst)):
        out[dst[i]] = fac[i] * x[src[i]] + out[dst[i]]
    return out


def mechanism_terms(m):
    """The production-rate sum omega_i += nu_ij q_j of a mechanism: one
    term per species slot of every reaction (reactants negative), in
    reaction order within a species."""
    dst, src, fac = [], [], []
    for j in range(m.nr):
        for idx, nu, sign in ((m.rf_idx, m.rf_nu, -1.0), (m.rr_idx, m.rr_nu, 1.0)):
            for s in range(3):
                if idx[j, s] >= 0:
                    dst.append(int(idx[j, s]))
                    src.append(j)
                    fac.append(sign * nu[j, s])
    order = np.arange(len(dst))
    return np.array(dst), np.array(src), np.array(fac), order


def skewed_terms(rng, n_dst, n_src):
    """Runs of very different lengths: a few dense rows (like the third-body
    column of a Jacobian) among many short ones, in shuffled order."""
    lens = np.concatenate([rng.integers(1, 4, n_dst - 3), [n_src, n_src // 2, 40]])
    dst = np.repeat(np.arange(n_dst) * 7 + 3, lens)
    src = rng.integers(0, n_src, len(dst))
    fac = rng.normal(size=len(dst))
    order = rng.permutation(len(dst))
    p = rng.permutation(len(dst))
    return dst[p], src[p], fac[p], order[p]


def check_schedule(terms, lanes, rng):
    dst, src, fac, order = terms
    sched = chemgb.cgx_schedule(dst, src, fac, order, lanes)
    n, sd, sf, ss, sc = sched
    # ownership: every destination lives in one lane, as one contiguous run
    # flagged first ... last, in its terms' order
    owner = {}
    for l in range(lanes):
        t, seen = 0, set()
        while t < n and sf[t, l] & FIRST:
            d = sd[t, l]
            assert d not in owner and d not in seen
            seen.add(d)
            owner[d] = l
            run = [t]
            while not sf[run[-1], l] & LAST:
                run.append(run[-1] + 1)
                assert sd[run[-1], l] == d and not sf[run[-1], l] & FIRST
            mine = np.nonzero(dst == d)[0]
            mine = mine[np.argsort(order[mine], kind="stable")]
            np.testing.assert_array_equal(ss[run, l], src[mine])
            np.testing.assert_array_equal(sc[run, l], fac[mine])
            t = run[-1] + 1
        # padding after the lane's last run
        assert np.all(sf[t:, l] == 0) and np.all(sc[t:, l] == 0.0) and np.all(sd[t:, l] == 0)
    assert set(owner) == set(np.unique(dst).tolist())
    # longest-run-first onto the least-loaded lane: the longest lane exceeds
    # the mean by less than the longest run
    runs = np.bincount(np.unique(dst, return_inverse=True)[1])
    assert n == 0 or n < len(dst) / lanes + runs.max()
    # walked as the kernels walk it, the sums equal the direct ones exactly
    x = rng.normal(size=int(src.max()) + 1 if len(src) else 1)
    out0 = rng.normal(size=int(dst.max()) + 1 if len(dst) else 1)
    np.testing.assert_array_equal(walk(sched, out0, x, lanes), direct(terms, out0, x))
    return sched


@pytest.mark.parametrize("kind", ["h2", "ch4", "c7"])
@pytest.mark.parametrize("lanes", [32, 64, 256])
def test_schedule_of_production_rates(kind, lanes):
    m = inputs.gen_mechanism(kind)
    check_schedule(mechanism_terms(m), lanes, np.random.default_rng(1))


@pytest.mark.parametrize("lanes", [1, 5, 32, 128])
def test_schedule_with_skewed_runs(lanes):
    rng = np.random.default_rng(lanes)
    check_schedule(skewed_terms(rng, 90, 300), lanes, rng)


def test_schedule_edge_cases():
    rng = np.random.default_rng(3)
    e = np.zeros(0, np.int64)
    n, *_ = chemgb.cgx_schedule(e, e, np.zeros(0), e, 32)   # no terms
    assert n == 0
    one = (np.array([5]), np.array([0]), np.array([2.0]), np.array([0]))
    n, sd, sf, ss, sc = check_schedule(one, 64, rng)        # more lanes than destinations
    assert n == 1 and (sf == (FIRST | LAST)).sum() == 1
    with pytest.raises(chemgb.ChemgbError):
        chemgb.cgx_schedule(np.array([-1]), np.array([0]), np.array([1.0]), np.array([0]), 32)
    with pytest.raises(chemgb.ChemgbError):
        chemgb.cgx_schedule(np.array([1 << 29]), np.array([0]), np.array([1.0]), np.array([0]), 32)
    with pytest.raises(chemgb.ChemgbError):
        chemgb.cgx_schedule(*one, 0)


def rxn_kind(t):
    return 2 if t == inputs.RXN_PLOG else (1 if t >= inputs.RXN_LINDEMANN else 0)


@pytest.mark.parametrize("team", [32, 64, 128, 256])
@pytest.mark.parametrize("case", ["ch4", "c7", "sri_plog", "mixed"])
def test_rate_chunks(team, case):
    if case == "mixed":   # kinds interleaved, not sorted (every run boundary)
        types = np.random.default_rng(5).choice([0, 1, 2, 3, 4, 5], size=301)
    else:
        m = inputs.gen_mechanism("ch4" if case != "c7" else "c7")
        if case == "sri_plog":
            m = inputs.with_sri_plog(m, n_sri=8, n_plog=20, seed=3)
        types = np.sort(m.rtype, kind="stable")   # the library's internal order is by type
    ptr, first, ln = chemgb.cgx_rate_chunks(types, team)
    nw = team // 32
    assert len(ptr) == nw + 1 and ptr[0] == 0 and ptr[-1] == len(first) and np.all(np.diff(ptr) >= 0)
    # an exact cover of the reactions by chunks of 1-32 of one kind
    cover = np.zeros(len(types), int)
    for f, n in zip(first, ln):
        assert 1 <= n <= 32
        cover[f:f + n] += 1
        assert len({rxn_kind(t) for t in types[f:f + n]}) == 1
    assert np.all(cover == 1)
    # chunks are maximal: a chunk shorter than 32 ends at a change of kind
    for f, n in zip(first, ln):
        if n < 32 and f + n < len(types):
            assert rxn_kind(types[f + n]) != rxn_kind(types[f + n - 1])
    # each warp walks its chunks in reaction order; the loads (falloff and
    # PLOG chunks 3, plain 1) differ by at most one chunk's cost
    cost = np.array([1.0 if rxn_kind(types[f]) == 0 else 3.0 for f in first])
    loads = []
    for w in range(nw):
        fw = first[ptr[w]:ptr[w + 1]]
        assert np.all(np.diff(fw) > 0)
        loads.append(cost[ptr[w]:ptr[w + 1]].sum())
    if len(first) >= nw:
        assert max(loads) - min(loads) <= 3.0


def test_rate_chunks_arguments():
    with pytest.raises(chemgb.ChemgbError):
        chemgb.cgx_rate_chunks(np.zeros(5, np.int32), 48)
    ptr, first, ln = chemgb.cgx_rate_chunks(np.zeros(0, np.int32), 64)
    assert len(first) == 0 and list(ptr) == [0, 0, 0]


def check_layout(L, smem_limit):
    off, size, glob = L["offset"], L["size"], L["in_global"]
    assert np.all(off % 2 == 0) and np.all(size % 2 == 0)          # 16-byte aligned arrays
    for space, total in ((False, L["smem"]), (True, L["glob"])):
        idx = [a for a in range(len(off)) if glob[a] == space and size[a] > 0]
        spans = sorted((off[a], off[a] + size[a]) for a in idx)
        for (b0, e0), (b1, e1) in zip(spans, spans[1:]):
            assert e0 <= b1                                         # no overlap
        assert all(e <= total for _, e in spans)
        assert total == sum(size[a] for a in range(len(off)) if glob[a] == space)
    budget = max(smem_limit - 1024, 1024) // 8
    pri = list(L["priority"])
    red = pri[0]
    assert not glob[red]                                            # the reduction scratch stays shared
    rest = [a for a in pri if a != red]
    spilled = [glob[a] for a in rest]
    if any(spilled):                                                # one spill moves all later arrays
        k = spilled.index(True)
        assert all(spilled[k:])
        assert L["smem"] + size[rest[k]] > budget
    assert L["smem"] <= max(budget, size[red])


@pytest.mark.parametrize("ns,nr", [(9, 21), (53, 325), (160, 900)])
@pytest.mark.parametrize("mat_bytes", [8, 4])
@pytest.mark.parametrize("adjoint,gmres_m", [(False, 0), (True, 0), (False, 30)])
def test_layout(ns, nr, mat_bytes, adjoint, gmres_m):
    n = ns + 1
    for limit in (227 * 1024, 40 * 1024, 4 * 1024, 0, 1 << 30):
        L = chemgb.cgx_layout(ns, nr, mat_bytes, limit, adjoint, gmres_m)
        assert L["ld"] % 2 == 1 and L["ld"] >= n
        check_layout(L, limit)
        # some array holds the Newton matrix: n rows of ld entries of mat_bytes
        assert np.any(L["size"] >= n * L["ld"] * mat_bytes / 8)
    # placement never changes the sizes; with room for all, nothing spills
    a = chemgb.cgx_layout(ns, nr, mat_bytes, 1 << 30, adjoint, gmres_m)
    b = chemgb.cgx_layout(ns, nr, mat_bytes, 4 * 1024, adjoint, gmres_m)
    np.testing.assert_array_equal(a["size"], b["size"])
    assert not a["in_global"].any() and a["smem"] + a["glob"] == b["smem"] + b["glob"]


def test_layout_arguments():
    with pytest.raises(chemgb.ChemgbError):
        chemgb.cgx_layout(0, 10, 8, 1024)
    with pytest.raises(chemgb.ChemgbError):
        chemgb.cgx_layout(9, 21, 2, 1024)


def device_thermo(P, th, T):
    """The kernels' evaluation of a thermo table at T (c_p/R, h/(RT), s/R,
    d(c_p/R)/dT): the NASA-7 expressions when P = 4, Horner's rule above."""
    lnT, invT = np.log(T), 1.0 / T
    if P == 4:
        cp = th[0] + T * (th[1] + T * (th[2] + T * (th[3] + T * th[4])))
        h = th[0] + T * (th[5] + T * (th[6] + T * (th[7] + T * th[8]))) + th[9] * invT
        s = th[0] * lnT + T * (th[1] + T * (th[10] + T * (th[11] + T * th[12]))) + th[13]
        dcp = th[1] + T * (th[14] + T * (th[15] + T * th[16]))
        return cp, h, s, dcp
    cp = th[P].copy()
    for k in range(P - 1, -1, -1):
        cp = cp * T + th[k]
    hp = th[2 * P].copy()
    for k in range(P - 1, 0, -1):
        hp = hp * T + th[P + k]
    sp = th[3 * P].copy()
    for k in range(P - 1, 1, -1):
        sp = sp * T + th[2 * P + k]
    dp = th[4 * P].copy()
    for k in range(P - 1, 1, -1):
        dp = dp * T + th[3 * P + k]
    return cp, th[0] + T * hp + th[2 * P + 1] * invT, th[0] * lnT + T * (th[1] + T * sp) + th[3 * P + 1], \
        th[1] + T * dp


@pytest.mark.parametrize("n_p", [0, 2, 4, 7, 15])
def test_thermo_table_evaluates_to_the_oracles_thermo(n_p):
    """The table cg_mech_set_thermo uploads, evaluated as the kernels
    evaluate it, gives the oracle's c_p, h and s (Horner against the
    oracle's sum of powers: 1e-12 relative, 1e-10 at n_p = 15 where the
    terms are ~5e3 times the value), and d c_p/dT agrees with the oracle's
    c_p by finite differences; n_p = 4 reproduces the NASA-7 table."""
    import oracle
    m = inputs.with_thermo_degree(inputs.gen_mechanism("ch4"), n_p)
    r = oracle.RefMech(m)
    P, th = chemgb.cgx_thermo_table(m.thermo)
    assert P == max(n_p, 4) and th.shape == (4 * P + 1, m.ns)
    tol = 1e-10 if n_p == 15 else 1e-12
    Ri = inputs.R_UNIV / m.W
    for T in (300.0, 800.0, 1500.0, 2900.0):
        cp, h, s, dcp = device_thermo(P, th, T)
        o = r.thermo(T)
        np.testing.assert_allclose(cp * Ri, o["cp"], rtol=tol)
        np.testing.assert_allclose(h * Ri * T, o["h"], rtol=tol, atol=tol * np.abs(o["cp"] * T).max())
        np.testing.assert_allclose(s * Ri, o["s"], rtol=tol)
        fd = (r.thermo(T + 0.5)["cp"] - r.thermo(T - 0.5)["cp"]) / 1.0
        np.testing.assert_allclose(dcp * Ri, fd, rtol=1e-5, atol=1e-9 * np.abs(o["cp"]).max())
    if n_p == 4:
        P0, th0 = chemgb.cgx_thermo_table(m.nasa7)
        np.testing.assert_array_equal(th, th0)


def test_thermo_table_arguments():
    with pytest.raises(chemgb.ChemgbError):
        chemgb.cgx_thermo_table(np.zeros((3, 19)))          # degree 16
    bad = np.zeros((3, 10))
    bad[1, 2] = np.nan
    with pytest.raises(chemgb.ChemgbError):
        chemgb.cgx_thermo_table(bad)


@pytest.mark.parametrize("method", [0, 1, 2])
def test_library_tableaux_equal_the_oracles(method):
    """The Butcher tableaux the kernels use (computed by the library on the
    host, SDIRK-4 as the long-double root of its order conditions) equal the
    oracle's independently computed ones to rounding, and SDIRK-4 keeps the
    seven digits Appendix A.2 prints."""
    from oracle import tableau
    lib_t, ref = chemgb.cgx_tableau(method), tableau.tableau(method)
    assert lib_t["s"] == ref["s"] and lib_t["err_order"] == ref["err_order"]
    np.testing.assert_allclose(lib_t["A"], ref["A"], rtol=0, atol=1e-14)
    np.testing.assert_allclose(lib_t["b"], ref["b"], rtol=0, atol=1e-14)
    np.testing.assert_allclose(lib_t["bhat"], ref["bhat"], rtol=0, atol=1e-13)
    if method == 2:
        import os
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sdirk4_appendix_a2.txt")
        printed = dict((k, float(v)) for k, v in (ln.split() for ln in open(path)
                                                  if ln.strip() and not ln.startswith("#")))
        A = lib_t["A"]
        for k, v in printed.items():
            if k[0] == "a" and k != "aii":
                got = A[int(k[1]) - 1, int(k[2]) - 1]
            elif k[0] == "b":
                got = lib_t["b"][int(k[1]) - 1]
            else:
                got = A[0, 0]
            assert got == pytest.approx(v, rel=5e-7, abs=5e-9), k


def test_tableau_arguments():
    with pytest.raises(chemgb.ChemgbError):
        chemgb.cgx_tableau(99)
