"""Pins of the oracle's reaction rates and source term (Section 2.2).

Closed forms and limits: third-body with unit efficiencies, Lindemann low and
high pressure limits, Troe at f1 = 0, the extreme Troe parameters of
Appendix C.1, the reverse reaction's equilibrium constant, and conservation
of mass and of every element by omega."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2510_10005_gb300 import inputs

R = inputs.R_UNIV


def edit(mech, j, rtype=None, effs=None, troe=None, reverse=False):
    """Copy of mech with reaction j changed (type, efficiencies, Troe data)."""
    m = mech.copy()
    if rtype is not None:
        m.rtype[j] = rtype
    if troe is not None:
        m.troe[j] = troe
    if reverse:
        m.rf_idx[j], m.rr_idx[j] = mech.rr_idx[j].copy(), mech.rf_idx[j].copy()
        m.rf_nu[j], m.rr_nu[j] = mech.rr_nu[j].copy(), mech.rf_nu[j].copy()
    if effs is not None:
        idx, val, ptr = [], [], [0]
        for k in range(m.nr):
            if k == j:
                pairs = effs
            else:
                pairs = list(zip(mech.eff_idx[mech.eff_ptr[k]:mech.eff_ptr[k + 1]],
                                 mech.eff_val[mech.eff_ptr[k]:mech.eff_ptr[k + 1]]))
            for s, v in pairs:
                idx.append(int(s)); val.append(float(v))
            ptr.append(len(idx))
        m.eff_ptr = np.array(ptr, dtype=np.int32)
        m.eff_idx = np.array(idx, dtype=np.int32)
        m.eff_val = np.array(val)
    return m


def first(mech, t):
    return int(np.nonzero(mech.rtype == t)[0][0])


def test_third_body_unit_efficiencies(mechs):
    m = mechs["ch4"]
    j = first(m, inputs.RXN_THREE_BODY)
    T, C, p = inputs.random_states(m, 4, seed=2)
    tb = oracle.RefMech(edit(m, j, effs=[]))
    el = oracle.RefMech(edit(m, j, rtype=inputs.RXN_ELEMENTARY, effs=[]))
    for c in range(4):
        kf_tb = tb.rates(T[c], C[c])[0][j]
        kA = el.rates(T[c], C[c])[0][j]
        assert kf_tb == pytest.approx(C[c].sum() * kA, rel=1e-14)
    # with efficiencies: [M] = sum_i alpha_i C_i
    effs = [(0, 2.5), (3, 0.5)]
    tbe = oracle.RefMech(edit(m, j, effs=effs))
    for c in range(4):
        M = C[c].sum() + 1.5 * C[c][0] - 0.5 * C[c][3]
        assert tbe.rates(T[c], C[c])[0][j] == pytest.approx(M * el.rates(T[c], C[c])[0][j], rel=1e-14)


def _arrhenius(tr, T):
    return math.exp(tr[0] + tr[1] * math.log(T) - tr[2] / (R * T))


def test_lindemann_limits(mechs):
    m = mechs["ch4"]
    j = first(m, inputs.RXN_TROE)
    lm = oracle.RefMech(edit(m, j, rtype=inputs.RXN_LINDEMANN, effs=[]))
    T = 1300.0
    kinf, k0 = _arrhenius(m.arr[j], T), _arrhenius(m.arr0[j], T)
    X = np.full(m.ns, 1.0 / m.ns)
    lo = X * 1e-12   # Pr -> 0: k_f -> k_0 [M]
    hi = X * 1e12    # Pr -> infinity: k_f -> k_inf
    assert lm.rates(T, lo)[0][j] == pytest.approx(k0 * lo.sum(), rel=1e-8)
    assert lm.rates(T, hi)[0][j] == pytest.approx(kinf, rel=1e-8)
    # in between: k_inf Pr/(1+Pr)
    mid = X * 0.02
    Pr = k0 * mid.sum() / kinf
    assert lm.rates(T, mid)[0][j] == pytest.approx(kinf * Pr / (1 + Pr), rel=1e-13)


def test_troe_at_f1_zero_gives_fcent(mechs):
    """log10 Pr = -c makes f1 = 0, so F = F_cent exactly (eq. f_and_fcent)."""
    m = mechs["ch4"]
    j = first(m, inputs.RXN_TROE)
    alpha, T3, T1, T2 = 0.6, 200.0, 2000.0, 5000.0
    tm = oracle.RefMech(edit(m, j, effs=[], troe=[alpha, T3, T1, T2]))
    T = 1100.0
    Fc = (1 - alpha) * math.exp(-T / T3) + alpha * math.exp(-T / T1) + math.exp(-T2 / T)
    c = -0.4 - 0.67 * math.log10(Fc)
    kinf, k0 = _arrhenius(m.arr[j], T), _arrhenius(m.arr0[j], T)
    Pr = 10.0 ** (-c)
    Mtot = Pr * kinf / k0
    C = np.full(m.ns, Mtot / m.ns)
    kf = tm.rates(T, C)[0][j]
    assert kf == pytest.approx(kinf * Pr / (1 + Pr) * Fc, rel=1e-12)


def test_troe_extreme_parameters_and_missing_T2(mechs):
    """T3 = 1e-30, T1 = 1e30 (Appendix C.1): first F_cent term 0, second alpha;
    a missing T2 drops the third term."""
    m = mechs["ch4"]
    j = first(m, inputs.RXN_TROE)
    alpha = 0.3
    tm = oracle.RefMech(edit(m, j, effs=[], troe=[alpha, 1e-30, 1e30, np.nan]))
    T = 1500.0
    kinf, k0 = _arrhenius(m.arr[j], T), _arrhenius(m.arr0[j], T)
    C = np.full(m.ns, 0.01 / m.ns)
    Pr = k0 * C.sum() / kinf
    L = math.log10(alpha)
    c, n = -0.4 - 0.67 * L, 0.75 - 1.27 * L
    P = math.log10(Pr)
    f1 = (P + c) / (n - 0.14 * (P + c))
    F = 10.0 ** (L / (1 + f1 * f1))
    kf = tm.rates(T, C)[0][j]
    assert np.isfinite(kf)
    assert kf == pytest.approx(kinf * Pr / (1 + Pr) * F, rel=1e-12)


@pytest.mark.parametrize("kind", ["h2", "ch4"])
def test_reverse_reaction_inverts_equilibrium_constant(mechs, kind):
    """Writing a reaction backwards inverts K: (kf/kr) * (kf'/kr') = 1."""
    m = mechs[kind]
    T, C, p = inputs.random_states(m, 3, seed=5)
    base = oracle.RefMech(m)
    for j in range(0, m.nr, max(1, m.nr // 12)):
        rev = oracle.RefMech(edit(m, j, reverse=True))
        for c in range(3):
            kf, kr, _ = base.rates(T[c], C[c])
            kf2, kr2, _ = rev.rates(T[c], C[c])
            assert (kf[j] / kr[j]) * (kf2[j] / kr2[j]) == pytest.approx(1.0, rel=1e-11)


def test_equilibrium_constant_from_gibbs(mechs, ref):
    """K = kf/kr equals exp(-sum nu W g / RT) (p_ref/RT)^{sum nu} computed with
    numpy's power on the oracle's own species Gibbs energies: pins the
    integer-power expansion for sum(nu) = -1, 0, +1."""
    m, r = mechs["ch4"], ref["ch4"]
    T, C, p = inputs.random_states(m, 2, seed=7)
    seen = set()
    for c in range(2):
        g = r.thermo(T[c])["g"]
        kf, kr, _ = r.rates(T[c], C[c])
        for j in range(m.nr):
            nu = np.zeros(m.ns)
            for s in range(3):
                if m.rf_idx[j, s] >= 0:
                    nu[m.rf_idx[j, s]] -= m.rf_nu[j, s]
                if m.rr_idx[j, s] >= 0:
                    nu[m.rr_idx[j, s]] += m.rr_nu[j, s]
            dG = nu @ (m.W * g)
            K = np.exp(-dG / (R * T[c])) * np.power(101325.0 / (R * T[c]), nu.sum())
            assert kf[j] / kr[j] == pytest.approx(K, rel=1e-9)
            seen.add(int(nu.sum()))
    assert {-1, 0, 1} <= seen


@pytest.mark.parametrize("kind", ["h2", "ch4"])
@pytest.mark.parametrize("reactor", [oracle.CONV, oracle.CONP_LITERAL])
def test_mass_and_element_conservation(mechs, ref, kind, reactor):
    """sum_i W_i omega_i = 0 (eq. chemical-reaction-mass-conservation) and
    sum_i e_ki omega_i = 0 for every element k, relative to the magnitudes."""
    m, r = mechs[kind], ref[kind]
    T, C, p = inputs.random_states(m, 64, seed=11)
    S = r.source(T, C, reactor)
    w = S[:, 1:]
    mass = w * m.W
    assert np.all(np.abs(mass.sum(1)) <= 1e-13 * np.abs(mass).sum(1))
    for k in range(len(m.elements)):
        el = w * m.comp[:, k]
        assert np.all(np.abs(el.sum(1)) <= 1e-13 * np.abs(el).sum(1) + 1e-300)


def test_conservation_160_species():
    """Mass and every element conserved by omega at 160 species / 900
    reactions (C, H, O, N, Ar), on random states."""
    m = inputs.gen_mechanism("c7")
    r = oracle.RefMech(m)
    T, C, p = inputs.random_states(m, 16, seed=19)
    w = r.source(T, C, oracle.CONV)[:, 1:]
    mass = w * m.W
    assert np.all(np.abs(mass.sum(1)) <= 1e-13 * np.abs(mass).sum(1))
    for k in range(len(m.elements)):
        el = w * m.comp[:, k]
        assert np.all(np.abs(el.sum(1)) <= 1e-13 * np.abs(el).sum(1) + 1e-300)


def test_production_rates_are_stoichiometric_sums(mechs, ref):
    """omega_i = sum_j nu_ij q_j with the oracle's own q_j; omega_T from the
    oracle's own mass-specific u and c_v (eq. temperature_source)."""
    m, r = mechs["h2"], ref["h2"]
    T, C, p = inputs.random_states(m, 4, seed=13)
    nu = np.zeros((m.ns, m.nr))
    for j in range(m.nr):
        for s in range(3):
            if m.rf_idx[j, s] >= 0:
                nu[m.rf_idx[j, s], j] -= m.rf_nu[j, s]
            if m.rr_idx[j, s] >= 0:
                nu[m.rr_idx[j, s], j] += m.rr_nu[j, s]
    S = r.source(T, C, oracle.CONV)
    for c in range(4):
        q = r.rates(T[c], C[c])[2]
        w = nu @ q
        np.testing.assert_allclose(S[c, 1:], w, rtol=1e-12, atol=1e-14 * np.abs(nu).dot(np.abs(q)).max())
        th = r.thermo(T[c])
        wT = -np.sum(m.W * th["u"] * w) / np.sum(m.W * C[c] * th["cv"])
        assert S[c, 0] == pytest.approx(wT, rel=1e-10, abs=1e-12 * np.abs(m.W * th["u"] * w).sum())


def test_conp_keeps_pressure_and_enthalpy_rates_zero(mechs, ref):
    """Constant-pressure form: d(T sum C)/dt = 0 (p fixed), and with the
    chemical production omega (the CONP_LITERAL rows) the parcel enthalpy
    rate sum W_i h_i omega_i + rho c_p omega_T vanishes (Appendix B)."""
    m, r = mechs["ch4"], ref["ch4"]
    T, C, p = inputs.random_states(m, 16, seed=17)
    S = r.source(T, C, oracle.CONP)
    L = r.source(T, C, oracle.CONP_LITERAL)
    for c in range(16):
        th = r.thermo(T[c])
        dpdt = S[c, 0] * C[c].sum() + T[c] * S[c, 1:].sum()
        assert abs(dpdt) <= 1e-12 * (abs(S[c, 0] * C[c].sum()) + T[c] * np.abs(S[c, 1:]).sum())
        w, wT = L[c, 1:], L[c, 0]
        assert S[c, 0] == wT
        s_dil = wT / T[c] + w.sum() / C[c].sum()
        np.testing.assert_allclose(S[c, 1:], w - C[c] * s_dil, rtol=1e-12,
                                   atol=1e-13 * np.abs(w).max())
        dH = np.sum(m.W * th["h"] * w) + np.sum(m.W * C[c] * th["cp"]) * wT
        assert abs(dH) <= 1e-12 * np.abs(m.W * th["h"] * w).sum()


def _golden_h_o2():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "h_o2_section_4_3.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    (name, A, b, Ea), = rows
    return name, float(A), float(b), float(Ea)


def test_golden_h_o2_example_of_section_4_3(mechs):
    """The printed example of the generation process (Section 4.3): H + O2
    <=> O + OH with A = 1.0399e11 m^3/kmol/s, b = 0, Ea = 6.405704e7 J/kmol
    in SI-kmol units. The oracle's k_f is A exp(-Ea/(R T)) at every T, and
    the rate of progress is the printed form [H][O2] k_f - [O][OH] k_f / K
    with K = exp(-Delta G/RT) and no pressure factor (sum nu = 0)."""
    name, A, b, Ea = _golden_h_o2()
    assert name == "H+O2<=>O+OH"
    m = mechs["h2"].copy()
    sp = {s: m.index(s) for s in ("H", "O2", "O", "OH")}
    m.rtype[0] = inputs.RXN_ELEMENTARY
    m.rf_idx[0], m.rf_nu[0] = [sp["H"], sp["O2"], -1], [1, 1, 0]
    m.rr_idx[0], m.rr_nu[0] = [sp["O"], sp["OH"], -1], [1, 1, 0]
    m.arr[0] = (math.log(A), b, Ea)
    m.eff_idx = m.eff_idx[m.eff_ptr[1] - m.eff_ptr[0]:]
    m.eff_val = m.eff_val[m.eff_ptr[1] - m.eff_ptr[0]:]
    m.eff_ptr = m.eff_ptr - m.eff_ptr[1]
    m.eff_ptr[0] = 0
    m.validate()
    r = oracle.RefMech(m)
    T, C, p = inputs.random_states(m, 4, seed=11)
    for Tc in (800.0, 1500.0, 2500.0):
        for c in range(4):
            kf, kr, q = r.rates(Tc, C[c])
            assert kf[0] == pytest.approx(A * math.exp(-Ea / (R * Tc)), rel=1e-13)
            g = r.thermo(Tc)["g"]
            dG = (m.W[sp["O"]] * g[sp["O"]] + m.W[sp["OH"]] * g[sp["OH"]]
                  - m.W[sp["H"]] * g[sp["H"]] - m.W[sp["O2"]] * g[sp["O2"]])
            K = math.exp(-dG / (R * Tc))
            expect = C[c, sp["H"]] * C[c, sp["O2"]] * kf[0] - C[c, sp["O"]] * C[c, sp["OH"]] * kf[0] / K
            assert q[0] == pytest.approx(expect, rel=1e-10, abs=1e-12 * abs(kf[0] * C[c, sp["H"]] * C[c, sp["O2"]]))
    # about 4.7e7 m^3/kmol/s at 1000 K (1.0399e11 e^-7.70)
    assert r.rates(1000.0, C[0])[0][0] == pytest.approx(4.7e7, rel=0.02)


@pytest.mark.parametrize("reverse", [False, True])
def test_equilibrium_constant_sum_nu_two(mechs, reverse):
    """The integer-power form of (p_ref/RT)^{sum nu} agrees with pow() at
    sum nu = -2 (2 H + O <=> H2O) and +2 (the reaction reversed), which the
    generated mechanisms never reach (Section 2.2, eq. equilibrium-constant-1)."""
    m = mechs["h2"].copy()
    H, O, H2O = m.index("H"), m.index("O"), m.index("H2O")
    m.rtype[0] = inputs.RXN_ELEMENTARY
    lhs, rhs = ([H, O, -1], [2, 1, 0]), ([H2O, -1, -1], [1, 0, 0])
    if reverse:
        lhs, rhs = rhs, lhs
    m.rf_idx[0], m.rf_nu[0] = lhs
    m.rr_idx[0], m.rr_nu[0] = rhs
    n0 = m.eff_ptr[1] - m.eff_ptr[0]
    m.eff_idx, m.eff_val = m.eff_idx[n0:], m.eff_val[n0:]
    m.eff_ptr = np.concatenate([[0], m.eff_ptr[1:] - n0]).astype(np.int32)
    m.validate()
    r = oracle.RefMech(m)
    nu = np.zeros(m.ns)
    for idx, n, sgn in ((m.rf_idx[0], m.rf_nu[0], -1), (m.rr_idx[0], m.rr_nu[0], 1)):
        for s in range(3):
            if idx[s] >= 0:
                nu[idx[s]] += sgn * n[s]
    assert nu.sum() == (2 if reverse else -2)
    T, C, _ = inputs.random_states(m, 3, seed=12)
    for c in range(3):
        kf, kr, _ = r.rates(T[c], C[c])
        g = r.thermo(T[c])["g"]
        K = np.exp(-(nu @ (m.W * g)) / (R * T[c])) * np.power(101325.0 / (R * T[c]), nu.sum())
        assert kf[0] / kr[0] == pytest.approx(K, rel=1e-12)


def test_three_species_sides():
    """Reactions with three species on one side (H + OH + H2 <=> H2O + H2,
    HO2 + N2 <=> H + O2 + N2): k_f is the Arrhenius closed form, q is the
    mass-action difference with all three concentration factors, K = kf/kr
    carries (p_ref/RT)^{sum nu} at sum nu = -1 and +1 from the three-slot
    side, and the oracle's Jacobian equals complex-step derivatives of its S
    (CONV and CONP)."""
    from test_oracle_jacobian import complex_step_jacobian
    m = inputs.with_three_species_sides(inputs.gen_mechanism("h2"))
    r = oracle.RefMech(m)
    sp = {s: m.names.index(s) for s in ("H", "OH", "H2", "H2O", "HO2", "O2", "N2")}
    T, C, _ = inputs.random_states(m, 4, seed=13)
    j1, j2 = m.nr - 2, m.nr - 1
    for c in range(4):
        kf, kr, q = r.rates(T[c], C[c])
        assert kf[j1] == pytest.approx(1e10, rel=1e-13)
        assert kf[j2] == pytest.approx(1e12 * math.exp(-48.0 * inputs.CAL / (R * T[c])), rel=1e-12)
        x = C[c]
        fwd1, rev1 = kf[j1] * x[sp["H"]] * x[sp["OH"]] * x[sp["H2"]], kr[j1] * x[sp["H2O"]] * x[sp["H2"]]
        fwd2, rev2 = kf[j2] * x[sp["HO2"]] * x[sp["N2"]], kr[j2] * x[sp["H"]] * x[sp["O2"]] * x[sp["N2"]]
        assert q[j1] == pytest.approx(fwd1 - rev1, rel=1e-12, abs=1e-13 * (fwd1 + rev1))
        assert q[j2] == pytest.approx(fwd2 - rev2, rel=1e-12, abs=1e-13 * (fwd2 + rev2))
        g = r.thermo(T[c])["g"]
        for j, dG, snu in ((j1, g[sp["H2O"]] * m.W[sp["H2O"]] - g[sp["H"]] * m.W[sp["H"]]
                            - g[sp["OH"]] * m.W[sp["OH"]], -1),
                           (j2, g[sp["H"]] * m.W[sp["H"]] + g[sp["O2"]] * m.W[sp["O2"]]
                            - g[sp["HO2"]] * m.W[sp["HO2"]], 1)):
            K = math.exp(-dG / (R * T[c])) * (101325.0 / (R * T[c])) ** snu
            assert kf[j] / kr[j] == pytest.approx(K, rel=1e-11)
        y = np.concatenate([[T[c]], C[c]])
        for reactor in (oracle.CONV, oracle.CONP):
            Ja = r.jacobian(T[c], C[c], reactor)[0]
            Jc = complex_step_jacobian(r, y, reactor)
            scale = np.maximum(np.abs(Jc), 1e-13 * np.abs(Jc).max(axis=1, keepdims=True) + 1e-300)
            assert np.max(np.abs(Ja - Jc) / scale) < 1e-10
