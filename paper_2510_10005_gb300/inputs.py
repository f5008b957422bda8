"""Seeded synthetic inputs: reaction mechanisms and cell fields.

This module is shared by the CUDA path, the oracle and the tests. It holds
no arithmetic of the integration method itself: it never evaluates
thermodynamic properties of cells, rates, source terms or Jacobians. It
draws mechanism parameters (and fits the c_p polynomials of a mechanism to
its drawn curves, anchored at 298.15 K) and cell states from seeded
distributions shaped like the workloads the paper studies (Table 2:
mechanisms of 10-96 species and 27-1054 reactions; Section 5.1 random-state
recipe; Section 5.3 homogeneous reactor initial conditions).

Units are SI-kmol throughout: concentrations in kmol/m^3, activation
energies in J/kmol, pressures in Pa, molecular masses in kg/kmol, and the
pre-exponential factor A in (m^3/kmol)^(order-1)/s (Section 4.3: the H+O2
example states its Arrhenius data in these units).

Mechanism arrays (all numpy):
  names[ns], elements[ne], comp[ns, ne] (int atom counts), W[ns] kg/kmol,
  nasa7[ns, 7]  (a1..a5: cp/R polynomial; a6: h/R constant; a7: s/R constant,
                 one range used over the whole temperature domain),
  thermo[ns, n_p + 3] or None  a c_p/R polynomial of another degree n_p in the
                 same layout (a_0..a_np, h/R constant, s/R constant; Section 2.1,
                 Appendix C.1); None means nasa7 (n_p = 4) is the thermodynamics,
  cp_src[ns, 5] or None  the drawn curve the polynomials are fitted to:
                 (c_lo, c_hi, theta, h_f(298.15 K) J/kmol, s(298.15 K) J/(kmol K)),
  rtype[nr]     (0 elementary, 1 third-body, 2 Lindemann, 3 Troe, 4 SRI falloff,
                 5 pressure-dependent Arrhenius "PLOG"),
  reversible[nr],
  rf_idx[nr,3], rf_nu[nr,3], rr_idx[nr,3], rr_nu[nr,3]  (-1 / 0 padded),
  arr[nr,3]     (ln A, b, Ea)      high-pressure / plain Arrhenius triple,
  arr0[nr,3]    (ln A0, b0, Ea0)   low-pressure triple of falloff reactions,
  troe[nr,4]    (alpha, T3, T1, T2); T2 = NaN means the term is absent,
  eff_ptr[nr+1], eff_idx[...], eff_val[...]  CSR of efficiencies != 1,
  sri[nr,5]     (a, b, c, d, e) of SRI falloff reactions (zeros otherwise),
  plog_ptr[nr+1], plog[K,4]  CSR of PLOG rate expressions (p in Pa, ln A, b,
                 Ea), sorted by pressure; equal pressures may repeat.
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np

R_UNIV = 8314.46261815324      # J/(kmol K)
P_ATM = 101325.0               # Pa
CAL = 4.184e6                  # J/kmol per kcal/mol

RXN_ELEMENTARY, RXN_THREE_BODY, RXN_LINDEMANN, RXN_TROE, RXN_SRI, RXN_PLOG = 0, 1, 2, 3, 4, 5

_ATOMIC_MASS = {"C": 12.011, "H": 1.008, "O": 15.999, "N": 14.007, "Ar": 39.95}
_VALENCE = {"C": 4, "H": 1, "O": 2, "N": 3, "Ar": 0}
_INIT_EA = (30.0, 50.0)   # kcal/mol, activation energy of initiation steps


@dataclasses.dataclass
class Mechanism:
    names: list
    elements: list
    comp: np.ndarray
    W: np.ndarray
    nasa7: np.ndarray
    rtype: np.ndarray
    reversible: np.ndarray
    rf_idx: np.ndarray
    rf_nu: np.ndarray
    rr_idx: np.ndarray
    rr_nu: np.ndarray
    arr: np.ndarray
    arr0: np.ndarray
    troe: np.ndarray
    eff_ptr: np.ndarray
    eff_idx: np.ndarray
    eff_val: np.ndarray
    sri: np.ndarray = None
    plog_ptr: np.ndarray = None
    plog: np.ndarray = None
    thermo: np.ndarray = None
    cp_src: np.ndarray = None

    def __post_init__(self):
        nr = int(self.rtype.shape[0])
        if self.sri is None:
            self.sri = np.zeros((nr, 5))
        if self.plog_ptr is None:
            self.plog_ptr = np.zeros(nr + 1, dtype=np.int32)
        if self.plog is None:
            self.plog = np.zeros((0, 4))

    @property
    def thermo_np(self) -> int:
        """Degree n_p of the c_p polynomial (4 for NASA-7)."""
        return 4 if self.thermo is None else int(self.thermo.shape[1]) - 3

    @property
    def thermo_coef(self) -> np.ndarray:
        """[ns, n_p + 3]: a_0..a_np of c_p/R, then the h/R and s/R constants."""
        return self.nasa7 if self.thermo is None else self.thermo

    @property
    def ns(self) -> int:
        return len(self.names)

    @property
    def nr(self) -> int:
        return int(self.rtype.shape[0])

    def index(self, name: str) -> int:
        return self.names.index(name)

    def copy(self) -> "Mechanism":
        def dup(v):
            if isinstance(v, np.ndarray):
                return np.array(v, copy=True)
            return list(v) if isinstance(v, list) else v
        return dataclasses.replace(self, **{f.name: dup(getattr(self, f.name)) for f in dataclasses.fields(self)})

    def validate(self) -> None:
        """Structural checks: index ranges, padding and element balance."""
        ns, nr = self.ns, self.nr
        assert self.nasa7.shape == (ns, 7) and self.W.shape == (ns,)
        if self.thermo is not None:
            assert self.thermo.ndim == 2 and self.thermo.shape[0] == ns and 3 <= self.thermo.shape[1] <= 18
        assert self.cp_src is None or self.cp_src.shape == (ns, 5)
        for a in (self.rf_idx, self.rf_nu, self.rr_idx, self.rr_nu):
            assert a.shape == (nr, 3)
        assert self.arr.shape == (nr, 3) and self.arr0.shape == (nr, 3)
        assert self.troe.shape == (nr, 4) and self.eff_ptr.shape == (nr + 1,)
        assert self.sri.shape == (nr, 5) and self.plog_ptr.shape == (nr + 1,)
        assert self.plog_ptr[0] == 0 and self.plog_ptr[-1] == len(self.plog) and np.all(np.diff(self.plog_ptr) >= 0)
        for idx, nu in ((self.rf_idx, self.rf_nu), (self.rr_idx, self.rr_nu)):
            assert np.all((idx >= -1) & (idx < ns))
            assert np.all((idx >= 0) == (nu > 0))
        assert np.all(np.diff(self.eff_ptr) >= 0) and self.eff_ptr[0] == 0
        assert self.eff_ptr[-1] == len(self.eff_idx) == len(self.eff_val)
        assert np.all((self.eff_idx >= 0) & (self.eff_idx < ns))
        for j in range(nr):
            bal = np.zeros(len(self.elements), dtype=np.int64)
            for s in range(3):
                if self.rf_idx[j, s] >= 0:
                    bal -= self.rf_nu[j, s] * self.comp[self.rf_idx[j, s]]
                if self.rr_idx[j, s] >= 0:
                    bal += self.rr_nu[j, s] * self.comp[self.rr_idx[j, s]]
            assert not bal.any(), f"reaction {j} is not element balanced"
            if self.rtype[j] in (RXN_ELEMENTARY, RXN_PLOG):
                assert self.eff_ptr[j + 1] == self.eff_ptr[j]
            if self.rtype[j] == RXN_PLOG:
                pts = self.plog[self.plog_ptr[j]:self.plog_ptr[j + 1]]
                assert len(pts) >= 1 and np.all(np.diff(pts[:, 0]) >= 0) and np.all(pts[:, 0] > 0)
            else:
                assert self.plog_ptr[j + 1] == self.plog_ptr[j]

    def equation(self, j: int) -> str:
        def side(idx, nu):
            t = []
            for s in range(3):
                if idx[j, s] >= 0:
                    t.append((f"{nu[j, s]} " if nu[j, s] > 1 else "") + self.names[idx[j, s]])
            return " + ".join(t)
        tb = {1: " + M", 2: " (+M)", 3: " (+M)", 4: " (+M)"}.get(int(self.rtype[j]), "")
        arrow = " <=> " if self.reversible[j] else " => "
        return side(self.rf_idx, self.rf_nu) + tb + arrow + side(self.rr_idx, self.rr_nu) + tb

    def save(self, path: str) -> None:
        np.savez(path, names=np.array(self.names), elements=np.array(self.elements),
                 **{f.name: getattr(self, f.name) for f in dataclasses.fields(self)
                    if f.name not in ("names", "elements") and getattr(self, f.name) is not None})

    @staticmethod
    def load(path: str) -> "Mechanism":
        z = np.load(path, allow_pickle=False)
        kw = {f.name: z[f.name] for f in dataclasses.fields(Mechanism) if f.name in z}
        kw["names"] = [str(s) for s in kw["names"]]
        kw["elements"] = [str(s) for s in kw["elements"]]
        return Mechanism(**kw)


# ----------------------------------------------------------------------------
# species sets


def _formula(counts: dict) -> str:
    s = ""
    for e in ("C", "H", "O", "N", "Ar"):
        c = counts.get(e, 0)
        if c:
            s += e + (str(c) if c > 1 else "")
    return s


def _parse(formula: str) -> dict:
    out, i = {}, 0
    while i < len(formula):
        e = "Ar" if formula.startswith("Ar", i) else formula[i]
        i += len(e)
        j = i
        while j < len(formula) and formula[j].isdigit():
            j += 1
        out[e] = out.get(e, 0) + (int(formula[i:j]) if j > i else 1)
        i = j
    return out


def _lattice(cmax, hmax, omax, nmax):
    out = []
    for c, h, o, n in itertools.product(range(cmax + 1), range(hmax + 1),
                                        range(omax + 1), range(nmax + 1)):
        nat = c + h + o + n
        if nat == 0 or h > 2 * c + 2 + n:
            continue
        if nat == 1 and h == 1:
            pass
        out.append({"C": c, "H": h, "O": o, "N": n})
    return out


def _species_set(kind: str, rng: np.random.Generator) -> list:
    if kind == "h2":
        return ["H2", "O2", "H2O", "H", "O", "OH", "HO2", "H2O2", "N2"]
    if kind == "ch4":
        required = ["H2", "O2", "H2O", "CO", "CO2", "N2", "Ar", "H", "O", "OH", "CH4"]
        lattice, total = _lattice(2, 6, 2, 1), 53
    elif kind == "c7":
        required = ["H2", "O2", "H2O", "CO", "CO2", "N2", "H", "O", "OH", "HO2", "C7H16"]
        lattice, total = _lattice(7, 16, 2, 1), 160
    else:
        raise ValueError(kind)
    req_f = {_formula(_parse(s)) for s in required}
    pool = [d for d in lattice if _formula(d) not in req_f]
    pick = rng.choice(len(pool), size=total - len(required), replace=False)
    return required + [_formula(pool[i]) for i in sorted(pick)]


# ----------------------------------------------------------------------------
# thermodynamic data (drawn, then fitted to the NASA-7 form)


T_FIT = (300.0, 3000.0)   # K, range of the c_p fits
T_ANCHOR = 298.15         # K, where h and s of a fit equal the drawn values


def fit_thermo(src: np.ndarray, n_p: int) -> np.ndarray:
    """Coefficients [n_p + 3] of one species fitted to its drawn curve
    src = (c_lo, c_hi, theta, h_f, s_298): c_p/R = c_lo + (c_hi - c_lo)
    (1 - exp(-T/theta)) fitted by least squares on 200 points over 300-3000 K
    with a polynomial of degree n_p (Section 2.1, eq.
    specific_heat_polynomial); the h/R and s/R constants make h and s equal
    h_f and s_298 at 298.15 K (eq. enthalpy-adjustment and its entropy
    analogue). n_p = 4 gives the NASA-7 row of the same species."""
    c_lo, c_hi, theta, hf, s298 = (float(v) for v in src)
    Tg = np.linspace(T_FIT[0], T_FIT[1], 200)
    cp = c_lo + (c_hi - c_lo) * (1.0 - np.exp(-Tg / theta))
    V = np.vander(Tg / 1000.0, n_p + 1, increasing=True)
    coef = np.linalg.lstsq(V, cp, rcond=None)[0] / 1000.0 ** np.arange(n_p + 1)
    T0 = T_ANCHOR
    h_int = sum(coef[k] * T0 ** (k + 1) / (k + 1) for k in range(n_p + 1))
    s_int = coef[0] * math.log(T0) + sum(coef[k] * T0 ** k / k for k in range(1, n_p + 1))
    return np.concatenate([coef, [hf / R_UNIV - h_int, s298 / R_UNIV - s_int]])


def with_thermo_degree(mech: Mechanism, n_p: int) -> Mechanism:
    """A copy of `mech` whose thermodynamics is refitted with a c_p
    polynomial of degree n_p (Appendix C.1 refits to n_p = 7 and 15) to the
    same drawn curves; needs `cp_src` (generated mechanisms carry it)."""
    if mech.cp_src is None:
        raise ValueError("the mechanism carries no source curves (cp_src) to refit")
    if not 0 <= n_p <= 15:
        raise ValueError("n_p must lie in [0, 15]")
    m = mech.copy()
    m.thermo = np.array([fit_thermo(src, n_p) for src in m.cp_src])
    m.validate()
    return m


def _nasa7_for(counts: dict, rng: np.random.Generator) -> np.ndarray:
    """Draw a smooth cp/R(T) curve, h_f(298) and s(298); fit NASA-7 to it.

    cp/R(T) = c_lo + (c_hi - c_lo) (1 - exp(-T/theta)) on 300-3000 K, fitted
    by least squares with a quartic (Section 2.1, eq. specific_heat_polynomial
    with n_p = 4); a6 and a7 anchor h and s at 298.15 K as the paper's
    enthalpy adjustment (eq. enthalpy-adjustment) does for h_ref.
    Returns (NASA-7 row, h_f, s_298, radical, source curve).
    """
    nat = sum(counts.values())
    if nat == 1:
        c_lo = c_hi = 2.5
    elif nat == 2:
        c_lo, c_hi = 3.5, 4.5
    else:
        c_lo, c_hi = 4.0, 3.0 * nat - 2.0
    theta = rng.uniform(500.0, 1500.0)

    # formation enthalpy: oxidised species are stable, open-shell ones are not
    h_, c_, o_, n_ = counts.get("H", 0), counts.get("C", 0), counts.get("O", 0), counts.get("N", 0)
    valence = sum(_VALENCE[e] * k for e, k in counts.items())
    radical = (valence % 2 == 1) or (nat == 1 and counts.get("Ar", 0) == 0)
    if _formula(counts) in ("H2", "O2", "N2", "Ar"):
        hf = 0.0
    else:
        ox = min(o_, h_ / 2.0 + 2.0 * c_)
        hf = -250e6 * ox + (rng.uniform(150e6, 250e6) if radical else 0.0)
        hf += rng.uniform(-30e6, 30e6) + 10e6 * (nat - 1) * rng.uniform(-1, 1)
    s298 = (rng.uniform(110e3, 150e3) + 25e3 * (nat - 1))        # J/(kmol K)

    src = np.array([c_lo, c_hi, theta, hf, s298])
    return fit_thermo(src, 4), hf, s298, radical, src


# ----------------------------------------------------------------------------
# reaction network


_SIZES = {"h2": (9, 21, 4, 1, 0), "ch4": (53, 325, 32, 24, 2), "c7": (160, 900, 60, 44, 4)}


def gen_mechanism(kind: str = "h2", seed: int | None = None) -> Mechanism:
    """Synthetic element-balanced mechanism.

    kind: "h2"  9 species of H/O/N, 21 reactions (4 third-body, 1 Troe);
          "ch4" 53 species of C/H/O/N/Ar, 325 reactions (~10% third-body,
                ~8% falloff);
          "c7"  160 species, 900 reactions (~12% third-body/falloff).
    All reactions are reversible and written in their exergonic direction at
    1000 K. A is log-uniform in [1e6, 1e14] SI-kmol as the rate scale at
    1000 K, b in U[-1.5, 1.5], Ea in U[0, 40] kcal/mol (converted to J/kmol),
    except reactions whose reactants are all closed-shell: U[30, 50] kcal/mol.
    """
    default_seed = {"h2": 0, "ch4": 1, "c7": 2}[kind]
    rng = np.random.default_rng(default_seed if seed is None else seed)
    ns_target, nr, n_tb, n_troe, n_lind = _SIZES[kind]
    names = _species_set(kind, rng)
    assert len(names) == ns_target
    elements = [e for e in ("C", "H", "O", "N", "Ar") if any(e in _parse(s) for s in names)]
    counts = [_parse(s) for s in names]
    comp = np.array([[c.get(e, 0) for e in elements] for c in counts], dtype=np.int64)
    W = np.array([sum(_ATOMIC_MASS[e] * k for e, k in c.items()) for c in counts])
    thermo = [_nasa7_for(c, rng) for c in counts]
    nasa7 = np.array([t[0] for t in thermo])
    hf = np.array([t[1] for t in thermo])
    s298 = np.array([t[2] for t in thermo])
    radical = np.array([t[3] for t in thermo])
    cp_src = np.array([t[4] for t in thermo])
    ns = len(names)

    # candidate reactions: 1<->2 (dissociation) and 2<->2 (exchange)
    keys = {}
    for i in range(ns):
        for j in range(i, ns):
            keys.setdefault(tuple(comp[i] + comp[j]), []).append((i, j))
    single = {tuple(comp[k]): k for k in range(ns)}
    diss, exch = [], []
    for key, pairs in keys.items():
        k = single.get(key)
        if k is not None:
            for (i, j) in pairs:
                if k not in (i, j):
                    diss.append(((k,), (i, j)))
        for a in range(len(pairs)):
            for b in range(a + 1, len(pairs)):
                if not set(pairs[a]) & set(pairs[b]):
                    exch.append((pairs[a], pairs[b]))

    def dG1000(lhs, rhs):
        # estimate from the drawn 298 K data only: (dH - T dS) / (R T) at 1000 K
        dh = sum(hf[i] for i in rhs) - sum(hf[i] for i in lhs)
        ds = sum(s298[i] for i in rhs) - sum(s298[i] for i in lhs)
        return (dh - 1000.0 * ds) / (R_UNIV * 1000.0)

    def dG_ok(lhs, rhs):
        return abs(dG1000(lhs, rhs)) <= 60.0

    diss = [c for c in diss if dG_ok(*c)]
    exch = [c for c in exch if dG_ok(*c)]
    n_fall = n_troe + n_lind
    n_press = n_tb + n_fall
    assert len(diss) >= n_press, "not enough dissociation candidates"

    di = rng.permutation(len(diss))
    chosen = [diss[i] for i in di[:n_press]]
    pool = [(c, 1) for c in (diss[i] for i in di[n_press:])] + [(c, 2) for c in exch]
    pool_order = rng.permutation(len(pool))
    # calibration: the H/O radical core and the fuel's reactions with radicals
    # come first, so that the larger mechanisms keep a chain that can run away
    rest = []
    if kind != "h2":
        core = {i for i, nm in enumerate(names)
                if nm in ("H2", "O2", "H2O", "H", "O", "OH", "HO2", "H2O2")}
        fuel = names.index("CH4" if kind == "ch4" else "C7H16")
        for p in pool_order:
            c, _ = pool[p]
            sp = set(c[0]) | set(c[1])
            fuel_rad = fuel in sp and any(radical[x] for x in sp if x != fuel)
            if (sp <= core or fuel_rad) and c not in rest and len(rest) < nr // 3:
                rest.append(c)
    # then make every species that has a candidate appear at least once
    used = set(s for c in chosen + rest for side in c for s in side)
    for p in pool_order:
        c, _ = pool[p]
        sp = set(c[0]) | set(c[1])
        if len(chosen) + len(rest) < nr and not sp <= used:
            rest.append(c)
            used |= sp
    for p in pool_order:
        if len(chosen) + len(rest) >= nr:
            break
        c, _ = pool[p]
        if c not in rest:
            rest.append(c)
    chosen = chosen + rest[: nr - len(chosen)]
    assert len(chosen) == nr

    rtype = np.zeros(nr, dtype=np.int32)
    rtype[:n_tb] = RXN_THREE_BODY
    rtype[n_tb:n_tb + n_troe] = RXN_TROE
    rtype[n_tb + n_troe:n_press] = RXN_LINDEMANN
    perm = rng.permutation(nr)
    chosen = [chosen[i] for i in perm]
    rtype = rtype[perm]

    rf_idx = -np.ones((nr, 3), dtype=np.int32)
    rr_idx = -np.ones((nr, 3), dtype=np.int32)
    rf_nu = np.zeros((nr, 3), dtype=np.int32)
    rr_nu = np.zeros((nr, 3), dtype=np.int32)
    for j, (lhs, rhs) in enumerate(chosen):
        # written in the exergonic direction at 1000 K, so that the reverse
        # rate k_f / K never exceeds the forward one there
        if dG1000(lhs, rhs) > 0.0:
            lhs, rhs = rhs, lhs
        for idx, nu, side in ((rf_idx, rf_nu, lhs), (rr_idx, rr_nu, rhs)):
            uniq = sorted(set(side))
            for s, sp in enumerate(uniq):
                idx[j, s] = sp
                nu[j, s] = side.count(sp)

    # A is drawn as the rate scale at T_ref = 1000 K, k = A (T/T_ref)^b exp(-E/RT),
    # and stored in the paper's form A' T^b exp(-E/RT) with A' = A T_ref^-b
    b = rng.uniform(-1.5, 1.5, nr)
    lnA = np.log(10.0 ** rng.uniform(6.0, 14.0, nr)) - b * math.log(1000.0)
    Ea = rng.uniform(0.0, 40.0, nr) * CAL
    # calibration: a reaction among closed-shell molecules only (an initiation
    # step) gets Ea in U[30, 50] kcal/mol, so that unburnt gas stays frozen at
    # 300-800 K while the radical chain still runs away above ~1000 K
    for j in range(nr):
        if not any(radical[rf_idx[j, s]] for s in range(3) if rf_idx[j, s] >= 0):
            Ea[j] = rng.uniform(*_INIT_EA) * CAL
    arr = np.stack([lnA, b, Ea], axis=1)
    arr0 = np.zeros((nr, 3))
    troe = np.zeros((nr, 4))
    eff_ptr = np.zeros(nr + 1, dtype=np.int32)
    eff_idx, eff_val = [], []
    for j in range(nr):
        if rtype[j] in (RXN_LINDEMANN, RXN_TROE):
            # k0/kinf = U[1e1, 1e4] m^3/kmol at 1000 K, with its own b and Ea
            b0 = b[j] + rng.uniform(-1.0, 0.0)
            Ea0 = max(0.0, Ea[j] - rng.uniform(0.0, 10.0) * CAL)
            ratio = rng.uniform(1e1, 1e4)
            lnA0 = lnA[j] + math.log(ratio) + (b[j] - b0) * math.log(1000.0) \
                - (Ea[j] - Ea0) / (R_UNIV * 1000.0)
            arr0[j] = (lnA0, b0, Ea0)
        if rtype[j] == RXN_TROE:
            T2 = rng.uniform(1000.0, 10000.0) if rng.random() < 0.5 else np.nan
            troe[j] = (rng.uniform(0.1, 0.9), rng.uniform(50.0, 500.0),
                       rng.uniform(500.0, 5000.0), T2)
        if rtype[j] != RXN_ELEMENTARY:
            k = int(rng.integers(3, 7))
            sp = sorted(rng.choice(ns, size=min(k, ns), replace=False))
            eff_idx.extend(int(s) for s in sp)
            eff_val.extend(float(v) for v in rng.uniform(0.5, 3.0, len(sp)))
        eff_ptr[j + 1] = len(eff_idx)

    mech = Mechanism(names=names, elements=elements, comp=comp, W=W, nasa7=nasa7,
                     rtype=rtype, reversible=np.ones(nr, dtype=np.int32),
                     rf_idx=rf_idx, rf_nu=rf_nu, rr_idx=rr_idx, rr_nu=rr_nu,
                     arr=arr, arr0=arr0, troe=troe, eff_ptr=eff_ptr,
                     eff_idx=np.array(eff_idx, dtype=np.int32),
                     eff_val=np.array(eff_val, dtype=np.float64), cp_src=cp_src)
    mech.validate()
    return mech


def with_sri_plog(mech: Mechanism, n_sri: int, n_plog: int, seed: int = 0) -> Mechanism:
    """A copy of `mech` in which n_sri Troe reactions take SRI broadening
    (Section 2.2.3: a in U[0.5, 2], b in U[100, 1000] K, c in U[500, 5000] K,
    d in U[0.8, 1.2], e in U[-0.5, 0.5]) and n_plog elementary reactions
    become pressure-dependent Arrhenius (PLOG, Section 2.2.4) with 3-6
    pressures log-spaced over 0.1-100 atm, each rate the original one
    perturbed (ln A + N(0, 0.5), b + N(0, 0.1), Ea + N(0, 1 kcal/mol)); every
    other PLOG reaction repeats one pressure with a second, smaller rate
    (the rule that rates given at one pressure add)."""
    rng = np.random.default_rng(seed)
    m = mech.copy()
    nr = m.nr
    troe = [j for j in range(nr) if m.rtype[j] == RXN_TROE]
    elem = [j for j in range(nr) if m.rtype[j] == RXN_ELEMENTARY]
    for j in rng.choice(troe, size=min(n_sri, len(troe)), replace=False):
        m.rtype[j] = RXN_SRI
        m.sri[j] = (rng.uniform(0.5, 2.0), rng.uniform(100.0, 1000.0), rng.uniform(500.0, 5000.0),
                    rng.uniform(0.8, 1.2), rng.uniform(-0.5, 0.5))
        m.troe[j] = 0.0
    chosen = set(int(j) for j in rng.choice(elem, size=min(n_plog, len(elem)), replace=False))
    ptr, rows, count = [0], [], 0
    for j in range(nr):
        if j in chosen:
            count += 1
            m.rtype[j] = RXN_PLOG
            k = int(rng.integers(3, 7))
            ps = np.exp(np.linspace(math.log(0.1), math.log(100.0), k)) * P_ATM
            pts = [(p, m.arr[j, 0] + rng.normal(0.0, 0.5), m.arr[j, 1] + rng.normal(0.0, 0.1),
                    max(0.0, m.arr[j, 2] + rng.normal(0.0, 1.0) * CAL)) for p in ps]
            if count % 2 == 1:
                i = int(rng.integers(0, k))
                pts.insert(i + 1, (ps[i], pts[i][1] - 2.0, pts[i][2] + 0.3, pts[i][3] + 2.0 * CAL))
            rows.extend(pts)
        ptr.append(len(rows))
    m.plog_ptr = np.array(ptr, dtype=np.int32)
    m.plog = np.array(rows, dtype=np.float64).reshape(-1, 4)
    m.validate()
    return m


def with_three_species_sides(mech: Mechanism) -> Mechanism:
    """A copy of a mechanism holding H, OH, H2, H2O, HO2, O2 and N2 (the
    9-species set) with two more reversible elementary reactions that have
    three species on one side (the stoichiometric slots the generated
    mechanisms never fill): H + OH + H2 <=> H2O + H2 (a termolecular
    recombination with H2 as a named collider; A = 1e10 m^6/(kmol^2 s),
    b = 0, Ea = 0) and HO2 + N2 <=> H + O2 + N2 (a dissociation; A = 1e12
    m^3/(kmol s), b = 0, Ea = 48 kcal/mol)."""
    m = mech.copy()
    ix = {s: m.names.index(s) for s in ("H", "OH", "H2", "H2O", "HO2", "O2", "N2")}
    add = [((ix["H"], ix["OH"], ix["H2"]), (ix["H2O"], ix["H2"], -1), (math.log(1e10), 0.0, 0.0)),
           ((ix["HO2"], ix["N2"], -1), (ix["H"], ix["O2"], ix["N2"]), (math.log(1e12), 0.0, 48.0 * CAL))]
    k = len(add)

    def rows(idx):
        a = np.array(idx, dtype=np.int32)
        return a, (a >= 0).astype(np.int32)

    rf = [rows(f) for f, _, _ in add]
    rr = [rows(r) for _, r, _ in add]
    m.rtype = np.concatenate([m.rtype, np.full(k, RXN_ELEMENTARY, dtype=m.rtype.dtype)])
    m.reversible = np.concatenate([m.reversible, np.ones(k, dtype=m.reversible.dtype)])
    m.rf_idx = np.vstack([m.rf_idx] + [a for a, _ in rf]).astype(np.int32)
    m.rf_nu = np.vstack([m.rf_nu] + [n for _, n in rf]).astype(np.int32)
    m.rr_idx = np.vstack([m.rr_idx] + [a for a, _ in rr]).astype(np.int32)
    m.rr_nu = np.vstack([m.rr_nu] + [n for _, n in rr]).astype(np.int32)
    m.arr = np.vstack([m.arr, [a for _, _, a in add]])
    m.arr0 = np.vstack([m.arr0, np.zeros((k, 3))])
    m.troe = np.vstack([m.troe, np.zeros((k, 4))])
    m.eff_ptr = np.concatenate([m.eff_ptr, np.full(k, m.eff_ptr[-1], dtype=m.eff_ptr.dtype)])
    m.sri = np.vstack([m.sri, np.zeros((k, 5))])
    m.plog_ptr = np.concatenate([m.plog_ptr, np.full(k, m.plog_ptr[-1], dtype=m.plog_ptr.dtype)])
    m.validate()
    return m


# ----------------------------------------------------------------------------
# small hand-built mechanisms used by closed-form tests


def isomer_mechanism(k_f: float, reversible: bool, ds_over_R: float = 0.0) -> Mechanism:
    """Two isomers A and B with identical cp and h, so u_A = u_B and the
    temperature source vanishes; one reaction A -> B (or A <=> B) with a
    temperature-independent rate constant k_f (b = 0, Ea = 0).

    B's entropy constant exceeds A's by ds_over_R (in units of R), so the
    equilibrium constant is exp(ds_over_R) (the reaction has sum(nu) = 0).
    """
    c = np.array([3.5, 1e-4, -2e-8, 1e-12, -1e-16, -1000.0, 5.0])
    nasa7 = np.stack([c, c + np.array([0, 0, 0, 0, 0, 0, ds_over_R])])
    e1 = np.zeros(1, dtype=np.int32)
    return Mechanism(
        names=["A", "B"], elements=["C"], comp=np.array([[2], [2]]),
        W=np.array([28.0, 28.0]), nasa7=nasa7,
        rtype=np.zeros(1, dtype=np.int32), reversible=np.array([int(reversible)], dtype=np.int32),
        rf_idx=np.array([[0, -1, -1]], dtype=np.int32), rf_nu=np.array([[1, 0, 0]], dtype=np.int32),
        rr_idx=np.array([[1, -1, -1]], dtype=np.int32), rr_nu=np.array([[1, 0, 0]], dtype=np.int32),
        arr=np.array([[math.log(k_f), 0.0, 0.0]]), arr0=np.zeros((1, 3)), troe=np.zeros((1, 4)),
        eff_ptr=np.zeros(2, dtype=np.int32), eff_idx=e1[:0], eff_val=np.zeros(0))


# ----------------------------------------------------------------------------
# cell fields


def random_states(mech: Mechanism, n: int, seed: int = 0):
    """Random chemical states of Section 5.1 (eq. chemical_state_01):
    T = 1000 + 1500 r_T K, p = 0.1 + 9.9 r_p atm, X_i = r_i renormalised,
    C_i = X_i p / (R T).  Returns (T[n], C[n, ns], p[n])."""
    rng = np.random.default_rng(seed)
    T = 1000.0 + 1500.0 * rng.random(n)
    p = (0.1 + 9.9 * rng.random(n)) * P_ATM
    X = rng.random((n, mech.ns))
    X /= X.sum(axis=1, keepdims=True)
    C = X * (p / (R_UNIV * T))[:, None]
    return T, C, p


def _fuel_air_X(mech: Mechanism, fuel: str, phi: np.ndarray, argon: float = 0.0):
    """Mole fractions of fuel/air at equivalence ratio phi (air O2:N2 = 21:79,
    optional argon share of the air). X_fuel/X_O2 = phi/(c + h/4 - o/2)."""
    cnt = _parse(fuel)
    stoich = cnt.get("C", 0) + cnt.get("H", 0) / 4.0 - cnt.get("O", 0) / 2.0
    X = np.zeros((len(phi), mech.ns))
    xo2 = 0.21 * (1.0 - argon)
    xn2 = 0.79 * (1.0 - argon)
    X[:, mech.index(fuel)] = phi / stoich * xo2
    X[:, mech.index("O2")] = xo2
    X[:, mech.index("N2")] = xn2
    if argon:
        X[:, mech.index("Ar")] = argon
    X /= X.sum(axis=1, keepdims=True)
    return X


def _burnt_X(mech: Mechanism, X_unburnt: np.ndarray, radicals: float = 1e-4):
    """Complete-combustion products by element balance: carbon to CO, hydrogen
    to H2O with the oxygen left, the rest of H to H2, then leftover oxygen turns
    CO into CO2 and finally O2; N to N2, Ar unchanged. Adds H, O, OH at the
    given mole fraction and renormalises."""
    el = {e: X_unburnt @ mech.comp[:, i] for i, e in enumerate(mech.elements)}
    n = X_unburnt.shape[0]
    C_ = el.get("C", np.zeros(n)); H_ = el.get("H", np.zeros(n)); O_ = el.get("O", np.zeros(n))
    N_ = el.get("N", np.zeros(n)); Ar_ = el.get("Ar", np.zeros(n))
    co = C_.copy(); o_left = O_ - co
    h2o = np.minimum(H_ / 2.0, np.maximum(o_left, 0.0)); o_left -= h2o
    h2 = H_ / 2.0 - h2o
    co2 = np.minimum(co, np.maximum(o_left, 0.0)); co -= co2; o_left -= co2
    o2 = np.maximum(o_left, 0.0) / 2.0
    X = np.zeros_like(X_unburnt)
    for name, val in (("CO", co), ("CO2", co2), ("H2O", h2o), ("H2", h2), ("O2", o2),
                      ("N2", N_ / 2.0), ("Ar", Ar_)):
        if name in mech.names:
            X[:, mech.index(name)] += val
    X /= X.sum(axis=1, keepdims=True)
    for r in ("H", "O", "OH"):
        X[:, mech.index(r)] += radicals
    X /= X.sum(axis=1, keepdims=True)
    return X


def X_to_Y(mech: Mechanism, X: np.ndarray) -> np.ndarray:
    Y = X * mech.W[None, :]
    return Y / Y.sum(axis=1, keepdims=True)


def field_reactor(mech: Mechanism, n: int, T_range, p_range_atm, phi_range, fuel: str,
                  seed: int = 0, argon: float = 0.0):
    """Independent fuel/air cells: T, p and phi uniform in the given ranges.
    Returns (T[n], Y[n, ns], p[n] in Pa)."""
    rng = np.random.default_rng(seed)
    T = rng.uniform(*T_range, n)
    p = rng.uniform(*p_range_atm, n) * P_ATM
    phi = rng.uniform(*phi_range, n)
    return T, X_to_Y(mech, _fuel_air_X(mech, fuel, phi, argon)), p


def field_mixed(mech: Mechanism, n: int, fuel: str, seed: int = 0, argon: float = 0.0,
                frozen=(300.0, 600.0), burnt=(1800.0, 2400.0), active=(1000.0, 1700.0),
                shares=(0.90, 0.05, 0.05)):
    """Cells of very uneven cost, randomly interleaved: `shares` of frozen
    fuel/air (T in `frozen`), burnt gas (complete-combustion products plus
    radicals, T in `burnt`) and reacting cells (T in `active` with the
    composition blended linearly in T between unburnt and burnt, as in a
    flame front). p in U[1, 10] atm, phi in U[0.5, 1.5] per cell."""
    rng = np.random.default_rng(seed)
    kind = rng.choice(3, size=n, p=np.asarray(shares) / np.sum(shares))
    phi = rng.uniform(0.5, 1.5, n)
    p = rng.uniform(1.0, 10.0, n) * P_ATM
    Xu = _fuel_air_X(mech, fuel, phi, argon)
    Xb = _burnt_X(mech, Xu)
    T = np.where(kind == 0, rng.uniform(*frozen, n),
                 np.where(kind == 1, rng.uniform(*burnt, n), rng.uniform(*active, n)))
    w = np.where(kind == 0, 0.0, np.where(kind == 1, 1.0, (T - active[0]) / (active[1] - active[0])))
    X = (1.0 - w[:, None]) * Xu + w[:, None] * Xb
    return T, X_to_Y(mech, X), p, kind


def field_flames(mech: Mechanism, n: int, seed: int = 0, cells_per_flame: int = 4096,
                 fuel: str = "CH4", argon: float = 0.0093):
    """Contiguous 1-D flame-like field, one flame per block of cells: 60% unburnt
    fuel/air (T in U[300, 800] K), 10% front (T ramps from 1000 to 1700 K with
    the composition blended linearly in T between unburnt and burnt), 30% burnt
    (T in U[1800, 2400] K, complete-combustion products plus radicals). Each
    flame draws p in U[1, 10] atm and phi in U[0.5, 1.5]; small per-cell jitter.
    Cell order is kept so that neighbouring cells hold similar states."""
    rng = np.random.default_rng(seed)
    T = np.empty(n); p = np.empty(n); Y = np.empty((n, mech.ns))
    for start in range(0, n, cells_per_flame):
        m = min(cells_per_flame, n - start)
        pf = rng.uniform(1.0, 10.0) * P_ATM
        phi = rng.uniform(0.5, 1.5)
        Tu = rng.uniform(300.0, 800.0)
        Tb = rng.uniform(1800.0, 2400.0)
        Xu = _fuel_air_X(mech, fuel, np.array([phi]), argon)
        Xb = _burnt_X(mech, Xu)
        nu_, nf = int(round(0.6 * m)), int(round(0.1 * m))
        nb = m - nu_ - nf
        Tc = np.concatenate([np.full(nu_, Tu), np.linspace(1000.0, 1700.0, nf), np.full(nb, Tb)])
        Tc *= 1.0 + 0.002 * rng.standard_normal(m)
        w = np.concatenate([np.zeros(nu_), (np.linspace(1000.0, 1700.0, nf) - 1000.0) / 700.0,
                            np.ones(nb)])[:, None]
        X = (1.0 - w) * Xu + w * Xb
        T[start:start + m] = Tc
        p[start:start + m] = pf
        Y[start:start + m] = X_to_Y(mech, X)
    return T, Y, p

