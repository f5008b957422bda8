"""Pins of the SDIRK tableaux (Appendix A) and invariants of the seeded
input generator."""
import os

import numpy as np
import pytest

from oracle import tableau
from paper_2510_10005_gb300 import inputs


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_sdirk4_reproduces_printed_coefficients():
    """Full-precision coefficients agree with the seven printed digits of
    Appendix A.2 (tests/golden/sdirk4_appendix_a2.txt), and a_52 (missing
    from the print) equals b_2."""
    A = tableau.sdirk4_full_precision()
    p = read_golden("sdirk4_appendix_a2.txt")
    assert np.all(np.diag(A) == p.pop("aii"))
    got = {"a21": A[1, 0], "a31": A[2, 0], "a32": A[2, 1], "a41": A[3, 0], "a42": A[3, 1],
           "a43": A[3, 2], "a51": A[4, 0], "a53": A[4, 2], "a54": A[4, 3], "b1": A[4, 0],
           "b2": A[4, 1], "b3": A[4, 2], "b4": A[4, 3], "b5": A[4, 4]}
    for k, v in p.items():
        assert got[k] == pytest.approx(v, rel=5e-7, abs=5e-9), k
    assert np.all(np.diag(A) == 4.0 / 15.0)


def test_sdirk4_order_conditions_and_abscissae():
    t = tableau.tableau(2)
    A, b, bh = t["A"], t["b"], t["bhat"]
    assert np.max(np.abs(tableau.order_conditions(A, b, 4))) < 1e-15
    c = A.sum(axis=1)
    np.testing.assert_allclose(c[:3], [4 / 15, 23 / 30, 17 / 30], atol=1e-15)
    assert c[4] == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_array_equal(b, A[4])             # stiffly accurate
    assert bh[4] == 0.0
    assert np.max(np.abs(tableau.order_conditions(A, bh, 3))) < 1e-14
    assert abs(tableau.order_conditions(A, bh, 4)[4]) > 1e-3   # genuinely third order


def test_sdirk2_and_be():
    t = tableau.tableau(1)
    g = 1 - np.sqrt(2) / 2
    assert t["A"][0, 0] == g and t["A"][1, 1] == g
    assert np.max(np.abs(tableau.order_conditions(t["A"][:2, :2], t["b"][:2], 2))) < 1e-15
    assert tableau.tableau(0)["A"][0, 0] == 1.0


@pytest.mark.parametrize("kind,ns,nr", [("h2", 9, 21), ("ch4", 53, 325), ("c7", 160, 900)])
def test_generated_mechanism_shape_and_balance(kind, ns, nr):
    m = inputs.gen_mechanism(kind)
    m.validate()   # index ranges, padding, element balance of every reaction
    assert (m.ns, m.nr) == (ns, nr)
    frac_press = np.mean(m.rtype != inputs.RXN_ELEMENTARY)
    if kind == "h2":
        assert (m.rtype == 1).sum() == 4 and (m.rtype == 3).sum() == 1
    else:
        assert 0.1 < frac_press < 0.2
    b = m.arr[:, 1]
    assert np.all(np.abs(b) <= 1.5)
    k1000 = np.exp(m.arr[:, 0] + b * np.log(1000.0))
    assert np.all((k1000 >= 1e6 * 0.999) & (k1000 <= 1e14 * 1.001))
    assert np.all((m.arr[:, 2] >= 0) & (m.arr[:, 2] <= 50.0 * inputs.CAL))
    assert len(set(m.names)) == ns


def test_generator_is_seeded():
    a, b = inputs.gen_mechanism("ch4"), inputs.gen_mechanism("ch4")
    np.testing.assert_array_equal(a.arr, b.arr)
    np.testing.assert_array_equal(a.nasa7, b.nasa7)
    c = inputs.gen_mechanism("ch4", seed=99)
    assert not np.array_equal(a.arr, c.arr)


def test_mechanism_save_load_keeps_thermo_degree(tmp_path):
    """A refitted mechanism (c_p polynomial of degree 7) and its source
    curves survive save and load; a NASA-7 mechanism comes back without a
    refit."""
    m = inputs.gen_mechanism("h2")
    m7 = inputs.with_thermo_degree(m, 7)
    assert m7.thermo_np == 7 and m7.thermo.shape == (m.ns, 10) and m.thermo_np == 4
    for mech, name in ((m, "a.npz"), (m7, "b.npz")):
        mech.save(str(tmp_path / name))
        back = inputs.Mechanism.load(str(tmp_path / name))
        assert back.thermo_np == mech.thermo_np
        np.testing.assert_array_equal(back.thermo_coef, mech.thermo_coef)
        np.testing.assert_array_equal(back.cp_src, mech.cp_src)
        np.testing.assert_array_equal(back.arr, mech.arr)


def test_fields():
    m = inputs.gen_mechanism("ch4")
    T, Y, p = inputs.field_flames(m, 10000, seed=0)
    assert T.shape == (10000,) and Y.shape == (10000, m.ns)
    np.testing.assert_allclose(Y.sum(1), 1.0, rtol=1e-13)
    assert np.all(Y >= 0) and np.all((p >= 1 * 101325) & (p <= 10 * 101325))
    frac_unburnt = np.mean(T < 900)
    assert 0.55 < frac_unburnt < 0.65
    assert 0.25 < np.mean(T > 1750) < 0.35
    Tr, Yr, pr = inputs.field_reactor(m, 100, (700, 1600), (20, 40), (0.5, 1.5), "CH4", seed=1)
    assert np.all((Tr >= 700) & (Tr <= 1600))
    # element ratios of fuel/air: O/N fixed by air
    el = (Yr / m.W) @ m.comp
    iO, iN = m.elements.index("O"), m.elements.index("N")
    np.testing.assert_allclose(el[:, iO] / el[:, iN], 0.21 * 2 / (0.79 * 2), rtol=1e-12)
