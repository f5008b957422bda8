"""The debug build of the library (CG_DEBUG), which stands in for a memory
checker on this GPU: every array of a cell's working memory is followed by
two guard words and poisoned before each cell (NaN, so a value read before
it is written spoils the result; zero for the pivot and reduction integers,
so that such a read cannot index out of bounds), and the guards are checked
after each cell. Mechanisms of 2, 3 and 9 species (the isomer pair, a
dissociation H2 + M <=> 2 H with a third-body efficiency, the synthetic
H2/O2 set) are integrated by backward Euler (FP64 and FP32 Newton matrix)
and adaptive SDIRK-4 in a child process that loads the debug library; the
results must match the oracle and no guard may have changed.

The child process is needed because a process loads one build of the
library. Building the debug library takes one to three minutes."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
sys.path.insert(0, ROOT + "/tests")
import oracle
from paper_2510_10005_gb300 import chemgb, inputs
from parity import check_adaptive, check_fixed

def dissociation():
    """H2 + M <=> H + H with an N2 efficiency of 0.7 (the 9-species set's
    thermo rows for H2, H and N2)."""
    m9 = inputs.gen_mechanism("h2")
    ix = [m9.names.index(s) for s in ("H2", "H", "N2")]
    return inputs.Mechanism(
        names=["H2", "H", "N2"], elements=list(m9.elements), comp=m9.comp[ix], W=m9.W[ix], nasa7=m9.nasa7[ix],
        rtype=np.array([1], np.int32), reversible=np.array([1], np.int32),
        rf_idx=np.array([[0, -1, -1]], np.int32), rf_nu=np.array([[1, 0, 0]], np.int32),
        rr_idx=np.array([[1, -1, -1]], np.int32), rr_nu=np.array([[2, 0, 0]], np.int32),
        arr=np.array([[np.log(4.6e15), -1.4, 2.0e8]]), arr0=np.zeros((1, 3)), troe=np.zeros((1, 4)),
        eff_ptr=np.array([0, 1], np.int32), eff_idx=np.array([2], np.int32), eff_val=np.array([0.7]))

def cells(m, n):
    rng = np.random.default_rng(5)
    if m.ns == 2:
        T = rng.uniform(900, 1100, n); Y = np.tile([0.9, 0.1], (n, 1)); p = np.full(n, 101325.0)
    elif m.ns == 3:
        T = rng.uniform(2500, 3500, n); X = np.tile([0.5, 0.01, 0.49], (n, 1)); Y = inputs.X_to_Y(m, X)
        p = np.full(n, 101325.0)
    else:
        T, Y, p = inputs.field_reactor(m, n, (1000, 1500), (1, 1), (0.5, 2), "H2", seed=4)
    return T, Y, p

BE = dict(method=oracle.BE, adaptive=0, dt=1e-6, rtol=1e-10, atol=1e-16, newton_tol=1.0, max_newton=20,
          max_halvings=10, reactor=oracle.CONP)
AD = dict(method=oracle.SDIRK4, adaptive=1, dt=1e-5, rtol=1e-6, atol=1e-12, newton_tol=0.03, max_newton=7,
          reactor=oracle.CONP)
out = {}
dev = "cuda:0"
for m in (inputs.isomer_mechanism(2e4, True, 0.3), dissociation(), inputs.gen_mechanism("h2")):
    r, h = oracle.RefMech(m), chemgb.cg_mech_create(m)
    T, Y, p = cells(m, 45)
    for name, o, prec in (("be", BE, 0), ("be_fp32", BE, 1), ("sdirk4", AD, 0)):
        To, Yo, so, _ = r.integrate(T, Y, p, o, nthreads=4)
        Tt = torch.tensor(T, device=dev); Yt = torch.tensor(np.ascontiguousarray(Y.T), device=dev)
        st = torch.empty(len(T), dtype=torch.int32, device=dev)
        chemgb.cg_integrate(h, chemgb.make_opts(**o, precision=prec), Tt, Yt, torch.tensor(p, device=dev), st)
        torch.cuda.synchronize()
        Tg, Yg = Tt.cpu().numpy(), Yt.cpu().numpy().T
        assert np.array_equal(st.cpu().numpy(), so), (m.ns, name)
        if o["adaptive"]:
            check_adaptive(name, m, Tg, Yg, To, Yo, p, o["reactor"], o["rtol"], o["atol"])
        else:
            check_fixed(name, Tg, Yg, To, Yo, 1e-10 if prec == 0 else 1e-8, 1e-22 if prec == 0 else 1e-18)
        out[f"{m.ns}sp_{name}"] = chemgb.cgx_debug_flags(h)
print(json.dumps(out))
'''


def test_debug_build_guards_and_parity():
    r = subprocess.run([sys.executable, "-m", "paper_2510_10005_gb300.build", "--debug"], cwd=ROOT,
                       capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    from paper_2510_10005_gb300 import build
    env = dict(os.environ, CHEMGB_LIB=build.LIB_DEBUG)
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    flags = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(flags) == 9
    for case, (arrays, first_cell) in flags.items():
        assert arrays == 0 and first_cell == -1, (case, hex(arrays), first_cell)


def test_release_build_has_no_debug_flags():
    """The normal library refuses the debug hook (no guard words there)."""
    torch = pytest.importorskip("torch")  # noqa: F841
    from paper_2510_10005_gb300 import chemgb, inputs
    chemgb.load(build_if_missing=True)
    h = chemgb.cg_mech_create(inputs.gen_mechanism("h2"))
    with pytest.raises(chemgb.ChemgbError) as e:
        chemgb.cgx_debug_flags(h)
    assert e.value.code == chemgb.CG_EUNSUPPORTED
