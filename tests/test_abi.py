"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point the headers in include/ declare; argument validation that
happens before any CUDA call is exercised here (no compute call needs a
GPU)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_2510_10005_gb300 import build, chemgb, inputs

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
HEADERS = sorted(glob.glob(os.path.join(INCLUDE, "*.h")))


def declared_functions():
    names = set()
    for h in HEADERS:
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(cgx?_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return chemgb.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(HEADERS) >= 2 and len(names) >= 20 and "cgx_exp_check" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(chemgb.EXPORTED) <= set(names)


def test_opts_default(lib):
    o = chemgb.cg_integrate_opts_default()
    assert (o.method, o.reactor, o.adaptive, o.precision) == (chemgb.CG_SDIRK4, chemgb.CG_CONP, 1, 0)
    assert o.rtol == 1e-6 and o.atol == 1e-12 and o.newton_tol == 0.03 and o.neg_tol == 1e-6
    assert ctypes.sizeof(chemgb.cg_integrate_opts) == 10 * 4 + 7 * 8 + 4 * 4 + 8
    assert (o.linear_solver, o.preconditioner, o.gmres_restart, o.gmres_maxit, o.gmres_tol) == \
        (chemgb.CG_LU, chemgb.CG_PC_GAUSS_SEIDEL, 30, 200, 1e-10)


def _desc(mech):
    keep = dict(W=mech.W.astype(np.float64), nasa7=mech.nasa7.astype(np.float64),
                rxn_type=mech.rtype.astype(np.int32), reversible=mech.reversible.astype(np.int32),
                rf_idx=mech.rf_idx.astype(np.int32), rf_nu=mech.rf_nu.astype(np.int32),
                rr_idx=mech.rr_idx.astype(np.int32), rr_nu=mech.rr_nu.astype(np.int32),
                arr=mech.arr.astype(np.float64), arr0=mech.arr0.astype(np.float64),
                troe=mech.troe.astype(np.float64), eff_ptr=mech.eff_ptr.astype(np.int32),
                eff_idx=mech.eff_idx.astype(np.int32), eff_val=mech.eff_val.astype(np.float64))
    d = chemgb.cg_mech_desc(mech.ns, mech.nr, *[keep[k].ctypes.data for k in (
        "W", "nasa7", "rxn_type", "reversible", "rf_idx", "rf_nu", "rr_idx", "rr_nu", "arr", "arr0",
        "troe", "eff_ptr", "eff_idx", "eff_val")])
    return d, keep


@pytest.mark.parametrize("field,value,needle", [
    ("rf_idx", 99, "species index out of range"),
    ("rf_nu", 0, "coefficients"),
    ("rtype", 7, "bad type"),
])
def test_mech_create_rejects_bad_data(lib, field, value, needle):
    m = inputs.gen_mechanism("h2").copy()
    getattr(m, field).flat[0] = value
    d, keep = _desc(m)
    h = ctypes.c_void_p()
    code = lib.cg_mech_create(ctypes.byref(d), ctypes.byref(h))
    assert code == chemgb.CG_EINVAL and h.value is None
    assert needle in lib.cg_last_error().decode()


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.cg_mech_create(None, ctypes.byref(h)) == chemgb.CG_EINVAL
    o = chemgb.cg_integrate_opts_default()
    assert lib.cg_integrate(None, ctypes.byref(o), 4, None, None, None, None, None, None) == chemgb.CG_EINVAL
    assert "mech is NULL" in lib.cg_last_error().decode()
    assert lib.cg_mech_n_species(None) == -1


def test_mech_create_checks_sri_and_plog(lib):
    """SRI and PLOG reactions (Section 2.2.3, 2.2.4): their parameter
    arrays are required and checked before anything reaches the GPU."""
    base = inputs.with_sri_plog(inputs.gen_mechanism("h2"), n_sri=1, n_plog=2, seed=1)
    j_sri = int(np.flatnonzero(base.rtype == inputs.RXN_SRI)[0])
    j_plog = int(np.flatnonzero(base.rtype == inputs.RXN_PLOG)[0])
    cases = []
    m = base.copy(); m.sri[j_sri, 2] = 0.0; cases.append((m, "SRI needs"))
    m = base.copy(); m.plog[m.plog_ptr[j_plog] + 1, 0] = m.plog[m.plog_ptr[j_plog], 0] / 2
    cases.append((m, "must not decrease"))
    m = base.copy(); m.plog[m.plog_ptr[j_plog], 0] = -1.0; cases.append((m, "PLOG entry"))
    for mech, needle in cases:
        with pytest.raises(chemgb.ChemgbError) as e:
            chemgb.cg_mech_create(mech)
        assert e.value.code == chemgb.CG_EINVAL and needle in str(e.value)
    d, keep = _desc(base)   # no sri / plog arrays given
    h = ctypes.c_void_p()
    assert lib.cg_mech_create(ctypes.byref(d), ctypes.byref(h)) == chemgb.CG_EINVAL
    assert b"SRI but sri is NULL" in lib.cg_last_error()


def test_set_thermo_checks_arguments(lib):
    """The degree entry point refuses a NULL mechanism before any device work."""
    coef = np.zeros(10)
    assert lib.cg_mech_set_thermo(None, 7, coef.ctypes.data) == chemgb.CG_EINVAL
    assert b"mech is NULL" in lib.cg_last_error()


def test_check_hooks_refuse_bad_arguments(lib):
    """The reciprocal hook refuses bad arguments before any device work."""
    assert lib.cgx_rcp_check(-1, None, None, None) == chemgb.CG_EINVAL
    assert lib.cgx_rcp_check(4, None, None, None) == chemgb.CG_EINVAL
    assert lib.cgx_rcp_check(0, None, None, None) == chemgb.CG_OK


def test_noalloc_capacity_plan(lib):
    """cg_integrate_noalloc's capacity check (host planner): the 53-species
    mechanism needs no scratch with its arrays in shared memory, and one
    slot per cell of a block when they spill; a layout too large for the
    fixed 32 MiB array (1023 species, 400,000 reactions, everything spilled)
    gets CG_ECAPACITY with both sizes in the message; teams per block that
    the launcher lowers for shared memory are lowered here too."""
    assert chemgb.cgx_noalloc_plan(53, 325, 8, 227 * 1024, 64, 1) == 0
    one = chemgb.cgx_noalloc_plan(53, 325, 8, 16 * 1024, 64, 1)
    assert one > 0 and one % 256 == 0
    assert chemgb.cgx_noalloc_plan(53, 325, 8, 16 * 1024, 32, 4) == 4 * one
    # GMRES(64) with a 100 KB limit: 97 KB of shared memory per cell, so of
    # four cells per block requested two fit in 227 KB, each with its slot
    lay = chemgb.cgx_layout(53, 325, 8, 100 * 1024, gmres_m=64)
    assert lay["glob"] > 0 and 2 * lay["smem"] * 8 <= 227 * 1024 < 3 * lay["smem"] * 8
    slot = chemgb.cgx_noalloc_plan(53, 325, 8, 100 * 1024, 32, 1, gmres_m=64)
    assert slot > 0 and chemgb.cgx_noalloc_plan(53, 325, 8, 100 * 1024, 32, 4, gmres_m=64) == 2 * slot
    with pytest.raises(chemgb.ChemgbError) as e:
        chemgb.cgx_noalloc_plan(1023, 400000, 8, 1024, 64, 1)
    assert e.value.code == chemgb.CG_ECAPACITY
    assert "cg_integrate_noalloc has 33554176" in str(e.value)
    with pytest.raises(chemgb.ChemgbError) as e:
        chemgb.cgx_noalloc_plan(53, 325, 8, 16 * 1024, 48, 1)
    assert e.value.code == chemgb.CG_EINVAL
