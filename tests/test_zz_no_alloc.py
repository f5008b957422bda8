"""cg_integrate_noalloc: integration for callers that cannot allocate device
memory while they run. It must give what cg_integrate gives, on repeated
calls (the library's fixed device array keeps the previous call's contents,
so each call must start from a cleared work counter).

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test. It builds its own handles and
inputs and runs the same alone in a fresh process or after other tests."""
import ctypes

import numpy as np
import pytest

from paper_2510_10005_gb300 import chemgb, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"

ADAPT = dict(method=chemgb.CG_SDIRK4, adaptive=1, dt=1e-6, rtol=1e-6, atol=1e-12, newton_tol=0.03,
             max_newton=7, reactor=chemgb.CG_CONP)


def d(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def call(fn, h, o, T, Y, p):
    """Run one entry point through the C ABI on fresh device copies."""
    N = len(T)
    Tt, Yt, pt = d(T), d(Y.T), d(p)
    st = torch.full((N,), -1, dtype=torch.int32, device=DEV)
    stats = torch.full((4, N), -1, dtype=torch.int32, device=DEV)
    lib = chemgb.load(build_if_missing=True)
    code = getattr(lib, fn)(h.ptr, ctypes.byref(o), N, Tt.data_ptr(), Yt.data_ptr(), pt.data_ptr(),
                            st.data_ptr(), stats.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert code == chemgb.CG_OK, lib.cg_last_error().decode()
    torch.cuda.synchronize()
    return Tt.cpu().numpy(), Yt.cpu().numpy().T, st.cpu().numpy(), stats.cpu().numpy().T


def test_noalloc_setup_call_with_no_cells():
    """A call with N = 0 is the set-up call: it loads the fixed array on the
    device (and so does the allocation a caller's memory manager must see
    before it takes over the heap), and integrates nothing."""
    mech = inputs.gen_mechanism("h2")
    h = chemgb.cg_mech_create(mech)
    lib = chemgb.load(build_if_missing=True)
    o = chemgb.make_opts(**ADAPT)
    code = lib.cg_integrate_noalloc(h.ptr, ctypes.byref(o), 0, None, None, None, None, None,
                                    torch.cuda.current_stream().cuda_stream)
    assert code == chemgb.CG_OK, lib.cg_last_error().decode()
    torch.cuda.synchronize()


@pytest.mark.parametrize("smem_limit", [None, 16 * 1024])
@pytest.mark.parametrize("precision", [chemgb.CG_FP64, chemgb.CG_FP32LU])
def test_noalloc_matches_integrate_twice(smem_limit, precision):
    """Two calls in a row (different cells, then the first cells again) give
    cg_integrate's results; with a 16 KiB shared-memory limit the cells'
    per-reaction data, thermo and stage vectors live in the fixed array."""
    mech = inputs.gen_mechanism("ch4")
    h = chemgb.cg_mech_create(mech)
    if smem_limit:
        chemgb.cg_mech_set_smem_limit(h, smem_limit)
    T, Y, p = inputs.field_flames(mech, 4096, seed=11)
    a = np.concatenate([np.arange(0, 4096, 64), np.arange(2430, 2470)])
    b = np.arange(1, 4096, 97)
    o = chemgb.make_opts(**ADAPT, precision=precision)
    for idx in (a, b, a):
        ref = call("cg_integrate", h, o, T[idx], Y[idx], p[idx])
        got = call("cg_integrate_noalloc", h, o, T[idx], Y[idx], p[idx])
        np.testing.assert_array_equal(got[2], ref[2])
        np.testing.assert_allclose(got[0], ref[0], rtol=1e-12)
        np.testing.assert_allclose(got[1], ref[1], rtol=1e-12, atol=1e-18)
        np.testing.assert_array_equal(got[3], ref[3])


def test_noalloc_large_mechanism():
    """160 species: the Newton matrix fills shared memory, the rest of each
    cell's arrays goes to the fixed array; backward Euler on a few cells."""
    mech = inputs.gen_mechanism("c7")
    h = chemgb.cg_mech_create(mech)
    T, Y, p = inputs.field_reactor(mech, 10, (700, 1600), (20, 40), (0.5, 1.5), "C7H16", seed=1)
    o = chemgb.make_opts(method=chemgb.CG_BE, adaptive=0, dt=1e-6, rtol=1e-10, atol=1e-16,
                         newton_tol=1.0, max_newton=20, reactor=chemgb.CG_CONP)
    for _ in range(2):
        ref = call("cg_integrate", h, o, T, Y, p)
        got = call("cg_integrate_noalloc", h, o, T, Y, p)
        np.testing.assert_array_equal(got[2], ref[2])
        np.testing.assert_allclose(got[0], ref[0], rtol=1e-12)
        np.testing.assert_allclose(got[1], ref[1], rtol=1e-12, atol=1e-18)
