"""Python binding of the chemgb C ABI (include/chemgb.h).

Argument marshalling only: every function passes raw device pointers of
torch tensors (float64 / int32, contiguous, on a CUDA device) and the
current CUDA stream to the library, where all of the computation happens.
The names are those of the C entry points. Importing this module does not
need a GPU; calling into it needs the built library (see build.py) and
fails loudly if it is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

CG_OK, CG_EINVAL, CG_ENOMEM, CG_ECUDA, CG_ECAPACITY, CG_EUNSUPPORTED = range(6)
(CG_CELL_OK, CG_CELL_NEWTON_FAIL, CG_CELL_STEP_TOO_SMALL, CG_CELL_MAX_STEPS, CG_CELL_NONFINITE,
 CG_CELL_NO_RECORD) = range(6)
CG_CONV, CG_CONP, CG_CONP_LITERAL = 0, 1, 2
CG_BE, CG_SDIRK2, CG_SDIRK4, CG_ROS2, CG_YASS = 0, 1, 2, 3, 4
CG_FP64, CG_FP32LU = 0, 1
CG_LU, CG_GMRES = 0, 1
CG_PC_NONE, CG_PC_JACOBI, CG_PC_GAUSS_SEIDEL = 0, 1, 2

_lib = None


class ChemgbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"chemgb error {code}: {msg}")
        self.code = code


class cg_mech_desc(ctypes.Structure):
    _fields_ = [("n_species", ctypes.c_int), ("n_reactions", ctypes.c_int)] + [
        (name, ctypes.c_void_p) for name in (
            "W", "nasa7", "rxn_type", "reversible", "rf_idx", "rf_nu", "rr_idx", "rr_nu",
            "arr", "arr0", "troe", "eff_ptr", "eff_idx", "eff_val", "sri", "plog_ptr", "plog")]


class cg_integrate_opts(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int) for k in (
        "method", "reactor", "adaptive", "precision", "nsub", "max_newton", "max_steps",
        "max_halvings", "err_filter", "persistent")] + [(k, ctypes.c_double) for k in (
            "dt", "rtol", "atol", "newton_tol", "h0", "hmin", "neg_tol")] + [(k, ctypes.c_int) for k in (
                "linear_solver", "preconditioner", "gmres_restart", "gmres_maxit")] + [
        ("gmres_tol", ctypes.c_double)]


EXPORTED = ("cg_mech_create", "cg_mech_destroy", "cg_mech_n_species", "cg_mech_n_reactions",
            "cg_mech_set_launch", "cg_mech_get_launch", "cg_mech_set_smem_limit",
            "cg_eval_rates", "cg_eval_jacobian", "cg_temperature_from_energy",
            "cg_integrate_opts_default", "cg_integrate", "cg_integrate_batch", "cg_integrate_host",
            "cg_integrate_noalloc", "cg_autotune", "cg_last_error", "cg_integrate_ckpt",
            "cg_integrate_adjoint", "cg_mech_set_arrhenius", "cgx_exp_check", "cg_react_split",
            "cgx_schedule", "cgx_rate_chunks", "cgx_layout", "cg_mech_set_thermo",
            "cgx_thermo_table", "cgx_tableau", "cgx_rcp_check", "cgx_noalloc_plan", "cg_mech_set_lu_panel",
            "cg_mech_get_lu_panel", "cgx_debug_flags")


def library_path() -> str:
    """The library this process loads: libchemgb.so, or the build named by
    the CHEMGB_LIB environment variable (the debug build in its tests)."""
    return os.environ.get("CHEMGB_LIB") or _build.LIB


def load(build_if_missing: bool = False):
    """Load libchemgb.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if build_if_missing and path == _build.LIB:
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"chemgb CUDA library not built ({path}); run "
                           "python -m paper_2510_10005_gb300.build")
    lib = ctypes.CDLL(path)
    P, I, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    lib.cg_mech_create.argtypes = [ctypes.POINTER(cg_mech_desc), ctypes.POINTER(P)]
    lib.cg_mech_destroy.argtypes = [P]
    lib.cg_mech_destroy.restype = None
    lib.cg_mech_n_species.argtypes = [P]
    lib.cg_mech_n_reactions.argtypes = [P]
    lib.cg_mech_set_launch.argtypes = [P, I, I]
    lib.cg_mech_get_launch.argtypes = [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.cg_mech_set_smem_limit.argtypes = [P, L]
    lib.cg_mech_set_lu_panel.argtypes = [P, I]
    lib.cg_mech_get_lu_panel.argtypes = [P]
    lib.cg_integrate_batch.argtypes = [I, P, P, P, P, P, P, P, ctypes.POINTER(cg_integrate_opts), P]
    lib.cg_integrate_noalloc.argtypes = [P, ctypes.POINTER(cg_integrate_opts), L, P, P, P, P, P, P]
    lib.cg_autotune.argtypes = [P, ctypes.POINTER(cg_integrate_opts), L, P, P, P, ctypes.c_char_p, P,
                                ctypes.POINTER(ctypes.c_double)]
    lib.cg_eval_rates.argtypes = [P, I, L, P, P, P, P]
    lib.cg_eval_jacobian.argtypes = [P, I, L, P, P, P, P]
    lib.cg_temperature_from_energy.argtypes = [P, I, L, P, P, P, I, P]
    lib.cg_integrate_opts_default.argtypes = [ctypes.POINTER(cg_integrate_opts)]
    lib.cg_integrate_opts_default.restype = None
    lib.cg_integrate.argtypes = [P, ctypes.POINTER(cg_integrate_opts), L, P, P, P, P, P, P]
    lib.cg_integrate_host.argtypes = [P, ctypes.POINTER(cg_integrate_opts), L, P, P, P, P, P]
    lib.cg_integrate_ckpt.argtypes = [P, ctypes.POINTER(cg_integrate_opts), L, P, P, P, P, P, P, P, I, P]
    lib.cg_integrate_adjoint.argtypes = [P, ctypes.POINTER(cg_integrate_opts), L, P, P, I, P, P, P, P, P, P,
                                         P, P]
    lib.cg_mech_set_arrhenius.argtypes = [P, P]
    lib.cg_mech_set_thermo.argtypes = [P, I, P]
    lib.cgx_thermo_table.argtypes = [I, I, P, P, P, L]
    lib.cgx_exp_check.argtypes = [P, L, P, P, P, P]
    lib.cgx_schedule.argtypes = [L, P, P, P, P, I, P, P, P, P, P, L]
    lib.cgx_rate_chunks.argtypes = [I, P, I, P, P, P, P, I]
    lib.cgx_layout.argtypes = [I, I, I, L, I, I] + [P] * 8
    lib.cgx_rcp_check.argtypes = [L, P, P, P]
    lib.cgx_debug_flags.argtypes = [P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int64)]
    lib.cgx_noalloc_plan.argtypes = [I, I, I, L, I, I, I, ctypes.POINTER(ctypes.c_int64)]
    lib.cgx_tableau.argtypes = [I, P, P, P, P, P]
    lib.cg_react_split.argtypes = [P, ctypes.POINTER(cg_integrate_opts), L, P, P, P, P, P, I, P, P, P]
    lib.cg_last_error.restype = ctypes.c_char_p
    lib.cg_last_error.argtypes = []
    _lib = lib
    return lib


def _check(code: int):
    if code != CG_OK:
        raise ChemgbError(code, load().cg_last_error().decode())


def _ptr(t) -> int:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    if isinstance(t, int):
        return t
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _dev(t, dtype_name="float64"):
    import torch
    dt = {"float64": torch.float64, "int32": torch.int32}[dtype_name]
    if not (t.is_cuda and t.dtype == dt and t.is_contiguous()):
        raise ValueError(f"expected a contiguous CUDA {dtype_name} tensor, got {t.dtype} on {t.device}")
    return t.data_ptr()


def _stream(stream):
    if stream is not None:
        return int(stream)
    import torch
    return torch.cuda.current_stream().cuda_stream


# ---------------------------------------------------------------------------
# C entry points


def cg_mech_create(mech) -> "MechHandle":
    """Upload a paper_2510_10005_gb300.inputs.Mechanism (host arrays)."""
    return MechHandle(mech)


def cg_mech_destroy(handle: "MechHandle"):
    handle.close()


def cg_mech_set_launch(h, team: int, teams_per_block: int = 1):
    _check(load().cg_mech_set_launch(h.ptr, team, teams_per_block))


def cg_mech_get_launch(h):
    t, b = ctypes.c_int(), ctypes.c_int()
    load().cg_mech_get_launch(h.ptr, ctypes.byref(t), ctypes.byref(b))
    return t.value, b.value


def cg_integrate_opts_default() -> cg_integrate_opts:
    o = cg_integrate_opts()
    load().cg_integrate_opts_default(ctypes.byref(o))
    return o


def make_opts(**kw) -> cg_integrate_opts:
    o = cg_integrate_opts_default()
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def cg_eval_rates(h, reactor, T, C, S, stream=None):
    _check(load().cg_eval_rates(h.ptr, reactor, T.shape[0], _dev(T), _dev(C), _dev(S), _stream(stream)))


def cg_eval_jacobian(h, reactor, T, C, J, stream=None):
    _check(load().cg_eval_jacobian(h.ptr, reactor, T.shape[0], _dev(T), _dev(C), _dev(J), _stream(stream)))


def cg_temperature_from_energy(h, reactor, e, Y, T, iters=5, stream=None):
    _check(load().cg_temperature_from_energy(h.ptr, reactor, T.shape[0], _dev(e), _dev(Y), _dev(T),
                                             iters, _stream(stream)))


def cg_integrate(h, opts, T, Y, p_or_rho, status=None, stats=None, stream=None):
    _check(load().cg_integrate(h.ptr, ctypes.byref(opts), T.shape[0], _dev(T), _dev(Y), _dev(p_or_rho),
                               None if status is None else _dev(status, "int32"),
                               None if stats is None else _dev(stats, "int32"), _stream(stream)))


def cg_integrate_noalloc(h, opts, T, Y, p_or_rho, status=None, stats=None, stream=None):
    """cg_integrate through the library's fixed device array instead of any
    allocation (for callers that cannot allocate device memory while they
    run; see include/chemgb.h for its limits)."""
    _check(load().cg_integrate_noalloc(h.ptr, ctypes.byref(opts), T.shape[0], _dev(T), _dev(Y),
                                       _dev(p_or_rho), None if status is None else _dev(status, "int32"),
                                       None if stats is None else _dev(stats, "int32"), _stream(stream)))


def cg_autotune(h, opts, T, Y, p_or_rho, cache_json=None, stream=None) -> float:
    """Pick the fastest launch shape on a sample (device tensors); returns its
    time in ms."""
    ms = ctypes.c_double(0.0)
    _check(load().cg_autotune(h.ptr, ctypes.byref(opts), T.shape[0], _dev(T), _dev(Y), _dev(p_or_rho),
                              cache_json.encode() if cache_json else None, _stream(stream), ctypes.byref(ms)))
    return ms.value


def cg_mech_set_smem_limit(h, nbytes: int):
    _check(load().cg_mech_set_smem_limit(h.ptr, int(nbytes)))


def cg_mech_set_lu_panel(h, nb: int):
    """Panel width of the blocked LU (0: unblocked; identical results)."""
    _check(load().cg_mech_set_lu_panel(h.ptr, int(nb)))


def cg_mech_get_lu_panel(h) -> int:
    return int(load().cg_mech_get_lu_panel(h.ptr))


def cg_integrate_batch(handles, opts, Ts, Ys, ps, statuses=None, stats=None, stream=None):
    """One persistent launch over the cells of several mechanisms; the k-th
    tensors belong to handles[k]."""
    k = len(handles)
    P = ctypes.c_void_p
    arr = lambda vals: (P * k)(*vals)
    Ns = (ctypes.c_int64 * k)(*[t.shape[0] for t in Ts])
    st = arr([_dev(s, "int32") for s in statuses]) if statuses is not None else None
    sa = arr([_dev(s, "int32") for s in stats]) if stats is not None else None
    _check(load().cg_integrate_batch(k, arr([h.ptr for h in handles]), Ns, arr([_dev(t) for t in Ts]),
                                     arr([_dev(y) for y in Ys]), arr([_dev(p) for p in ps]), st, sa,
                                     ctypes.byref(opts), _stream(stream)))


def cg_integrate_host(h, opts, T, Y, p_or_rho, status=None, stats=None):
    """Host numpy arrays (float64 / int32, C-contiguous; Y as [ns, N])."""
    for a in (T, Y, p_or_rho):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    _check(load().cg_integrate_host(h.ptr, ctypes.byref(opts), T.shape[0], _ptr(T), _ptr(Y),
                                    _ptr(p_or_rho), _ptr(status), _ptr(stats)))


def cg_integrate_ckpt(h, opts, T, Y, p_or_rho, ckpt, ckpt_n, status=None, stats=None, stream=None):
    """cg_integrate that records the adjoint's checkpoints: ckpt is a CUDA
    float64 tensor [N, cap, ns + 2], ckpt_n int32 [N]."""
    N = T.shape[0]
    if ckpt.dim() != 3 or ckpt.shape[0] != N or ckpt.shape[2] != h.n + 1:
        raise ValueError(f"ckpt must be [N, cap, {h.n + 1}]")
    _check(load().cg_integrate_ckpt(h.ptr, ctypes.byref(opts), N, _dev(T), _dev(Y), _dev(p_or_rho),
                                    None if status is None else _dev(status, "int32"),
                                    None if stats is None else _dev(stats, "int32"), _dev(ckpt),
                                    _dev(ckpt_n, "int32"), ckpt.shape[1], _stream(stream)))


def cg_integrate_adjoint(h, opts, ckpt, ckpt_n, dT_end, dY_end, dT0, dY0, dtheta=None, dtheta_cells=None,
                         status=None, stream=None):
    """Backward sweep over the checkpoints of cg_integrate_ckpt (CUDA
    tensors; dtheta [nr, 3], dtheta_cells [nr, 3, N] may be None)."""
    _check(load().cg_integrate_adjoint(h.ptr, ctypes.byref(opts), dT_end.shape[0], _dev(ckpt),
                                       _dev(ckpt_n, "int32"), ckpt.shape[1], _dev(dT_end), _dev(dY_end),
                                       _dev(dT0), _dev(dY0), None if dtheta is None else _dev(dtheta),
                                       None if dtheta_cells is None else _dev(dtheta_cells),
                                       None if status is None else _dev(status, "int32"), _stream(stream)))


def cg_mech_set_thermo(h, coef):
    """Thermodynamics of another degree: coef [ns, n_p + 3] (a_0..a_np of
    c_p/R, then the h/R and s/R constants)."""
    c = np.ascontiguousarray(coef, dtype=np.float64)
    if c.ndim != 2 or c.shape[0] != h.ns or c.shape[1] < 3:
        raise ValueError(f"coef must be [{h.ns}, n_p + 3]")
    _check(load().cg_mech_set_thermo(h.ptr, c.shape[1] - 3, c.ctypes.data))


def cg_mech_set_arrhenius(h, arr):
    """Replace (ln A, b, Ea) of every reaction (host array [nr, 3])."""
    a = np.ascontiguousarray(arr, dtype=np.float64).reshape(h.nr, 3)
    _check(load().cg_mech_set_arrhenius(h.ptr, a.ctypes.data))
    h.arr = a.copy()


def cg_react_split(h, opts, rho, e, rhoY, T, R, iters=5, status=None, stats=None, stream=None):
    """Operator-split reaction step: rho [N], e [N], rhoY [ns, N] in; T [N]
    guess in, temperature after dt out; R [ns, N] out (CUDA tensors)."""
    _check(load().cg_react_split(h.ptr, ctypes.byref(opts), rho.shape[0], _dev(rho), _dev(e), _dev(rhoY),
                                 _dev(T), _dev(R), int(iters), None if status is None else _dev(status, "int32"),
                                 None if stats is None else _dev(stats, "int32"), _stream(stream)))


def cgx_exp_check(h, x, y_tab, y_lib, stream=None):
    """Test hook: the library's table-driven exp and CUDA's exp of x."""
    _check(load().cgx_exp_check(h.ptr, x.shape[0], _dev(x), _dev(y_tab), _dev(y_lib), _stream(stream)))


def cgx_schedule(dst, src, fac, order, lanes: int):
    """Test hook (host only): the thread-owned assembly schedule of the terms
    out[dst] += fac * in[src]; returns (len, dst, flags, src, fac), each of
    the four arrays [len, lanes] (slot t of lane l at [t, l])."""
    lib = load()
    dst, src = np.ascontiguousarray(dst, np.int32), np.ascontiguousarray(src, np.int32)
    fac, order = np.ascontiguousarray(fac, np.float64), np.ascontiguousarray(order, np.int64)
    n = ctypes.c_int(0)
    _check(lib.cgx_schedule(len(dst), _ptr(dst), _ptr(src), _ptr(fac), _ptr(order), lanes, ctypes.byref(n),
                            None, None, None, None, 0))
    slots = n.value * lanes
    out = [np.zeros(slots, np.int32), np.zeros(slots, np.int32), np.zeros(slots, np.int32), np.zeros(slots)]
    _check(lib.cgx_schedule(len(dst), _ptr(dst), _ptr(src), _ptr(fac), _ptr(order), lanes, ctypes.byref(n),
                            *[_ptr(a) for a in out], slots))
    return (n.value,) + tuple(a.reshape(n.value, lanes) for a in out)


def cgx_rate_chunks(rxn_type, team: int):
    """Test hook (host only): the rate loop's reaction chunks; returns
    (warp_ptr, first, len)."""
    lib = load()
    t = np.ascontiguousarray(rxn_type, np.int32)
    n = ctypes.c_int(0)
    ptr = np.zeros(team // 32 + 1, np.int32)
    _check(lib.cgx_rate_chunks(len(t), _ptr(t), team, ctypes.byref(n), _ptr(ptr), None, None, 0))
    first, ln = np.zeros(n.value, np.int32), np.zeros(n.value, np.int32)
    _check(lib.cgx_rate_chunks(len(t), _ptr(t), team, ctypes.byref(n), _ptr(ptr), _ptr(first), _ptr(ln), n.value))
    return ptr, first, ln


def cgx_thermo_table(coef):
    """Test hook (host only): the device thermo table for coef [ns, n_p + 3];
    returns (P, table [4 P + 1, ns])."""
    lib = load()
    c = np.ascontiguousarray(coef, dtype=np.float64)
    ns, np_ = c.shape[0], c.shape[1] - 3
    P = ctypes.c_int(0)
    _check(lib.cgx_thermo_table(ns, np_, c.ctypes.data, ctypes.byref(P), None, 0))
    t = np.zeros((4 * P.value + 1) * ns)
    _check(lib.cgx_thermo_table(ns, np_, c.ctypes.data, ctypes.byref(P), t.ctypes.data, t.size))
    return P.value, t.reshape(4 * P.value + 1, ns)


def cgx_rcp_check(x, y, stream=None):
    """Test hook: the library's pivot reciprocal of x (CUDA tensors)."""
    _check(load().cgx_rcp_check(x.shape[0], _dev(x), _dev(y), _stream(stream)))


def cgx_debug_flags(h):
    """Debug build only: (arrays whose guard words changed as a bit mask,
    first such cell or -1), cleared by the call."""
    a, c = ctypes.c_uint64(0), ctypes.c_int64(-1)
    _check(load().cgx_debug_flags(h.ptr, ctypes.byref(a), ctypes.byref(c)))
    return a.value, c.value


def cgx_noalloc_plan(ns: int, nr: int, mat_bytes: int, smem_limit: int, team: int, teams_per_block: int,
                     gmres_m: int = 0) -> int:
    """Test hook (host only): the scratch bytes cg_integrate_noalloc needs
    for such a mechanism and launch shape (raises ChemgbError with
    CG_ECAPACITY when the library's fixed array is too small)."""
    need = ctypes.c_int64(0)
    _check(load().cgx_noalloc_plan(ns, nr, mat_bytes, int(smem_limit), gmres_m, team, teams_per_block,
                                   ctypes.byref(need)))
    return need.value


def cgx_tableau(method: int) -> dict:
    """Test hook (host only): the kernels' Butcher tableau of `method`."""
    s, e = np.zeros(1, np.int32), np.zeros(1, np.int32)
    A, b, bh = np.zeros(25), np.zeros(5), np.zeros(5)
    _check(load().cgx_tableau(method, _ptr(s), _ptr(A), _ptr(b), _ptr(bh), _ptr(e)))
    return dict(s=int(s[0]), A=A.reshape(5, 5), b=b, bhat=bh, err_order=int(e[0]))


def cgx_layout(ns: int, nr: int, mat_bytes: int, smem_limit: int, adjoint: bool = False, gmres_m: int = 0) -> dict:
    """Test hook (host only): one cell's memory layout; returns ld, and per
    array offset, size, in_global, plus the priority order and the totals (in
    doubles)."""
    lib = load()
    ints = [np.zeros(1, np.int32) for _ in range(2)] + [np.zeros(32, np.int32) for _ in range(4)] + \
        [np.zeros(1, np.int32) for _ in range(2)]
    _check(lib.cgx_layout(ns, nr, mat_bytes, int(smem_limit), int(adjoint), gmres_m, *[_ptr(a) for a in ints]))
    k = int(ints[1][0])
    return dict(ld=int(ints[0][0]), offset=ints[2][:k], size=ints[3][:k], in_global=ints[4][:k].astype(bool),
                priority=ints[5][:k], smem=int(ints[6][0]), glob=int(ints[7][0]))


class MechHandle:
    """Owns one cg_mech."""

    def __init__(self, mech):
        thermo = getattr(mech, "thermo", None)
        lib = load()
        f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
        self._keep = dict(
            W=f64(mech.W), nasa7=f64(mech.nasa7 if thermo is None or thermo.shape[1] != 7 else thermo), rxn_type=i32(mech.rtype), reversible=i32(mech.reversible),
            rf_idx=i32(mech.rf_idx), rf_nu=i32(mech.rf_nu), rr_idx=i32(mech.rr_idx), rr_nu=i32(mech.rr_nu),
            arr=f64(mech.arr), arr0=f64(mech.arr0), troe=f64(mech.troe), eff_ptr=i32(mech.eff_ptr),
            eff_idx=i32(mech.eff_idx) if len(mech.eff_idx) else np.zeros(1, np.int32),
            eff_val=f64(mech.eff_val) if len(mech.eff_val) else np.zeros(1),
            sri=f64(mech.sri), plog_ptr=i32(mech.plog_ptr),
            plog=f64(mech.plog) if len(mech.plog) else np.zeros(4))
        d = cg_mech_desc(mech.ns, mech.nr, *[self._keep[k].ctypes.data for k in (
            "W", "nasa7", "rxn_type", "reversible", "rf_idx", "rf_nu", "rr_idx", "rr_nu", "arr", "arr0",
            "troe", "eff_ptr", "eff_idx", "eff_val", "sri", "plog_ptr", "plog")])
        h = ctypes.c_void_p()
        _check(lib.cg_mech_create(ctypes.byref(d), ctypes.byref(h)))
        self.ptr = h.value
        self.ns, self.nr, self.n = mech.ns, mech.nr, mech.ns + 1
        self.mech = mech
        self.arr = np.array(self._keep["arr"]).reshape(mech.nr, 3)   # current (ln A, b, Ea)
        if thermo is not None and thermo.shape[1] != 7:   # a c_p polynomial of another degree
            cg_mech_set_thermo(self, thermo)

    def close(self):
        if getattr(self, "ptr", None):
            load().cg_mech_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
