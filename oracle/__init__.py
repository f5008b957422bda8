"""ORACLE -- test infrastructure only.

Python front end of the plain FP64 CPU oracle (`cgref.cpp`) for the per-cell
chemistry of ChemGen (arXiv 2510.10005). Only the tests, the smoke check and
the CPU baseline of the benchmark may import this package; the product path
never does. It shares no code with the CUDA library: the only module both
sides use is the seeded input generator (`paper_2510_10005_gb300.inputs`),
which holds none of the method's arithmetic.

State layout here: cell-major, y[c] = (T, C_1..C_ns) (eq. extracted_problem-1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import tableau as _tableau

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libcgref.so")
R_UNIV = 8314.46261815324

CONV, CONP, CONP_LITERAL = 0, 1, 2
BE, SDIRK2, SDIRK4, ROS2, YASS = 0, 1, 2, 3, 4

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (portable flags only)."""
    src = os.path.join(_HERE, "cgref.cpp")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread",
                           "-o", tmp, src])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.cgref_mech_create.restype = P
        lib.cgref_mech_create.argtypes = [ctypes.c_int, ctypes.c_int] + [P] * 17
        lib.cgref_mech_destroy.argtypes = [P]
        lib.cgref_mech_set_thermo.restype = ctypes.c_int
        lib.cgref_mech_set_thermo.argtypes = [P, ctypes.c_int, P]
        lib.cgref_thermo.argtypes = [P, ctypes.c_double] + [P] * 6
        lib.cgref_rates.argtypes = [P, ctypes.c_double, P, P, P, P]
        lib.cgref_source.argtypes = [P, ctypes.c_int, ctypes.c_long, P, P]
        lib.cgref_source_complex.argtypes = [P, ctypes.c_int, P, P, P, P]
        lib.cgref_jacobian.argtypes = [P, ctypes.c_int, ctypes.c_long, P, P]
        lib.cgref_lu_solve.restype = ctypes.c_int
        lib.cgref_lu_solve.argtypes = [ctypes.c_int, P, P]
        lib.cgref_gmres.restype = ctypes.c_int
        lib.cgref_gmres.argtypes = [ctypes.c_int, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, P]
        lib.cgref_temperature.argtypes = [P, ctypes.c_int, ctypes.c_long, P, P, P, ctypes.c_int, P]
        lib.cgref_integrate.argtypes = [P, P, P, P, ctypes.c_long, P, P, P, ctypes.c_int]
        I = ctypes.c_int
        lib.cgref_integrate_hist.argtypes = [P, P, P, P, ctypes.c_long, P, P, P, P, I, I]
        lib.cgref_replay.argtypes = [P, P, P, P, ctypes.c_long, P, P, P, I, P, I]
        lib.cgref_adjoint.argtypes = [P, P, P, P, ctypes.c_long, P, P, P, P, P, I]
        lib.cgref_tangent.argtypes = [P, P, P, P, ctypes.c_long, P, P, I, I, P, P, I]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def lu_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Dense solve with LU and partial pivoting (Section 3.4)."""
    lib = _load()
    A = _f64(A).copy(); x = _f64(b).copy()
    if not lib.cgref_lu_solve(A.shape[0], _p(A), _p(x)):
        raise np.linalg.LinAlgError("singular matrix")
    return x


LU, GMRES = 0, 1
PC_NONE, PC_JACOBI, PC_GAUSS_SEIDEL = 0, 1, 2


def gmres(A: np.ndarray, b: np.ndarray, prec: int = PC_NONE, m: int = 30, maxit: int = 1000,
          tol: float = 1e-12):
    """Restarted, left-preconditioned GMRES of Section 3.4 on a dense system;
    returns (x, converged, iterations)."""
    A = _f64(A)
    x = _f64(b).copy()
    it = ctypes.c_int(0)
    ok = _load().cgref_gmres(A.shape[0], _p(A), _p(x), prec, m, maxit, tol, ctypes.byref(it))
    return x, bool(ok), it.value


def default_opts(**kw) -> dict:
    o = dict(method=SDIRK4, reactor=CONP, adaptive=1, nsub=1, max_newton=7, max_steps=100000,
             max_halvings=10, err_filter=1, dt=1e-6, rtol=1e-6, atol=1e-12, newton_tol=0.03,
             h0=0.0, hmin=1e-20, neg_tol=1e-6, linear_solver=LU, preconditioner=PC_GAUSS_SEIDEL,
             gmres_restart=30, gmres_maxit=200, gmres_tol=1e-10)
    o.update(kw)
    return o


class RefMech:
    """Oracle handle of one mechanism (host copy)."""

    def __init__(self, mech):
        self.mech = mech
        lib = _load()
        self._keep = [_f64(mech.W), _f64(mech.nasa7), _i32(mech.rtype), _i32(mech.reversible),
                      _i32(mech.rf_idx), _i32(mech.rf_nu), _i32(mech.rr_idx), _i32(mech.rr_nu),
                      _f64(mech.arr), _f64(mech.arr0), _f64(mech.troe), _i32(mech.eff_ptr),
                      _i32(mech.eff_idx) if len(mech.eff_idx) else np.zeros(1, np.int32),
                      _f64(mech.eff_val) if len(mech.eff_val) else np.zeros(1),
                      _f64(mech.sri), _i32(mech.plog_ptr),
                      _f64(mech.plog) if len(mech.plog) else np.zeros(4)]
        self.h = lib.cgref_mech_create(mech.ns, mech.nr, *[_p(a) for a in self._keep])
        if getattr(mech, "thermo", None) is not None:   # a c_p polynomial of degree n_p != NASA-7's
            coef = _f64(mech.thermo)
            if lib.cgref_mech_set_thermo(self.h, coef.shape[1] - 3, _p(coef)) != 0:
                raise ValueError("thermo degree n_p must lie in [0, 15]")
        self.ns, self.nr = mech.ns, mech.nr
        self.n = mech.ns + 1

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.cgref_mech_destroy(self.h)
            self.h = None

    # -- single-state helpers -------------------------------------------
    def thermo(self, T: float) -> dict:
        """Mass-specific cp, h, u, s, g, cv of every species at T (Table 1)."""
        out = {k: np.zeros(self.ns) for k in ("cp", "h", "u", "s", "g", "cv")}
        _load().cgref_thermo(self.h, float(T), *[_p(out[k]) for k in ("cp", "h", "u", "s", "g", "cv")])
        return out

    def rates(self, T: float, C: np.ndarray):
        kf, kr, q = np.zeros(self.nr), np.zeros(self.nr), np.zeros(self.nr)
        C = _f64(C)
        _load().cgref_rates(self.h, float(T), _p(C), _p(kf), _p(kr), _p(q))
        return kf, kr, q

    # -- batched over cells (cell-major) -----------------------------------
    @staticmethod
    def _state(T, C):
        T = np.atleast_1d(np.asarray(T, dtype=np.float64))
        C = np.atleast_2d(np.asarray(C, dtype=np.float64))
        return np.ascontiguousarray(np.concatenate([T[:, None], C], axis=1))

    def source(self, T, C, reactor: int = CONV) -> np.ndarray:
        """S = (omega_T, dC/dt) for each cell; returns [N, ns+1]."""
        y = self._state(T, C)
        S = np.zeros_like(y)
        _load().cgref_source(self.h, reactor, y.shape[0], _p(y), _p(S))
        return S

    def source_complex(self, y: np.ndarray, reactor: int = CONV) -> np.ndarray:
        y = np.asarray(y, dtype=np.complex128)
        yr, yi = _f64(y.real), _f64(y.imag)
        Sr, Si = np.zeros(self.n), np.zeros(self.n)
        _load().cgref_source_complex(self.h, reactor, _p(yr), _p(yi), _p(Sr), _p(Si))
        return Sr + 1j * Si

    def jacobian(self, T, C, reactor: int = CONV) -> np.ndarray:
        """Analytical J = dS/dy, [N, n, n]."""
        y = self._state(T, C)
        J = np.zeros((y.shape[0], self.n, self.n))
        _load().cgref_jacobian(self.h, reactor, y.shape[0], _p(y), _p(J))
        return J

    def temperature(self, e, Y, T0, iters: int = 5, reactor: int = CONV) -> np.ndarray:
        e = _f64(np.atleast_1d(e)); Y = _f64(np.atleast_2d(Y)); T0 = _f64(np.atleast_1d(T0))
        T = np.zeros_like(e)
        _load().cgref_temperature(self.h, reactor, e.shape[0], _p(e), _p(Y), _p(T0), iters, _p(T))
        return T

    # -- state conversions (Section 2 definitions) -------------------------
    def concentrations(self, T, Y, p_or_rho, reactor: int):
        """C_i = rho Y_i / W_i; rho given (CONV) or rho = p/(R T sum Y/W)."""
        T = np.asarray(T, dtype=np.float64); Y = np.asarray(Y, dtype=np.float64)
        if reactor == CONV:
            rho = np.asarray(p_or_rho, dtype=np.float64)
        else:
            rho = np.asarray(p_or_rho) / (R_UNIV * T * (Y / self.mech.W).sum(axis=1))
        return rho[:, None] * Y / self.mech.W

    def mass_fractions(self, C):
        rho_i = np.asarray(C) * self.mech.W
        return rho_i / rho_i.sum(axis=1, keepdims=True)

    @staticmethod
    def _packed(opts: dict):
        o = default_opts(**opts)
        iopt = _i32([o["method"], o["reactor"], o["adaptive"], o["nsub"], o["max_newton"],
                     o["max_steps"], o["max_halvings"], o["err_filter"], o["linear_solver"],
                     o["preconditioner"], o["gmres_restart"], o["gmres_maxit"]])
        dopt = _f64([o["dt"], o["rtol"], o["atol"], o["newton_tol"], o["h0"], o["hmin"],
                     o["neg_tol"], o["gmres_tol"]])
        tab = _tableau.pack(_tableau.tableau(o["method"]))
        return iopt, dopt, tab

    def integrate_hist(self, y, opts: dict, cap: int = 4096, nthreads: int = 1):
        """Integrate y[N, n] and return (y_end, status, step sizes hs[N, cap],
        accepted-step counts hn[N])."""
        iopt, dopt, tab = self._packed(opts)
        y = _f64(y).copy()
        N = y.shape[0]
        st = np.zeros(N, np.int32)
        hs = np.zeros((N, cap))
        hn = np.zeros(N, np.int32)
        _load().cgref_integrate_hist(self.h, _p(iopt), _p(dopt), _p(tab), N, _p(y), _p(st), _p(hs), _p(hn),
                                     cap, int(nthreads))
        return y, st, hs, hn

    def replay(self, y, opts: dict, hs, hn, nthreads: int = 1):
        """Steps of the given sizes (no step-size control) from y[N, n]."""
        iopt, dopt, tab = self._packed(opts)
        y = _f64(y).copy()
        hs = _f64(hs)
        hn = _i32(hn)
        N = y.shape[0]
        st = np.zeros(N, np.int32)
        _load().cgref_replay(self.h, _p(iopt), _p(dopt), _p(tab), N, _p(y), _p(hs), _p(hn), hs.shape[1],
                             _p(st), int(nthreads))
        return y, st

    def adjoint(self, y0, lam_end, opts: dict, nthreads: int = 1):
        """Discrete adjoint of the integration from y0[N, n] with
        lam_end = dL/dy_end[N, n]; returns (dL/dy0 [N, n],
        dL/dtheta [N, nr, 3] for (ln A, b, Ea), status)."""
        iopt, dopt, tab = self._packed(opts)
        y0 = _f64(y0)
        lam = _f64(lam_end)
        N = y0.shape[0]
        dy0 = np.zeros_like(y0)
        grad = np.zeros((N, self.nr, 3))
        st = np.zeros(N, np.int32)
        _load().cgref_adjoint(self.h, _p(iopt), _p(dopt), _p(tab), N, _p(y0), _p(lam), _p(dy0), _p(grad),
                              _p(st), int(nthreads))
        return dy0, grad, st

    def adjoint_TY(self, T0, Y0, p_or_rho, dT_end, dY_end, opts: dict, nthreads: int = 1):
        """The adjoint in the variables a flow solver holds: cells given by
        (T0, Y0[N, ns], p) (or rho at constant volume), loss gradients
        dL/dT_end[N], dL/dY_end[N, ns]. Chains the state adjoint through
        Y_k = W_k C_k / rho with rho = sum W_i C_i (Section 2) at the end and
        C_k = rho Y_k / W_k at the start (rho given, or p / (R T sum Y/W)).
        Returns (dL/dT0 [N], dL/dY0 [N, ns], dL/dtheta [N, nr, 3], status)."""
        reactor = default_opts(**opts)["reactor"]
        T0 = _f64(T0)
        Y0 = _f64(Y0)
        W = self.mech.W
        C0 = self.concentrations(T0, Y0, p_or_rho, reactor)
        y0 = self._state(T0, C0)
        y_end, _, _ = self.integrate_y(y0, opts, nthreads)
        # dL/dC_end by the chain rule of Y_end(C_end)
        Cend = y_end[:, 1:]
        rho_end = (W * Cend).sum(axis=1)
        Yend = W * Cend / rho_end[:, None]
        dY_end = _f64(dY_end)
        J_YC = (W[None, None, :] * (np.eye(self.ns)[None] - Yend[:, :, None])) / rho_end[:, None, None]
        lam = np.zeros_like(y_end)
        lam[:, 0] = dT_end
        lam[:, 1:] = np.einsum("ck,ckm->cm", dY_end, J_YC)   # J_YC[c, k, m] = dY_k / dC_m
        dy0, g, st = self.adjoint(y0, lam, opts, nthreads)
        # dC0/dY0 and dC0/dT0
        if reactor == CONV:
            rho0 = np.asarray(p_or_rho, dtype=np.float64) * np.ones(len(T0))
            dC_dY = rho0[:, None, None] * np.eye(self.ns)[None] / W[None, :, None]
            dC_dT = np.zeros_like(C0)
        else:
            sig = (Y0 / W).sum(axis=1)
            rho0 = np.asarray(p_or_rho, dtype=np.float64) / (R_UNIV * T0 * sig)
            # C_m = rho Y_m / W_m, d rho / d Y_k = -rho / (W_k sig), d rho / d T0 = -rho / T0
            dC_dY = (rho0[:, None, None] * np.eye(self.ns)[None] / W[None, :, None]
                     - (C0[:, :, None] / (W[None, None, :] * sig[:, None, None])))
            dC_dT = -C0 / T0[:, None]
        dY0 = np.einsum("cm,cmk->ck", dy0[:, 1:], dC_dY)     # dC_dY[c, m, k] = dC_m / dY_k
        dT0 = dy0[:, 0] + (dy0[:, 1:] * dC_dT).sum(axis=1)
        return dT0, dY0, g, st

    def react_split(self, rho, e, rhoY, T_guess, opts: dict, iters: int = 5, nthreads: int = 1):
        """Operator-split reaction step of a flow solver (Section 5.5): T from
        (e, Y = rhoY / rho) by the Newton of Section 2.1, then C = rhoY / W
        integrated at constant volume over dt; returns (T after dt,
        R = W (C^{n+1} - C^n) / dt [N, ns], status, stats)."""
        rho = _f64(rho)
        rhoY = _f64(rhoY)
        Y = rhoY / rho[:, None]
        T = self.temperature(e, Y, T_guess, iters, CONV)
        C = rhoY / self.mech.W
        o = dict(opts, reactor=CONV)
        y, status, stats = self.integrate_y(self._state(T, C), o, nthreads)
        R = (self.mech.W * y[:, 1:] - rhoY) / default_opts(**o)["dt"]
        return y[:, 0].copy(), R, status, stats

    def tangent(self, y0, dy0, opts: dict, pj: int = -1, pk: int = 0, nthreads: int = 1):
        """Forward sensitivity dy_end for the initial perturbation dy0 and
        the parameter (reaction pj, kind pk: 0 ln A, 1 b, 2 Ea)."""
        iopt, dopt, tab = self._packed(opts)
        y0 = _f64(y0)
        dy0 = _f64(dy0)
        N = y0.shape[0]
        dyend = np.zeros_like(y0)
        st = np.zeros(N, np.int32)
        _load().cgref_tangent(self.h, _p(iopt), _p(dopt), _p(tab), N, _p(y0), _p(dy0), int(pj), int(pk),
                              _p(dyend), _p(st), int(nthreads))
        return dyend, st

    def integrate_y(self, y: np.ndarray, opts: dict, nthreads: int = 1):
        """Integrate states y[N, ns+1] over opts['dt']; returns (y, status, stats)."""
        iopt, dopt, tab = self._packed(opts)
        y = _f64(y).copy()
        N = y.shape[0]
        status = np.zeros(N, dtype=np.int32)
        stats = np.zeros((N, 4), dtype=np.int32)
        _load().cgref_integrate(self.h, _p(iopt), _p(dopt), _p(tab), N, _p(y), _p(status),
                                _p(stats), int(nthreads))
        return y, status, stats

    def integrate(self, T, Y, p_or_rho, opts: dict, nthreads: int = 1):
        """Integrate cells given (T, Y, p) (CONP) or (T, Y, rho) (CONV) over
        opts['dt']; returns (T, Y, status, stats)."""
        reactor = default_opts(**opts)["reactor"]
        C = self.concentrations(T, Y, p_or_rho, reactor)
        y = self._state(T, C)
        y, status, stats = self.integrate_y(y, opts, nthreads)
        return y[:, 0].copy(), self.mass_fractions(y[:, 1:]), status, stats
