// Pieces shared by the forward integration and the adjoint sweep: the team's
// position in a launch and its cell loop, one implicit Runge-Kutta step
// (Section 3.2, Appendix A), checkpoints, and the host-side launch helpers.
#pragma once

#include "chem_device.cuh"
#include "chem_internal.h"

namespace cg {

constexpr double kR = 8314.46261815324;   // J/(kmol K)

// Position of this team in the launch.
template <int TEAM>
struct TeamPos {
    int lane, tib, tpb;
    int64_t id, count;
    __device__ __forceinline__ TeamPos() {
        lane = team_lane<TEAM>();
        tpb = blockDim.x / TEAM;
        tib = threadIdx.x / TEAM;
        id = (int64_t)blockIdx.x * tpb + tib;
        count = (int64_t)gridDim.x * tpb;
    }
};

// Next global cell index: from the work counter (every thread of the team
// gets the same value) or the fixed stride.
template <int TEAM>
__device__ __forceinline__ int64_t next_cell(unsigned long long* counter, int64_t prev, int64_t stride,
                                             int lane) {
    if (!counter) return prev + stride;
    if constexpr (TEAM == 32) {
        unsigned long long v = 0;
        if (lane == 0) v = atomicAdd(counter, 1ull);
        return (int64_t)__shfl_sync(kFull, v, 0);
    } else {
        __shared__ unsigned long long slot;
        __syncthreads();
        if (lane == 0) slot = atomicAdd(counter, 1ull);
        __syncthreads();
        return (int64_t)slot;
    }
}

template <int TEAM>
__device__ __forceinline__ int64_t first_cell(unsigned long long* counter, int64_t id, int lane) {
    return counter ? next_cell<TEAM>(counter, 0, 0, lane) : id;
}

// Registers per thread of the cell kernels (integration, split, adjoint), by
// team size and Newton-matrix type: the most that still lets the intended
// number of cells share an SM's 65,536 registers. Left to itself the
// compiler gives every kernel about 254, because the register tiles of the
// blocked LU raise the whole kernel's allocation even where that path does
// not run, and then only four 64-thread cells fit on an SM.
//   TEAM 32: 168 (12 one-warp cells)      TEAM 64: 128 (8 cells)
//   TEAM 128: 128 (4 cells)               TEAM 256 FP32: 128 (2 cells)
//   TEAM 256 FP64: 255 (the 207 KB FP64 Newton matrix of 161 unknowns
//   allows one cell per SM)
// At 53 species (team 64, FP64) 128 registers spill about 1 KB per thread
// and still run 1.08 times faster than 168 (8 cells per SM instead of 6).
template <int TEAM, class MT>
struct KernelRegs {
    static constexpr int value = TEAM == 32 ? 168
                                 : TEAM == 64 ? 128
                                 : TEAM == 128 ? 128
                                 : (sizeof(MT) == 8 ? 255 : 128);
};

// ---------------------------------------------------------------------------
// integration

struct Counters {
    int steps, rejects, newton, lu;
};

// Linear solver of the Newton systems (Section 3.4): the dense LU of G, or
// GMRES on G as assembled (one warp of the team; the others wait). Counter
// `lu` counts factorisations or GMRES iterations.
template <int TEAM, class MT>
__device__ __forceinline__ bool lin_prepare(const DevMech& M, const Ws& W, const IntParams& P, int n,
                                            Counters& cnt, int lane) {
    MT* G = reinterpret_cast<MT*>(W.G);
    if (P.linear_solver == 0) {
        cnt.lu++;
        return lu_factor_nb<TEAM, MT>(G, n, W.ld, M.lu_nb, W.piv, W.rinv, W.red, lane);
    }
    bool zero = false;   // inverse diagonal for the preconditioner
    for (int i = lane; i < n; i += TEAM) {
        const double d = static_cast<double>(G[i * W.ld + i]);
        zero |= d == 0.0;
        W.rinv[i] = d != 0.0 ? rcp_nr(d) : 0.0;
    }
    team_sync<TEAM>();
    zero = team_any<TEAM>(zero, W.red);
    return P.prec == 0 || !zero;
}

template <int TEAM, class MT>
__device__ __forceinline__ bool lin_solve(const Ws& W, const IntParams& P, int n, double* x, Counters& cnt,
                                          int lane) {
    const MT* G = reinterpret_cast<const MT*>(W.G);
    if (P.linear_solver == 0) {
        if constexpr (sizeof(MT) == 4)   // colB is free while a step solves
            lu_solve_f32<TEAM>(G, n, W.ld, W.piv, reinterpret_cast<const float*>(W.rinv), x,
                               reinterpret_cast<float*>(W.colB), lane);
        else
            lu_solve<TEAM, MT>(G, n, W.ld, W.piv, W.rinv, x, lane);
        return true;
    }
    int* flag = reinterpret_cast<int*>(W.red + 20);
    if (lane < 32) {
        GmresWs K;
        K.m = P.gmres_m;
        K.vs = n | 1;
        K.V = W.kv;
        K.H = W.kh;
        K.cs = K.H + (K.m + 1) * K.m;
        K.sn = K.cs + K.m;
        K.g = K.sn + K.m;
        K.t = K.g + K.m + 1;
        K.bb = W.colA;
        K.w = W.colB;
        int it = 0;
        const bool ok = warp_gmres<MT>(G, n, W.ld, W.rinv, P.prec, P.gmres_maxit, P.gmres_tol, x, K, lane, it);
        if (lane == 0) {
            flag[0] = ok ? 1 : 0;
            flag[1] = it;
        }
    }
    team_sync<TEAM>();
    const bool ok = flag[0] != 0;
    cnt.lu += flag[1];
    team_sync<TEAM>();
    return ok;
}

// One step of size h from W.yn: stages of the tableau in stage-derivative
// form (Appendix A), each by full Newton with G = I - a_pp h J(Y_p). On
// success y1 holds the new state and err the (filtered) embedded estimate.
// MT = float: G is assembled and factored in FP32 (an inexact Newton whose
// residual, update and convergence test stay in FP64).
template <int TEAM, class MT>
__device__ bool rk_step(const DevMech& M, const Ws& W, const IntParams& P, double h, Counters& cnt,
                        int lane) {
    const int n = M.n;
    double* yn = W.yn;
    double* Y = W.Y;
    double* base = W.base;
    double* S = W.S;
    double* S0 = W.S0;
    double* f = W.f;
    MT* G = reinterpret_cast<MT*>(W.G);
    if (!P.start_zero) {   // first Newton iterate of every stage: Gamma = S(y_n)
        const double Mc = rates<TEAM>(M, W, yn, false, lane);
        assemble_source<TEAM>(M, W, yn, P.reactor, Mc, lane);
        for (int i = lane; i < n; i += TEAM) S0[i] = S[i];
        team_sync<TEAM>();
    }
    for (int p = 0; p < P.s; ++p) {
        const double gh = P.A[p][p] * h;
        double* Gp = W.Gam + p * n;
        for (int i = lane; i < n; i += TEAM) {
            double b = yn[i];
            for (int j = 0; j < p; ++j) b = fma(h * P.A[p][j], W.Gam[j * n + i], b);
            base[i] = b;
            Gp[i] = P.start_zero ? 0.0 : S0[i];
        }
        team_sync<TEAM>();
        bool conv = false;
        for (int k = 0; k < P.max_newton; ++k) {
            for (int i = lane; i < n; i += TEAM) Y[i] = fma(gh, Gp[i], base[i]);
            team_sync<TEAM>();
            const double Mc = rates<TEAM>(M, W, Y, true, lane);
            const SrcInfo si = assemble_source<TEAM>(M, W, Y, P.reactor, Mc, lane);
            assemble_jacobian<TEAM, MT>(M, W, Y, P.reactor, si, gh, nullptr, lane);
            for (int i = lane; i < n; i += TEAM) f[i] = S[i] - Gp[i];   // -f(Gamma)
            team_sync<TEAM>();
            cnt.newton++;
            if (!lin_prepare<TEAM, MT>(M, W, P, n, cnt, lane)) return false;
            if (!lin_solve<TEAM, MT>(W, P, n, f, cnt, lane)) return false;
            for (int i = lane; i < n; i += TEAM) {
                const double g = Gp[i] + f[i];
                Gp[i] = g;
                f[i] *= gh;                  // change of the stage state
                Y[i] = fma(gh, g, base[i]);
            }
            team_sync<TEAM>();
            const double nrm = wrms<TEAM>(f, yn, Y, n, P.rtol, P.atol, W.red, lane);
            if (!isfinite(nrm)) return false;
            if (nrm <= P.newton_tol) { conv = true; break; }
        }
        if (!conv) return false;
    }
    double* y1 = W.y1;
    double* err = W.err;
    bool bad = false;
    for (int i = lane; i < n; i += TEAM) {
        double v = yn[i], e = 0.0;
        for (int p = 0; p < P.s; ++p) {
            const double g = W.Gam[p * n + i];
            v = fma(h * P.b[p], g, v);
            e = fma(h * (P.b[p] - P.bh[p]), g, e);
        }
        y1[i] = v;
        err[i] = e;
        bad |= !isfinite(v);
    }
    team_sync<TEAM>();
    if (team_any<TEAM>(bad, W.red)) return false;
    if (P.adaptive && P.err_filter && !lin_solve<TEAM, MT>(W, P, n, err, cnt, lane)) return false;
    // admissible: T > 0 and C_i >= -neg_tol sum C
    double cs = 0.0;
    for (int i = 1 + lane; i < n; i += TEAM) cs += y1[i];
    cs = team_sum<TEAM>(cs, W.red);
    bool neg = false;
    for (int i = 1 + lane; i < n; i += TEAM) neg |= y1[i] < -P.neg_tol * cs;
    neg = team_any<TEAM>(neg, W.red) || !(y1[0] > 0.0);
    return !neg;
}

// Second-order Rosenbrock step (Appendix A.3, coefficients of FATODE's Ros2
// as the appendix quotes them): with G = I - h gamma J(y_n),
//   G Gamma_1 = h gamma S(y_n),
//   G Gamma_2 = h gamma S(y_n + alpha Gamma_1) + gamma beta Gamma_1,
//   y_{n+1} = y_n + m1 Gamma_1 + m2 Gamma_2,
// (the appendix's (I/(h gamma) - J) form multiplied through by h gamma; its
// printed extra -S(y_n) in the second stage is not taken: it makes the
// scheme inconsistent). One Jacobian, one factorisation, two solves.
// Embedded first-order error (Gamma_1 + Gamma_2)/(2 gamma) into W.err.
// P.A[0][0] = gamma, P.A[1][0] = alpha, P.A[1][1] = beta, P.b = (m1, m2).
template <int TEAM, class MT>
__device__ bool ros2_step(const DevMech& M, const Ws& W, const IntParams& P, double h, Counters& cnt,
                          int lane) {
    const int n = M.n;
    const double g = P.A[0][0], al = P.A[1][0], be = P.A[1][1];
    const double hg = h * g;
    double* yn = W.yn;
    double* G1 = W.Gam;
    double* G2 = W.Gam + n;
    MT* G = reinterpret_cast<MT*>(W.G);
    const double Mc = rates<TEAM>(M, W, yn, true, lane);
    const SrcInfo si = assemble_source<TEAM>(M, W, yn, P.reactor, Mc, lane);
    assemble_jacobian<TEAM, MT>(M, W, yn, P.reactor, si, hg, nullptr, lane);
    for (int i = lane; i < n; i += TEAM) G1[i] = hg * W.S[i];
    team_sync<TEAM>();
    cnt.newton++;
    if (!lin_prepare<TEAM, MT>(M, W, P, n, cnt, lane)) return false;
    if (!lin_solve<TEAM, MT>(W, P, n, G1, cnt, lane)) return false;
    bool bad = false;
    for (int i = lane; i < n; i += TEAM) {
        const double v = fma(al, G1[i], yn[i]);
        W.Y[i] = v;
        bad |= !isfinite(v);
    }
    team_sync<TEAM>();
    if (team_any<TEAM>(bad, W.red)) return false;
    const double Mc2 = rates<TEAM>(M, W, W.Y, false, lane);
    assemble_source<TEAM>(M, W, W.Y, P.reactor, Mc2, lane);
    for (int i = lane; i < n; i += TEAM) G2[i] = fma(hg, W.S[i], g * be * G1[i]);
    team_sync<TEAM>();
    if (!lin_solve<TEAM, MT>(W, P, n, G2, cnt, lane)) return false;
    const double e = 0.5 / g;
    for (int i = lane; i < n; i += TEAM) {
        const double v = fma(P.b[1], G2[i], fma(P.b[0], G1[i], yn[i]));
        W.y1[i] = v;
        W.err[i] = e * (G1[i] + G2[i]);
        bad |= !isfinite(v);
    }
    team_sync<TEAM>();
    if (team_any<TEAM>(bad, W.red)) return false;
    double cs = 0.0;
    for (int i = 1 + lane; i < n; i += TEAM) cs += W.y1[i];
    cs = team_sum<TEAM>(cs, W.red);
    bool neg = false;
    for (int i = 1 + lane; i < n; i += TEAM) neg |= W.y1[i] < -P.neg_tol * cs;
    neg = team_any<TEAM>(neg, W.red) || !(W.y1[0] > 0.0);
    return !neg;
}

// One step of the configured integrator: Rosenbrock-2, or the implicit
// Runge-Kutta step (backward Euler, SDIRK-2/4; YASS is backward Euler with a
// single Newton iteration whose decrement norm must stay below alpha).
template <int TEAM, class MT>
__device__ __forceinline__ bool step(const DevMech& M, const Ws& W, const IntParams& P, double h,
                                     Counters& cnt, int lane) {
    if (P.method == 3) return ros2_step<TEAM, MT>(M, W, P, h, cnt, lane);
    return rk_step<TEAM, MT>(M, W, P, h, cnt, lane);
}

template <int TEAM>
__device__ __forceinline__ void copy_vec(double* dst, const double* src, int n, int lane) {
    for (int i = lane; i < n; i += TEAM) dst[i] = src[i];
    team_sync<TEAM>();
}

// Checkpoint k of a cell: (y_k, h_k) when 0 <= k < cap (the record after
// the last step holds the final state and the density that converted the
// initial mass fractions).
template <int TEAM>
__device__ __forceinline__ void save_step(double* ck, int cap, int k, const double* y, double h, int n,
                                          int lane) {
    if (!ck || k < 0 || k >= cap) return;
    double* e = ck + (int64_t)k * (n + 1);
    for (int i = lane; i < n; i += TEAM) e[i] = y[i];
    if (lane == 0) e[n] = h;
}

// The integrators below record accepted step k as checkpoint k - rec_from
// of ck (cap entries) and return after stop_after accepted steps: the
// forward pass records from step 0 and never stops early; the adjoint's
// replay of a segment records [rec_from, stop_after) of the same steps.

// Fixed steps with deterministic halving: a failed step of level d is
// replaced by two steps of level d+1 (recursively, at most max_halvings
// deep), walked iteratively with a position counter.
template <int TEAM, class MT>
__device__ int integrate_fixed(const DevMech& M, const Ws& W, const IntParams& P, Counters& cnt, double* ck,
                               int cap, int lane, int rec_from = 0, int stop_after = 0x7fffffff) {
    const int D = P.max_halvings;
    const double hsub = P.dt / P.nsub;
    for (int s = 0; s < P.nsub; ++s) {
        unsigned long long pos = 0ull;
        const unsigned long long total = 1ull << D;
        int d = 0;
        while (pos < total) {
            const double h = ldexp(hsub, -d);
            if (step<TEAM, MT>(M, W, P, h, cnt, lane)) {
                save_step<TEAM>(ck, cap, cnt.steps - rec_from, W.yn, h, M.n, lane);
                copy_vec<TEAM>(W.yn, W.y1, M.n, lane);
                if (++cnt.steps >= stop_after) return CELL_OK;
                pos += 1ull << (D - d);
                while (d > 0 && ((pos >> (D - d)) & 1ull) == 0ull) --d;
            } else {
                cnt.rejects++;
                if (d >= D) return CELL_NEWTON_FAIL;
                ++d;
            }
        }
    }
    return CELL_OK;
}

// Error-controlled steps: accept when WRMS(err) <= 1; next step
// h min(5, max(0.2, 0.9 err^(-1/(q+1)))); Newton failure: h / 4.
template <int TEAM, class MT>
__device__ int integrate_adaptive(const DevMech& M, const Ws& W, const IntParams& P, Counters& cnt, double* ck,
                                  int cap, int lane, int rec_from = 0, int stop_after = 0x7fffffff) {
    const double expo = -1.0 / (P.err_order + 1.0);
    double t = 0.0;
    double h = P.h0 > 0.0 ? fmin(P.h0, P.dt) : P.dt;
    int attempts = 0;
    while (t < P.dt) {
        if (attempts++ >= P.max_steps) return CELL_MAX_STEPS;
        if (h < P.hmin) return CELL_STEP_TOO_SMALL;
        const bool last = t + h >= P.dt;
        const double hh = last ? P.dt - t : h;
        if (!step<TEAM, MT>(M, W, P, hh, cnt, lane)) {
            cnt.rejects++;
            h = 0.25 * hh;
            continue;
        }
        const double e = wrms<TEAM>(W.err, W.yn, W.y1, M.n, P.rtol, P.atol, W.red, lane);
        double fac = e > 0.0 ? 0.9 * pow(e, expo) : 5.0;
        fac = fmin(5.0, fmax(0.2, fac));
        if (e <= 1.0) {
            save_step<TEAM>(ck, cap, cnt.steps - rec_from, W.yn, hh, M.n, lane);
            copy_vec<TEAM>(W.yn, W.y1, M.n, lane);
            t = last ? P.dt : t + hh;
            if (++cnt.steps >= stop_after) return CELL_OK;
        } else {
            cnt.rejects++;
        }
        h = hh * fac;
    }
    return CELL_OK;
}

// ---------------------------------------------------------------------------
// host-side launch helpers

static inline cudaError_t set_smem(const void* fn, size_t smem) {
    if (smem > 48 * 1024)
        return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

// Blocks that keep every SM full (persistent launches).
static inline cudaError_t resident_blocks(const void* fn, int threads, size_t smem, int64_t* out) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
    if (e != cudaSuccess) return e;
    *out = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    return cudaSuccess;
}

__host__ __device__ static inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Global scratch slots (one per team) and the work counter, allocated
// stream-ordered for this launch and released after it.
struct LaunchMem {
    double* gscratch = nullptr;
    unsigned long long* counter = nullptr;
};

static inline cudaError_t get_mem(int64_t teams, int64_t gstride, bool need_counter, cudaStream_t st,
                           LaunchMem& m) {
    cudaError_t e;
    if (gstride) {
        void* p = nullptr;
        if ((e = cudaMallocAsync(&p, (size_t)(teams * gstride) * sizeof(double), st)) != cudaSuccess)
            return e;
        m.gscratch = static_cast<double*>(p);
    }
    if (need_counter) {   // two counters: whole-team cells, and cells of split tasks
        void* p = nullptr;
        if ((e = cudaMallocAsync(&p, 2 * sizeof(unsigned long long), st)) != cudaSuccess) return e;
        m.counter = static_cast<unsigned long long*>(p);
        return cudaMemsetAsync(m.counter, 0, 2 * sizeof(unsigned long long), st);
    }
    return cudaSuccess;
}

static inline cudaError_t put_mem(LaunchMem& m, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (m.gscratch) e = cudaFreeAsync(m.gscratch, st);
    if (m.counter && e == cudaSuccess) e = cudaFreeAsync(m.counter, st);
    return e;
}

#ifndef CG_DEBUG
#define CG_DISPATCH_TEAM(team, CALL)                         \
    switch (team) {                                          \
        case 32: return CALL(32);                            \
        case 64: return CALL(64);                            \
        case 128: return CALL(128);                          \
        case 256: return CALL(256);                          \
        default: return cudaErrorInvalidValue;               \
    }
#else   // the debug build holds the one-warp teams only
#define CG_DISPATCH_TEAM(team, CALL)                         \
    switch (team) {                                          \
        case 32: return CALL(32);                            \
        default: return cudaErrorInvalidValue;               \
    }
#endif

}  // namespace cg
