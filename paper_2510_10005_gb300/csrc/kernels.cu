// Kernels of chemgb: one team of TEAM threads per cell (TEAM = 32: one warp,
// several teams per block; TEAM = 64..256: one team per block).
//
//   eval_rates_kernel      S(y) for N cells (Section 2.2, Section 3, App. B)
//   eval_jacobian_kernel   dS/dy for N cells (Section 3.2)
//   temperature_kernel     T from (e, Y) by Newton (Section 2.1)
//   integrate_kernel       backward Euler / SDIRK over dt (Section 3.2, App. A)
#include "chem_device.cuh"
#include "chem_internal.h"

namespace cg {

constexpr double kR = 8314.46261815324;   // J/(kmol K)

template <int TEAM>
__device__ __forceinline__ double* team_smem(const Layout& L) {
    extern __shared__ double smem_all[];
    return smem_all + (size_t)(threadIdx.x / TEAM) * L.total;
}

template <int TEAM>
__device__ __forceinline__ int64_t team_cell() {
    return (int64_t)blockIdx.x * (blockDim.x / TEAM) + threadIdx.x / TEAM;
}

// ---------------------------------------------------------------------------

template <int TEAM>
__global__ void eval_rates_kernel(DevMech M, Layout L, int reactor, int64_t N,
                                  const double* __restrict__ T, const double* __restrict__ C,
                                  double* __restrict__ S) {
    const int lane = team_lane<TEAM>();
    const int64_t cell = team_cell<TEAM>();
    if (cell >= N) return;   // whole team (a team never straddles this bound)
    double* sm = team_smem<TEAM>(L);
    double* y = sm + L.Y;
    if (lane == 0) y[0] = T[cell];
    for (int i = lane; i < M.ns; i += TEAM) y[1 + i] = C[(int64_t)i * N + cell];
    team_sync<TEAM>();
    const double Mc = rates<TEAM>(M, L, sm, y, false, lane);
    assemble_source<TEAM>(M, L, sm, y, reactor, Mc, lane);
    const double* Sv = sm + L.S;
    for (int i = lane; i < M.n; i += TEAM) S[(int64_t)i * N + cell] = Sv[i];
}

template <int TEAM>
__global__ void eval_jacobian_kernel(DevMech M, Layout L, int reactor, int64_t N,
                                     const double* __restrict__ T, const double* __restrict__ C,
                                     double* __restrict__ J) {
    const int lane = team_lane<TEAM>();
    const int64_t cell = team_cell<TEAM>();
    if (cell >= N) return;
    double* sm = team_smem<TEAM>(L);
    double* y = sm + L.Y;
    if (lane == 0) y[0] = T[cell];
    for (int i = lane; i < M.ns; i += TEAM) y[1 + i] = C[(int64_t)i * N + cell];
    team_sync<TEAM>();
    const double Mc = rates<TEAM>(M, L, sm, y, true, lane);
    const SrcInfo si = assemble_source<TEAM>(M, L, sm, y, reactor, Mc, lane);
    assemble_jacobian<TEAM, double>(M, L, sm, y, reactor, si, 0.0, J + cell * (int64_t)M.n * M.n, lane);
}

// Newton on sum_i Y_i e_i(T) = e, e = u (constant volume) or h (otherwise),
// molar e_i = R T h/RT (minus R T for u), mass-specific = molar / W_i.
// One warp per cell.
__global__ void temperature_kernel(DevMech M, int reactor, int64_t N, const double* __restrict__ e,
                                   const double* __restrict__ Y, double* __restrict__ Tio,
                                   int iters) {
    const int lane = threadIdx.x & 31;
    const int64_t cell = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (cell >= N) return;
    const int ns = M.ns;
    const double sub = reactor == R_CONV ? 1.0 : 0.0;
    double T = Tio[cell];
    const double target = e[cell];
    for (int it = 0; it < iters; ++it) {
        const double invT = 1.0 / T;
        double ev = 0.0, cv = 0.0;
        for (int i = lane; i < ns; i += 32) {
            const double* th = M.th + i;
#define TH(k) __ldg(th + (k) * ns)
            const double cp = TH(TH_A1) + T * (TH(TH_A2) + T * (TH(TH_A3) + T * (TH(TH_A4) + T * TH(TH_A5))));
            const double h = TH(TH_A1) + T * (TH(TH_H2) + T * (TH(TH_H3) + T * (TH(TH_H4) + T * TH(TH_H5))))
                             + TH(TH_A6) * invT;
#undef TH
            const double yw = Y[(int64_t)i * N + cell] * __ldg(M.invW + i);
            ev = fma(yw, h - sub, ev);
            cv = fma(yw, cp - sub, cv);
        }
        ev = warp_sum(ev) * kR * T;
        cv = warp_sum(cv) * kR;
        T += (target - ev) / cv;
    }
    if (lane == 0) Tio[cell] = T;
}

// ---------------------------------------------------------------------------
// integration

struct Counters {
    int steps, rejects, newton, lu;
};

// One step of size h from sm[yn]: stages of the tableau in stage-derivative
// form (Appendix A), each by full Newton with G = I - a_pp h J(Y_p). On
// success y1 holds the new state and err the (filtered) embedded estimate.
// MT = float: G is assembled and factored in FP32 (an inexact Newton whose
// residual, update and convergence test stay in FP64).
template <int TEAM, class MT>
__device__ bool rk_step(const DevMech& M, const Layout& L, const IntParams& P, double* sm, double h,
                        Counters& cnt, int lane) {
    const int n = M.n;
    double* yn = sm + L.yn;
    double* Y = sm + L.Y;
    double* base = sm + L.base;
    double* S = sm + L.S;
    double* S0 = sm + L.S0;
    double* f = sm + L.f;
    MT* G = reinterpret_cast<MT*>(sm + L.G);
    double* rinv = sm + L.rinv;
    double* red = sm + L.red;
    int* piv = reinterpret_cast<int*>(sm + L.piv);
    if (!P.start_zero) {   // first Newton iterate of every stage: Gamma = S(y_n)
        const double Mc = rates<TEAM>(M, L, sm, yn, false, lane);
        assemble_source<TEAM>(M, L, sm, yn, P.reactor, Mc, lane);
        for (int i = lane; i < n; i += TEAM) S0[i] = S[i];
        team_sync<TEAM>();
    }
    for (int p = 0; p < P.s; ++p) {
        const double gh = P.A[p][p] * h;
        double* Gp = sm + L.Gam + p * n;
        for (int i = lane; i < n; i += TEAM) {
            double b = yn[i];
            for (int j = 0; j < p; ++j) b = fma(h * P.A[p][j], sm[L.Gam + j * n + i], b);
            base[i] = b;
            Gp[i] = P.start_zero ? 0.0 : S0[i];
        }
        team_sync<TEAM>();
        bool conv = false;
        for (int k = 0; k < P.max_newton; ++k) {
            for (int i = lane; i < n; i += TEAM) Y[i] = fma(gh, Gp[i], base[i]);
            team_sync<TEAM>();
            const double Mc = rates<TEAM>(M, L, sm, Y, true, lane);
            const SrcInfo si = assemble_source<TEAM>(M, L, sm, Y, P.reactor, Mc, lane);
            assemble_jacobian<TEAM, MT>(M, L, sm, Y, P.reactor, si, gh, nullptr, lane);
            for (int i = lane; i < n; i += TEAM) f[i] = S[i] - Gp[i];   // -f(Gamma)
            team_sync<TEAM>();
            cnt.newton++;
            cnt.lu++;
            if (!lu_factor<TEAM, MT>(G, n, L.ld, piv, rinv, red, lane)) return false;
            lu_solve<TEAM, MT>(G, n, L.ld, piv, rinv, f, lane);
            for (int i = lane; i < n; i += TEAM) {
                const double g = Gp[i] + f[i];
                Gp[i] = g;
                f[i] *= gh;                  // change of the stage state
                Y[i] = fma(gh, g, base[i]);
            }
            team_sync<TEAM>();
            const double nrm = wrms<TEAM>(f, yn, Y, n, P.rtol, P.atol, red, lane);
            if (!isfinite(nrm)) return false;
            if (nrm <= P.newton_tol) { conv = true; break; }
        }
        if (!conv) return false;
    }
    double* y1 = sm + L.y1;
    double* err = sm + L.err;
    bool bad = false;
    for (int i = lane; i < n; i += TEAM) {
        double v = yn[i], e = 0.0;
        for (int p = 0; p < P.s; ++p) {
            const double g = sm[L.Gam + p * n + i];
            v = fma(h * P.b[p], g, v);
            e = fma(h * (P.b[p] - P.bh[p]), g, e);
        }
        y1[i] = v;
        err[i] = e;
        bad |= !isfinite(v);
    }
    team_sync<TEAM>();
    if (team_any<TEAM>(bad, red)) return false;
    if (P.adaptive && P.err_filter) lu_solve<TEAM, MT>(G, n, L.ld, piv, rinv, err, lane);
    // admissible: T > 0 and C_i >= -neg_tol sum C
    double cs = 0.0;
    for (int i = 1 + lane; i < n; i += TEAM) cs += y1[i];
    cs = team_sum<TEAM>(cs, red);
    bool neg = false;
    for (int i = 1 + lane; i < n; i += TEAM) neg |= y1[i] < -P.neg_tol * cs;
    neg = team_any<TEAM>(neg, red) || !(y1[0] > 0.0);
    return !neg;
}

template <int TEAM>
__device__ __forceinline__ void copy_vec(double* dst, const double* src, int n, int lane) {
    for (int i = lane; i < n; i += TEAM) dst[i] = src[i];
    team_sync<TEAM>();
}

// Fixed steps with deterministic halving: a failed step of level d is
// replaced by two steps of level d+1 (recursively, at most max_halvings
// deep), walked iteratively with a position counter.
template <int TEAM, class MT>
__device__ int integrate_fixed(const DevMech& M, const Layout& L, const IntParams& P, double* sm,
                               Counters& cnt, int lane) {
    const int D = P.max_halvings;
    const double hsub = P.dt / P.nsub;
    for (int s = 0; s < P.nsub; ++s) {
        unsigned long long pos = 0ull;
        const unsigned long long total = 1ull << D;
        int d = 0;
        while (pos < total) {
            const double h = ldexp(hsub, -d);
            if (rk_step<TEAM, MT>(M, L, P, sm, h, cnt, lane)) {
                copy_vec<TEAM>(sm + L.yn, sm + L.y1, M.n, lane);
                cnt.steps++;
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
__device__ int integrate_adaptive(const DevMech& M, const Layout& L, const IntParams& P, double* sm,
                                  Counters& cnt, int lane) {
    const double expo = -1.0 / (P.err_order + 1.0);
    double t = 0.0;
    double h = P.h0 > 0.0 ? fmin(P.h0, P.dt) : P.dt;
    int attempts = 0;
    while (t < P.dt) {
        if (attempts++ >= P.max_steps) return CELL_MAX_STEPS;
        if (h < P.hmin) return CELL_STEP_TOO_SMALL;
        const bool last = t + h >= P.dt;
        const double hh = last ? P.dt - t : h;
        if (!rk_step<TEAM, MT>(M, L, P, sm, hh, cnt, lane)) {
            cnt.rejects++;
            h = 0.25 * hh;
            continue;
        }
        const double e = wrms<TEAM>(sm + L.err, sm + L.yn, sm + L.y1, M.n, P.rtol, P.atol, sm + L.red, lane);
        double fac = e > 0.0 ? 0.9 * pow(e, expo) : 5.0;
        fac = fmin(5.0, fmax(0.2, fac));
        if (e <= 1.0) {
            copy_vec<TEAM>(sm + L.yn, sm + L.y1, M.n, lane);
            t = last ? P.dt : t + hh;
            cnt.steps++;
        } else {
            cnt.rejects++;
        }
        h = hh * fac;
    }
    return CELL_OK;
}

template <int TEAM, class MT>
__global__ void integrate_kernel(DevMech M, Layout L, IntParams P, int64_t N, double* __restrict__ T,
                                 double* __restrict__ Yio, const double* __restrict__ p_or_rho,
                                 int32_t* __restrict__ status, int32_t* __restrict__ stats) {
    const int lane = team_lane<TEAM>();
    const int64_t cell = team_cell<TEAM>();
    if (cell >= N) return;
    const int ns = M.ns, n = M.n;
    double* sm = team_smem<TEAM>(L);
    double* yn = sm + L.yn;
    double* red = sm + L.red;
    // load and unpack: C_i = rho Y_i / W_i
    const double T0 = T[cell];
    const double pr = p_or_rho[cell];
    double ysum = 0.0;
    for (int i = lane; i < ns; i += TEAM) {
        const double Yi = Yio[(int64_t)i * N + cell];
        yn[1 + i] = Yi;
        ysum = fma(Yi, __ldg(M.invW + i), ysum);
    }
    ysum = team_sum<TEAM>(ysum, red);
    const double rho = P.reactor == R_CONV ? pr : pr / (kR * T0 * ysum);
    bool fin = isfinite(T0);
    for (int i = lane; i < ns; i += TEAM) {
        const double c = rho * yn[1 + i] * __ldg(M.invW + i);
        yn[1 + i] = c;
        fin &= isfinite(c);
    }
    if (lane == 0) yn[0] = T0;
    team_sync<TEAM>();
    fin = !team_any<TEAM>(!fin, red);
    Counters cnt = {0, 0, 0, 0};
    int st;
    if (!fin) {
        st = CELL_NONFINITE;
    } else {
        st = P.adaptive ? integrate_adaptive<TEAM, MT>(M, L, P, sm, cnt, lane)
                        : integrate_fixed<TEAM, MT>(M, L, P, sm, cnt, lane);
        bool bad = false;
        for (int i = lane; i < n; i += TEAM) bad |= !isfinite(yn[i]);
        if (team_any<TEAM>(bad, red) && st == CELL_OK) st = CELL_NONFINITE;
    }
    // store: T, Y_i = W_i C_i / sum W_j C_j (the input is kept for non-finite cells)
    if (st != CELL_NONFINITE) {
        double ms = 0.0;
        for (int i = lane; i < ns; i += TEAM) ms = fma(__ldg(M.W + i), yn[1 + i], ms);
        const double inv = 1.0 / team_sum<TEAM>(ms, red);
        for (int i = lane; i < ns; i += TEAM) Yio[(int64_t)i * N + cell] = __ldg(M.W + i) * yn[1 + i] * inv;
        if (lane == 0) T[cell] = yn[0];
    }
    if (lane == 0) {
        if (status) status[cell] = st;
        if (stats) {
            stats[cell] = cnt.steps;
            stats[N + cell] = cnt.rejects;
            stats[2 * N + cell] = cnt.newton;
            stats[3 * N + cell] = cnt.lu;
        }
    }
}

// ---------------------------------------------------------------------------
// launchers: teams_per_block teams of TEAM threads (TEAM > 32: one per block)

static cudaError_t prepare(const void* fn, size_t smem) {
    if (smem > 48 * 1024)
        return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

template <int TEAM, class K, class... Args>
static cudaError_t launch_team(K kernel, const Layout& L, int tpb, int64_t N, cudaStream_t st,
                               Args... args) {
    if (TEAM > 32) tpb = 1;
    const size_t smem = (size_t)tpb * L.total * sizeof(double);
    cudaError_t e = prepare((const void*)kernel, smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (N + tpb - 1) / tpb;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    kernel<<<(unsigned)blocks, TEAM * tpb, smem, st>>>(args...);
    return cudaGetLastError();
}

#define CG_DISPATCH_TEAM(team, CALL)                         \
    switch (team) {                                          \
        case 32: return CALL(32);                            \
        case 64: return CALL(64);                            \
        case 128: return CALL(128);                          \
        case 256: return CALL(256);                          \
        default: return cudaErrorInvalidValue;               \
    }

cudaError_t launch_eval_rates(const DevMech& M, const Layout& L, int tpb, int reactor, int64_t N,
                              const double* T, const double* C, double* S, cudaStream_t st) {
#define CALL(TM) launch_team<TM>(eval_rates_kernel<TM>, L, tpb, N, st, M, L, reactor, N, T, C, S)
    CG_DISPATCH_TEAM(M.team, CALL)
#undef CALL
}

cudaError_t launch_eval_jacobian(const DevMech& M, const Layout& L, int tpb, int reactor, int64_t N,
                                 const double* T, const double* C, double* J, cudaStream_t st) {
#define CALL(TM) launch_team<TM>(eval_jacobian_kernel<TM>, L, tpb, N, st, M, L, reactor, N, T, C, J)
    CG_DISPATCH_TEAM(M.team, CALL)
#undef CALL
}

cudaError_t launch_temperature(const DevMech& M, int reactor, int64_t N, const double* e,
                               const double* Y, double* T, int iters, cudaStream_t st) {
    const int wpb = 4;
    const int64_t blocks = (N + wpb - 1) / wpb;
    temperature_kernel<<<(unsigned)blocks, 32 * wpb, 0, st>>>(M, reactor, N, e, Y, T, iters);
    return cudaGetLastError();
}

cudaError_t launch_integrate(const DevMech& M, const Layout& L, const IntParams& P, int tpb,
                             int64_t N, double* T, double* Y, const double* p_or_rho,
                             int32_t* status, int32_t* stats, cudaStream_t st) {
    if (P.precision == 1) {
#define CALL(TM) \
    launch_team<TM>(integrate_kernel<TM, float>, L, tpb, N, st, M, L, P, N, T, Y, p_or_rho, status, stats)
        CG_DISPATCH_TEAM(M.team, CALL)
#undef CALL
    }
#define CALL(TM) \
    launch_team<TM>(integrate_kernel<TM, double>, L, tpb, N, st, M, L, P, N, T, Y, p_or_rho, status, stats)
    CG_DISPATCH_TEAM(M.team, CALL)
#undef CALL
}

}  // namespace cg
