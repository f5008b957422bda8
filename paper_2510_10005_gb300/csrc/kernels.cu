// Kernels of chemgb outside the per-team instantiations, and the host-side
// dispatch of every launch to the instantiation of its team size and
// Newton-matrix type (instances.cu compiles the integration, split and
// adjoint kernels once per combination, so that they build in parallel).
//
//   temperature_kernel     T from (e, Y) by Newton (Section 2.1)
//   sum_rows_kernel        fixed-order sum of the adjoint's per-cell gradients
//   exp_check_kernel, rcp_check_kernel   test hooks: exp_tab, rcp_nr
#include "stepper.cuh"

namespace cg {

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
            double cp, h;
            if (M.th_np == 4) {
#define TH(k) __ldg(th + (k) * ns)
                cp = TH(TH_A1) + T * (TH(TH_A2) + T * (TH(TH_A3) + T * (TH(TH_A4) + T * TH(TH_A5))));
                h = TH(TH_A1) + T * (TH(TH_H2) + T * (TH(TH_H3) + T * (TH(TH_H4) + T * TH(TH_H5))))
                    + TH(TH_A6) * invT;
#undef TH
            } else {
                thermo_cp_h_deg(th, ns, M.th_np, T, invT, cp, h);
            }
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

// exp_tab next to the library exp on the same arguments (test hook).
__global__ void exp_check_kernel(int64_t n, const double* __restrict__ tab, const double* __restrict__ x,
                                 double* __restrict__ y_tab, double* __restrict__ y_lib) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        y_tab[i] = exp_tab(x[i], tab);
        y_lib[i] = exp(x[i]);
    }
}

// rcp_nr on the same arguments (test hook).
__global__ void rcp_check_kernel(int64_t n, const double* __restrict__ x, double* __restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = rcp_nr(x[i]);
}

// out[r] = sum_c g[r * N + c]: one block per row, a fixed order of
// additions for a given N (strided partial sums, then a fixed tree).
__global__ void sum_rows_kernel(int64_t N, const double* __restrict__ g, double* __restrict__ out) {
    const double* row = g + (int64_t)blockIdx.x * N;
    double s = 0.0;
    for (int64_t c = threadIdx.x; c < N; c += blockDim.x) s += row[c];
    __shared__ double red[32];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        out[blockIdx.x] = t;
    }
}

// ---------------------------------------------------------------------------
// launch planning

int64_t integrate_slot_doubles(const Tasks& tasks, int team) {
    int64_t g = 0;
    for (int k = 0; k < tasks.count; ++k) {
        const Task& t = tasks.t[k];
        const int64_t need = t.split ? (team / 32) * round_up(t.L.gtotal, 32) : round_up(t.L.gtotal, 32);
        g = g > need ? g : need;
    }
    return g;
}

int integrate_sstride(const Tasks& tasks, int team) {
    int sstride = 0;
    for (int k = 0; k < tasks.count; ++k) {
        const Task& t = tasks.t[k];
        const int need = t.split ? (team / 32) * t.L.stotal : t.L.stotal;
        sstride = sstride > need ? sstride : need;
    }
    return sstride;
}

int integrate_tpb(const Tasks& tasks, int team, int tpb) {
    if (team > 32) return 1;
    const int sstride = integrate_sstride(tasks, team);
    while (tpb > 1 && (size_t)tpb * sstride * sizeof(double) > 227 * 1024) --tpb;   // larger layouts (GMRES)
    return tpb;
}

// ---------------------------------------------------------------------------
// dispatch

cudaError_t launch_eval_rates(const DevMech& M, const Layout& L, int tpb, int reactor, int64_t N,
                              const double* T, const double* C, double* S, cudaStream_t st) {
#define CALL(TM) launch_eval_team<TM>(false, M, L, tpb, reactor, N, T, C, S, st)
    CG_DISPATCH_TEAM(M.team, CALL)
#undef CALL
}

cudaError_t launch_eval_jacobian(const DevMech& M, const Layout& L, int tpb, int reactor, int64_t N,
                                 const double* T, const double* C, double* J, cudaStream_t st) {
#define CALL(TM) launch_eval_team<TM>(true, M, L, tpb, reactor, N, T, C, J, st)
    CG_DISPATCH_TEAM(M.team, CALL)
#undef CALL
}

cudaError_t launch_exp_check(const DevMech& M, int64_t n, const double* x, double* y_tab, double* y_lib,
                             cudaStream_t st) {
    const int64_t blocks = n > 0 ? (n + 255) / 256 : 0;
    if (blocks == 0) return cudaSuccess;
    exp_check_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(n, M.exp2j, x, y_tab, y_lib);
    return cudaGetLastError();
}

cudaError_t launch_rcp_check(int64_t n, const double* x, double* y, cudaStream_t st) {
    const int64_t blocks = n > 0 ? (n + 255) / 256 : 0;
    if (blocks == 0) return cudaSuccess;
    rcp_check_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(n, x, y);
    return cudaGetLastError();
}

cudaError_t launch_temperature(const DevMech& M, int reactor, int64_t N, const double* e,
                               const double* Y, double* T, int iters, cudaStream_t st) {
    const int wpb = 4;
    const int64_t blocks = (N + wpb - 1) / wpb;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    temperature_kernel<<<(unsigned)blocks, 32 * wpb, 0, st>>>(M, reactor, N, e, Y, T, iters);
    return cudaGetLastError();
}

cudaError_t launch_integrate(const Tasks& tasks, const IntParams& P, int team, int tpb, bool persistent,
                             cudaStream_t st) {
    if (P.precision == 1) {
#define CALL(TM) launch_integrate_team<TM, float>(tasks, P, tpb, persistent, st)
        CG_DISPATCH_TEAM(team, CALL)
#undef CALL
    }
#define CALL(TM) launch_integrate_team<TM, double>(tasks, P, tpb, persistent, st)
    CG_DISPATCH_TEAM(team, CALL)
#undef CALL
}

cudaError_t launch_integrate_on(const Tasks& tasks, const IntParams& P, int team, int tpb, double* scratch,
                                int64_t scratch_doubles, unsigned long long* counter, cudaStream_t st) {
    if (P.precision == 1) {
#define CALL(TM) launch_integrate_on_team<TM, float>(tasks, P, tpb, scratch, scratch_doubles, counter, st)
        CG_DISPATCH_TEAM(team, CALL)
#undef CALL
    }
#define CALL(TM) launch_integrate_on_team<TM, double>(tasks, P, tpb, scratch, scratch_doubles, counter, st)
    CG_DISPATCH_TEAM(team, CALL)
#undef CALL
}

cudaError_t launch_react_split(const SplitTask& t, const IntParams& P, int team, int tpb, cudaStream_t st) {
    if (P.precision == 1) {
#define CALL(TM) launch_split_team<TM, float>(t, P, tpb, st)
        CG_DISPATCH_TEAM(team, CALL)
#undef CALL
    }
#define CALL(TM) launch_split_team<TM, double>(t, P, tpb, st)
    CG_DISPATCH_TEAM(team, CALL)
#undef CALL
}

static cudaError_t launch_adjoint_sweep(const AdjTask& t, const IntParams& P, int team, int tpb,
                                        cudaStream_t st) {
    if (P.precision == 1) {
#define CALL(TM) launch_adjoint_team<TM, float>(t, P, tpb, st)
        CG_DISPATCH_TEAM(team, CALL)
#undef CALL
    }
#define CALL(TM) launch_adjoint_team<TM, double>(t, P, tpb, st)
    CG_DISPATCH_TEAM(team, CALL)
#undef CALL
}

cudaError_t launch_adjoint(const AdjTask& t, const IntParams& P, int team, int tpb, double* dtheta,
                           cudaStream_t st) {
    cudaError_t e = launch_adjoint_sweep(t, P, team, tpb, st);
    if (e != cudaSuccess || !dtheta || t.M.nr == 0) return e;
    sum_rows_kernel<<<3 * t.M.nr, 256, 0, st>>>(t.N, t.grad_cells, dtheta);
    return cudaGetLastError();
}

}  // namespace cg
