// Kernels of chemgb: one team of TEAM threads per cell (TEAM = 32: one warp,
// several teams per block; TEAM = 64..256: one team per block). Every
// kernel walks the cells in a loop: a team takes cell `team id` and then
// either the next cell of a fixed stride or, in the persistent form, the
// next cell of an atomic work counter shared by the whole launch (work
// stealing: a team that finishes a cheap cell takes the next one at once).
// Arrays of a cell that do not fit in shared memory live in the team's slot
// of a global scratch buffer.
//
//   eval_rates_kernel      S(y) for N cells (Section 2.2, Section 3, App. B)
//   eval_jacobian_kernel   dS/dy for N cells (Section 3.2)
//   temperature_kernel     T from (e, Y) by Newton (Section 2.1)
//   integrate_kernel       backward Euler / SDIRK over dt (Section 3.2, App. A),
//                          for up to kMaxTasks mechanisms in one launch
//   exp_check_kernel, rcp_check_kernel   test hooks: exp_tab, rcp_nr
#include "stepper.cuh"

namespace cg {

// ---------------------------------------------------------------------------

template <int TEAM>
__global__ void eval_rates_kernel(DevMech M, Layout L, int reactor, int64_t N,
                                  const double* __restrict__ T, const double* __restrict__ C,
                                  double* __restrict__ S, double* gscratch, int64_t gstride) {
    extern __shared__ double smem_all[];
    const TeamPos<TEAM> tp;
    const Ws W = make_ws(L, smem_all + (size_t)tp.tib * L.stotal,
                         gscratch ? gscratch + tp.id * gstride : nullptr);
    const int lane = tp.lane;
    for (int64_t cell = tp.id; cell < N; cell += tp.count) {
        double* y = W.Y;
        if (lane == 0) y[0] = T[cell];
        for (int i = lane; i < M.ns; i += TEAM) y[1 + i] = C[(int64_t)i * N + cell];
        team_sync<TEAM>();
        const double Mc = rates<TEAM>(M, W, y, false, lane);
        assemble_source<TEAM>(M, W, y, reactor, Mc, lane);
        for (int i = lane; i < M.n; i += TEAM) S[(int64_t)i * N + cell] = W.S[i];
        team_sync<TEAM>();
    }
}

template <int TEAM>
__global__ void eval_jacobian_kernel(DevMech M, Layout L, int reactor, int64_t N,
                                     const double* __restrict__ T, const double* __restrict__ C,
                                     double* __restrict__ J, double* gscratch, int64_t gstride) {
    extern __shared__ double smem_all[];
    const TeamPos<TEAM> tp;
    const Ws W = make_ws(L, smem_all + (size_t)tp.tib * L.stotal,
                         gscratch ? gscratch + tp.id * gstride : nullptr);
    const int lane = tp.lane;
    for (int64_t cell = tp.id; cell < N; cell += tp.count) {
        double* y = W.Y;
        if (lane == 0) y[0] = T[cell];
        for (int i = lane; i < M.ns; i += TEAM) y[1 + i] = C[(int64_t)i * N + cell];
        team_sync<TEAM>();
        const double Mc = rates<TEAM>(M, W, y, true, lane);
        const SrcInfo si = assemble_source<TEAM>(M, W, y, reactor, Mc, lane);
        assemble_jacobian<TEAM, double>(M, W, y, reactor, si, 0.0, J + cell * (int64_t)M.n * M.n, lane);
    }
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

// ---------------------------------------------------------------------------
// integration

// Load, integrate and store one cell of one task.
template <int TEAM, class MT>
__device__ void integrate_cell(const Task& tk, const Ws& W, const IntParams& P, int64_t cell,
                               int lane) {
    const DevMech& M = tk.M;
    const int64_t N = tk.N;
    const int ns = M.ns, n = M.n;
    double* yn = W.yn;
    // load and unpack: C_i = rho Y_i / W_i
    const double T0 = tk.T[cell];
    const double pr = tk.p[cell];
    double ysum = 0.0;
    for (int i = lane; i < ns; i += TEAM) {
        const double Yi = tk.Y[(int64_t)i * N + cell];
        yn[1 + i] = Yi;
        ysum = fma(Yi, __ldg(M.invW + i), ysum);
    }
    ysum = team_sum<TEAM>(ysum, W.red);
    const double rho = P.reactor == R_CONV ? pr : pr / (kR * T0 * ysum);
    bool fin = isfinite(T0);
    for (int i = lane; i < ns; i += TEAM) {
        const double c = rho * yn[1 + i] * __ldg(M.invW + i);
        yn[1 + i] = c;
        fin &= isfinite(c);
    }
    if (lane == 0) yn[0] = T0;
    team_sync<TEAM>();
    fin = !team_any<TEAM>(!fin, W.red);
    Counters cnt = {0, 0, 0, 0};
    int st;
    if (!fin) {
        st = CELL_NONFINITE;
        if (tk.ckpt && lane == 0) tk.ckpt_n[cell] = -1;
    } else {
        double* ck = tk.ckpt ? tk.ckpt + cell * (int64_t)tk.ckpt_cap * (n + 1) : nullptr;
        st = P.adaptive ? integrate_adaptive<TEAM, MT>(M, W, P, cnt, ck, tk.ckpt_cap, lane)
                        : integrate_fixed<TEAM, MT>(M, W, P, cnt, ck, tk.ckpt_cap, lane);
        if (ck) {   // the final state closes the record
            save_step<TEAM>(ck, tk.ckpt_cap, cnt.steps, yn, rho, n, lane);
            if (lane == 0) tk.ckpt_n[cell] = (st == CELL_OK && cnt.steps < tk.ckpt_cap) ? cnt.steps : -1;
        }
        bool bad = false;
        for (int i = lane; i < n; i += TEAM) bad |= !isfinite(yn[i]);
        if (team_any<TEAM>(bad, W.red) && st == CELL_OK) st = CELL_NONFINITE;
    }
    // store: T, Y_i = W_i C_i / sum W_j C_j (the input is kept for non-finite cells)
    if (st != CELL_NONFINITE) {
        double ms = 0.0;
        for (int i = lane; i < ns; i += TEAM) ms = fma(__ldg(M.W + i), yn[1 + i], ms);
        const double inv = 1.0 / team_sum<TEAM>(ms, W.red);
        for (int i = lane; i < ns; i += TEAM) tk.Y[(int64_t)i * N + cell] = __ldg(M.W + i) * yn[1 + i] * inv;
        if (lane == 0) tk.T[cell] = yn[0];
    }
    if (lane == 0) {
        if (tk.status) tk.status[cell] = st;
        if (tk.stats) {
            tk.stats[cell] = cnt.steps;
            tk.stats[N + cell] = cnt.rejects;
            tk.stats[2 * N + cell] = cnt.newton;
            tk.stats[3 * N + cell] = cnt.lu;
        }
    }
    team_sync<TEAM>();
}

template <int TEAM, class MT>
__global__ void integrate_kernel(Tasks tasks, IntParams P, int sstride, double* gscratch,
                                 int64_t gstride, unsigned long long* counter) {
    extern __shared__ double smem_all[];
    const TeamPos<TEAM> tp;
    double* sbase = smem_all + (size_t)tp.tib * sstride;
    double* gbase = gscratch ? gscratch + tp.id * gstride : nullptr;
    for (int64_t g = first_cell<TEAM>(counter, tp.id, tp.lane); g < tasks.total;
         g = next_cell<TEAM>(counter, g, tp.count, tp.lane)) {
        int k = 0;
        while (k + 1 < tasks.count && g >= tasks.t[k + 1].first) ++k;
        const Task& tk = tasks.t[k];
        const Ws W = make_ws(tk.L, sbase, gbase);
        integrate_cell<TEAM, MT>(tk, W, P, g - tk.first, tp.lane);
    }
}

// ---------------------------------------------------------------------------
// launchers

template <int TEAM, class K>
static cudaError_t launch_eval(K kernel, const DevMech& M, const Layout& L, int tpb, int reactor,
                               int64_t N, const double* T, const double* C, double* out,
                               cudaStream_t st) {
    if (TEAM > 32) tpb = 1;
    const size_t smem = (size_t)tpb * L.stotal * sizeof(double);
    cudaError_t e = set_smem((const void*)kernel, smem);
    if (e != cudaSuccess) return e;
    int64_t blocks = (N + tpb - 1) / tpb;
    const int64_t gstride = round_up(L.gtotal, 32);
    if (gstride) {
        int64_t res = 0;
        if ((e = resident_blocks((const void*)kernel, TEAM * tpb, smem, &res)) != cudaSuccess) return e;
        blocks = blocks < res ? blocks : res;
    }
    if (blocks > 0x7fffffffLL) blocks = 0x7fffffffLL;   // the cell loop covers the rest
    LaunchMem mem;
    if ((e = get_mem(blocks * tpb, gstride, false, st, mem)) != cudaSuccess) return e;
    kernel<<<(unsigned)blocks, TEAM * tpb, smem, st>>>(M, L, reactor, N, T, C, out, mem.gscratch, gstride);
    e = cudaGetLastError();
    cudaError_t e2 = put_mem(mem, st);
    return e != cudaSuccess ? e : e2;
}

cudaError_t launch_eval_rates(const DevMech& M, const Layout& L, int tpb, int reactor, int64_t N,
                              const double* T, const double* C, double* S, cudaStream_t st) {
#define CALL(TM) launch_eval<TM>(eval_rates_kernel<TM>, M, L, tpb, reactor, N, T, C, S, st)
    CG_DISPATCH_TEAM(M.team, CALL)
#undef CALL
}

cudaError_t launch_eval_jacobian(const DevMech& M, const Layout& L, int tpb, int reactor, int64_t N,
                                 const double* T, const double* C, double* J, cudaStream_t st) {
#define CALL(TM) launch_eval<TM>(eval_jacobian_kernel<TM>, M, L, tpb, reactor, N, T, C, J, st)
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

// Global scratch of one team's slot (doubles, a multiple of 32 so that slots
// stay 256-byte aligned): the largest of the tasks.
int64_t integrate_slot_doubles(const Tasks& tasks) {
    int64_t g = 0;
    for (int k = 0; k < tasks.count; ++k) g = g > tasks.t[k].L.gtotal ? g : tasks.t[k].L.gtotal;
    return round_up(g, 32);
}

// Shared-memory stride (doubles) of one team's slice: the largest of the tasks.
static int integrate_sstride(const Tasks& tasks) {
    int sstride = 0;
    for (int k = 0; k < tasks.count; ++k) sstride = sstride > tasks.t[k].L.stotal ? sstride : tasks.t[k].L.stotal;
    return sstride;
}

int integrate_tpb(const Tasks& tasks, int team, int tpb) {
    if (team > 32) return 1;
    const int sstride = integrate_sstride(tasks);
    while (tpb > 1 && (size_t)tpb * sstride * sizeof(double) > 227 * 1024) --tpb;   // larger layouts (GMRES)
    return tpb;
}

template <int TEAM, class MT>
static cudaError_t launch_integrate_t(const Tasks& tasks, const IntParams& P, int tpb, bool persistent,
                                      cudaStream_t st) {
    tpb = integrate_tpb(tasks, TEAM, tpb);
    const int sstride = integrate_sstride(tasks);
    const int64_t gstride = integrate_slot_doubles(tasks);   // 256-byte aligned slots
    const void* fn = (const void*)integrate_kernel<TEAM, MT>;
    const size_t smem = (size_t)tpb * sstride * sizeof(double);
    cudaError_t e = set_smem(fn, smem);
    if (e != cudaSuccess) return e;
    int64_t blocks = (tasks.total + tpb - 1) / tpb;
    const bool queue = persistent || gstride > 0;
    if (queue) {
        int64_t res = 0;
        if ((e = resident_blocks(fn, TEAM * tpb, smem, &res)) != cudaSuccess) return e;
        blocks = blocks < res ? blocks : res;
    }
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    LaunchMem mem;
    if ((e = get_mem(blocks * tpb, gstride, queue, st, mem)) != cudaSuccess) return e;
    integrate_kernel<TEAM, MT><<<(unsigned)blocks, TEAM * tpb, smem, st>>>(tasks, P, sstride, mem.gscratch,
                                                                           gstride, mem.counter);
    e = cudaGetLastError();
    cudaError_t e2 = put_mem(mem, st);
    return e != cudaSuccess ? e : e2;
}

// Persistent launch on caller-provided memory: `scratch` holds
// scratch_doubles doubles for the teams' slots, `counter` must be zero when
// the kernel starts (the caller clears it on the stream). The grid is
// limited so that every team's slot fits. Allocates nothing.
template <int TEAM, class MT>
static cudaError_t launch_integrate_on_t(const Tasks& tasks, const IntParams& P, int tpb, double* scratch,
                                         int64_t scratch_doubles, unsigned long long* counter,
                                         cudaStream_t st) {
    tpb = integrate_tpb(tasks, TEAM, tpb);
    const int sstride = integrate_sstride(tasks);
    const int64_t gstride = integrate_slot_doubles(tasks);
    const void* fn = (const void*)integrate_kernel<TEAM, MT>;
    const size_t smem = (size_t)tpb * sstride * sizeof(double);
    cudaError_t e = set_smem(fn, smem);
    if (e != cudaSuccess) return e;
    int64_t blocks = (tasks.total + tpb - 1) / tpb, res = 0;
    if ((e = resident_blocks(fn, TEAM * tpb, smem, &res)) != cudaSuccess) return e;
    blocks = blocks < res ? blocks : res;
    if (gstride) {
        const int64_t fit = scratch_doubles / (gstride * tpb);   // blocks whose slots fit
        if (fit < 1) return cudaErrorMemoryAllocation;
        blocks = blocks < fit ? blocks : fit;
    }
    integrate_kernel<TEAM, MT><<<(unsigned)blocks, TEAM * tpb, smem, st>>>(tasks, P, sstride,
                                                                           gstride ? scratch : nullptr,
                                                                           gstride, counter);
    return cudaGetLastError();
}

cudaError_t launch_integrate_on(const Tasks& tasks, const IntParams& P, int team, int tpb, double* scratch,
                                int64_t scratch_doubles, unsigned long long* counter, cudaStream_t st) {
    if (P.precision == 1) {
#define CALL(TM) launch_integrate_on_t<TM, float>(tasks, P, tpb, scratch, scratch_doubles, counter, st)
        CG_DISPATCH_TEAM(team, CALL)
#undef CALL
    }
#define CALL(TM) launch_integrate_on_t<TM, double>(tasks, P, tpb, scratch, scratch_doubles, counter, st)
    CG_DISPATCH_TEAM(team, CALL)
#undef CALL
}

cudaError_t launch_integrate(const Tasks& tasks, const IntParams& P, int team, int tpb, bool persistent,
                             cudaStream_t st) {
    if (P.precision == 1) {
#define CALL(TM) launch_integrate_t<TM, float>(tasks, P, tpb, persistent, st)
        CG_DISPATCH_TEAM(team, CALL)
#undef CALL
    }
#define CALL(TM) launch_integrate_t<TM, double>(tasks, P, tpb, persistent, st)
    CG_DISPATCH_TEAM(team, CALL)
#undef CALL
}

}  // namespace cg
