// Integration kernels of chemgb, included only by instances.cu, which
// compiles them once per team size and Newton-matrix type: one team of TEAM
// threads per cell (TEAM = 32: one warp, several teams per block; TEAM =
// 64..256: one team per block). Every kernel walks the cells in a loop: a
// team takes cell `team id` and then either the next cell of a fixed stride
// or, in the persistent form, the next cell of an atomic work counter
// shared by the whole launch (work stealing: a team that finishes a cheap
// cell takes the next one at once). Arrays of a cell that do not fit in
// shared memory live in the team's slot of a global scratch buffer.
//
//   eval_rates_kernel      S(y) for N cells (Section 2.2, Section 3, App. B)
//   eval_jacobian_kernel   dS/dy for N cells (Section 3.2)
//   integrate_kernel       backward Euler / SDIRK / Rosenbrock-2 / YASS over
//                          dt (Section 3.2, App. A), for up to kMaxTasks
//                          mechanisms in one launch
#pragma once

#include "stepper.cuh"

namespace cg {

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
            // after the last step, or in the last slot when the steps did not
            // fit (the adjoint then recomputes them from record 0)
            const bool fits = cnt.steps < tk.ckpt_cap;
            if (st == CELL_OK) save_step<TEAM>(ck, tk.ckpt_cap, fits ? cnt.steps : tk.ckpt_cap - 1, yn, rho, n, lane);
            if (lane == 0) tk.ckpt_n[cell] = st != CELL_OK ? -1 : (fits ? cnt.steps : -(cnt.steps + 2));
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
__global__ void __maxnreg__((KernelRegs<TEAM, MT>::value)) integrate_kernel(Tasks tasks, IntParams P, int sstride,
                                                                              double* gscratch, int64_t gstride,
                                                                              unsigned long long* counter) {
    extern __shared__ double smem_all[];
    const TeamPos<TEAM> tp;
    double* sbase = smem_all + (size_t)tp.tib * sstride;
    double* gbase = gscratch ? gscratch + tp.id * gstride : nullptr;
    for (int64_t g = first_cell<TEAM>(counter, tp.id, tp.lane); g < tasks.total;
         g = next_cell<TEAM>(counter, g, tp.count, tp.lane)) {
        int k = 0;   // the whole-team task holding g (tasks of no cells are skipped)
        while (tasks.t[k].split || g >= tasks.t[k].first + tasks.t[k].N) ++k;
        const Task& tk = tasks.t[k];
#ifdef CG_DEBUG
        debug_poison<TEAM>(tk.L, sbase, gbase, tp.lane);
#endif
        integrate_cell<TEAM, MT>(tk, make_ws(tk.L, sbase, gbase), P, g - tk.first, tp.lane);
#ifdef CG_DEBUG
        debug_check<TEAM>(tk.L, sbase, gbase, tk.M.dbg, g - tk.first, tp.lane);
#endif
    }
    if constexpr (TEAM > 32) {
        // Split tasks (one-warp mechanisms in this wider launch), once the
        // whole-team cells are taken: every warp of the team claims cells on
        // its own from the second counter, in its own part of the team's
        // shared slice and scratch slot, with no barrier across the team.
        if (tasks.total_split > 0 && counter) {
            const int w = tp.lane >> 5, l = tp.lane & 31;
            for (int64_t c = next_cell<32>(counter + 1, 0, 0, l); c < tasks.total_split;
                 c = next_cell<32>(counter + 1, 0, 0, l)) {
                int k = 0;
                while (!tasks.t[k].split || c >= tasks.t[k].first + tasks.t[k].N) ++k;
                const Task& tk = tasks.t[k];
                double* ws = sbase + (size_t)w * tk.L.stotal;
                double* wg = gbase ? gbase + (int64_t)w * round_up(tk.L.gtotal, 32) : nullptr;
                integrate_cell<32, MT>(tk, make_ws(tk.L, ws, wg), P, c - tk.first, l);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// launchers of one team size (instantiated in instances.cu)

template <int TEAM>
cudaError_t launch_eval_team(bool jacobian, const DevMech& M, const Layout& L, int tpb, int reactor, int64_t N,
                             const double* T, const double* C, double* out, cudaStream_t st) {
    if (TEAM > 32) tpb = 1;
    const void* fn = jacobian ? (const void*)eval_jacobian_kernel<TEAM> : (const void*)eval_rates_kernel<TEAM>;
    const size_t smem = (size_t)tpb * L.stotal * sizeof(double);
    cudaError_t e = set_smem(fn, smem);
    if (e != cudaSuccess) return e;
    int64_t blocks = (N + tpb - 1) / tpb;
    const int64_t gstride = round_up(L.gtotal, 32);
    if (gstride) {
        int64_t res = 0;
        if ((e = resident_blocks(fn, TEAM * tpb, smem, &res)) != cudaSuccess) return e;
        blocks = blocks < res ? blocks : res;
    }
    if (blocks > 0x7fffffffLL) blocks = 0x7fffffffLL;   // the cell loop covers the rest
    LaunchMem mem;
    if ((e = get_mem(blocks * tpb, gstride, false, st, mem)) != cudaSuccess) return e;
    if (jacobian)
        eval_jacobian_kernel<TEAM><<<(unsigned)blocks, TEAM * tpb, smem, st>>>(M, L, reactor, N, T, C, out,
                                                                               mem.gscratch, gstride);
    else
        eval_rates_kernel<TEAM><<<(unsigned)blocks, TEAM * tpb, smem, st>>>(M, L, reactor, N, T, C, out,
                                                                            mem.gscratch, gstride);
    e = cudaGetLastError();
    cudaError_t e2 = put_mem(mem, st);
    return e != cudaSuccess ? e : e2;
}

template <int TEAM, class MT>
cudaError_t launch_integrate_team(const Tasks& tasks, const IntParams& P, int tpb, bool persistent,
                                  cudaStream_t st) {
    tpb = integrate_tpb(tasks, TEAM, tpb);
    const int sstride = integrate_sstride(tasks, TEAM);
    const int64_t gstride = integrate_slot_doubles(tasks, TEAM);   // 256-byte aligned slots
    const void* fn = (const void*)integrate_kernel<TEAM, MT>;
    const size_t smem = (size_t)tpb * sstride * sizeof(double);
    cudaError_t e = set_smem(fn, smem);
    if (e != cudaSuccess) return e;
    const int64_t units = tasks.total > tasks.total_split / (TEAM / 32) ? tasks.total
                                                                        : tasks.total_split / (TEAM / 32) + 1;
    int64_t blocks = (units + tpb - 1) / tpb;
    int64_t res = 0;
    if ((e = resident_blocks(fn, TEAM * tpb, smem, &res)) != cudaSuccess) return e;
    // the work queue (resident teams take cells from a counter) whenever it
    // is asked for, needed (scratch slots, split tasks), or the cells would
    // take more than one wave of blocks: cells of very different cost then
    // balance across the teams (9 species, 4096 cells: 13.3 instead of
    // 15.3 ms, against 9.7 ms for the slowest cell alone)
    const bool queue = persistent || gstride > 0 || tasks.total_split > 0 || blocks > res;
    if (queue) blocks = blocks < res ? blocks : res;
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
cudaError_t launch_integrate_on_team(const Tasks& tasks, const IntParams& P, int tpb, double* scratch,
                                     int64_t scratch_doubles, unsigned long long* counter, cudaStream_t st) {
    tpb = integrate_tpb(tasks, TEAM, tpb);
    const int sstride = integrate_sstride(tasks, TEAM);
    const int64_t gstride = integrate_slot_doubles(tasks, TEAM);
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

}  // namespace cg
