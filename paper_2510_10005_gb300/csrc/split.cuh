// Operator-split chemistry for a compressible flow solver (Section 5.5):
// the flow solver holds per cell the density rho, the mass-specific internal
// energy u and the species densities rho Y_i; for its reaction sub-step it
// needs the temperature (recovered from u by Newton, Section 2.1) and the
// species source R_i = W_i (C_i^{n+1} - C_i^n) / dt of eq. openfom_fvm, with
// C integrated at constant volume over dt (Section 3, eq.
// temperature_source).
//
//   react_split_kernel   one team per cell: load, temperature recovery,
//                        integration, source
// (included only by instances.cu, which compiles it once per team size and
// Newton-matrix type)
#pragma once

#include "stepper.cuh"

namespace cg {

template <int TEAM, class MT>
__device__ void split_cell(const SplitTask& tk, const Ws& W, const IntParams& P, int64_t cell, int lane) {
    const DevMech& M = tk.M;
    const int64_t N = tk.N;
    const int ns = M.ns, n = M.n;
    double* yn = W.yn;
    const double rho = tk.rho[cell];
    const double e = tk.e[cell];
    const double irho = 1.0 / rho;
    // Y_i = rho Y_i / rho (kept in yn[1 + i] for the temperature Newton)
    bool fin = isfinite(rho) && rho > 0.0 && isfinite(e);
    for (int i = lane; i < ns; i += TEAM) {
        const double y = tk.rhoY[(int64_t)i * N + cell] * irho;
        yn[1 + i] = y;
        fin &= isfinite(y);
    }
    team_sync<TEAM>();
    fin = !team_any<TEAM>(!fin, W.red);
    // T from sum_i Y_i u_i(T) = u: Newton from the caller's guess,
    // u_i = R T (h_i/(RT) - 1) / W_i, c_v,i = R (c_p,i/R - 1) / W_i
    double T = tk.T[cell];
    for (int it = 0; it < tk.iters && fin; ++it) {
        const double invT = 1.0 / T;
        double ev = 0.0, cv = 0.0;
        for (int i = lane; i < ns; i += TEAM) {
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
            const double yw = yn[1 + i] * __ldg(M.invW + i);
            ev = fma(yw, h - 1.0, ev);
            cv = fma(yw, cp - 1.0, cv);
        }
        ev = team_sum<TEAM>(ev, W.red) * kR * T;
        cv = team_sum<TEAM>(cv, W.red) * kR;
        T += (e - ev) / cv;
    }
    fin = fin && isfinite(T) && T > 0.0;
    // C_i = rho Y_i / W_i
    for (int i = lane; i < ns; i += TEAM) yn[1 + i] = tk.rhoY[(int64_t)i * N + cell] * __ldg(M.invW + i);
    if (lane == 0) yn[0] = T;
    team_sync<TEAM>();
    Counters cnt = {0, 0, 0, 0};
    int st = CELL_NONFINITE;
    if (fin) {
        st = P.adaptive ? integrate_adaptive<TEAM, MT>(M, W, P, cnt, nullptr, 0, lane)
                        : integrate_fixed<TEAM, MT>(M, W, P, cnt, nullptr, 0, lane);
        bool bad = false;
        for (int i = lane; i < n; i += TEAM) bad |= !isfinite(yn[i]);
        if (team_any<TEAM>(bad, W.red) && st == CELL_OK) st = CELL_NONFINITE;
    }
    // R_i = (W_i C_i^{n+1} - rho Y_i^n) / dt; zero for cells that were not integrated
    const double idt = 1.0 / P.dt;
    for (int i = lane; i < ns; i += TEAM) {
        const int64_t k = (int64_t)i * N + cell;
        tk.R[k] = st == CELL_NONFINITE ? 0.0 : (__ldg(M.W + i) * yn[1 + i] - tk.rhoY[k]) * idt;
    }
    if (lane == 0) {
        if (st != CELL_NONFINITE) tk.T[cell] = yn[0];
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
__global__ void __maxnreg__((KernelRegs<TEAM, MT>::value)) react_split_kernel(SplitTask tk, IntParams P, int sstride, double* gscratch, int64_t gstride,
                                   unsigned long long* counter) {
    extern __shared__ double smem_all[];
    const TeamPos<TEAM> tp;
    const Ws W = make_ws(tk.L, smem_all + (size_t)tp.tib * sstride,
                         gscratch ? gscratch + tp.id * gstride : nullptr);
    for (int64_t c = first_cell<TEAM>(counter, tp.id, tp.lane); c < tk.N;
         c = next_cell<TEAM>(counter, c, tp.count, tp.lane))
        split_cell<TEAM, MT>(tk, W, P, c, tp.lane);
}

template <int TEAM, class MT>
cudaError_t launch_split_team(const SplitTask& t, const IntParams& P, int tpb, cudaStream_t st) {
    if (TEAM > 32) tpb = 1;
    const int sstride = t.L.stotal;
    const int64_t gstride = round_up(t.L.gtotal, 32);
    while (tpb > 1 && (size_t)tpb * sstride * sizeof(double) > 227 * 1024) --tpb;
    const void* fn = (const void*)react_split_kernel<TEAM, MT>;
    const size_t smem = (size_t)tpb * sstride * sizeof(double);
    cudaError_t e = set_smem(fn, smem);
    if (e != cudaSuccess) return e;
    int64_t blocks = (t.N + tpb - 1) / tpb, res = 0;
    if ((e = resident_blocks(fn, TEAM * tpb, smem, &res)) != cudaSuccess) return e;
    blocks = blocks < res ? blocks : res;
    LaunchMem mem;
    if ((e = get_mem(blocks * tpb, gstride, true, st, mem)) != cudaSuccess) return e;
    react_split_kernel<TEAM, MT><<<(unsigned)blocks, TEAM * tpb, smem, st>>>(t, P, sstride, mem.gscratch, gstride,
                                                                             mem.counter);
    e = cudaGetLastError();
    cudaError_t e2 = put_mem(mem, st);
    return e != cudaSuccess ? e : e2;
}

}  // namespace cg
