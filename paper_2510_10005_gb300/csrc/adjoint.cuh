// Discrete adjoint of the implicit integration: gradients of a loss L of
// the final state (T, Y) of every cell with respect to the initial state and
// to (ln A, b, Ea) of every reaction. The paper builds ChemGen for use inside
// a differentiable code base (Section 1); this is the reverse-mode
// derivative of the integrators of Section 3.2 and Appendix A taken on the
// converged stage equations, with the accepted steps (y_n, h_n) frozen to
// those of the forward integration and Newton not differentiated.
//
// For a step of s stages with G_p = I - h a_pp J(Y_p) and lam = dL/dy_{n+1}:
//   G_p^T nu_p = h b_p lam + sum_{q>p} h a_qp J_q^T nu_q     (p = s-1 .. 0)
//   dL/dy_n    = lam + sum_p J_p^T nu_p
//   dL/dtheta += sum_p nu_p^T dS/dtheta (Y_p)
// and J_p^T nu_p = (nu_p - rhs_p) / (h a_pp) needs no second product with J.
//
//   adjoint_kernel   one team per cell: stages recomputed from the cell's
//                    checkpoints, transposed solves on the FP64 LU of G_p,
//                    per-cell gradients
//   sum_rows_kernel  fixed-order sum of the per-cell parameter gradients
//                    (kernels.cu)
// (included only by instances.cu, which compiles it once per team size and
// Newton-matrix type)
#pragma once

#include "stepper.cuh"

namespace cg {

// Backward sweep over one step from W.yn with size h. On entry W.lam holds
// dL/dy_{n+1}, on exit dL/dy_n; W.grad accumulates the parameter gradient.
// The stages W.Gam are those of the forward step (rk_step just recomputed
// them). Returns false when a Newton matrix is singular.
template <int TEAM>
__device__ bool adjoint_step(const DevMech& M, const Ws& W, const IntParams& P, double h, int lane) {
    const int n = M.n, ns = M.ns, nr = M.nr, s = P.s;
    double* lam = W.lam;
    double* lamn = W.lamn;
    double* nu = W.nu;
    double* rhs = W.rhs;
    double* acc = W.acc;
    double* at = W.f;   // effective adjoint weight of each species' production rate
    for (int i = lane; i < s * n; i += TEAM) acc[i] = 0.0;
    for (int i = lane; i < n; i += TEAM) lamn[i] = lam[i];
    team_sync<TEAM>();
    const double sub = P.reactor == R_CONV ? 1.0 : 0.0;
    for (int p = s - 1; p >= 0; --p) {
        const double gh = h * P.A[p][p];
        // converged stage state Y_p = y_n + h sum_{j <= p} a_pj Gamma_j
        for (int i = lane; i < n; i += TEAM) {
            double v = W.yn[i];
            for (int j = 0; j <= p; ++j) v = fma(h * P.A[p][j], W.Gam[j * n + i], v);
            W.Y[i] = v;
        }
        team_sync<TEAM>();
        const double Mc = rates<TEAM>(M, W, W.Y, true, lane, W.xf);
        const SrcInfo si = assemble_source<TEAM>(M, W, W.Y, P.reactor, Mc, lane);
        assemble_jacobian<TEAM, double>(M, W, W.Y, P.reactor, si, gh, nullptr, lane);
        for (int i = lane; i < n; i += TEAM) {
            const double v = fma(h * P.b[p], lam[i], acc[p * n + i]);
            nu[i] = v;
            rhs[i] = v;
        }
        team_sync<TEAM>();
        if (!lu_factor_nb<TEAM, double>(W.G, n, W.ld, M.lu_nb, W.piv, W.rinv, W.red, lane)) return false;
        lu_solve_t<TEAM, double>(W.G, n, W.ld, W.piv, W.rinv, nu, lane);
        const double igh = 1.0 / gh;
        for (int i = lane; i < n; i += TEAM) {
            const double w = (nu[i] - rhs[i]) * igh;   // (J_p^T nu_p)_i
            lamn[i] += w;
            for (int q = 0; q < p; ++q) acc[q * n + i] = fma(h * P.A[p][q], w, acc[q * n + i]);
        }
        // nu^T dS/domega_m: omega_T = -T sum_i e_i omega_i / D (e = u/RT or
        // h/RT, D = sum C c, molar), and at constant pressure the dilution
        // -C_k (omega_T / T + sum omega / sum C) of every species row
        const double T = W.Y[0];
        const double* eRT = W.SP;
        double cnu = 0.0;
        if (P.reactor == R_CONP) {
            for (int k = lane; k < ns; k += TEAM) cnu = fma(nu[1 + k], W.Y[1 + k], cnu);
            cnu = team_sum<TEAM>(cnu, W.red);
        }
        const double invD = 1.0 / si.Dt, invM = 1.0 / si.Mc, invT = 1.0 / T;
        for (int m = lane; m < ns; m += TEAM) {
            const double dwT = -T * (eRT[m] - sub) * invD;   // d omega_T / d omega_m
            double a = fma(nu[0], dwT, nu[1 + m]);
            if (P.reactor == R_CONP) a = fma(-cnu, fma(dwT, invT, invM), a);
            at[m] = a;
        }
        team_sync<TEAM>();
        // dS/dtheta_j = dS/dq_j dq_j/d ln k_j (1, ln T, -1/(R T)); dS/dq_j is
        // the net stoichiometric column of reaction j through at
        const double lnT = log(T);
        const double mRT = -invT / kR;
        for (int j = lane; j < nr; j += TEAM) {
            double g = 0.0;
#pragma unroll
            for (int sl = 0; sl < 6; ++sl) {
                const int sp = __ldg(M.sidx + sl * nr + j);
                if (sp >= 0) {
                    const double c = (double)__ldg(M.snu + sl * nr + j);
                    g = fma(sl < 3 ? -c : c, at[sp], g);
                }
            }
            const double dq = g * W.RD[j] * W.xf[j];
            W.grad[3 * j + 0] += dq;
            W.grad[3 * j + 1] = fma(dq, lnT, W.grad[3 * j + 1]);
            W.grad[3 * j + 2] = fma(dq, mRT, W.grad[3 * j + 2]);
        }
        team_sync<TEAM>();
    }
    for (int i = lane; i < n; i += TEAM) lam[i] = lamn[i];
    team_sync<TEAM>();
    return true;
}

// The whole backward sweep of one cell, from its checkpoints.
template <int TEAM, class MT>
__device__ void adjoint_cell(const AdjTask& tk, const Ws& W, const IntParams& P, int64_t cell, int lane) {
    const DevMech& M = tk.M;
    const int64_t N = tk.N;
    const int ns = M.ns, n = M.n, nr = M.nr;
    const int K = tk.ckpt_n[cell];
    const double* ck = tk.ckpt + cell * (int64_t)tk.ckpt_cap * (n + 1);
    double* lam = W.lam;
    for (int j = lane; j < 3 * nr; j += TEAM) W.grad[j] = 0.0;
    int st = CELL_OK;
    double rho0 = 0.0;
    // K >= 0: all K steps recorded, the final state in record K. K <= -2:
    // S = -K - 2 steps did not fit; record 0 holds the initial state and the
    // last record the final one, and the steps are recomputed from record 0
    // in segments of kSegSteps (the forward integration replayed in its own
    // arithmetic, so each segment's states are those of the forward pass),
    // last segment first, each swept backwards from the team's scratch.
    const bool full = K >= 0 && K < tk.ckpt_cap;
    const int S = full ? K : -K - 2;
    if (!full && (K > -2 || tk.ckpt_cap < 2)) {
        st = CELL_NO_RECORD;
    } else {
        // lam = dL/dy at the end: dL/dT_end and, from Y_k = W_k C_k / rho,
        // dL/dC_m = W_m / rho (dL/dY_m - sum_k Y_k dL/dY_k)
        const double* ye = ck + (int64_t)(full ? K : tk.ckpt_cap - 1) * (n + 1);
        rho0 = ye[n];
        double ms = 0.0;
        for (int i = lane; i < ns; i += TEAM) ms = fma(__ldg(M.W + i), ye[1 + i], ms);
        const double irho = 1.0 / team_sum<TEAM>(ms, W.red);
        double ys = 0.0;
        for (int i = lane; i < ns; i += TEAM)
            ys = fma(__ldg(M.W + i) * ye[1 + i] * irho, tk.dY_end[(int64_t)i * N + cell], ys);
        ys = team_sum<TEAM>(ys, W.red);
        for (int i = lane; i < ns; i += TEAM)
            lam[1 + i] = __ldg(M.W + i) * irho * (tk.dY_end[(int64_t)i * N + cell] - ys);
        if (lane == 0) lam[0] = tk.dT_end[cell];
        team_sync<TEAM>();
        Counters cnt = {0, 0, 0, 0};
        for (int end = S; end > 0 && st == CELL_OK;) {
            const int from = full ? 0 : (end > kSegSteps ? end - kSegSteps : 0);
            if (!full) {   // replay steps 0 .. end - 1 from the initial state, recording from .. end - 1
                for (int i = lane; i < n; i += TEAM) W.yn[i] = ck[i];
                team_sync<TEAM>();
                Counters rc = {0, 0, 0, 0};
                const int rs = P.adaptive ? integrate_adaptive<TEAM, MT>(M, W, P, rc, W.seg, kSegSteps, lane, from, end)
                                          : integrate_fixed<TEAM, MT>(M, W, P, rc, W.seg, kSegSteps, lane, from, end);
                if (rs != CELL_OK || rc.steps != end) {
                    st = CELL_NEWTON_FAIL;
                    break;
                }
            }
            for (int k = end - 1; k >= from; --k) {
                const double* e = full ? ck + (int64_t)k * (n + 1) : W.seg + (int64_t)(k - from) * (n + 1);
                for (int i = lane; i < n; i += TEAM) W.yn[i] = e[i];
                const double h = e[n];
                team_sync<TEAM>();
                // the forward step's stages, recomputed in its own arithmetic
                if (!rk_step<TEAM, MT>(M, W, P, h, cnt, lane) || !adjoint_step<TEAM>(M, W, P, h, lane)) {
                    st = CELL_NEWTON_FAIL;
                    break;
                }
            }
            end = from;
        }
    }
    // dL/dy_0 -> dL/dT_0, dL/dY_0 through C_m = rho Y_m / W_m with rho
    // fixed (constant volume) or rho = p / (R T_0 sum Y / W) (otherwise):
    // dL/dY_k = rho / W_k (lam_k - sum_m lam_m C_m / sum C),
    // dL/dT_0 = lam_T - sum_m lam_m C_m / T_0
    const bool ok = st == CELL_OK;
    double lc = 0.0, cs = 0.0;
    if (ok && P.reactor != R_CONV) {
        for (int i = lane; i < ns; i += TEAM) {
            lc = fma(lam[1 + i], ck[1 + i], lc);
            cs += ck[1 + i];
        }
        lc = team_sum<TEAM>(lc, W.red);
        cs = team_sum<TEAM>(cs, W.red);
    }
    const double shift = P.reactor != R_CONV && ok ? lc / cs : 0.0;
    for (int i = lane; i < ns; i += TEAM)
        tk.dY0[(int64_t)i * N + cell] = ok ? rho0 * __ldg(M.invW + i) * (lam[1 + i] - shift) : 0.0;
    if (lane == 0) {
        tk.dT0[cell] = ok ? lam[0] - (P.reactor != R_CONV ? lc / ck[0] : 0.0) : 0.0;
        if (tk.status) tk.status[cell] = st;
    }
    for (int j = lane; j < nr; j += TEAM) {
        const int64_t o = (int64_t)3 * __ldg(tk.perm + j) * N + cell;
#pragma unroll
        for (int k = 0; k < 3; ++k) tk.grad_cells[o + k * N] = ok ? W.grad[3 * j + k] : 0.0;
    }
    team_sync<TEAM>();
}

template <int TEAM, class MT>
__global__ void __maxnreg__((KernelRegs<TEAM, MT>::value)) adjoint_kernel(AdjTask tk, IntParams P, int sstride, double* gscratch, int64_t gstride,
                               unsigned long long* counter) {
    extern __shared__ double smem_all[];
    const TeamPos<TEAM> tp;
    const Ws W = make_ws(tk.L, smem_all + (size_t)tp.tib * sstride,
                         gscratch ? gscratch + tp.id * gstride : nullptr);
    for (int64_t c = first_cell<TEAM>(counter, tp.id, tp.lane); c < tk.N;
         c = next_cell<TEAM>(counter, c, tp.count, tp.lane))
        adjoint_cell<TEAM, MT>(tk, W, P, c, tp.lane);
}

template <int TEAM, class MT>
cudaError_t launch_adjoint_team(const AdjTask& t, const IntParams& P, int tpb, cudaStream_t st) {
    if (TEAM > 32) tpb = 1;
    const int sstride = t.L.stotal;
    const int64_t gstride = round_up(t.L.gtotal, 32);
    const void* fn = (const void*)adjoint_kernel<TEAM, MT>;
    const size_t smem = (size_t)tpb * sstride * sizeof(double);
    cudaError_t e = set_smem(fn, smem);
    if (e != cudaSuccess) return e;
    int64_t blocks = (t.N + tpb - 1) / tpb, res = 0;
    if ((e = resident_blocks(fn, TEAM * tpb, smem, &res)) != cudaSuccess) return e;
    blocks = blocks < res ? blocks : res;
    LaunchMem mem;
    if ((e = get_mem(blocks * tpb, gstride, true, st, mem)) != cudaSuccess) return e;
    adjoint_kernel<TEAM, MT><<<(unsigned)blocks, TEAM * tpb, smem, st>>>(t, P, sstride, mem.gscratch, gstride,
                                                                         mem.counter);
    e = cudaGetLastError();
    cudaError_t e2 = put_mem(mem, st);
    return e != cudaSuccess ? e : e2;
}

}  // namespace cg
