// Device side of chemgb: per-cell chemistry and implicit integration, one
// warp per cell, everything a cell touches during a Newton iteration staged
// in that warp's slice of shared memory.
//
// Method (arXiv 2510.10005): thermodynamics of Section 2.1 (NASA-7 form,
// molar, in units of R and R T), rates of Section 2.2 (Arrhenius,
// third-body eq. TB_optimization, falloff eq. falloff-reaction with Troe
// broadening eq. f_and_fcent, equilibrium constants eq.
// equilibrium-constant-1), temperature source of Section 3 (eq.
// temperature_source) and Appendix B, analytical Jacobian of Section 3.2 with
// (T, C) independent, Newton on (I - gamma h J) (Section 3.2, Appendix A)
// and a dense LU with partial pivoting (Section 3.4).
//
// GB300 notes that shape the code: FP64 runs at 2 lanes per clock per SM and
// a warp instruction costs the same whether 1 or 32 lanes are active, so
// every FP64 loop is flattened across all 32 lanes; omega and J are
// assembled by host-scheduled rounds in which the 32 lanes add 32 terms into
// 32 distinct entries (no atomics, deterministic order); reactions are
// sorted by type so that lanes of a warp take the same branch.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cg {

constexpr double kLn10 = 2.302585092994045684;
constexpr double kInvLn10 = 0.43429448190325182765;
constexpr unsigned kFull = 0xffffffffu;

enum { RXN_ELEM = 0, RXN_TB = 1, RXN_LIND = 2, RXN_TROE = 3 };
enum { R_CONV = 0, R_CONP = 1, R_CONP_LIT = 2 };
enum { CELL_OK = 0, CELL_NEWTON_FAIL = 1, CELL_STEP_TOO_SMALL = 2, CELL_MAX_STEPS = 3,
       CELL_NONFINITE = 4 };

// rows of the per-species thermo table th[k * ns + i]
enum {
    TH_A1 = 0, TH_A2, TH_A3, TH_A4, TH_A5,       // c_p / R = a1 + a2 T + .. + a5 T^4
    TH_H2, TH_H3, TH_H4, TH_H5, TH_A6,           // h/(RT) = a1 + a2/2 T + .. + a6 / T
    TH_S3, TH_S4, TH_S5, TH_A7,                  // s/R = a1 ln T + a2 T + a3/2 T^2 + .. + a7
    TH_D3, TH_D4, TH_D5,                         // d(c_p/R)/dT = a2 + 2 a3 T + ..
    TH_ROWS
};

// A mechanism as the kernels see it. All pointers are device memory.
// Reactions are in the library's internal order (sorted by type).
struct DevMech {
    int ns, nr, n;               // species, reactions, n = ns + 1
    double ln_pref_R;            // ln(p_ref / R)
    const double *th;            // [TH_ROWS][ns]
    const double *W, *invW;      // [ns]
    const int *rtype, *rev, *sumnu;
    const int *sidx, *snu;       // [6][nr]: slots 0..2 reactants, 3..5 products; -1 empty
    const double *lnA, *beta, *Ta;        // Ta = Ea / R
    const double *dlnA0, *dbeta0, *dTa0;  // low-pressure minus high-pressure
    const double *talpha, *tiT3, *tiT1, *tT2;
    const int *hasT2;
    const int *eff_ptr, *eff_idx;
    const double *eff_am1;       // alpha - 1
    // assembly schedules: rounds of 32 (dst, src, factor) terms
    int w_rounds, v_rounds, j_rounds;
    const int *w_dst, *w_src, *v_dst, *v_src, *j_dst, *j_src;
    const double *w_fac, *v_fac, *j_fac;
};

// Offsets (in doubles) of the arrays in one warp's shared-memory slice.
struct Layout {
    int ld;                  // row stride of the n x n matrix (odd)
    int G;                   // n x ld: Newton matrix / LU factors
    int RD;                  // 9 nr: q, dq/dT, w, d[6] per reaction
    int SP;                  // 4 ns: h/RT, g/RT, c_p/R, d(c_p/R)/dT
    int V;                   // ns: dense third-body column of dOmega/dC
    int yn, Y, base, S, S0, f, err, y1, colA, colB, rinv;   // n each
    int Gam;                 // 5 n: stage derivatives
    int piv;                 // ints, n of them (in ceil(n/2) doubles)
    int total;               // doubles per warp
};

// Integration parameters and the Butcher tableau (stage-derivative form).
struct IntParams {
    int method, reactor, adaptive, nsub, max_newton, max_steps, max_halvings, err_filter;
    double dt, rtol, atol, newton_tol, h0, hmin, neg_tol;
    int s, err_order, start_zero;   // stages; embedded order; BE starts Newton at y_n
    double A[5][5], b[5], bh[5];
};

// ---------------------------------------------------------------------------
// warp helpers

static __device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return __shfl_sync(kFull, v, 0);   // one value for every lane
}

// Walks a rows x ncol row-major index space with stride 32 from `lane`.
struct Flat2D {
    int r, c, dr, dc, ncol;
    __device__ __forceinline__ Flat2D(int lane, int ncol_) : ncol(ncol_) {
        r = lane / ncol;
        c = lane - r * ncol;
        dr = 32 / ncol;
        dc = 32 - dr * ncol;
    }
    __device__ __forceinline__ void next() {
        r += dr;
        c += dc;
        if (c >= ncol) { c -= ncol; ++r; }
    }
};

// out[dst] += fac * in[src], one round of 32 distinct destinations at a time.
static __device__ __forceinline__ void run_schedule(int rounds, const int* __restrict__ dst,
                                             const int* __restrict__ src,
                                             const double* __restrict__ fac, double* out,
                                             const double* in, int lane) {
    for (int r = 0; r < rounds; ++r) {
        const int k = r * 32 + lane;
        const int d = __ldg(dst + k);
        if (d >= 0) out[d] = fma(__ldg(fac + k), in[__ldg(src + k)], out[d]);
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// thermodynamics and rates of progress (Sections 2.1, 2.2)

// Fills SP (species thermo) and RD (q_j and, with deriv, dq_j/dT, the
// third-body weight w_j and the mass-action partials). Returns sum C.
static __device__ double rates(const DevMech& M, const Layout& L, double* sm, const double* y,
                        bool deriv, int lane) {
    const int ns = M.ns, nr = M.nr;
    const double T = y[0];
    const double* C = y + 1;
    const double lnT = log(T);
    const double invT = 1.0 / T;
    double* hRT = sm + L.SP;
    double* gRT = hRT + ns;
    double* cpR = gRT + ns;
    double* dcpR = cpR + ns;
    double csum = 0.0;
    for (int i = lane; i < ns; i += 32) {
        const double* th = M.th + i;
#define TH(k) __ldg(th + (k) * ns)
        const double cp = TH(TH_A1) + T * (TH(TH_A2) + T * (TH(TH_A3) + T * (TH(TH_A4) + T * TH(TH_A5))));
        const double h = TH(TH_A1) + T * (TH(TH_H2) + T * (TH(TH_H3) + T * (TH(TH_H4) + T * TH(TH_H5))))
                         + TH(TH_A6) * invT;
        const double s = TH(TH_A1) * lnT
                         + T * (TH(TH_A2) + T * (TH(TH_S3) + T * (TH(TH_S4) + T * TH(TH_S5)))) + TH(TH_A7);
        const double dcp = TH(TH_A2) + T * (TH(TH_D3) + T * (TH(TH_D4) + T * TH(TH_D5)));
#undef TH
        hRT[i] = h;
        gRT[i] = h - s;
        cpR[i] = cp;
        dcpR[i] = dcp;
        csum += C[i];
    }
    const double Mc = warp_sum(csum);
    __syncwarp();
    const double lnPRT = M.ln_pref_R - lnT;   // ln(p_ref / (R T))
    double* q = sm + L.RD;
    double* dqdT = q + nr;
    double* wv = dqdT + nr;
    double* dd = wv + nr;
    for (int j = lane; j < nr; j += 32) {
        const int type = __ldg(M.rtype + j);
        const double bj = __ldg(M.beta + j), Taj = __ldg(M.Ta + j);
        const double kA = exp(__ldg(M.lnA + j) + bj * lnT - Taj * invT);
        const double dlnkA = (bj + Taj * invT) * invT;
        double kf, dkf_dT, dkf_dM = 0.0;
        if (type == RXN_ELEM) {
            kf = kA;
            dkf_dT = kA * dlnkA;
        } else {
            double Mx = Mc;
            const int e1 = __ldg(M.eff_ptr + j + 1);
            for (int e = __ldg(M.eff_ptr + j); e < e1; ++e)
                Mx = fma(__ldg(M.eff_am1 + e), C[__ldg(M.eff_idx + e)], Mx);
            if (type == RXN_TB) {
                kf = Mx * kA;
                dkf_dT = kf * dlnkA;
                dkf_dM = kA;
            } else {
                const double db = __ldg(M.dbeta0 + j), dTa = __ldg(M.dTa0 + j);
                const double ratio = exp(__ldg(M.dlnA0 + j) + db * lnT - dTa * invT);   // k0 / kinf
                const double Pr = ratio * Mx;
                const double dlnr = (db + dTa * invT) * invT;
                double F = 1.0, dlogF_dP = 0.0, dlogF_dT = 0.0;   // log = log10
                if (type == RXN_TROE) {
                    const double al = __ldg(M.talpha + j);
                    const double i3 = __ldg(M.tiT3 + j), i1 = __ldg(M.tiT1 + j);
                    const double e3 = exp(-T * i3), e1x = exp(-T * i1);
                    double Fc = (1.0 - al) * e3 + al * e1x;
                    double dFc = -(1.0 - al) * i3 * e3 - al * i1 * e1x;
                    if (__ldg(M.hasT2 + j)) {
                        const double T2 = __ldg(M.tT2 + j);
                        const double e2 = exp(-T2 * invT);
                        Fc += e2;
                        dFc += T2 * invT * invT * e2;
                    }
                    const double Lc = log(Fc) * kInvLn10;
                    const double dL_dT = dFc / Fc * kInvLn10;
                    const double c = -0.4 - 0.67 * Lc;
                    const double nn = 0.75 - 1.27 * Lc;
                    const bool clamp = !(Pr >= 1e-300);
                    const double P = log(clamp ? 1e-300 : Pr) * kInvLn10;
                    const double x = P + c;
                    const double rden = 1.0 / (nn - 0.14 * x);
                    const double f1 = x * rden;
                    const double ig = 1.0 / (1.0 + f1 * f1);
                    const double logF = Lc * ig;
                    F = exp(kLn10 * logF);
                    const double df1_dx = nn * rden * rden;
                    const double df1_dn = -x * rden * rden;
                    const double t2 = 2.0 * Lc * f1 * ig * ig;
                    dlogF_dP = clamp ? 0.0 : -t2 * df1_dx;
                    dlogF_dT = (ig - t2 * (-0.67 * df1_dx - 1.27 * df1_dn)) * dL_dT;
                }
                const double ip = 1.0 / (1.0 + Pr);
                kf = kA * (Pr * ip) * F;
                const double dkf_dPr = kA * F * ip * (ip + dlogF_dP);
                dkf_dT = kf * dlnkA + dkf_dPr * Pr * dlnr + kf * kLn10 * dlogF_dT;
                dkf_dM = dkf_dPr * ratio;
            }
        }
        // mass-action products and their slot partials
        double p[6], dp[6];
        int sp[6];
#pragma unroll
        for (int s = 0; s < 6; ++s) {
            sp[s] = __ldg(M.sidx + s * nr + j);
            p[s] = 1.0;
            dp[s] = 0.0;
            if (sp[s] >= 0) {
                const int nu = __ldg(M.snu + s * nr + j);
                const double c = C[sp[s]];
                double pw = 1.0;
                for (int k = 1; k < nu; ++k) pw *= c;
                dp[s] = nu * pw;
                p[s] = pw * c;
            }
        }
        const double Pf = p[0] * p[1] * p[2];
        const double Pb = p[3] * p[4] * p[5];
        double invK = 0.0, dlnK = 0.0;
        if (__ldg(M.rev + j)) {
            double dG = 0.0, dH = 0.0;
#pragma unroll
            for (int s = 0; s < 6; ++s) {
                if (sp[s] >= 0) {
                    const double nu = (s < 3 ? -1.0 : 1.0) * __ldg(M.snu + s * nr + j);
                    dG = fma(nu, gRT[sp[s]], dG);
                    dH = fma(nu, hRT[sp[s]], dH);
                }
            }
            const double snu = (double)__ldg(M.sumnu + j);
            invK = exp(dG - snu * lnPRT);      // 1 / K_c
            dlnK = (dH - snu) * invT;          // d ln K_c / dT
        }
        const double kr = kf * invK;
        q[j] = kf * Pf - kr * Pb;
        if (deriv) {
            const double phi = Pf - invK * Pb;
            dqdT[j] = dkf_dT * phi + kr * Pb * dlnK;
            wv[j] = dkf_dM * phi;
            if (sp[0] >= 0) dd[0 * nr + j] = kf * dp[0] * p[1] * p[2];
            if (sp[1] >= 0) dd[1 * nr + j] = kf * p[0] * dp[1] * p[2];
            if (sp[2] >= 0) dd[2 * nr + j] = kf * p[0] * p[1] * dp[2];
            if (sp[3] >= 0) dd[3 * nr + j] = -kr * dp[3] * p[4] * p[5];
            if (sp[4] >= 0) dd[4 * nr + j] = -kr * p[3] * dp[4] * p[5];
            if (sp[5] >= 0) dd[5 * nr + j] = -kr * p[3] * p[4] * dp[5];
        }
    }
    __syncwarp();
    return Mc;
}

struct SrcInfo {
    double wT, Dt, Ws, Mc, sdil, cw, cdc;
};

// S = (omega_T, dC/dt) into sm[L.S..]; y = (T, C).
static __device__ SrcInfo assemble_source(const DevMech& M, const Layout& L, double* sm, const double* y,
                                   int reactor, double Mc, int lane) {
    const int ns = M.ns;
    double* S = sm + L.S;
    const double* hRT = sm + L.SP;
    const double* cpR = hRT + 2 * ns;
    const double* dcpR = cpR + ns;
    const double T = y[0];
    const double* C = y + 1;
    for (int i = lane; i < ns; i += 32) S[1 + i] = 0.0;
    __syncwarp();
    run_schedule(M.w_rounds, M.w_dst, M.w_src, M.w_fac, S, sm + L.RD, lane);
    const double sub = reactor == R_CONV ? 1.0 : 0.0;   // u/RT = h/RT - 1, c_v/R = c_p/R - 1
    double qe = 0.0, den = 0.0, ws = 0.0, cw = 0.0, cdc = 0.0;
    for (int i = lane; i < ns; i += 32) {
        const double w = S[1 + i];
        const double c = cpR[i] - sub;
        qe = fma(hRT[i] - sub, w, qe);
        den = fma(C[i], c, den);
        ws += w;
        cw = fma(c, w, cw);
        cdc = fma(C[i], dcpR[i], cdc);
    }
    SrcInfo si;
    si.Mc = Mc;
    const double Qt = warp_sum(qe);
    si.Dt = warp_sum(den);
    si.Ws = warp_sum(ws);
    si.cw = warp_sum(cw);
    si.cdc = warp_sum(cdc);
    si.wT = -T * Qt / si.Dt;   // -sum e_i omega_i / (rho c), volumetric c
    si.sdil = 0.0;
    if (reactor == R_CONP) {
        si.sdil = si.wT / T + si.Ws / Mc;
        for (int i = lane; i < ns; i += 32) S[1 + i] = fma(-C[i], si.sdil, S[1 + i]);
    }
    if (lane == 0) S[0] = si.wT;
    __syncwarp();
    return si;
}

// Analytical Jacobian. With out == nullptr, writes the Newton matrix
// G = I - gh J into sm[L.G] (row stride L.ld); otherwise writes J to out
// (row-major n x n, global memory).
static __device__ void assemble_jacobian(const DevMech& M, const Layout& L, double* sm, const double* y,
                                  int reactor, const SrcInfo& si, double gh, double* out, int lane) {
    const int ns = M.ns, n = M.n, ld = L.ld;
    double* G = sm + L.G;
    double* V = sm + L.V;
    const double* hRT = sm + L.SP;
    const double* cpR = hRT + 2 * ns;
    const double* RD = sm + L.RD;
    const double T = y[0];
    const double* C = y + 1;
    const double sub = reactor == R_CONV ? 1.0 : 0.0;

    // dense part of d omega / d C from third-body and falloff reactions
    for (int i = lane; i < ns; i += 32) V[i] = 0.0;
    __syncwarp();
    run_schedule(M.v_rounds, M.v_dst, M.v_src, M.v_fac, V, RD, lane);
    for (Flat2D it(lane, n); it.r < ns; it.next())
        G[(1 + it.r) * ld + it.c] = it.c == 0 ? 0.0 : V[it.r];
    __syncwarp();
    // sparse part, reaction by reaction in a fixed order
    run_schedule(M.j_rounds, M.j_dst, M.j_src, M.j_fac, G, RD, lane);

    // temperature row: J_T,m = -(T A_m + omega_T c_m) / D (m > 0),
    // J_T,0 = -(sum c_i omega_i + T A_0 + omega_T sum C_i dc_i/dT) / D,
    // A_m = sum_i e_i dOmega_i/dy_m (e = u/RT or h/RT, c = c_v/R or c_p/R)
    double* JT = sm + L.colA;
    double* ds = sm + L.colB;
    const double invD = 1.0 / si.Dt;
    for (int m = lane; m < n; m += 32) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < ns; ++i) {
            const double g = G[(1 + i) * ld + m];
            a = fma(hRT[i] - sub, g, a);
            b += g;
        }
        double jt;
        if (m == 0) jt = -(si.cw + T * a + si.wT * si.cdc) * invD;
        else jt = -(T * a + si.wT * (cpR[m - 1] - sub)) * invD;
        JT[m] = jt;
        if (reactor == R_CONP) {
            // s = omega_T / T + sum omega / sum C;  ds/dy_m
            double d = jt / T + b / si.Mc;
            if (m == 0) d -= si.wT / (T * T);
            else d -= si.Ws / (si.Mc * si.Mc);
            ds[m] = d;
        }
    }
    __syncwarp();
    const bool conp = reactor == R_CONP;
    for (Flat2D it(lane, n); it.r < n; it.next()) {
        const int r = it.r, c = it.c;
        double J;
        if (r == 0) {
            J = JT[c];
        } else {
            J = G[r * ld + c];
            if (conp) {
                J = fma(-C[r - 1], ds[c], J);
                if (c == r) J -= si.sdil;
            }
        }
        if (out) out[r * n + c] = J;
        else G[r * ld + c] = fma(-gh, J, r == c ? 1.0 : 0.0);
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// dense LU with partial pivoting (Section 3.4), in place, warp-cooperative

static __device__ bool lu_factor(double* G, int n, int ld, int* piv, double* rinv, int lane) {
    for (int k = 0; k < n; ++k) {
        // pivot: largest |G_ik|, i >= k; ties to the lowest row (non-negative
        // doubles order like their bit patterns)
        unsigned long long best = 0ull;
        int bi = n;
        for (int i = k + lane; i < n; i += 32) {
            const unsigned long long b =
                (unsigned long long)__double_as_longlong(G[i * ld + k]) & 0x7fffffffffffffffull;
            if (bi == n || b > best) { best = b; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ob = __shfl_xor_sync(kFull, best, o);
            const int oi = __shfl_xor_sync(kFull, bi, o);
            if (oi < n && (bi == n || ob > best || (ob == best && oi < bi))) { best = ob; bi = oi; }
        }
        if (lane == 0) piv[k] = bi;
        if (bi != k)
            for (int j = lane; j < n; j += 32) {
                const double t = G[k * ld + j];
                G[k * ld + j] = G[bi * ld + j];
                G[bi * ld + j] = t;
            }
        __syncwarp();
        const double pv = G[k * ld + k];
        if (pv == 0.0) return false;
        const double r = 1.0 / pv;
        if (lane == 0) rinv[k] = r;
        for (int i = k + 1 + lane; i < n; i += 32) G[i * ld + k] *= r;
        __syncwarp();
        const int m = n - k - 1;
        if (m > 0) {
            const int k1 = k + 1;
            for (Flat2D it(lane, m); it.r < m; it.next()) {
                const int i = k1 + it.r, j = k1 + it.c;
                G[i * ld + j] = fma(-G[i * ld + k], G[k * ld + j], G[i * ld + j]);
            }
        }
        __syncwarp();
    }
    return true;
}

// x <- G^{-1} x with the factors of lu_factor.
static __device__ void lu_solve(const double* G, int n, int ld, const int* piv, const double* rinv,
                         double* x, int lane) {
    if (lane == 0)
        for (int k = 0; k < n; ++k) {
            const int p = piv[k];
            if (p != k) { const double t = x[k]; x[k] = x[p]; x[p] = t; }
        }
    __syncwarp();
    for (int j = 0; j < n - 1; ++j) {           // unit lower triangle, by columns
        const double xj = x[j];
        for (int i = j + 1 + lane; i < n; i += 32) x[i] = fma(-G[i * ld + j], xj, x[i]);
        __syncwarp();
    }
    for (int j = n - 1; j >= 0; --j) {          // upper triangle, by columns
        const double xj = x[j] * rinv[j];
        __syncwarp();
        if (lane == 0) x[j] = xj;
        for (int i = lane; i < j; i += 32) x[i] = fma(-G[i * ld + j], xj, x[i]);
        __syncwarp();
    }
}

// weighted RMS norm with w_i = atol + rtol max(|a_i|, |b_i|)
static __device__ __forceinline__ double wrms(const double* v, const double* a, const double* b, int n,
                                       double rtol, double atol, int lane) {
    double s = 0.0;
    for (int i = lane; i < n; i += 32) {
        const double w = atol + rtol * fmax(fabs(a[i]), fabs(b[i]));
        const double r = v[i] / w;
        s = fma(r, r, s);
    }
    return sqrt(warp_sum(s) / n);
}

}  // namespace cg
