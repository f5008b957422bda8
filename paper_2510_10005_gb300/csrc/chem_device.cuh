// Device side of chemgb: per-cell chemistry and implicit integration. One
// team of TEAM threads (a warp, or a whole block of 2-8 warps) owns one cell;
// everything the cell touches during a Newton iteration is staged in the
// team's slice of shared memory.
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
// GB300 notes that shape the code: each SM sub-partition has its own FP64
// unit retiring half a lane per clock, and a warp instruction costs the same
// whatever its active-lane count. So every FP64 loop is flattened across
// the whole team, a team of two warps keeps two instruction streams per
// sub-partition, and omega and J are assembled by host-built schedules in
// which every thread owns a set of destination entries and accumulates their
// terms in a register (no atomics, no synchronisation, deterministic order);
// reactions are sorted by type so that neighbouring threads take the same
// branch.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cg {

constexpr double kLn10 = 2.302585092994045684;
constexpr double kInvLn10 = 0.43429448190325182765;
constexpr unsigned kFull = 0xffffffffu;

enum { RXN_ELEM = 0, RXN_TB = 1, RXN_LIND = 2, RXN_TROE = 3, RXN_SRI = 4, RXN_PLOG = 5 };
enum { R_CONV = 0, R_CONP = 1, R_CONP_LIT = 2 };
enum { CELL_OK = 0, CELL_NEWTON_FAIL = 1, CELL_STEP_TOO_SMALL = 2, CELL_MAX_STEPS = 3,
       CELL_NONFINITE = 4, CELL_NO_RECORD = 5 };

// rows of the per-species thermo table th[k * ns + i] for the NASA-7 form
// (c_p polynomial of degree P = 4)
enum {
    TH_A1 = 0, TH_A2, TH_A3, TH_A4, TH_A5,       // c_p / R = a1 + a2 T + .. + a5 T^4
    TH_H2, TH_H3, TH_H4, TH_H5, TH_A6,           // h/(RT) = a1 + a2/2 T + .. + a6 / T
    TH_S3, TH_S4, TH_S5, TH_A7,                  // s/R = a1 ln T + a2 T + a3/2 T^2 + .. + a7
    TH_D3, TH_D4, TH_D5,                         // d(c_p/R)/dT = a2 + 2 a3 T + ..
    TH_ROWS
};
// The same table for a c_p polynomial of degree P >= 4 (Section 2.1, eq.
// specific_heat_polynomial; Appendix C.1), c_p/R = sum_{k=0}^{P} a_k T^k:
// 4 P + 1 rows, a_k at k, a_k/(k+1) at P + k (k >= 1), the h/R constant at
// 2 P + 1, a_k/k at 2 P + k (k >= 2), the s/R constant at 3 P + 1, k a_k at
// 3 P + k (k >= 2). P = 4 is the layout above.
__host__ __device__ constexpr int th_rows(int P) { return 4 * P + 1; }

// A mechanism as the kernels see it. All pointers are device memory.
// Reactions are in the library's internal order (sorted by type).
struct DevMech {
    int ns, nr, n;               // species, reactions, n = ns + 1
    int team;                    // threads per cell the schedules were built for
    int lu_nb;                   // panel width of the blocked LU (0: unblocked)
    double ln_pref_R;            // ln(p_ref / R)
    const double *th;            // [th_rows(th_np)][ns]
    int th_np;                   // degree P of the c_p polynomial (4: NASA-7)
    const double *W, *invW;      // [ns]
    const int *rtype, *rev, *sumnu;
    const int *sidx, *snu;       // [6][nr]: slots 0..2 reactants, 3..5 products; -1 empty
    int slots;                   // slots used on either side by some reaction: 2 (slots 2 and 5
                                 // empty everywhere, rates compiled without them) or 3
    const double *snud, *sumnud; // the coefficients as doubles ([6][nr], 0 on empty slots) and sum nu
    const double *lnA, *beta, *Ta;        // Ta = Ea / R
    const double *dlnA0, *dbeta0, *dTa0;  // low-pressure minus high-pressure
    const double *talpha, *tiT3, *tiT1, *tT2;
    const int *hasT2;
    const int *eff_ptr, *eff_idx;
    const double *eff_am1;       // alpha - 1
    // thread-owned assembly schedules: len terms per thread, (dst, src, factor)
    int w_len, v_len, j_len;
    const int *w_dst, *w_src, *v_dst, *v_src, *j_dst, *j_src;
    const double *w_fac, *v_fac, *j_fac;
    // reaction chunks of the rates loop: runs of at most 32 reactions of one
    // kind (with or without falloff); warp w of a team takes chunks
    // rc_ptr[w] .. rc_ptr[w+1]-1, chunk c = reactions rc_first[c] + 0 .. rc_len[c]-1
    const int *rc_ptr, *rc_first, *rc_len;
    const double* exp2j;         // 2^(j/64), j = 0..63 (exp_tab)
    // SRI falloff: [5][nr] = a, b, 1/c, ln d, e
    const double* sri;
    // PLOG: pressure levels of reaction j are pl_lev[j] .. pl_lev[j+1]-1,
    // each with ln p and its Arrhenius rates pl_rate[l] .. pl_rate[l+1]-1
    int has_plog;
    const int *pl_lev, *pl_rate;
    const double *pl_lnp, *pl_lnA, *pl_b, *pl_Ta;
#ifdef CG_DEBUG
    unsigned long long* dbg;     // [2]: arrays whose guard words changed (bit a), first such cell + 1
#endif
};

// Working arrays of one cell. Each lives in the team's slice of shared
// memory or, when the cell's arrays do not fit there (large mechanisms), in
// the team's slot of a global scratch buffer (L2-resident).
enum {
    A_G = 0,    // n x ld Newton matrix / LU factors (FP64 or FP32)
    A_RD,       // 9 nr: q, dq/dT, w, d[6] per reaction
    A_SP,       // 4 ns: h/RT, g/RT, c_p/R, d(c_p/R)/dT
    A_V,        // ns: dense third-body column of dOmega/dC
    A_YN, A_Y, A_BASE, A_S, A_S0, A_F, A_ERR, A_Y1, A_COLA, A_COLB, A_RINV,   // n each
    A_GAM,      // 5 n: stage derivatives
    A_PIV,      // n ints
    A_RED,      // 24 doubles: cross-warp reduction scratch (always shared)
    // adjoint only (size 0 in the forward layouts)
    A_XF,       // nr: d ln q_j / d ln k_j
    A_GRAD,     // 3 nr: dL/d(ln A, b, Ea), reaction-major
    A_LAM, A_LAMN, A_NU, A_RHS,   // n each
    A_ACC,      // 5 n: sum over later stages of h a_qp J_q^T nu_q
    A_SEG,      // kSegSteps (n + 1): records of a replayed segment of steps
    // GMRES only (size 0 with the LU)
    A_KV,       // (m+1) x vs Krylov basis
    A_KH,       // (m+1) m Hessenberg + 2 m rotations + 2 (m+1) (g, projections)
    A_COUNT
};

// Steps per segment when the adjoint recomputes a cell whose checkpoints
// did not fit in the caller's record.
constexpr int kSegSteps = 32;

struct Layout {
    int ld;                  // row stride of the n x n matrix (odd)
    int off[A_COUNT];        // offset in doubles within shared or global slot
    unsigned gmask;          // bit a set: array a is in global scratch
    int stotal;              // doubles of shared memory per team
    int gtotal;              // doubles of global scratch per team
#ifdef CG_DEBUG
    int size[A_COUNT];       // doubles of each array; kGuard guard words follow it
#endif
};

#ifdef CG_DEBUG
// Debug build (stands in for a memory checker): two guard words after each
// array of a cell, every array poisoned before each cell (NaN, so that a
// value read before it is written spoils the result; zero for the pivot
// and reduction arrays, whose integers index rows), guards checked after it.
constexpr int kGuard = 2;
constexpr unsigned long long kCanary = 0x7ff4c0ffee000000ull;   // a signalling-NaN pattern
constexpr unsigned long long kPoison = 0x7ff4deadbeef0000ull;

#endif

struct Ws {
    int ld;
    double *G, *RD, *SP, *V, *yn, *Y, *base, *S, *S0, *f, *err, *y1, *colA, *colB, *rinv, *Gam, *red;
    int* piv;
    double *xf, *grad, *lam, *lamn, *nu, *rhs, *acc, *seg;
    double *kv, *kh;
};

__device__ __forceinline__ Ws make_ws(const Layout& L, double* sbase, double* gbase) {
    double* p[A_COUNT];
#pragma unroll
    for (int a = 0; a < A_COUNT; ++a) p[a] = ((L.gmask >> a) & 1u ? gbase : sbase) + L.off[a];
    Ws w;
    w.ld = L.ld;
    w.G = p[A_G]; w.RD = p[A_RD]; w.SP = p[A_SP]; w.V = p[A_V];
    w.yn = p[A_YN]; w.Y = p[A_Y]; w.base = p[A_BASE]; w.S = p[A_S]; w.S0 = p[A_S0];
    w.f = p[A_F]; w.err = p[A_ERR]; w.y1 = p[A_Y1]; w.colA = p[A_COLA]; w.colB = p[A_COLB];
    w.rinv = p[A_RINV]; w.Gam = p[A_GAM]; w.red = p[A_RED];
    w.piv = reinterpret_cast<int*>(p[A_PIV]);
    w.xf = p[A_XF]; w.grad = p[A_GRAD]; w.lam = p[A_LAM]; w.lamn = p[A_LAMN];
    w.nu = p[A_NU]; w.rhs = p[A_RHS]; w.acc = p[A_ACC]; w.seg = p[A_SEG];
    w.kv = p[A_KV]; w.kh = p[A_KH];
    return w;
}

// Integration parameters and the Butcher tableau (stage-derivative form).
struct IntParams {
    int method, reactor, adaptive, nsub, max_newton, max_steps, max_halvings, err_filter;
    int precision;                  // 0: FP64 Newton matrix, 1: FP32 Newton matrix
    int linear_solver, prec, gmres_m, gmres_maxit;   // 0 LU, 1 GMRES; preconditioner; restart; limit
    double gmres_tol;
    double dt, rtol, atol, newton_tol, h0, hmin, neg_tol;
    int s, err_order, start_zero;   // stages; embedded order; BE starts Newton at y_n
    double A[5][5], b[5], bh[5];
};

// ---------------------------------------------------------------------------
// team helpers (TEAM = 32: one warp; TEAM > 32: the whole block)

template <int TEAM>
__device__ __forceinline__ void team_sync() {
    if constexpr (TEAM == 32) __syncwarp();
    else __syncthreads();
}

template <int TEAM>
__device__ __forceinline__ int team_lane() { return threadIdx.x & (TEAM - 1); }

static __device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return __shfl_sync(kFull, v, 0);   // one value for every lane
}

// Sum over the team, the same value in every thread (fixed order).
template <int TEAM>
__device__ __forceinline__ double team_sum(double v, double* red) {
    v = warp_sum(v);
    if constexpr (TEAM == 32) {
        return v;
    } else {
        const int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) red[w] = v;
        __syncthreads();
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < TEAM / 32; ++k) s += red[k];
        __syncthreads();
        return s;
    }
}

// K sums over the team at once, each in team_sum's order (the same bits),
// with one pair of block barriers instead of K pairs.
template <int TEAM, int K>
__device__ __forceinline__ void team_sums(double (&v)[K], double* red) {
    constexpr int NW = TEAM / 32;
    if constexpr (TEAM == 32 || NW * K > 24) {   // the 24 words of the scratch
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = team_sum<TEAM>(v[k], red);
    } else {
        const int w = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const double x = warp_sum(v[k]);
            if ((threadIdx.x & 31) == 0) red[k * NW + w] = x;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double s = 0.0;
#pragma unroll
            for (int u = 0; u < NW; ++u) s += red[k * NW + u];
            v[k] = s;
        }
        __syncthreads();
    }
}

template <int TEAM>
__device__ __forceinline__ bool team_any(bool b, double* red) {
    b = __any_sync(kFull, b);
    if constexpr (TEAM == 32) {
        return b;
    } else {
        int* ri = reinterpret_cast<int*>(red + 16);
        const int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) ri[w] = b ? 1 : 0;
        __syncthreads();
        int r = 0;
#pragma unroll
        for (int k = 0; k < TEAM / 32; ++k) r |= ri[k];
        __syncthreads();
        return r != 0;
    }
}

#ifdef CG_DEBUG
template <int TEAM>
__device__ void debug_poison(const Layout& L, double* sbase, double* gbase, int lane) {
    for (int a = 0; a < A_COUNT; ++a) {
        if (L.size[a] == 0) continue;
        double* p = ((L.gmask >> a) & 1u ? gbase : sbase) + L.off[a];
        const unsigned long long fill = (a == A_PIV || a == A_RED) ? 0ull : kPoison;
        for (int i = lane; i < L.size[a] + kGuard; i += TEAM)
            p[i] = __longlong_as_double((long long)(i < L.size[a] ? fill : kCanary + a));
    }
    team_sync<TEAM>();
}

template <int TEAM>
__device__ void debug_check(const Layout& L, double* sbase, double* gbase, unsigned long long* dbg,
                            int64_t cell, int lane) {
    team_sync<TEAM>();
    unsigned long long bad = 0ull;
    for (int a = lane; a < A_COUNT; a += TEAM) {
        if (L.size[a] == 0) continue;
        const double* p = ((L.gmask >> a) & 1u ? gbase : sbase) + L.off[a] + L.size[a];
        for (int g = 0; g < kGuard; ++g)
            if ((unsigned long long)__double_as_longlong(p[g]) != kCanary + a) bad |= 1ull << a;
    }
    if (bad) {
        atomicOr(dbg, bad);
        atomicCAS(dbg + 1, 0ull, (unsigned long long)cell + 1ull);
    }
    team_sync<TEAM>();
}
#endif

// Walks a rows x ncol row-major index space with stride S from `lane`.
struct Flat2D {
    int r, c, dr, dc, ncol;
    __device__ __forceinline__ Flat2D(int lane, int ncol_, int S) : ncol(ncol_) {
        r = lane / ncol;
        c = lane - r * ncol;
        dr = S / ncol;
        dc = S - dr * ncol;
    }
    __device__ __forceinline__ void next() {
        r += dr;
        c += dc;
        if (c >= ncol) { c -= ncol; ++r; }
    }
};

// Thread-owned assembly schedule: term t of thread l is at [t * TEAM + l];
// each thread owns a set of destinations and walks their terms in a fixed
// order, accumulating in a register. Every term carries its destination with
// two flags: kSchedFirst (the run of a destination starts: the register
// takes the destination's current value) and kSchedLast (the run ends: the
// register is stored back). Padding terms (after a thread's last run) have
// fac 0, src 0 and no flags. No two threads share a destination, so no
// synchronisation is needed inside the walk, and a thread's destinations
// never repeat, so the loads of a group of terms may precede its stores.
// `in` is read-only while the schedule runs. The sum is formed in FP64 (one
// FMA per term, no separate add) and stored in the destination's type.
constexpr int kSchedFirst = 1 << 30, kSchedLast = 1 << 29, kSchedIndex = kSchedLast - 1;

template <int TEAM, class OT>
__device__ __forceinline__ void run_schedule(int len, const int* __restrict__ dst,
                                             const int* __restrict__ src,
                                             const double* __restrict__ fac, OT* out,
                                             const double* in, int lane) {
    double acc = 0.0;
    int t = 0;
    for (; t + 4 <= len; t += 4) {
        int d[4], s[4];
        double f[4], x[4], o[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int k = (t + u) * TEAM + lane;
            d[u] = __ldg(dst + k);
            s[u] = __ldg(src + k);
            f[u] = __ldg(fac + k);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            x[u] = in[s[u]];
            o[u] = (d[u] & kSchedFirst) ? static_cast<double>(out[d[u] & kSchedIndex]) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (d[u] & kSchedFirst) acc = o[u];
            acc = fma(f[u], x[u], acc);
            if (d[u] & kSchedLast) out[d[u] & kSchedIndex] = static_cast<OT>(acc);
        }
    }
    for (; t < len; ++t) {
        const int k = t * TEAM + lane;
        const int d = __ldg(dst + k);
        if (d & kSchedFirst) acc = static_cast<double>(out[d & kSchedIndex]);
        acc = fma(__ldg(fac + k), in[__ldg(src + k)], acc);
        if (d & kSchedLast) out[d & kSchedIndex] = static_cast<OT>(acc);
    }
    team_sync<TEAM>();
}

// 1/x by two Newton-Raphson steps r <- r + r (1 - x r) (quadratic
// convergence) from the hardware's approximate single-precision reciprocal
// of x truncated to 20 mantissa bits; the conversions between the formats
// are done on the bit patterns. Falls back to division outside the
// single-precision exponent range. Within 1 ulp of the correctly rounded
// reciprocal (checked against 1.0/x in the tests).
static __device__ __forceinline__ double rcp_nr(double x) {
    const int hi = __double2hiint(x);
    const int e = ((hi >> 20) & 0x7ff) - 1023;
    if (e < -125 || e > 125) return 1.0 / x;
    const int fbits = (hi & 0x80000000) | ((e + 127) << 23) | ((hi & 0xfffff) << 3);
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(__int_as_float(fbits)));
    const int rb = __float_as_int(rf);
    const int re = ((rb >> 23) & 0xff) - 127;
    const int rhi = (rb & 0x80000000) | ((re + 1023) << 20) | ((rb & 0x7fffff) >> 3);
    const int rlo = (rb & 0x7) << 29;
    double r = __hiloint2double(rhi, rlo);
    double t = fma(-x, r, 1.0);
    r = fma(r, t, r);
    t = fma(-x, r, 1.0);
    return fma(r, t, r);
}

// e^x by Tang's table-driven method (ACM Trans. Math. Softw. 15(2), 1989):
// x = (64 m + j) ln2/64 + r with |r| <= ln2/128, e^x = 2^m 2^(j/64) e^r. The
// integer 64 m + j is round(x 64/ln2), taken from the low bits of
// x 64/ln2 + 1.5 2^52; ln2/64 is split in two parts (Cody and Waite) so that
// r keeps the rounding of x only; e^r - 1 is its Taylor polynomial to degree
// 5 (truncation below 3e-17 relative); 2^(j/64) comes from a 64-entry table
// of correctly rounded values built on the host; 2^m is added to the
// exponent field. Ten FP64 operations. |x| >= 707 (where 2^m would leave
// the normal range), infinities and NaN go to the library exp. Checked
// against the library exp to 2 ulp in the tests.
static __device__ __forceinline__ double exp_tab(double x, const double* __restrict__ tab) {
    const int hi = __double2hiint(x);
    if ((hi & 0x7fffffff) >= 0x40861800) return exp(x);
    const double shift = 0x1.8p52;
    const double t = fma(x, 0x1.71547652b82fep+6, shift);   // x 64/ln2 + 1.5 2^52
    const int k = __double2loint(t);
    const double kd = t - shift;
    double r = fma(kd, -0x1.62e42fefa39efp-7, x);          // leading part of ln2/64
    r = fma(kd, -0x1.abc9e3b39803fp-62, r);                 // remainder of ln2/64
    const double r2 = r * r;
    double q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
    q = fma(q, r, 1.0 / 6.0);
    q = fma(q, r, 0.5);
    const double em1 = fma(q, r2, r);                       // e^r - 1
    const double sj = __ldg(tab + (k & 63));
    const double y = fma(sj, em1, sj);
    return __hiloint2double(__double2hiint(y) + ((k >> 6) << 20), __double2loint(y));
}

// ---------------------------------------------------------------------------
// thermodynamics and rates of progress (Sections 2.1, 2.2)

// c_p/R and h/(RT) of species i from a table of degree P > 4, by Horner's rule
__device__ __forceinline__ void thermo_cp_h_deg(const double* th, int ns, int P, double T, double invT,
                                                double& cp, double& h) {
    double c = __ldg(th + P * ns);
    for (int k = P - 1; k >= 0; --k) c = fma(c, T, __ldg(th + k * ns));
    double hp = __ldg(th + 2 * P * ns);
    for (int k = P - 1; k >= 1; --k) hp = fma(hp, T, __ldg(th + (P + k) * ns));
    cp = c;
    h = fma(T, hp, __ldg(th)) + __ldg(th + (2 * P + 1) * ns) * invT;
}

// s/R and d(c_p/R)/dT of species i from a table of degree P > 4
__device__ __forceinline__ void thermo_s_dcp_deg(const double* th, int ns, int P, double T, double lnT,
                                                 double& s, double& dcp) {
    double sp = __ldg(th + 3 * P * ns);
    for (int k = P - 1; k >= 2; --k) sp = fma(sp, T, __ldg(th + (2 * P + k) * ns));
    double dp = __ldg(th + 4 * P * ns);
    for (int k = P - 1; k >= 2; --k) dp = fma(dp, T, __ldg(th + (3 * P + k) * ns));
    s = __ldg(th) * lnT + T * fma(T, sp, __ldg(th + ns)) + __ldg(th + (3 * P + 1) * ns);
    dcp = fma(T, dp, __ldg(th + ns));
}

// Fills SP (species thermo) and RD (q_j and, with deriv, dq_j/dT, the
// third-body weight w_j and the mass-action partials). Returns sum C.
// Rate of progress q_j = k_f prod C^nu' - k_r prod C^nu'' of reaction j
// from its forward rate constant (Section 2.2, K_c from the Gibbs energies
// with the integer power of p_ref / RT folded into the exponent) and, with
// deriv, its partials: dq/dT, the third-body weight dq/d[M], and the
// per-slot dq/dC (d[s][j]). NSL = 2 leaves out the third slot of each side
// at compile time (mechanisms whose reactions have at most two species on
// either side); the products over the remaining slots are the same.
template <int NSL>
__device__ __forceinline__ void progress_rate(const DevMech& M, int j, const double* C, const double* gRT,
                                              const double* hRT, double lnPRT, double invT, double kf,
                                              double dkf_dT, double dkf_dM, bool deriv, double* q, double* dqdT,
                                              double* wv, double* dd) {
    // mass-action products C^nu of every slot and their derivatives
    const int nr = M.nr;
    double p[6], dp[6], nd[6];
    int sp[6];
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        if (s % 3 >= NSL) {   // a slot no reaction uses: factor 1, no derivative
            sp[s] = -1;
            nd[s] = 0.0;
            p[s] = 1.0;
            dp[s] = 0.0;
            continue;
        }
        sp[s] = __ldg(M.sidx + s * nr + j);
        nd[s] = __ldg(M.snud + s * nr + j);
        p[s] = 1.0;
        dp[s] = 0.0;
        if (sp[s] >= 0) {
            const int nu = __ldg(M.snu + s * nr + j);
            const double c = C[sp[s]];
            double pw = 1.0;
            for (int k = 1; k < nu; ++k) pw *= c;
            dp[s] = nu == 1 ? 1.0 : nd[s] * pw;
            p[s] = pw * c;
        }
    }
    double invK = 0.0, dlnK = 0.0;
    if (__ldg(M.rev + j)) {
        double dG = 0.0, dH = 0.0;
#pragma unroll
        for (int s = 0; s < 6; ++s) {
            if (sp[s] >= 0) {
                const double nu = s < 3 ? -nd[s] : nd[s];
                dG = fma(nu, gRT[sp[s]], dG);
                dH = fma(nu, hRT[sp[s]], dH);
            }
        }
        const double snu = __ldg(M.sumnud + j);
        invK = exp_tab(fma(-snu, lnPRT, dG), M.exp2j);   // 1 / K_c
        dlnK = (dH - snu) * invT;                        // d ln K_c / dT
    }
    const double kr = kf * invK;
    // prefix and suffix products: kf p0 p1 p2 and the slot partials
    const double f01 = kf * p[0], f012 = f01 * p[1], fP = f012 * p[2];   // kf Pf
    const double f12 = p[1] * p[2];
    const double r01 = kr * p[3], r012 = r01 * p[4], rP = r012 * p[5];   // kr Pb
    const double r12 = p[4] * p[5];
    q[j] = fP - rP;
    if (deriv) {
        const double Pf = p[0] * f12, Pb = p[3] * r12;
        const double phi = fma(-invK, Pb, Pf);
        dqdT[j] = fma(dkf_dT, phi, rP * dlnK);
        wv[j] = dkf_dM * phi;
        if (sp[0] >= 0) dd[0 * nr + j] = dp[0] * (kf * f12);
        if (sp[1] >= 0) dd[1 * nr + j] = dp[1] * (f01 * p[2]);
        if (sp[2] >= 0) dd[2 * nr + j] = dp[2] * f012;
        if (sp[3] >= 0) dd[3 * nr + j] = -dp[3] * (kr * r12);
        if (sp[4] >= 0) dd[4 * nr + j] = -dp[4] * (r01 * p[5]);
        if (sp[5] >= 0) dd[5 * nr + j] = -dp[5] * r012;
    }
}

template <int TEAM>
__device__ double rates(const DevMech& M, const Ws& W,const double* y, bool deriv,
                        int lane, double* xf = nullptr) {   // xf: d ln q_j / d ln k_j (adjoint)
    const int ns = M.ns, nr = M.nr;
    const double T = y[0];
    const double* C = y + 1;
    const double lnT = log(T);
    const double invT = 1.0 / T;
    double* hRT = W.SP;
    double* gRT = hRT + ns;
    double* cpR = gRT + ns;
    double* dcpR = cpR + ns;
    double csum = 0.0;
    for (int i = lane; i < ns; i += TEAM) {
        const double* th = M.th + i;
        double cp, h, s, dcp;
        if (M.th_np == 4) {
#define TH(k) __ldg(th + (k) * ns)
            cp = TH(TH_A1) + T * (TH(TH_A2) + T * (TH(TH_A3) + T * (TH(TH_A4) + T * TH(TH_A5))));
            h = TH(TH_A1) + T * (TH(TH_H2) + T * (TH(TH_H3) + T * (TH(TH_H4) + T * TH(TH_H5))))
                + TH(TH_A6) * invT;
            s = TH(TH_A1) * lnT
                + T * (TH(TH_A2) + T * (TH(TH_S3) + T * (TH(TH_S4) + T * TH(TH_S5)))) + TH(TH_A7);
            dcp = TH(TH_A2) + T * (TH(TH_D3) + T * (TH(TH_D4) + T * TH(TH_D5)));
#undef TH
        } else {
            thermo_cp_h_deg(th, ns, M.th_np, T, invT, cp, h);
            thermo_s_dcp_deg(th, ns, M.th_np, T, lnT, s, dcp);
        }
        hRT[i] = h;
        gRT[i] = h - s;
        cpR[i] = cp;
        dcpR[i] = dcp;
        csum += C[i];
    }
    // SP visible to the whole team: the block barriers of team_sum, or one
    // warp barrier
    const double Mc = team_sum<TEAM>(csum, W.red);
    if constexpr (TEAM == 32) team_sync<TEAM>();
    const double lnPRT = M.ln_pref_R - lnT;   // ln(p_ref / (R T))
    const double lnP = M.has_plog ? log(8314.46261815324 * T * Mc) : 0.0;   // ln p = ln(R T sum C)
    double* q = W.RD;
    double* dqdT = q + nr;
    double* wv = dqdT + nr;
    double* dd = wv + nr;
    const int wt = lane >> 5, l32 = lane & 31;
    const int c1 = __ldg(M.rc_ptr + wt + 1);
    for (int c = __ldg(M.rc_ptr + wt); c < c1; ++c) {
        if (l32 >= __ldg(M.rc_len + c)) continue;
        const int j = __ldg(M.rc_first + c) + l32;
        const int type = __ldg(M.rtype + j);
        const double bj = __ldg(M.beta + j), Taj = __ldg(M.Ta + j);
        const double kA = type == RXN_PLOG ? 0.0 : exp_tab(__ldg(M.lnA + j) + bj * lnT - Taj * invT, M.exp2j);
        const double dlnkA = (bj + Taj * invT) * invT;
        double kf, dkf_dT, dkf_dM = 0.0;
        if (type == RXN_PLOG) {
            // Section 2.2.4: ln k linear in ln p between the bracketing levels
            // (sum of a level's rates), the nearest level outside the range;
            // p = R T sum C, so k depends on C through sum C (dkf_dM)
            const int l0 = __ldg(M.pl_lev + j), l1 = __ldg(M.pl_lev + j + 1);
            int lb = l0;
            while (lb < l1 && __ldg(M.pl_lnp + lb) < lnP) ++lb;
            auto level = [&](int l, double& dlnk) {
                double k = 0.0, dk = 0.0;
                const int r1 = __ldg(M.pl_rate + l + 1);
                for (int r = __ldg(M.pl_rate + l); r < r1; ++r) {
                    const double br = __ldg(M.pl_b + r), Tr = __ldg(M.pl_Ta + r);
                    const double kr = exp_tab(__ldg(M.pl_lnA + r) + br * lnT - Tr * invT, M.exp2j);
                    k += kr;
                    dk = fma(kr, (br + Tr * invT) * invT, dk);
                }
                dlnk = dk / k;
                return k;
            };
            if (lb == l0 || lb == l1) {
                double d0;
                kf = level(lb == l0 ? l0 : l1 - 1, d0);
                dkf_dT = kf * d0;
            } else {
                double d0, d1;
                const double k0 = level(lb - 1, d0), k1 = level(lb, d1);
                const double p0 = __ldg(M.pl_lnp + lb - 1);
                const double idl = 1.0 / (__ldg(M.pl_lnp + lb) - p0);
                const double lk0 = log(k0), dlk = log(k1) - lk0;
                const double w = (lnP - p0) * idl;
                kf = exp(fma(dlk, w, lk0));
                const double sl = dlk * idl;
                dkf_dT = kf * (fma(w, d1 - d0, d0) + sl * invT);
                dkf_dM = kf * sl / Mc;
            }
            if (xf) xf[j] = 0.0;   // not set by (ln A, b, Ea)
        } else if (type == RXN_ELEM) {
            kf = kA;
            dkf_dT = kA * dlnkA;
            if (xf) xf[j] = 1.0;
        } else {
            double Mx = Mc;
            const int e1 = __ldg(M.eff_ptr + j + 1);
            for (int e = __ldg(M.eff_ptr + j); e < e1; ++e)
                Mx = fma(__ldg(M.eff_am1 + e), C[__ldg(M.eff_idx + e)], Mx);
            if (type == RXN_TB) {
                kf = Mx * kA;
                dkf_dT = kf * dlnkA;
                dkf_dM = kA;
                if (xf) xf[j] = 1.0;
            } else {
                const double db = __ldg(M.dbeta0 + j), dTa = __ldg(M.dTa0 + j);
                const double ratio = exp_tab(__ldg(M.dlnA0 + j) + db * lnT - dTa * invT, M.exp2j);   // k0 / kinf
                const double Pr = ratio * Mx;
                const double dlnr = (db + dTa * invT) * invT;
                double F = 1.0, dlogF_dP = 0.0, dlogF_dT = 0.0;   // log = log10
                if (type == RXN_TROE) {
                    const double al = __ldg(M.talpha + j);
                    const double i3 = __ldg(M.tiT3 + j), i1 = __ldg(M.tiT1 + j);
                    const double e3 = exp_tab(-T * i3, M.exp2j), e1x = exp_tab(-T * i1, M.exp2j);
                    double Fc = (1.0 - al) * e3 + al * e1x;
                    double dFc = -(1.0 - al) * i3 * e3 - al * i1 * e1x;
                    if (__ldg(M.hasT2 + j)) {
                        const double T2 = __ldg(M.tT2 + j);
                        const double e2 = exp_tab(-T2 * invT, M.exp2j);
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
                    F = exp_tab(kLn10 * logF, M.exp2j);
                    const double df1_dx = nn * rden * rden;
                    const double df1_dn = -x * rden * rden;
                    const double t2 = 2.0 * Lc * f1 * ig * ig;
                    dlogF_dP = clamp ? 0.0 : -t2 * df1_dx;
                    dlogF_dT = (ig - t2 * (-0.67 * df1_dx - 1.27 * df1_dn)) * dL_dT;
                } else if (type == RXN_SRI) {
                    // Section 2.2.3: F = d [a e^(-b/T) + e^(-T/c)]^X T^e, X = 1/(1 + log10^2 Pr)
                    const double a = __ldg(M.sri + j), bb = __ldg(M.sri + nr + j), ic = __ldg(M.sri + 2 * nr + j);
                    const double lnd = __ldg(M.sri + 3 * nr + j), ee = __ldg(M.sri + 4 * nr + j);
                    const bool clamp = !(Pr >= 1e-300);
                    const double P = log(clamp ? 1e-300 : Pr) * kInvLn10;
                    const double X = 1.0 / fma(P, P, 1.0);
                    const double ea = exp_tab(-bb * invT, M.exp2j), ec = exp_tab(-T * ic, M.exp2j);
                    const double G = fma(a, ea, ec);
                    const double dG = fma(a * bb * invT * invT, ea, -ic * ec);
                    const double lnG = log(G);
                    F = exp_tab(fma(X, lnG, fma(ee, lnT, lnd)), M.exp2j);
                    dlogF_dP = clamp ? 0.0 : lnG * kInvLn10 * (-2.0 * P * X * X);
                    dlogF_dT = fma(X, dG / G, ee * invT) * kInvLn10;
                }
                const double ip = 1.0 / (1.0 + Pr);
                kf = kA * (Pr * ip) * F;
                const double dkf_dPr = kA * F * ip * (ip + dlogF_dP);
                dkf_dT = kf * dlnkA + dkf_dPr * Pr * dlnr + kf * kLn10 * dlogF_dT;
                dkf_dM = dkf_dPr * ratio;
                // ln k_f = ln k_inf + ln(Pr/(1+Pr)) + ln F, Pr proportional to 1/k_inf
                if (xf) xf[j] = Pr * ip - dlogF_dP;
            }
        }
        if (M.slots == 2)
            progress_rate<2>(M, j, C, gRT, hRT, lnPRT, invT, kf, dkf_dT, dkf_dM, deriv, q, dqdT, wv, dd);
        else
            progress_rate<3>(M, j, C, gRT, hRT, lnPRT, invT, kf, dkf_dT, dkf_dM, deriv, q, dqdT, wv, dd);
    }
    team_sync<TEAM>();
    return Mc;
}

struct SrcInfo {
    double wT, Dt, Ws, Mc, sdil, cw, cdc;
};

// S = (omega_T, dC/dt) into W.S; y = (T, C).
template <int TEAM>
__device__ SrcInfo assemble_source(const DevMech& M, const Ws& W,const double* y,
                                   int reactor, double Mc, int lane) {
    const int ns = M.ns;
    double* S = W.S;
    double* red = W.red;
    const double* hRT = W.SP;
    const double* cpR = hRT + 2 * ns;
    const double* dcpR = cpR + ns;
    const double T = y[0];
    const double* C = y + 1;
    for (int i = lane; i < ns; i += TEAM) S[1 + i] = 0.0;
    team_sync<TEAM>();
    run_schedule<TEAM>(M.w_len, M.w_dst, M.w_src, M.w_fac, S, W.RD, lane);
    const double sub = reactor == R_CONV ? 1.0 : 0.0;   // u/RT = h/RT - 1, c_v/R = c_p/R - 1
    double qe = 0.0, den = 0.0, ws = 0.0, cw = 0.0, cdc = 0.0;
    for (int i = lane; i < ns; i += TEAM) {
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
    double sums[5] = {qe, den, ws, cw, cdc};
    team_sums<TEAM, 5>(sums, red);
    const double Qt = sums[0];
    si.Dt = sums[1];
    si.Ws = sums[2];
    si.cw = sums[3];
    si.cdc = sums[4];
    si.wT = -T * Qt / si.Dt;   // -sum e_i omega_i / (rho c), volumetric c
    si.sdil = 0.0;
    if (reactor == R_CONP) {
        si.sdil = si.wT / T + si.Ws / Mc;
        for (int i = lane; i < ns; i += TEAM) S[1 + i] = fma(-C[i], si.sdil, S[1 + i]);
    }
    if (lane == 0) S[0] = si.wT;
    team_sync<TEAM>();
    return si;
}

// Analytical Jacobian. With out == nullptr, writes the Newton matrix
// G = I - gh J into W.G (row stride W.ld) in the matrix type MT (FP64,
// or FP32 for the mixed-precision Newton); otherwise writes J to out
// (row-major n x n, global memory, MT = double).
template <int TEAM, class MT>
__device__ void assemble_jacobian(const DevMech& M, const Ws& W,const double* y,
                                  int reactor, const SrcInfo& si, double gh, double* out, int lane) {
    const int ns = M.ns, n = M.n, ld = W.ld;
    MT* G = reinterpret_cast<MT*>(W.G);
    double* V = W.V;
    const double* hRT = W.SP;
    const double* cpR = hRT + 2 * ns;
    const double* RD = W.RD;
    const double T = y[0];
    const double* C = y + 1;
    const double sub = reactor == R_CONV ? 1.0 : 0.0;

    // dense part of d omega / d C from third-body and falloff reactions
    for (int i = lane; i < ns; i += TEAM) V[i] = 0.0;
    team_sync<TEAM>();
    run_schedule<TEAM>(M.v_len, M.v_dst, M.v_src, M.v_fac, V, RD, lane);
    for (Flat2D it(lane, n, TEAM); it.r < ns; it.next())
        G[(1 + it.r) * ld + it.c] = static_cast<MT>(it.c == 0 ? 0.0 : V[it.r]);
    team_sync<TEAM>();
    // sparse part, reaction by reaction in a fixed order
    run_schedule<TEAM>(M.j_len, M.j_dst, M.j_src, M.j_fac, G, RD, lane);

    // temperature row: J_T,m = -(T A_m + omega_T c_m) / D (m > 0),
    // J_T,0 = -(sum c_i omega_i + T A_0 + omega_T sum C_i dc_i/dT) / D,
    // A_m = sum_i e_i dOmega_i/dy_m (e = u/RT or h/RT, c = c_v/R or c_p/R)
    double* JT = W.colA;
    double* ds = W.colB;
    double* eb = W.y1;   // e_i = u_i/RT or h_i/RT (y1 is free while Newton iterates)
    for (int i = lane; i < ns; i += TEAM) eb[i] = hRT[i] - sub;
    team_sync<TEAM>();
    const double invD = 1.0 / si.Dt;
    const bool conp = reactor == R_CONP;
    for (int m = lane; m < n; m += TEAM) {
        double a = 0.0, b = 0.0;
        if (conp) {
            for (int i = 0; i < ns; ++i) {
                const double g = static_cast<double>(G[(1 + i) * ld + m]);
                a = fma(eb[i], g, a);
                b += g;
            }
        } else {
            for (int i = 0; i < ns; ++i) a = fma(eb[i], static_cast<double>(G[(1 + i) * ld + m]), a);
        }
        double jt;
        if (m == 0) jt = -(si.cw + T * a + si.wT * si.cdc) * invD;
        else jt = -(T * a + si.wT * (cpR[m - 1] - sub)) * invD;
        JT[m] = jt;
        if (conp) {
            // s = omega_T / T + sum omega / sum C;  ds/dy_m
            double d = jt / T + b / si.Mc;
            if (m == 0) d -= si.wT / (T * T);
            else d -= si.Ws / (si.Mc * si.Mc);
            ds[m] = d;
        }
    }
    team_sync<TEAM>();
    if (out) {
        for (Flat2D it(lane, n, TEAM); it.r < n; it.next()) {
            const int r = it.r, c = it.c;
            double J;
            if (r == 0) {
                J = JT[c];
            } else {
                J = static_cast<double>(G[r * ld + c]);
                if (conp) {
                    J = fma(-C[r - 1], ds[c], J);
                    if (c == r) J -= si.sdil;
                }
            }
            out[r * n + c] = J;
        }
    } else {
        // G = I - gh J: the off-diagonal entries, then the diagonal (with the
        // dilution term -s) in a pass of its own, so that the n^2 pass
        // carries no diagonal-only arithmetic; the same operations per entry
        for (Flat2D it(lane, n, TEAM); it.r < n; it.next()) {
            const int r = it.r, c = it.c;
            if (r == c) continue;
            double J;
            if (r == 0) {
                J = JT[c];
            } else {
                J = static_cast<double>(G[r * ld + c]);
                if (conp) J = fma(-C[r - 1], ds[c], J);
            }
            G[r * ld + c] = static_cast<MT>(fma(-gh, J, 0.0));
        }
        for (int r = lane; r < n; r += TEAM) {
            double J;
            if (r == 0) {
                J = JT[0];
            } else {
                J = static_cast<double>(G[r * ld + r]);
                if (conp) {
                    J = fma(-C[r - 1], ds[r], J);
                    J -= si.sdil;
                }
            }
            G[r * ld + r] = static_cast<MT>(fma(-gh, J, 1.0));
        }
    }
    team_sync<TEAM>();
}

// ---------------------------------------------------------------------------
// dense LU with partial pivoting (Section 3.4), in place, team-cooperative

// |x| as an unsigned integer with the order of |x| (non-negative IEEE values
// order like their bit patterns)
static __device__ __forceinline__ unsigned long long abs_key(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
static __device__ __forceinline__ unsigned long long abs_key(float x) {
    return (unsigned long long)((unsigned)__float_as_int(x) & 0x7fffffffu);
}

// Column k of the factorisation: pivot = the largest |G_ik|, i >= k (ties to
// the lowest row; non-negative IEEE values order like their bit patterns),
// whole rows k and pivot swapped, inverse pivot into rinv[k], column scaled
// below the pivot. False on an exact zero pivot. Ends synchronised.
template <int TEAM, class MT>
__device__ __forceinline__ bool lu_pivot_column(MT* G, int n, int ld, int k, int* piv, double* rinv, double* red,
                                                int lane) {
    unsigned long long best = 0ull;
    int bi = n;
    for (int i = k + lane; i < n; i += TEAM) {
        const unsigned long long b = abs_key(G[i * ld + k]);
        if (bi == n || b > best) { best = b; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(kFull, best, o);
        const int oi = __shfl_xor_sync(kFull, bi, o);
        if (oi < n && (bi == n || ob > best || (ob == best && oi < bi))) { best = ob; bi = oi; }
    }
    if constexpr (TEAM > 32) {
        unsigned long long* rb = reinterpret_cast<unsigned long long*>(red + 8);
        int* ri = reinterpret_cast<int*>(red + 16);
        const int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) { rb[w] = best; ri[w] = bi; }
        __syncthreads();
        best = rb[0];
        bi = ri[0];
#pragma unroll
        for (int v = 1; v < TEAM / 32; ++v) {
            const unsigned long long ob = rb[v];
            const int oi = ri[v];
            if (oi < n && (bi == n || ob > best || (ob == best && oi < bi))) { best = ob; bi = oi; }
        }
    }
    if (lane == 0) piv[k] = bi;
    if (bi != k) {
        for (int j = lane; j < n; j += TEAM) {
            const MT t = G[k * ld + j];
            G[k * ld + j] = G[bi * ld + j];
            G[bi * ld + j] = t;
        }
    }
    team_sync<TEAM>();
    const MT pv = G[k * ld + k];
    if (abs_key(pv) == 0ull) return false;   // exact zero pivot (integer test)
    // The first warp forms the reciprocal and scales the column; an FP64
    // instruction costs the same for one lane as for 32, so the other
    // warps of the team would only repeat it. The FP32 factorisation keeps
    // its inverse pivots in FP32 (in the first n floats of rinv): the
    // correctly rounded FP32 reciprocal, no FP64 instruction.
    if (lane < 32) {
        if constexpr (sizeof(MT) == 8) {
            const double r = rcp_nr(static_cast<double>(pv));
            if (lane == 0) rinv[k] = r;
            for (int i = k + 1 + lane; i < n; i += 32) G[i * ld + k] *= r;
        } else {
            const float r = __frcp_rn(pv);
            if (lane == 0) reinterpret_cast<float*>(rinv)[k] = r;
            for (int i = k + 1 + lane; i < n; i += 32) G[i * ld + k] *= r;
        }
    }
    team_sync<TEAM>();
    return true;
}

// MT = double: the FP64 factorisation; MT = float: the FP32 factorisation
// of the mixed-precision Newton (inverse pivots kept in FP64 for the solves).
// Unblocked: after each column, the rank-one update of the whole trailing
// block.
template <int TEAM, class MT>
__device__ bool lu_factor(MT* G, int n, int ld, int* piv, double* rinv, double* red, int lane) {
    for (int k = 0; k < n; ++k) {
        if (!lu_pivot_column<TEAM, MT>(G, n, ld, k, piv, rinv, red, lane)) return false;
        const int m = n - k - 1;
        if (m > 0) {
            const int k1 = k + 1;
            const MT* Uk = G + k * ld + k1;   // pivot row, right of the pivot
            MT* B = G + k1 * ld;              // trailing block, rows k+1 .. n-1
            const int total = m * m;
            Flat2D it(lane, m, TEAM);
            int e = lane;
            for (; e + 3 * TEAM < total; e += 4 * TEAM) {   // four elements, all in range, loads first
                int o[4], c[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    o[u] = it.r * ld;
                    c[u] = it.c;
                    it.next();
                }
                MT l[4], uu[4], a[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    l[u] = B[o[u] + k];
                    uu[u] = Uk[c[u]];
                    a[u] = B[o[u] + c[u] + k1];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) B[o[u] + c[u] + k1] = fma(-l[u], uu[u], a[u]);
            }
            for (; e < total; e += TEAM) {                   // the remaining 0-3 elements
                const int o = it.r * ld;
                B[o + it.c + k1] = fma(-B[o + k], Uk[it.c], B[o + it.c + k1]);
                it.next();
            }
        }
        team_sync<TEAM>();
    }
    return true;
}

// Right-looking blocked LU with partial pivoting (Section 3.4), in place,
// team-cooperative, panels of nb columns. Within a panel each column is
// pivoted (whole rows swapped) and scaled, and its rank-one update goes to
// the panel's own columns only; columns right of the panel are left as they
// are until the panel is done (a later pivot of the panel may swap any two
// of its rows). Then U12 = L11^{-1} A12 by forward substitution, one column
// per thread, and the trailing block takes the panel's nb rank-one updates
// at once: A22 -= L21 U12, each thread accumulating an RA x CB tile in
// registers (rows tr + a TRn, columns tc + b TCn of the tile grid, so that
// neighbouring threads touch neighbouring columns). Every element receives
// the same fused multiply-adds, in the same order and rounded to MT after
// each, as in lu_factor: the factors and pivots are identical to the last
// bit. The tile keeps the panel's rows and columns in registers, so the
// trailing update reads (RA + CB) / (RA CB) operands from shared memory per
// multiply-add instead of three reads and one write.
template <int TEAM, class MT, int RA, int CB>
__device__ bool lu_factor_blocked(MT* G, int n, int ld, int nb, int* piv, double* rinv, double* red, int lane) {
    for (int k0 = 0; k0 < n; k0 += nb) {
        const int kend = k0 + nb < n ? k0 + nb : n;
        for (int k = k0; k < kend; ++k) {
            if (!lu_pivot_column<TEAM, MT>(G, n, ld, k, piv, rinv, red, lane)) return false;
            const int w = kend - k - 1;   // panel columns right of k
            if (w > 0) {
                const int h = n - k - 1;
                for (Flat2D it(lane, w, TEAM); it.r < h; it.next()) {
                    MT* row = G + (k + 1 + it.r) * ld;
                    const int c = k + 1 + it.c;
                    row[c] = fma(-row[k], G[k * ld + c], row[c]);
                }
            }
            team_sync<TEAM>();
        }
        const int m = n - kend;
        if (m <= 0) break;
        // U12: rows k0+1 .. kend-1 of the columns right of the panel, each
        // element updated by the panel rows above it in order
        for (int c = kend + lane; c < n; c += TEAM)
            for (int i = k0 + 1; i < kend; ++i) {
                MT a = G[i * ld + c];
                for (int j = k0; j < i; ++j) a = fma(-G[i * ld + j], G[j * ld + c], a);
                G[i * ld + c] = a;
            }
        team_sync<TEAM>();
        const int kb = kend - k0;
        const int TRn = (m + RA - 1) / RA, TCn = (m + CB - 1) / CB;
        const MT* L21 = G + kend * ld + k0;   // L21[i * ld + j]: row kend + i, column k0 + j
        const MT* U12 = G + k0 * ld + kend;   // U12[j * ld + c]: row k0 + j, column kend + c
        MT* A22 = G + kend * ld + kend;
        for (int t = lane; t < TRn * TCn; t += TEAM) {
            const int tr = t / TCn, tc = t - tr * TCn;
            int ro[RA], co[CB];
            bool rv[RA], cv[CB];
#pragma unroll
            for (int a = 0; a < RA; ++a) {
                const int r = tr + a * TRn;
                rv[a] = r < m;
                ro[a] = (rv[a] ? r : m - 1) * ld;   // rows past the end read the last row, store nothing
            }
#pragma unroll
            for (int b = 0; b < CB; ++b) {
                const int c = tc + b * TCn;
                cv[b] = c < m;
                co[b] = cv[b] ? c : m - 1;
            }
            MT acc[RA][CB];
#pragma unroll
            for (int a = 0; a < RA; ++a)
#pragma unroll
                for (int b = 0; b < CB; ++b) acc[a][b] = A22[ro[a] + co[b]];
            for (int j = 0; j < kb; ++j) {
                MT l[RA], u[CB];
#pragma unroll
                for (int a = 0; a < RA; ++a) l[a] = L21[ro[a] + j];
#pragma unroll
                for (int b = 0; b < CB; ++b) u[b] = U12[j * ld + co[b]];
#pragma unroll
                for (int a = 0; a < RA; ++a)
#pragma unroll
                    for (int b = 0; b < CB; ++b)
                        acc[a][b] = fma(-l[a], u[b], acc[a][b]);
            }
#pragma unroll
            for (int a = 0; a < RA; ++a)
#pragma unroll
                for (int b = 0; b < CB; ++b)
                    if (rv[a] && cv[b]) A22[ro[a] + co[b]] = acc[a][b];
        }
        team_sync<TEAM>();
    }
    return true;
}

// The factorisation of the Newton matrix: blocked with panels of nb columns
// (register tiles of 4 x 4), or unblocked for nb = 0; identical factors.
template <int TEAM, class MT>
__device__ __forceinline__ bool lu_factor_nb(MT* G, int n, int ld, int nb, int* piv, double* rinv, double* red,
                                             int lane) {
    if (nb > 0) return lu_factor_blocked<TEAM, MT, 4, 4>(G, n, ld, nb, piv, rinv, red, lane);
    return lu_factor<TEAM, MT>(G, n, ld, piv, rinv, red, lane);
}

// x <- G^{-1} x with the FP64 factors of lu_factor (FP64 arithmetic on x).
template <int TEAM, class MT>
__device__ void lu_solve(const MT* G, int n, int ld, const int* piv, const double* rinv,
                         double* x, int lane) {
    if (lane == 0)
        for (int k = 0; k < n; ++k) {
            const int p = piv[k];
            if (p != k) { const double t = x[k]; x[k] = x[p]; x[p] = t; }
        }
    team_sync<TEAM>();
    for (int j = 0; j < n - 1; ++j) {           // unit lower triangle, by columns
        const double xj = x[j];
        for (int i = j + 1 + lane; i < n; i += TEAM)
            x[i] = fma(-static_cast<double>(G[i * ld + j]), xj, x[i]);
        team_sync<TEAM>();
    }
    for (int j = n - 1; j >= 0; --j) {          // upper triangle, by columns
        if (lane == 0) x[j] *= rinv[j];
        team_sync<TEAM>();
        const double xj = x[j];
        for (int i = lane; i < j; i += TEAM) x[i] = fma(-static_cast<double>(G[i * ld + j]), xj, x[i]);
        team_sync<TEAM>();
    }
}

// x <- G^{-1} x with FP32 factors, in FP32 arithmetic (xs: n floats of
// scratch): the application of the FP32 preconditioner of the inexact
// Newton. x (the FP64 residual) is permuted, rounded to FP32, solved, and
// widened back; the Newton update, residual and convergence test stay FP64,
// so the iteration's fixed point is the FP64 one. rinv: the FP32 inverse
// pivots of lu_pivot_column<TEAM, float>.
template <int TEAM>
__device__ void lu_solve_f32(const float* G, int n, int ld, const int* piv, const float* rinv, double* x, float* xs,
                             int lane) {
    if (lane == 0)
        for (int k = 0; k < n; ++k) {
            const int p = piv[k];
            if (p != k) { const double t = x[k]; x[k] = x[p]; x[p] = t; }
        }
    team_sync<TEAM>();
    for (int i = lane; i < n; i += TEAM) xs[i] = static_cast<float>(x[i]);
    team_sync<TEAM>();
    for (int j = 0; j < n - 1; ++j) {           // unit lower triangle, by columns
        const float xj = xs[j];
        for (int i = j + 1 + lane; i < n; i += TEAM) xs[i] = fmaf(-G[i * ld + j], xj, xs[i]);
        team_sync<TEAM>();
    }
    for (int j = n - 1; j >= 0; --j) {          // upper triangle, by columns
        if (lane == 0) xs[j] *= rinv[j];
        team_sync<TEAM>();
        const float xj = xs[j];
        for (int i = lane; i < j; i += TEAM) xs[i] = fmaf(-G[i * ld + j], xj, xs[i]);
        team_sync<TEAM>();
    }
    for (int i = lane; i < n; i += TEAM) x[i] = static_cast<double>(xs[i]);
    team_sync<TEAM>();
}

// x <- G^{-T} x with the factors of lu_factor: with P G = L U, G^T = U^T L^T P,
// so solve U^T v = x (forward, by rows of U), L^T z = v (backward, by rows
// of L), then undo the row interchanges in reverse order.
template <int TEAM, class MT>
__device__ void lu_solve_t(const MT* G, int n, int ld, const int* piv, const double* rinv, double* x,
                           int lane) {
    for (int j = 0; j < n; ++j) {               // U^T: column j of U^T is row j of U
        const double vj = x[j] * rinv[j];
        team_sync<TEAM>();
        if (lane == 0) x[j] = vj;
        for (int i = j + 1 + lane; i < n; i += TEAM)
            x[i] = fma(-static_cast<double>(G[j * ld + i]), vj, x[i]);
        team_sync<TEAM>();
    }
    for (int j = n - 1; j > 0; --j) {           // L^T (unit diagonal): row j of L, columns < j
        const double zj = x[j];
        for (int i = lane; i < j; i += TEAM) x[i] = fma(-static_cast<double>(G[j * ld + i]), zj, x[i]);
        team_sync<TEAM>();
    }
    if (lane == 0)
        for (int k = n - 1; k >= 0; --k) {
            const int p = piv[k];
            if (p != k) { const double t = x[k]; x[k] = x[p]; x[p] = t; }
        }
    team_sync<TEAM>();
}

// ---------------------------------------------------------------------------
// GMRES (Section 3.4), run by one warp (l = lane within the warp)

// v <- M^{-1} v for M = I (prec 0), diag(G) (Jacobi, prec 1) or the lower
// triangle of G with its diagonal (Gauss-Seidel, prec 2, forward
// substitution by columns); dinv = 1 / diag(G).
template <class MT>
__device__ void warp_precondition(const MT* G, int n, int ld, const double* dinv, int prec, double* v, int l) {
    if (prec == 1) {
        for (int i = l; i < n; i += 32) v[i] *= dinv[i];
    } else if (prec == 2) {
        for (int j = 0; j < n; ++j) {
            if (l == 0) v[j] *= dinv[j];
            __syncwarp();
            const double vj = v[j];
            for (int i = j + 1 + l; i < n; i += 32) v[i] = fma(-static_cast<double>(G[i * ld + j]), vj, v[i]);
        }
    }
    __syncwarp();
}

// out = G v, one row per lane at a time, four partial sums for independent FMAs.
template <class MT>
__device__ void warp_matvec(const MT* G, int n, int ld, const double* v, double* out, int l) {
    for (int i = l; i < n; i += 32) {
        const MT* row = G + i * ld;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int c = 0;
        for (; c + 4 <= n; c += 4) {
            s0 = fma(static_cast<double>(row[c]), v[c], s0);
            s1 = fma(static_cast<double>(row[c + 1]), v[c + 1], s1);
            s2 = fma(static_cast<double>(row[c + 2]), v[c + 2], s2);
            s3 = fma(static_cast<double>(row[c + 3]), v[c + 3], s3);
        }
        for (; c < n; ++c) s0 = fma(static_cast<double>(row[c]), v[c], s0);
        out[i] = (s0 + s1) + (s2 + s3);
    }
    __syncwarp();
}

static __device__ __forceinline__ double warp_dot(const double* a, const double* b, int n, int l) {
    double s = 0.0;
    for (int i = l; i < n; i += 32) s = fma(a[i], b[i], s);
    return warp_sum(s);
}

// Workspace of warp_gmres: V[(m+1) vs] (Krylov basis, odd row stride vs),
// K[(m+1) m + 2m + 2(m+1)] (Hessenberg matrix, Givens cosines and sines,
// right-hand side g, projections), bb and w: n each.
struct GmresWs {
    double *V, *H, *cs, *sn, *g, *t, *bb, *w;
    int vs, m;
};

// Restarted GMRES with left preconditioning: M^{-1} G x = M^{-1} b from
// x0 = 0; Arnoldi by classical Gram-Schmidt applied twice (each lane forms
// whole dot products with its basis vectors, so one pass needs no
// reduction); Givens rotations for the least-squares problem (lane 0);
// converged when the preconditioned residual is at most tol ||M^{-1} b||.
// x: b in, solution out. Returns false when maxit iterations do not
// converge or a rotation degenerates. `iters` receives the iterations.
template <class MT>
__device__ bool warp_gmres(const MT* G, int n, int ld, const double* dinv, int prec, int maxit, double tol,
                           double* x, const GmresWs& K, int l, int& iters) {
    const int m = K.m, vs = K.vs;
    double* const bb = K.bb;
    double* const w = K.w;
    iters = 0;
    for (int i = l; i < n; i += 32) {
        bb[i] = x[i];
        w[i] = x[i];
        x[i] = 0.0;
    }
    __syncwarp();
    warp_precondition<MT>(G, n, ld, dinv, prec, w, l);
    const double bnorm = sqrt(warp_dot(w, w, n, l));
    if (bnorm == 0.0) return true;
    const double stop = tol * bnorm;
    bool first = true;
    while (true) {
        if (!first) {   // w = M^{-1} (b - G x)
            warp_matvec<MT>(G, n, ld, x, w, l);
            for (int i = l; i < n; i += 32) w[i] = bb[i] - w[i];
            __syncwarp();
            warp_precondition<MT>(G, n, ld, dinv, prec, w, l);
        }
        first = false;
        const double beta = sqrt(warp_dot(w, w, n, l));
        if (beta <= stop) return true;
        if (iters >= maxit) return false;
        const double ib = 1.0 / beta;
        for (int i = l; i < n; i += 32) K.V[i] = w[i] * ib;
        for (int q = l; q <= m; q += 32) K.g[q] = q == 0 ? beta : 0.0;
        __syncwarp();
        int k = 0;
        for (int j = 0; j < m && iters < maxit; ++j) {
            const double* vj = K.V + j * vs;
            warp_matvec<MT>(G, n, ld, vj, w, l);
            warp_precondition<MT>(G, n, ld, dinv, prec, w, l);
            ++iters;
            for (int pass = 0; pass < 2; ++pass) {   // classical Gram-Schmidt, twice
                for (int q = l; q <= j; q += 32) {
                    const double* vq = K.V + q * vs;
                    double s = 0.0;
                    for (int i = 0; i < n; ++i) s = fma(w[i], vq[i], s);
                    K.t[q] = s;
                    K.H[q * m + j] = pass == 0 ? s : K.H[q * m + j] + s;
                }
                __syncwarp();
                for (int i = l; i < n; i += 32) {
                    double v = w[i];
                    for (int q = 0; q <= j; ++q) v = fma(-K.t[q], K.V[q * vs + i], v);
                    w[i] = v;
                }
                __syncwarp();
            }
            const double hn = sqrt(warp_dot(w, w, n, l));
            if (hn > 0.0) {
                const double ih = 1.0 / hn;
                for (int i = l; i < n; i += 32) K.V[(j + 1) * vs + i] = w[i] * ih;
            }
            if (l == 0) {
                double* Hc = K.H + j;   // column j, rows q at Hc[q * m]
                Hc[(j + 1) * m] = hn;
                for (int q = 0; q < j; ++q) {
                    const double a = Hc[q * m], b = Hc[(q + 1) * m];
                    Hc[q * m] = fma(K.cs[q], a, K.sn[q] * b);
                    Hc[(q + 1) * m] = fma(-K.sn[q], a, K.cs[q] * b);
                }
                const double a = Hc[j * m], b = hn;
                const double rho = sqrt(fma(a, a, b * b));
                const double c = rho > 0.0 ? a / rho : 0.0, s = rho > 0.0 ? b / rho : 0.0;
                K.cs[j] = c;
                K.sn[j] = s;
                Hc[j * m] = rho;
                Hc[(j + 1) * m] = 0.0;
                K.g[j + 1] = -s * K.g[j];
                K.g[j] *= c;
            }
            __syncwarp();
            if (!(K.H[j * m + j] > 0.0)) return false;   // degenerate rotation
            k = j + 1;
            if (fabs(K.g[j + 1]) <= stop || hn == 0.0) break;
        }
        if (l == 0)   // H y = g (upper triangular), y into t
            for (int q = k - 1; q >= 0; --q) {
                double s = K.g[q];
                for (int c = q + 1; c < k; ++c) s = fma(-K.H[q * m + c], K.t[c], s);
                K.t[q] = s / K.H[q * m + q];
            }
        __syncwarp();
        for (int i = l; i < n; i += 32) {
            double v = x[i];
            for (int q = 0; q < k; ++q) v = fma(K.t[q], K.V[q * vs + i], v);
            x[i] = v;
        }
        __syncwarp();
    }
}

// weighted RMS norm with w_i = atol + rtol max(|a_i|, |b_i|)
template <int TEAM>
__device__ __forceinline__ double wrms(const double* v, const double* a, const double* b, int n,
                                       double rtol, double atol, double* red, int lane) {
    double s = 0.0;
    for (int i = lane; i < n; i += TEAM) {
        const double w = atol + rtol * fmax(fabs(a[i]), fabs(b[i]));
        const double r = v[i] / w;
        s = fma(r, r, s);
    }
    return sqrt(team_sum<TEAM>(s, red) / n);
}

}  // namespace cg
