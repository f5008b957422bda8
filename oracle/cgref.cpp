// ORACLE -- test infrastructure only.
//
// A plain, slow, FP64 CPU restatement of the per-cell chemistry of ChemGen
// (arXiv 2510.10005): thermodynamics (Section 2.1, Table 1), reaction rates
// (Section 2.2), the temperature source (Section 3, eq. temperature_source;
// Appendix B, eq. temperature_source_h), the analytical Jacobian (Section 3.2,
// eqs. derivative_matrices_temp_evol ff.), a dense direct solver (Section 3.4),
// temperature recovery (Section 2.1, eqs. temperature-nonlinear ff.),
// backward Euler with Newton (Section 3.2, eqs. Backward_euler,
// newtons-method-2, jacobian) and the SDIRK schemes in stage-derivative form
// (Appendix A.1, A.2), plus the step-size control the paper leaves open.
//
// It is the reference the CUDA path is checked against. Only the tests, the
// smoke check and the CPU baseline of the benchmark may load it. It shares no
// code, header or table with the CUDA library: the two are written
// independently from the paper. One cell is processed at a time, in the
// order the paper writes the steps; there is no blocking, fusion or reordering.
//
// Units: SI-kmol (C in kmol/m^3, Ea in J/kmol, p in Pa, W in kg/kmol).
// State y = (T, C_1..C_ns) (eq. extracted_problem-1); S = (omega_T, omega_i).

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

typedef std::complex<double> cplx;

const double R_U = 8314.46261815324;   // universal gas constant, J/(kmol K)
const double P_REF = 101325.0;         // reference pressure, 1 atm (Section 2.1)
const double LN10 = 2.302585092994045684;

enum { ELEMENTARY = 0, THREE_BODY = 1, LINDEMANN = 2, TROE = 3, SRI = 4, PLOG = 5 };
enum { CONV = 0, CONP = 1, CONP_LITERAL = 2 };
enum { ST_OK = 0, ST_NEWTON_FAIL = 1, ST_STEP_TOO_SMALL = 2, ST_MAX_STEPS = 3, ST_NONFINITE = 4 };

inline double re(double x) { return x; }
inline double re(const cplx& x) { return x.real(); }

struct Reaction {
    int type = ELEMENTARY;
    int reversible = 1;
    int f_idx[3], f_nu[3], r_idx[3], r_nu[3];
    double lnA, b, Ea;          // Arrhenius (k_inf for falloff)
    double lnA0, b0, Ea0;       // low-pressure limit k_0
    double alpha, T3, T1, T2;   // Troe parameters
    bool has_T2 = false;
    std::vector<int> eff_sp;    // third-body efficiencies different from 1
    std::vector<double> eff_val;
    double sri[5] = {0, 0, 0, 0, 0};   // SRI a, b, c, d, e (Section 2.2.3)
    // PLOG rate expressions (Section 2.2.4), sorted by pressure; equal
    // pressures repeat (their rates add)
    std::vector<double> pl_lnp, pl_lnA, pl_b, pl_Ea;
    int sum_nu = 0;             // sum_i nu_ij = sum nu^r - sum nu^f
};

// Mechanism with the coefficient sets of Table 1 in mass-specific form for a
// c_p polynomial of degree n_p (eq. specific_heat_polynomial). A NASA-7 range
// is the n_p = 4 instance: a_k = R_i * a_{k+1}^{NASA}, h_ref = R_i * a6,
// s_ref = R_i * a7; Appendix C.1 refits to other degrees.
struct Mech {
    int ns = 0, nr = 0;
    int np = 4;                               // degree of the c_p polynomial
    std::vector<double> W, Ri;
    std::vector<double> a, bc, cc, dc, fc;   // a, d: ns x (n_p+1); b, c, f: ns x (n_p+2)
    std::vector<Reaction> rx;
};

// ---------------------------------------------------------------------------
// Thermodynamics, Table 1 (Section 2.1). Each quantity is an inner product of
// its coefficients with a monomial basis in T.

template <class S> S poly(const double* coef, int deg, const S& T) {
    S out = 0.0, Tk = 1.0;
    for (int k = 0; k <= deg; ++k) { out += coef[k] * Tk; Tk *= T; }
    return out;
}

// c_p,i = sum_{k=0}^{n_p} a_ik T^k   (eq. specific_heat_polynomial)
template <class S> S cp_i(const Mech& m, int i, const S& T) {
    return poly(&m.a[(m.np + 1) * i], m.np, T);
}
// h_i = sum_{k=0}^{n_p+1} b_ik T^k   (eq. enthalpy-polynomial)
template <class S> S h_i(const Mech& m, int i, const S& T) {
    return poly(&m.bc[(m.np + 2) * i], m.np + 1, T);
}
// u_i = sum_{k=0}^{n_p+1} c_ik T^k   (eq. internal-energy-polynomial)
template <class S> S u_i(const Mech& m, int i, const S& T) {
    return poly(&m.cc[(m.np + 2) * i], m.np + 1, T);
}
// s_i^o = a_i0 ln T + sum_{k=0}^{n_p} d_ik T^k   (eq. entropy_polynomial)
template <class S> S s_i(const Mech& m, int i, const S& T, const S& lnT) {
    return m.a[(m.np + 1) * i] * lnT + poly(&m.dc[(m.np + 1) * i], m.np, T);
}
// g_i^o = -a_i0 T ln T + sum_{k=0}^{n_p+1} f_ik T^k   (eq. gibbs-polynomial)
template <class S> S g_i(const Mech& m, int i, const S& T, const S& lnT) {
    return -m.a[(m.np + 1) * i] * T * lnT + poly(&m.fc[(m.np + 2) * i], m.np + 1, T);
}
// c_v,i = c_p,i - R_i   (eq. cv_equation)
template <class S> S cv_i(const Mech& m, int i, const S& T) { return cp_i(m, i, T) - m.Ri[i]; }
// d c_p,i / dT
double dcp_i(const Mech& m, int i, double T) {
    const double* a = &m.a[(m.np + 1) * i];
    double out = 0.0, Tk = 1.0;
    for (int k = 1; k <= m.np; ++k) { out += k * a[k] * Tk; Tk *= T; }
    return out;
}

// The coefficient sets of Table 1 from a c_p polynomial of degree n_p given
// in molar form over R: coef[i*stride + k] = a_k of c_p/R (k = 0..n_p), then
// the constants of h/R and s/R (the NASA-7 a6, a7 when n_p = 4).
void set_thermo(Mech& m, int np, const double* coef, int stride) {
    const int ns = m.ns;
    m.np = np;
    m.a.assign((np + 1) * ns, 0.0); m.dc.assign((np + 1) * ns, 0.0);
    m.bc.assign((np + 2) * ns, 0.0); m.cc.assign((np + 2) * ns, 0.0); m.fc.assign((np + 2) * ns, 0.0);
    for (int i = 0; i < ns; ++i) {
        const double Ri = m.Ri[i];
        const double* nc = coef + stride * i;
        double* a = &m.a[(np + 1) * i];
        for (int k = 0; k <= np; ++k) a[k] = Ri * nc[k];       // c_p fit coefficients
        double href = Ri * nc[np + 1], sref = Ri * nc[np + 2];
        double* b = &m.bc[(np + 2) * i];                         // Table 1, h_i
        b[0] = href;
        for (int k = 1; k <= np + 1; ++k) b[k] = a[k - 1] / k;
        double* c = &m.cc[(np + 2) * i];                         // Table 1, u_i
        c[0] = href;
        c[1] = a[0] - Ri;
        for (int k = 2; k <= np + 1; ++k) c[k] = a[k - 1] / k;
        double* d = &m.dc[(np + 1) * i];                         // Table 1, s_i^o
        d[0] = sref;
        for (int k = 1; k <= np; ++k) d[k] = a[k] / k;
        double* f = &m.fc[(np + 2) * i];                         // Table 1, g_i^o
        f[0] = href;
        f[1] = a[0] - sref;
        for (int k = 2; k <= np + 1; ++k) f[k] = (1.0 / k - 1.0 / (k - 1)) * a[k - 1];
    }
}

// ---------------------------------------------------------------------------
// Rates (Section 2.2).

template <class S> S clamp_pr(const S& Pr) { return re(Pr) < 1e-300 ? S(1e-300) : Pr; }

// PLOG (Section 2.2.4, eq. plog_rate): the sum of the rate expressions
// given at one pressure level, from index i0; i1 receives the next level.
template <class S> S plog_level(const Reaction& r, int i0, int& i1, const S& T, const S& lnT) {
    S k = 0.0;
    int i = i0;
    for (; i < (int)r.pl_lnp.size() && r.pl_lnp[i] == r.pl_lnp[i0]; ++i)
        k += exp(r.pl_lnA[i] + r.pl_b[i] * lnT - r.pl_Ea[i] / (R_U * T));
    i1 = i;
    return k;
}

// k at the state's own pressure p = R T sum C: ln k interpolated linearly in
// ln p between the bracketing levels; the nearest level outside the range.
template <class S> S plog_rate(const Reaction& r, const S& T, const S& lnT, const S& Mc) {
    const S lnp = log(R_U * T * Mc);
    const int n = (int)r.pl_lnp.size();
    int i0 = 0, i1 = 0;
    S k0 = plog_level(r, 0, i1, T, lnT);
    if (re(lnp) <= r.pl_lnp[0]) return k0;
    while (i1 < n) {   // level [i0, i1) and the next one
        int i2 = 0;
        S k1 = plog_level(r, i1, i2, T, lnT);
        if (re(lnp) <= r.pl_lnp[i1]) {
            S w = (lnp - r.pl_lnp[i0]) / (r.pl_lnp[i1] - r.pl_lnp[i0]);
            return exp(log(k0) + (log(k1) - log(k0)) * w);
        }
        i0 = i1;
        i1 = i2;
        k0 = k1;
    }
    return k0;   // above the highest pressure
}

// SRI broadening (Section 2.2.3): F = d [a exp(-b/T) + exp(-T/c)]^X T^e,
// X = 1 / (1 + log10^2 Pr).
template <class S> S sri_F(const Reaction& r, const S& T, const S& Pr) {
    S P = log(clamp_pr(Pr)) / LN10;
    S X = 1.0 / (1.0 + P * P);
    S G = r.sri[0] * exp(-r.sri[1] / T) + exp(-T / r.sri[2]);
    return r.sri[3] * exp(X * log(G)) * exp(r.sri[4] * log(T));
}

// forward rate constant k_f and the effective third-body concentration
template <class S>
S forward_rate(const Reaction& r, const S& T, const S& lnT, const S* C, const S& Mc) {
    if (r.type == PLOG) return plog_rate(r, T, lnT, Mc);
    // k_A = A exp(b ln T - E/(R T))  (Section 2.2.1)
    S kA = exp(r.lnA + r.b * lnT - r.Ea / (R_U * T));
    if (r.type == ELEMENTARY) return kA;
    // [M] = M_c + sum (alpha_ij - 1) C_i  (eq. TB_optimization)
    S M = Mc;
    for (size_t e = 0; e < r.eff_sp.size(); ++e) M += (r.eff_val[e] - 1.0) * C[r.eff_sp[e]];
    if (r.type == THREE_BODY) return M * kA;
    // falloff: k_f = k_inf Pr/(1+Pr) F  (eq. falloff-reaction)
    S k0 = exp(r.lnA0 + r.b0 * lnT - r.Ea0 / (R_U * T));
    S Pr = k0 * M / kA;
    S F = 1.0;
    if (r.type == TROE) {
        // eq. f_and_fcent; alpha used in both terms of F_cent, T2 term dropped
        // when T2 is absent (Appendix C.1)
        S Fc = (1.0 - r.alpha) * exp(-T / r.T3) + r.alpha * exp(-T / r.T1);
        if (r.has_T2) Fc += exp(-r.T2 / T);
        S logFc = log(Fc) / LN10;
        S c = -0.4 - 0.67 * logFc;
        S n = 0.75 - 1.27 * logFc;
        S P = log(clamp_pr(Pr)) / LN10;
        S f1 = (P + c) / (n - 0.14 * (P + c));
        S logF = logFc / (1.0 + f1 * f1);
        F = exp(LN10 * logF);
    } else if (r.type == SRI) {
        F = sri_F(r, T, Pr);
    }
    return kA * (Pr / (1.0 + Pr)) * F;
}

// equilibrium constant, eq. equilibrium-constant-1 with molar Gibbs energies
template <class S>
S equilibrium_constant(const Mech& m, const Reaction& r, const S& T, const S* g) {
    S dG = 0.0;   // Delta G'_j = sum_i nu_ij W_i g_i^o  (molar)
    for (int s = 0; s < 3; ++s) {
        if (r.r_idx[s] >= 0) dG += double(r.r_nu[s]) * m.W[r.r_idx[s]] * g[r.r_idx[s]];
        if (r.f_idx[s] >= 0) dG -= double(r.f_nu[s]) * m.W[r.f_idx[s]] * g[r.f_idx[s]];
    }
    S K = exp(-dG / (R_U * T));
    // (p_ref / (R T))^{sum nu} as repeated multiplication (Section 2.2)
    S base = r.sum_nu >= 0 ? P_REF / (R_U * T) : (R_U * T) / P_REF;
    for (int k = 0; k < std::abs(r.sum_nu); ++k) K *= base;
    return K;
}

template <class S> S prod_conc(const int* idx, const int* nu, const S* C) {
    S p = 1.0;
    for (int s = 0; s < 3; ++s)
        if (idx[s] >= 0)
            for (int k = 0; k < nu[s]; ++k) p *= C[idx[s]];
    return p;
}

// Rates of progress q_j (eq. chemical-reaction-rate-of-progress).
template <class S>
void progress_rates(const Mech& m, const S& T, const S* C, S* kf_out, S* kr_out, S* q) {
    S lnT = log(T);
    S Mc = 0.0;
    for (int i = 0; i < m.ns; ++i) Mc += C[i];
    std::vector<S> g(m.ns);
    for (int i = 0; i < m.ns; ++i) g[i] = g_i(m, i, T, lnT);
    for (int j = 0; j < m.nr; ++j) {
        const Reaction& r = m.rx[j];
        S kf = forward_rate(r, T, lnT, C, Mc);
        S kr = 0.0;
        if (r.reversible) kr = kf / equilibrium_constant(m, r, T, g.data());   // eq. reverse_rate
        q[j] = kf * prod_conc(r.f_idx, r.f_nu, C) - kr * prod_conc(r.r_idx, r.r_nu, C);
        if (kf_out) kf_out[j] = kf;
        if (kr_out) kr_out[j] = kr;
    }
}

// Source term S(y) = (omega_T, dC/dt).
//   omega_i = sum_j nu_ij q_j.
//   CONV: omega_T = -sum W_i u_i omega_i / (rho c_v)  (eq. temperature_source)
//   CONP_LITERAL: omega_T = -sum W_i h_i omega_i / (rho c_p), dC/dt = omega
//       (Appendix B, eq. temperature_source_h, the rest unchanged)
//   CONP: same omega_T; dC_i/dt = omega_i - C_i (omega_T/T + sum omega/sum C),
//       the dilution of an ideal gas held at constant pressure.
// The c_v and c_p of the temperature source are volumetric: rho c = sum W_i C_i c_i.
template <class S>
void source(const Mech& m, int reactor, const S* y, S* out) {
    const S T = y[0];
    const S* C = y + 1;
    std::vector<S> q(m.nr), w(m.ns, S(0.0));
    progress_rates(m, T, C, (S*)nullptr, (S*)nullptr, q.data());
    for (int j = 0; j < m.nr; ++j) {
        const Reaction& r = m.rx[j];
        for (int s = 0; s < 3; ++s) {
            if (r.r_idx[s] >= 0) w[r.r_idx[s]] += double(r.r_nu[s]) * q[j];
            if (r.f_idx[s] >= 0) w[r.f_idx[s]] -= double(r.f_nu[s]) * q[j];
        }
    }
    S num = 0.0, den = 0.0;
    for (int i = 0; i < m.ns; ++i) {
        S e = reactor == CONV ? u_i(m, i, T) : h_i(m, i, T);
        S c = reactor == CONV ? cv_i(m, i, T) : cp_i(m, i, T);
        num += m.W[i] * e * w[i];
        den += m.W[i] * C[i] * c;
    }
    S wT = -num / den;
    out[0] = wT;
    if (reactor == CONP) {
        S sw = 0.0, sc = 0.0;
        for (int i = 0; i < m.ns; ++i) { sw += w[i]; sc += C[i]; }
        S dil = wT / T + sw / sc;
        for (int i = 0; i < m.ns; ++i) out[1 + i] = w[i] - C[i] * dil;
    } else {
        for (int i = 0; i < m.ns; ++i) out[1 + i] = w[i];
    }
}

// ---------------------------------------------------------------------------
// Analytical Jacobian J_ij = dS_i/dy_j (eq. derivative_matrices_temp_evol),
// with T and C independent state variables, row/column 0 = T.

// derivative of prod_s C^nu with respect to C_m (product rule, exact at C = 0)
double dprod(const int* idx, const int* nu, const double* C, int mcol) {
    double total = 0.0;
    for (int s = 0; s < 3; ++s) {
        if (idx[s] != mcol) continue;
        double p = nu[s];
        for (int k = 0; k < nu[s] - 1; ++k) p *= C[mcol];
        for (int t = 0; t < 3; ++t)
            if (t != s && idx[t] >= 0)
                for (int k = 0; k < nu[t]; ++k) p *= C[idx[t]];
        total += p;
    }
    return total;
}

void jacobian(const Mech& m, int reactor, const double* y, double* J) {
    const int ns = m.ns, n = ns + 1;
    const double T = y[0];
    const double* C = y + 1;
    const double lnT = std::log(T), RT = R_U * T;
    double Mc = 0.0;
    for (int i = 0; i < ns; ++i) Mc += C[i];
    std::vector<double> g(ns), h(ns);
    for (int i = 0; i < ns; ++i) { g[i] = g_i(m, i, T, lnT); h[i] = h_i(m, i, T); }

    // dw[i*n + col] = d omega_i / d y_col ; w = omega
    std::vector<double> dw(ns * n, 0.0), w(ns, 0.0), dq(n);
    for (int j = 0; j < m.nr; ++j) {
        const Reaction& r = m.rx[j];
        std::fill(dq.begin(), dq.end(), 0.0);
        double kA = std::exp(r.lnA + r.b * lnT - r.Ea / RT);
        double dkA = kA * (r.b / T + r.Ea / (R_U * T * T));
        double M = Mc;
        std::vector<double> alpha(ns, 1.0);
        for (size_t e = 0; e < r.eff_sp.size(); ++e) {
            M += (r.eff_val[e] - 1.0) * C[r.eff_sp[e]];
            alpha[r.eff_sp[e]] = r.eff_val[e];
        }
        double kf, dkf_dT, dkf_dM;
        if (r.type == PLOG) {
            // ln k = (1 - w) ln k_l + w ln k_{l+1}, w = (ln p - ln p_l)/(ln p_{l+1} - ln p_l),
            // ln p = ln(R T M_c): d ln k/dT = (1-w) dln k_l/dT + w dln k_{l+1}/dT + s/T,
            // d ln k/d M_c = s/M_c with s = (ln k_{l+1} - ln k_l)/(ln p_{l+1} - ln p_l)
            auto level = [&](int i0, int& i1, double& dlnk) {
                double k = 0.0, dk = 0.0;
                int i = i0;
                for (; i < (int)r.pl_lnp.size() && r.pl_lnp[i] == r.pl_lnp[i0]; ++i) {
                    double ki = std::exp(r.pl_lnA[i] + r.pl_b[i] * lnT - r.pl_Ea[i] / RT);
                    k += ki;
                    dk += ki * (r.pl_b[i] / T + r.pl_Ea[i] / (R_U * T * T));
                }
                i1 = i;
                dlnk = dk / k;
                return k;
            };
            const double lnp = std::log(RT * Mc);
            const int np = (int)r.pl_lnp.size();
            int i0 = 0, i1 = 0;
            double d0 = 0.0;
            double k0 = level(0, i1, d0);
            kf = k0; dkf_dT = k0 * d0; dkf_dM = 0.0;
            if (lnp > r.pl_lnp[0]) {
                while (i1 < np) {
                    int i2 = 0;
                    double d1 = 0.0;
                    double k1 = level(i1, i2, d1);
                    if (lnp <= r.pl_lnp[i1]) {
                        const double dl = r.pl_lnp[i1] - r.pl_lnp[i0];
                        const double w = (lnp - r.pl_lnp[i0]) / dl;
                        const double sl = (std::log(k1) - std::log(k0)) / dl;
                        kf = std::exp(std::log(k0) + (std::log(k1) - std::log(k0)) * w);
                        dkf_dT = kf * ((1.0 - w) * d0 + w * d1 + sl / T);
                        dkf_dM = kf * sl / Mc;
                        break;
                    }
                    i0 = i1; i1 = i2; k0 = k1; d0 = d1;
                    kf = k0; dkf_dT = k0 * d0; dkf_dM = 0.0;   // above the range: the last level
                }
            }
        } else if (r.type == ELEMENTARY) {
            kf = kA; dkf_dT = dkA; dkf_dM = 0.0;
        } else if (r.type == THREE_BODY) {
            kf = M * kA; dkf_dT = M * dkA; dkf_dM = kA;
        } else {
            double k0 = std::exp(r.lnA0 + r.b0 * lnT - r.Ea0 / RT);
            double Pr = k0 * M / kA;
            double dPr_dT = Pr * ((r.b0 - r.b) / T + (r.Ea0 - r.Ea) / (R_U * T * T));
            double dPr_dM = k0 / kA;
            double F = 1.0, dlogF_dP = 0.0, dlogF_dT = 0.0;   // log = log10
            if (r.type == TROE) {
                double e3 = std::exp(-T / r.T3), e1 = std::exp(-T / r.T1);
                double Fc = (1.0 - r.alpha) * e3 + r.alpha * e1;
                double dFc = -(1.0 - r.alpha) / r.T3 * e3 - r.alpha / r.T1 * e1;
                if (r.has_T2) {
                    double e2 = std::exp(-r.T2 / T);
                    Fc += e2;
                    dFc += r.T2 / (T * T) * e2;
                }
                double L = std::log10(Fc);
                double dL_dT = dFc / (Fc * LN10);
                double c = -0.4 - 0.67 * L, nn = 0.75 - 1.27 * L;
                bool clamped = Pr < 1e-300;
                double P = std::log10(clamped ? 1e-300 : Pr);
                double x = P + c, den = nn - 0.14 * x;
                double f1 = x / den;
                double g1 = 1.0 + f1 * f1;
                double logF = L / g1;
                F = std::pow(10.0, logF);
                double df1_dx = nn / (den * den);
                double df1_dn = -x / (den * den);
                double df1_dL = df1_dx * (-0.67) + df1_dn * (-1.27);
                dlogF_dP = clamped ? 0.0 : -L * 2.0 * f1 / (g1 * g1) * df1_dx;
                double dlogF_dL = 1.0 / g1 - L * 2.0 * f1 / (g1 * g1) * df1_dL;
                dlogF_dT = dlogF_dL * dL_dT;   // at fixed Pr
            } else if (r.type == SRI) {
                // log10 F = log10 d + X log10 G + e log10 T, X = 1/(1 + P^2)
                bool clamped = Pr < 1e-300;
                double P = std::log10(clamped ? 1e-300 : Pr);
                double X = 1.0 / (1.0 + P * P);
                double ea = std::exp(-r.sri[1] / T), ec = std::exp(-T / r.sri[2]);
                double G = r.sri[0] * ea + ec;
                double dG = r.sri[0] * r.sri[1] / (T * T) * ea - ec / r.sri[2];
                double logG = std::log10(G);
                F = r.sri[3] * std::pow(G, X) * std::pow(T, r.sri[4]);
                dlogF_dP = clamped ? 0.0 : logG * (-2.0 * P * X * X);
                dlogF_dT = X * dG / (G * LN10) + r.sri[4] / (T * LN10);
            }
            double fr = Pr / (1.0 + Pr);
            kf = kA * fr * F;
            // d kf / d Pr = kA F [1/(1+Pr)^2 + dlog10F/dlog10Pr / (1+Pr)]
            double dkf_dPr = kA * F * (1.0 / ((1.0 + Pr) * (1.0 + Pr)) + dlogF_dP / (1.0 + Pr));
            dkf_dT = dkA * fr * F + dkf_dPr * dPr_dT + kf * LN10 * dlogF_dT;
            dkf_dM = dkf_dPr * dPr_dM;
        }
        double pf = prod_conc(r.f_idx, r.f_nu, C), pr = prod_conc(r.r_idx, r.r_nu, C);
        double invK = 0.0, dlnK = 0.0;
        if (r.reversible) {
            invK = 1.0 / equilibrium_constant(m, r, T, g.data());
            // d ln K / dT = sum nu_i W_i h_i / (R T^2) - sum nu / T
            double dH = 0.0;
            for (int s = 0; s < 3; ++s) {
                if (r.r_idx[s] >= 0) dH += r.r_nu[s] * m.W[r.r_idx[s]] * h[r.r_idx[s]];
                if (r.f_idx[s] >= 0) dH -= r.f_nu[s] * m.W[r.f_idx[s]] * h[r.f_idx[s]];
            }
            dlnK = dH / (R_U * T * T) - r.sum_nu / T;
        }
        double phi = pf - pr * invK;
        double q = kf * phi;
        dq[0] = dkf_dT * phi + kf * pr * invK * dlnK;
        for (int mm = 0; mm < ns; ++mm) {
            double d = dkf_dM * alpha[mm] * phi;
            d += kf * (dprod(r.f_idx, r.f_nu, C, mm) - invK * dprod(r.r_idx, r.r_nu, C, mm));
            dq[1 + mm] = d;
        }
        for (int s = 0; s < 3; ++s) {
            for (int side = 0; side < 2; ++side) {
                int sp = side ? r.r_idx[s] : r.f_idx[s];
                if (sp < 0) continue;
                double nu = side ? r.r_nu[s] : -r.f_nu[s];
                w[sp] += nu * q;
                for (int col = 0; col < n; ++col) dw[sp * n + col] += nu * dq[col];
            }
        }
    }

    // temperature row: omega_T = -Q/D, Q = sum W e omega, D = sum W C c
    double Q = 0.0, D = 0.0, dD_dT = 0.0, dQ_dT = 0.0;
    std::vector<double> e(ns), c(ns);
    for (int i = 0; i < ns; ++i) {
        e[i] = reactor == CONV ? u_i(m, i, T) : h_i(m, i, T);
        c[i] = reactor == CONV ? cv_i(m, i, T) : cp_i(m, i, T);
        Q += m.W[i] * e[i] * w[i];
        D += m.W[i] * C[i] * c[i];
        dD_dT += m.W[i] * C[i] * dcp_i(m, i, T);
        dQ_dT += m.W[i] * c[i] * w[i] + m.W[i] * e[i] * dw[i * n];
    }
    double wT = -Q / D;
    J[0] = -dQ_dT / D + Q * dD_dT / (D * D);
    for (int mm = 0; mm < ns; ++mm) {
        double dQ = 0.0;
        for (int i = 0; i < ns; ++i) dQ += m.W[i] * e[i] * dw[i * n + 1 + mm];
        J[1 + mm] = -dQ / D + Q * m.W[mm] * c[mm] / (D * D);
    }
    for (int i = 0; i < ns; ++i)
        for (int col = 0; col < n; ++col) J[(1 + i) * n + col] = dw[i * n + col];

    if (reactor == CONP) {
        // dC_i/dt = omega_i - C_i s, s = omega_T/T + sum omega / sum C
        double sw = 0.0, sc = Mc;
        for (int i = 0; i < ns; ++i) sw += w[i];
        double sdil = wT / T + sw / sc;
        std::vector<double> ds(n);
        for (int col = 0; col < n; ++col) {
            double dsw = 0.0;
            for (int i = 0; i < ns; ++i) dsw += dw[i * n + col];
            ds[col] = J[col] / T + dsw / sc;
        }
        ds[0] -= wT / (T * T);
        for (int col = 1; col < n; ++col) ds[col] -= sw / (sc * sc);
        for (int i = 0; i < ns; ++i) {
            for (int col = 0; col < n; ++col) J[(1 + i) * n + col] -= C[i] * ds[col];
            J[(1 + i) * n + 1 + i] -= sdil;
        }
    }
}

// ---------------------------------------------------------------------------
// Dense direct solver (Section 3.4): LU with partial pivoting.

bool lu_factor(int n, double* A, int* piv) {
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i < n; ++i)
            if (std::fabs(A[i * n + k]) > std::fabs(A[p * n + k])) p = i;
        piv[k] = p;
        if (p != k)
            for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[p * n + j]);
        if (A[k * n + k] == 0.0) return false;
        for (int i = k + 1; i < n; ++i) {
            A[i * n + k] /= A[k * n + k];
            for (int j = k + 1; j < n; ++j) A[i * n + j] -= A[i * n + k] * A[k * n + j];
        }
    }
    return true;
}

void lu_solve(int n, const double* LU, const int* piv, double* b) {
    for (int k = 0; k < n; ++k) std::swap(b[k], b[piv[k]]);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j) b[i] -= LU[i * n + j] * b[j];
    for (int i = n - 1; i >= 0; --i) {
        for (int j = i + 1; j < n; ++j) b[i] -= LU[i * n + j] * b[j];
        b[i] /= LU[i * n + i];
    }
}

// ---------------------------------------------------------------------------
// Iterative solver (Section 3.4): restarted GMRES (Saad and Schultz 1986) with
// left preconditioning, M^{-1} A x = M^{-1} b, M = I (prec 0), the diagonal
// of A (Jacobi, prec 1) or the lower triangle of A with its diagonal
// (Gauss-Seidel, prec 2, applied by forward substitution). x0 = 0; Arnoldi
// by modified Gram-Schmidt; the small least-squares problem by Givens
// rotations; restart after m iterations. Converged when the preconditioned
// residual norm is at most tol ||M^{-1} b||. b in, x out; false when not
// converged within maxit iterations (or on a zero diagonal with a
// preconditioner). *iters receives the iterations taken.

void precondition(int n, const double* A, int prec, double* v) {
    if (prec == 1) {
        for (int i = 0; i < n; ++i) v[i] /= A[i * n + i];
    } else if (prec == 2) {
        for (int i = 0; i < n; ++i) {
            double s = v[i];
            for (int k = 0; k < i; ++k) s -= A[i * n + k] * v[k];
            v[i] = s / A[i * n + i];
        }
    }
}

bool gmres(int n, const double* A, double* b, int prec, int m, int maxit, double tol, int* iters) {
    *iters = 0;
    if (prec != 0)
        for (int i = 0; i < n; ++i)
            if (A[i * n + i] == 0.0) return false;
    std::vector<double> x(n, 0.0), r(n), w(n), g(m + 1), cs(m), sn(m), y(m);
    std::vector<std::vector<double>> V(m + 1, std::vector<double>(n));
    std::vector<std::vector<double>> H(m + 1, std::vector<double>(m, 0.0));
    auto norm = [&](const std::vector<double>& v) {
        double s = 0.0;
        for (double e : v) s += e * e;
        return std::sqrt(s);
    };
    r.assign(b, b + n);
    precondition(n, A, prec, r.data());
    const double bnorm = norm(r);
    if (bnorm == 0.0) {
        std::fill(b, b + n, 0.0);
        return true;
    }
    while (true) {
        // r = M^{-1} (b - A x)
        for (int i = 0; i < n; ++i) {
            double s = b[i];
            for (int k = 0; k < n; ++k) s -= A[i * n + k] * x[k];
            r[i] = s;
        }
        precondition(n, A, prec, r.data());
        const double beta = norm(r);
        if (beta <= tol * bnorm) break;
        if (*iters >= maxit) return false;
        for (int i = 0; i < n; ++i) V[0][i] = r[i] / beta;
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int k = 0;
        for (int j = 0; j < m && *iters < maxit; ++j) {
            for (int i = 0; i < n; ++i) {
                double s = 0.0;
                for (int c = 0; c < n; ++c) s += A[i * n + c] * V[j][c];
                w[i] = s;
            }
            precondition(n, A, prec, w.data());
            ++*iters;
            for (int q = 0; q <= j; ++q) {
                double h = 0.0;
                for (int i = 0; i < n; ++i) h += w[i] * V[q][i];
                H[q][j] = h;
                for (int i = 0; i < n; ++i) w[i] -= h * V[q][i];
            }
            const double hn = norm(w);
            H[j + 1][j] = hn;
            if (hn > 0.0)
                for (int i = 0; i < n; ++i) V[j + 1][i] = w[i] / hn;
            for (int q = 0; q < j; ++q) {   // earlier rotations on the new column
                const double t = cs[q] * H[q][j] + sn[q] * H[q + 1][j];
                H[q + 1][j] = -sn[q] * H[q][j] + cs[q] * H[q + 1][j];
                H[q][j] = t;
            }
            const double rho = std::hypot(H[j][j], H[j + 1][j]);
            if (rho == 0.0) return false;
            cs[j] = H[j][j] / rho;
            sn[j] = H[j + 1][j] / rho;
            H[j][j] = rho;
            H[j + 1][j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            k = j + 1;
            if (std::fabs(g[j + 1]) <= tol * bnorm || hn == 0.0) break;
        }
        for (int q = k - 1; q >= 0; --q) {   // H y = g, upper triangular
            double s = g[q];
            for (int c = q + 1; c < k; ++c) s -= H[q][c] * y[c];
            y[q] = s / H[q][q];
        }
        for (int q = 0; q < k; ++q)
            for (int i = 0; i < n; ++i) x[i] += y[q] * V[q][i];
    }
    std::copy(x.begin(), x.end(), b);
    return true;
}

// ---------------------------------------------------------------------------
// Integrators.

struct Tableau {
    int s;                 // stages
    double A[5][5];        // lower triangular incl. diagonal
    double b[5], bhat[5];  // weights and embedded weights
    int err_order;         // order of the embedded solution (controller exponent 1/(q+1))
};

struct Opts {
    int method;            // 0 BE, 1 SDIRK-2, 2 SDIRK-4, 3 Rosenbrock-2, 4 YASS
    int linear_solver;     // 0 dense LU, 1 GMRES (Section 3.4)
    int prec, gmres_m, gmres_maxit;   // GMRES: preconditioner, restart length, iteration limit
    double gmres_tol;
    int reactor;
    int adaptive;
    int nsub;              // fixed-step mode: number of equal steps
    double dt, rtol, atol, newton_tol, h0, hmin, neg_tol;
    int max_newton, max_steps, max_halvings, err_filter;
};

struct Stats { int steps = 0, rejects = 0, newton = 0, lu = 0; };

bool finite_vec(const std::vector<double>& v) {
    for (double x : v) if (!std::isfinite(x)) return false;
    return true;
}

// A converged step is admissible when T > 0 and no concentration is below
// -neg_tol * sum(C) (the paper does not say what to do with a Newton root
// outside the physical domain; such a step is treated as a failed step).
bool admissible(const std::vector<double>& y, double neg_tol) {
    if (!(y[0] > 0.0)) return false;
    double sc = 0.0;
    for (size_t i = 1; i < y.size(); ++i) sc += y[i];
    for (size_t i = 1; i < y.size(); ++i)
        if (y[i] < -neg_tol * sc) return false;
    return true;
}

double wrms(int n, const double* v, const double* ya, const double* yb, double rtol, double atol) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) {
        double w = atol + rtol * std::max(std::fabs(ya[i]), std::fabs(yb[i]));
        double r = v[i] / w;
        s += r * r;
    }
    return std::sqrt(s / n);
}

// ---------------------------------------------------------------------------
// Parameter derivatives for the adjoint and the forward sensitivity. The
// differentiated parameters of reaction j are theta_j = (ln A, b, Ea) of its
// Arrhenius triple (k_inf for falloff reactions, k_0 held fixed).

// dq_j / d ln k_j (with k_j the Arrhenius triple's rate): q_j itself for
// elementary and third-body reactions; for falloff, ln k_f = ln k_inf +
// ln(Pr/(1+Pr)) + ln F with Pr = k_0 [M] / k_inf, so the factor is
// Pr/(1+Pr) - dlog10F/dlog10Pr.
double dq_dlnk(const Mech& m, int j, double T, const double* C) {
    std::vector<double> q(m.nr);
    progress_rates(m, T, C, (double*)nullptr, (double*)nullptr, q.data());
    const Reaction& r = m.rx[j];
    if (r.type == ELEMENTARY || r.type == THREE_BODY) return q[j];
    if (r.type == PLOG) return 0.0;   // its own rate table, not (ln A, b, Ea), sets k
    double M = 0.0;
    for (int i = 0; i < m.ns; ++i) M += C[i];
    for (size_t e = 0; e < r.eff_sp.size(); ++e) M += (r.eff_val[e] - 1.0) * C[r.eff_sp[e]];
    const double lnT = std::log(T);
    const double kinf = std::exp(r.lnA + r.b * lnT - r.Ea / (R_U * T));
    const double k0 = std::exp(r.lnA0 + r.b0 * lnT - r.Ea0 / (R_U * T));
    const double Pr = k0 * M / kinf;
    double dlogF_dP = 0.0;
    if (r.type == TROE && Pr >= 1e-300) {
        double Fc = (1.0 - r.alpha) * std::exp(-T / r.T3) + r.alpha * std::exp(-T / r.T1);
        if (r.has_T2) Fc += std::exp(-r.T2 / T);
        const double L = std::log10(Fc);
        const double c = -0.4 - 0.67 * L, nn = 0.75 - 1.27 * L;
        const double x = std::log10(Pr) + c, den = nn - 0.14 * x;
        const double f1 = x / den;
        dlogF_dP = -L * 2.0 * f1 / ((1.0 + f1 * f1) * (1.0 + f1 * f1)) * nn / (den * den);
    }
    if (r.type == SRI && Pr >= 1e-300) {
        const double P = std::log10(Pr), X = 1.0 / (1.0 + P * P);
        const double G = r.sri[0] * std::exp(-r.sri[1] / T) + std::exp(-T / r.sri[2]);
        dlogF_dP = std::log10(G) * (-2.0 * P * X * X);
    }
    return q[j] * (Pr / (1.0 + Pr) - dlogF_dP);
}

// dS/dq_j for every reaction: column j of an n x nr matrix (row-major).
// Species rows: net coefficients nu_kj (CONP adds the dilution terms);
// temperature row: -sum_k W_k e_k nu_kj / (rho c).
void dS_dq(const Mech& m, int reactor, const double* y, std::vector<double>& out) {
    const int ns = m.ns, n = ns + 1, nr = m.nr;
    const double T = y[0];
    const double* C = y + 1;
    out.assign((size_t)n * nr, 0.0);
    std::vector<double> e(ns);
    double D = 0.0, sc = 0.0;
    for (int i = 0; i < ns; ++i) {
        e[i] = reactor == CONV ? u_i(m, i, T) : h_i(m, i, T);
        D += m.W[i] * C[i] * (reactor == CONV ? cv_i(m, i, T) : cp_i(m, i, T));
        sc += C[i];
    }
    for (int j = 0; j < nr; ++j) {
        const Reaction& r = m.rx[j];
        std::vector<double> nu(ns, 0.0);
        for (int s = 0; s < 3; ++s) {
            if (r.r_idx[s] >= 0) nu[r.r_idx[s]] += r.r_nu[s];
            if (r.f_idx[s] >= 0) nu[r.f_idx[s]] -= r.f_nu[s];
        }
        double dwT = 0.0, snu = 0.0;
        for (int k = 0; k < ns; ++k) { dwT -= m.W[k] * e[k] * nu[k] / D; snu += nu[k]; }
        out[(size_t)0 * nr + j] = dwT;
        for (int k = 0; k < ns; ++k) {
            double v = nu[k];
            if (reactor == CONP) v -= C[k] * (dwT / T + snu / sc);
            out[(size_t)(1 + k) * nr + j] = v;
        }
    }
}

void transpose_solve(int n, const double* G, std::vector<double>& x) {
    std::vector<double> Gt((size_t)n * n);
    std::vector<int> piv(n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Gt[(size_t)i * n + j] = G[(size_t)j * n + i];
    lu_factor(n, Gt.data(), piv.data());
    lu_solve(n, Gt.data(), piv.data(), x.data());
}

struct Step {
    std::vector<double> y;   // state at the start of an accepted step
    double h;
};

struct Cell {
    const Mech& m;
    const Opts& o;
    Stats st;
    int n;
    std::vector<double> S, J, G, f, d;
    std::vector<int> piv;
    bool record = false;                     // keep the accepted steps in hist
    std::vector<Step> hist;
    std::vector<std::vector<double>> lastY;  // converged stage states of the last step
    Cell(const Mech& mm, const Opts& oo) : m(mm), o(oo), n(mm.ns + 1),
        S(n), J(n * n), G(n * n), f(n), d(n), piv(n) {}

    // The linear solver of the Newton systems with matrix G (Section 3.4):
    // dense LU (prepare = factorise), or GMRES on G as assembled. Stats.lu
    // counts factorisations, or GMRES iterations.
    bool lin_prepare() {
        if (o.linear_solver == 1) return true;
        st.lu++;
        return lu_factor(n, G.data(), piv.data());
    }
    bool lin_solve(double* v) {
        if (o.linear_solver == 1) {
            int it = 0;
            const bool ok = gmres(n, G.data(), v, o.prec, o.gmres_m, o.gmres_maxit, o.gmres_tol, &it);
            st.lu += it;
            return ok;
        }
        lu_solve(n, G.data(), piv.data(), v);
        return true;
    }

    // Backward Euler (eq. Backward_euler) with full Newton (eq. newtons-method-2):
    // G(y_k) (y_{k+1} - y_k) = -f(y_k), f = (y_k - y^n)/h - S(y_k),
    // G = I/h - J(y_k) (eq. jacobian), J re-evaluated at every iterate.
    // Starts from y^n; converged when WRMS(y_{k+1} - y_k) <= newton_tol.
    bool be_step(const std::vector<double>& yn, double h, std::vector<double>& y) {
        y = yn;
        for (int k = 0; k < o.max_newton; ++k) {
            source(m, o.reactor, y.data(), S.data());
            jacobian(m, o.reactor, y.data(), J.data());
            for (int i = 0; i < n; ++i) {
                f[i] = (y[i] - yn[i]) / h - S[i];
                for (int j = 0; j < n; ++j) G[i * n + j] = (i == j ? 1.0 / h : 0.0) - J[i * n + j];
            }
            st.newton++;
            if (!lin_prepare()) return false;
            for (int i = 0; i < n; ++i) d[i] = -f[i];
            if (!lin_solve(d.data())) return false;
            for (int i = 0; i < n; ++i) y[i] += d[i];
            if (!finite_vec(y)) return false;
            if (wrms(n, d.data(), yn.data(), y.data(), o.rtol, o.atol) <= o.newton_tol) {
                lastY.assign(1, y);   // the one stage state of backward Euler is y^{n+1}
                return admissible(y, o.neg_tol);
            }
        }
        return false;
    }

    // One SDIRK step in stage-derivative form (Appendix A.1/A.2):
    //   Gamma_p = S(y_n + h sum_{j<p} a_pj Gamma_j + h a_pp Gamma_p),
    //   Newton on f(Gamma_p) = Gamma_p - S(Y_p) with G = I - a_pp h J(Y_p),
    //   first iterate Gamma_{p,1} = S(y_n), converged when the change of the
    //   stage state, WRMS(h a_pp dGamma), is <= newton_tol;
    //   y_{n+1} = y_n + h sum b_i Gamma_i.
    // On success also returns the embedded error estimate
    //   e = h sum (b_i - bhat_i) Gamma_i, optionally filtered by the last
    //   Newton matrix: e <- (I - a_pp h J)^{-1} e.
    bool sdirk_step(const Tableau& tb, const std::vector<double>& yn, double h,
                    std::vector<double>& y1, std::vector<double>& err) {
        std::vector<std::vector<double>> Gam(tb.s, std::vector<double>(n));
        std::vector<double> S0(n), Y(n), base(n);
        lastY.assign(tb.s, std::vector<double>(n));
        source(m, o.reactor, yn.data(), S0.data());
        for (int p = 0; p < tb.s; ++p) {
            double gh = tb.A[p][p] * h;
            for (int i = 0; i < n; ++i) {
                base[i] = yn[i];
                for (int j = 0; j < p; ++j) base[i] += h * tb.A[p][j] * Gam[j][i];
            }
            std::vector<double>& Gp = Gam[p];
            Gp = S0;
            bool conv = false;
            for (int k = 0; k < o.max_newton; ++k) {
                for (int i = 0; i < n; ++i) Y[i] = base[i] + gh * Gp[i];
                source(m, o.reactor, Y.data(), S.data());
                jacobian(m, o.reactor, Y.data(), J.data());
                for (int i = 0; i < n; ++i) {
                    f[i] = Gp[i] - S[i];
                    for (int j = 0; j < n; ++j) G[i * n + j] = (i == j ? 1.0 : 0.0) - gh * J[i * n + j];
                }
                st.newton++;
                if (!lin_prepare()) return false;
                for (int i = 0; i < n; ++i) d[i] = -f[i];
                if (!lin_solve(d.data())) return false;
                for (int i = 0; i < n; ++i) { Gp[i] += d[i]; d[i] *= gh; Y[i] = base[i] + gh * Gp[i]; }
                if (!finite_vec(Gp)) return false;
                if (wrms(n, d.data(), yn.data(), Y.data(), o.rtol, o.atol) <= o.newton_tol) {
                    conv = true;
                    break;
                }
            }
            if (!conv) return false;
            lastY[p] = Y;
        }
        y1 = yn;
        err.assign(n, 0.0);
        for (int p = 0; p < tb.s; ++p)
            for (int i = 0; i < n; ++i) {
                y1[i] += h * tb.b[p] * Gam[p][i];
                err[i] += h * (tb.b[p] - tb.bhat[p]) * Gam[p][i];
            }
        if (o.err_filter && !lin_solve(err.data())) return false;
        return finite_vec(y1) && admissible(y1, o.neg_tol);
    }

    // Second-order Rosenbrock step (Appendix A.3) with the coefficients of
    // FATODE's Ros2 that the appendix quotes: gamma = 1 + sqrt(2)/2,
    // alpha = 1/gamma, beta = -2/gamma, m1 = 3/(2 gamma), m2 = 1/(2 gamma):
    //   (I/(h gamma) - J_n) Gamma_1 = S(y_n)
    //   (I/(h gamma) - J_n) Gamma_2 = S(y_n + alpha Gamma_1) + (beta/h) Gamma_1
    //   y_{n+1} = y_n + m1 Gamma_1 + m2 Gamma_2.
    // (The appendix prints a further -S(y_n) in the second right-hand side,
    // which makes the scheme inconsistent -- on y' = lambda y the first-order
    // term becomes lambda h y / 2 -- and which FATODE's Ros2 does not have.)
    // J is evaluated once, at y_n. Embedded first-order solution
    // y_n + Gamma_1/gamma: error e = (Gamma_1 + Gamma_2)/(2 gamma).
    bool ros2_step(const std::vector<double>& yn, double h, std::vector<double>& y1,
                   std::vector<double>& err) {
        const double g = 1.0 + std::sqrt(2.0) / 2.0;
        const double alpha = 1.0 / g, beta = -2.0 / g, m1 = 3.0 / (2.0 * g), m2 = 1.0 / (2.0 * g);
        std::vector<double> S0(n), G1(n), G2(n), Y2(n);
        source(m, o.reactor, yn.data(), S0.data());
        jacobian(m, o.reactor, yn.data(), J.data());
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) G[i * n + j] = (i == j ? 1.0 / (h * g) : 0.0) - J[i * n + j];
        st.newton++;
        if (!lin_prepare()) return false;
        G1 = S0;
        if (!lin_solve(G1.data())) return false;
        for (int i = 0; i < n; ++i) Y2[i] = yn[i] + alpha * G1[i];
        if (!finite_vec(Y2)) return false;
        source(m, o.reactor, Y2.data(), G2.data());
        for (int i = 0; i < n; ++i) G2[i] += beta / h * G1[i];
        if (!lin_solve(G2.data())) return false;
        y1.assign(n, 0.0);
        err.assign(n, 0.0);
        for (int i = 0; i < n; ++i) {
            y1[i] = yn[i] + m1 * G1[i] + m2 * G2[i];
            err[i] = (G1[i] + G2[i]) / (2.0 * g);
        }
        lastY.clear();
        return finite_vec(y1) && admissible(y1, o.neg_tol);
    }

    // YASS (Appendix A.4): one backward-Euler Newton step from y_n,
    //   (I - h J(y_n)) dy = h S(y_n),  y_{n+1} = y_n + dy,
    // rejected (and halved by the caller) when the decrement's norm exceeds
    // alpha: WRMS(dy; atol + rtol max(|y_n|, |y_{n+1}|)) > alpha, with alpha
    // passed as newton_tol.
    bool yass_step(const std::vector<double>& yn, double h, std::vector<double>& y1) {
        std::vector<double> dy(n);
        source(m, o.reactor, yn.data(), dy.data());
        jacobian(m, o.reactor, yn.data(), J.data());
        for (int i = 0; i < n; ++i) {
            dy[i] *= h;
            for (int j = 0; j < n; ++j) G[i * n + j] = (i == j ? 1.0 : 0.0) - h * J[i * n + j];
        }
        st.newton++;
        if (!lin_prepare()) return false;
        if (!lin_solve(dy.data())) return false;
        y1 = yn;
        for (int i = 0; i < n; ++i) y1[i] += dy[i];
        lastY.clear();
        if (!finite_vec(y1)) return false;
        if (wrms(n, dy.data(), yn.data(), y1.data(), o.rtol, o.atol) > o.newton_tol) return false;
        return admissible(y1, o.neg_tol);
    }

    bool step_with_error(const Tableau& tb, const std::vector<double>& yn, double h, std::vector<double>& y1,
                         std::vector<double>& err) {
        if (o.method == 3) return ros2_step(yn, h, y1, err);
        return sdirk_step(tb, yn, h, y1, err);
    }

    bool fixed_step(const Tableau& tb, const std::vector<double>& yn, double h, std::vector<double>& y) {
        if (o.method == 0) return be_step(yn, h, y);
        if (o.method == 4) return yass_step(yn, h, y);
        std::vector<double> err;
        return step_with_error(tb, yn, h, y, err);
    }

    // Fixed step with deterministic halving on Newton failure (after YASS,
    // Appendix A.4): a failed step is replaced by two steps of half the size,
    // recursively, at most max_halvings levels deep.
    int fixed_recursive(const Tableau& tb, std::vector<double>& y, double h, int depth) {
        std::vector<double> y1;
        if (fixed_step(tb, y, h, y1)) {
            if (record) hist.push_back({y, h});
            y = y1;
            st.steps++;
            return ST_OK;
        }
        st.rejects++;
        if (depth >= o.max_halvings) return ST_NEWTON_FAIL;
        int s = fixed_recursive(tb, y, 0.5 * h, depth + 1);
        if (s != ST_OK) return s;
        return fixed_recursive(tb, y, 0.5 * h, depth + 1);
    }

    // Adaptive step-size control (not specified by the paper): accept when the
    // WRMS error <= 1; h_new = h min(5, max(0.2, 0.9 err^{-1/(q+1)}));
    // Newton failure: h <- h/4; last step clipped to end at dt.
    int adaptive(const Tableau& tb, std::vector<double>& y) {
        double t = 0.0, h = o.h0 > 0.0 ? std::min(o.h0, o.dt) : o.dt;
        double expo = -1.0 / (tb.err_order + 1.0);
        std::vector<double> y1, err;
        int attempts = 0;
        while (t < o.dt) {
            if (attempts++ >= o.max_steps) return ST_MAX_STEPS;
            if (h < o.hmin) return ST_STEP_TOO_SMALL;
            bool last = t + h >= o.dt;
            double hh = last ? o.dt - t : h;
            if (!step_with_error(tb, y, hh, y1, err)) {
                st.rejects++;
                h = 0.25 * hh;
                continue;
            }
            double e = wrms(n, err.data(), y.data(), y1.data(), o.rtol, o.atol);
            double fac = e > 0.0 ? 0.9 * std::pow(e, expo) : 5.0;
            fac = std::min(5.0, std::max(0.2, fac));
            if (e <= 1.0) {
                if (record) hist.push_back({y, hh});
                y = y1;
                t = last ? o.dt : t + hh;
                st.steps++;
            } else {
                st.rejects++;
            }
            h = hh * fac;
        }
        return ST_OK;
    }

    int integrate(const Tableau& tb, std::vector<double>& y) {
        if (!finite_vec(y)) return ST_NONFINITE;
        if (o.adaptive && o.method >= 1 && o.method <= 3) return adaptive(tb, y);
        int ns = std::max(1, o.nsub);
        double h = o.dt / ns;
        for (int k = 0; k < ns; ++k) {
            int s = fixed_recursive(tb, y, h, 0);
            if (s != ST_OK) return s;
        }
        return ST_OK;
    }

    // Converged stage states of the step (y_n, h) into lastY.
    // (backward Euler and SDIRK only: the adjoint covers those integrators)
    bool stages(const Tableau& tb, const std::vector<double>& yn, double h) {
        std::vector<double> y1, err;
        if (o.method == 0) return be_step(yn, h, y1);
        if (o.method > 2) return false;
        return sdirk_step(tb, yn, h, y1, err);
    }

    // Steps of prescribed sizes (no step-size decisions).
    int replay(const Tableau& tb, std::vector<double>& y, const double* hs, int count) {
        std::vector<double> y1, err;
        for (int k = 0; k < count; ++k) {
            bool ok = fixed_step(tb, y, hs[k], y1);
            if (!ok) return ST_NEWTON_FAIL;
            y = y1;
        }
        return ST_OK;
    }

    // Discrete adjoint of the converged stage equations with the accepted
    // steps frozen: for a step (y_n, h) with stages Y_p, Gamma_p = S(Y_p),
    //   (I - h a_pp J_p)^T nu_p = h b_p lam + sum_{q>p} h a_qp J_q^T nu_q,
    //   lam_n = lam + sum_p J_p^T nu_p,  dL/dtheta += sum_p nu_p^T dS/dtheta(Y_p).
    // Backward Euler is the one-stage case a = b = 1. lam: dL/dy_end in,
    // dL/dy_0 out; grad[3 nr] accumulates (ln A, b, Ea) of every reaction.
    bool adjoint(const Tableau& tb, std::vector<double>& lam, std::vector<double>& grad) {
        const int s = o.method == 0 ? 1 : tb.s;
        const double A00 = 1.0;
        std::vector<double> dSq;
        for (int stp = (int)hist.size() - 1; stp >= 0; --stp) {
            const double h = hist[stp].h;
            if (!stages(tb, hist[stp].y, h)) return false;
            std::vector<std::vector<double>> acc(s, std::vector<double>(n, 0.0));
            std::vector<double> lam_n = lam;
            for (int p = s - 1; p >= 0; --p) {
                const double app = o.method == 0 ? A00 : tb.A[p][p];
                const double bp = o.method == 0 ? 1.0 : tb.b[p];
                std::vector<double> nu(n);
                for (int i = 0; i < n; ++i) nu[i] = h * bp * lam[i] + acc[p][i];
                jacobian(m, o.reactor, lastY[p].data(), J.data());
                for (int i = 0; i < n; ++i)
                    for (int j = 0; j < n; ++j) G[i * n + j] = (i == j ? 1.0 : 0.0) - h * app * J[i * n + j];
                transpose_solve(n, G.data(), nu);
                std::vector<double> w(n, 0.0);   // J_p^T nu_p
                for (int i = 0; i < n; ++i)
                    for (int j = 0; j < n; ++j) w[j] += J[i * n + j] * nu[i];
                for (int q = 0; q < p; ++q)
                    for (int i = 0; i < n; ++i) acc[q][i] += h * tb.A[p][q] * w[i];
                for (int i = 0; i < n; ++i) lam_n[i] += w[i];
                dS_dq(m, o.reactor, lastY[p].data(), dSq);
                const double T = lastY[p][0];
                for (int j = 0; j < m.nr; ++j) {
                    double g = 0.0;
                    for (int i = 0; i < n; ++i) g += nu[i] * dSq[(size_t)i * m.nr + j];
                    const double dq = g * dq_dlnk(m, j, T, lastY[p].data() + 1);
                    grad[3 * j + 0] += dq;
                    grad[3 * j + 1] += dq * std::log(T);
                    grad[3 * j + 2] -= dq / (R_U * T);
                }
            }
            lam = lam_n;
        }
        return true;
    }

    // Forward sensitivity (tangent linear) of the same frozen steps:
    //   (I - h a_pp J_p) dGamma_p = J_p (dy_n + h sum_{q<p} a_pq dGamma_q)
    //                               + dS/dtheta(Y_p),
    //   dy_{n+1} = dy_n + h sum_p b_p dGamma_p;
    // for the parameter (reaction pj, kind pk: 0 ln A, 1 b, 2 Ea; pj < 0: none).
    bool tangent(const Tableau& tb, std::vector<double>& dy, int pj, int pk) {
        const int s = o.method == 0 ? 1 : tb.s;
        std::vector<double> dSq;
        for (size_t stp = 0; stp < hist.size(); ++stp) {
            const double h = hist[stp].h;
            if (!stages(tb, hist[stp].y, h)) return false;
            std::vector<std::vector<double>> dG(s, std::vector<double>(n, 0.0));
            for (int p = 0; p < s; ++p) {
                const double app = o.method == 0 ? 1.0 : tb.A[p][p];
                std::vector<double> z = dy;
                for (int q = 0; q < p; ++q)
                    for (int i = 0; i < n; ++i) z[i] += h * tb.A[p][q] * dG[q][i];
                jacobian(m, o.reactor, lastY[p].data(), J.data());
                std::vector<double> rhs(n, 0.0);
                for (int i = 0; i < n; ++i)
                    for (int j = 0; j < n; ++j) rhs[i] += J[i * n + j] * z[j];
                if (pj >= 0) {
                    dS_dq(m, o.reactor, lastY[p].data(), dSq);
                    const double T = lastY[p][0];
                    double dq = dq_dlnk(m, pj, T, lastY[p].data() + 1);
                    if (pk == 1) dq *= std::log(T);
                    if (pk == 2) dq *= -1.0 / (R_U * T);
                    for (int i = 0; i < n; ++i) rhs[i] += dSq[(size_t)i * m.nr + pj] * dq;
                }
                for (int i = 0; i < n; ++i)
                    for (int j = 0; j < n; ++j) G[i * n + j] = (i == j ? 1.0 : 0.0) - h * app * J[i * n + j];
                lu_factor(n, G.data(), piv.data());
                lu_solve(n, G.data(), piv.data(), rhs.data());
                dG[p] = rhs;
            }
            for (int p = 0; p < s; ++p) {
                const double bp = o.method == 0 ? 1.0 : tb.b[p];
                for (int i = 0; i < n; ++i) dy[i] += h * bp * dG[p][i];
            }
        }
        return true;
    }
};

// ---------------------------------------------------------------------------
// Temperature recovery, eqs. temperature-nonlinear .. netwon_iteration_temperature.
// Solves sum_i Y_i e_i(T) = e (e = u for CONV, h for CONP) with n Newton
// iterations: T_k = T_{k-1} + (e - e(T_{k-1})) / c(T_{k-1}), where
// c = sum Y_i c_v,i (or c_p,i). (The printed update carries the opposite sign
// of the Newton step eq. netwons-method-temperature defines; the step is used.)
double recover_T(const Mech& m, int reactor, double e, const double* Y, double T, int iters) {
    for (int k = 0; k < iters; ++k) {
        double ev = 0.0, c = 0.0;
        for (int i = 0; i < m.ns; ++i) {
            ev += Y[i] * (reactor == CONV ? u_i(m, i, T) : h_i(m, i, T));
            c += Y[i] * (reactor == CONV ? cv_i(m, i, T) : cp_i(m, i, T));
        }
        T = T + (e - ev) / c;
    }
    return T;
}

// Cells are independent and their cost varies by two orders of magnitude
// (frozen vs igniting gas), so each thread takes the next unclaimed cell from
// a shared counter; the result of a cell does not depend on which thread
// computed it.
template <class F> void parallel_for(long N, int nthreads, F fn) {
    if (nthreads <= 1 || N < 2) {
        for (long c = 0; c < N; ++c) fn(c);
        return;
    }
    std::atomic<long> next(0);
    std::vector<std::thread> th;
    for (int t = 0; t < nthreads; ++t)
        th.emplace_back([&]() {
            for (long c = next.fetch_add(1); c < N; c = next.fetch_add(1)) fn(c);
        });
    for (auto& x : th) x.join();
}

}  // namespace

// ---------------------------------------------------------------------------
// C entry points (host pointers; arrays of cells are cell-major: cell c's
// state is y[c*n .. c*n+n-1]).

extern "C" {

void* cgref_mech_create(int ns, int nr, const double* W, const double* nasa7,
                        const int* rtype, const int* reversible,
                        const int* rf_idx, const int* rf_nu, const int* rr_idx, const int* rr_nu,
                        const double* arr, const double* arr0, const double* troe,
                        const int* eff_ptr, const int* eff_idx, const double* eff_val,
                        const double* sri, const int* plog_ptr, const double* plog) {
    Mech* m = new Mech();
    m->ns = ns;
    m->nr = nr;
    m->W.assign(W, W + ns);
    m->Ri.resize(ns);
    for (int i = 0; i < ns; ++i) m->Ri[i] = R_U / W[i];
    set_thermo(*m, 4, nasa7, 7);
    m->rx.resize(nr);
    for (int j = 0; j < nr; ++j) {
        Reaction& r = m->rx[j];
        r.type = rtype[j];
        r.reversible = reversible[j];
        r.sum_nu = 0;
        for (int s = 0; s < 3; ++s) {
            r.f_idx[s] = rf_idx[3 * j + s]; r.f_nu[s] = rf_nu[3 * j + s];
            r.r_idx[s] = rr_idx[3 * j + s]; r.r_nu[s] = rr_nu[3 * j + s];
            if (r.f_idx[s] >= 0) r.sum_nu -= r.f_nu[s];
            if (r.r_idx[s] >= 0) r.sum_nu += r.r_nu[s];
        }
        r.lnA = arr[3 * j]; r.b = arr[3 * j + 1]; r.Ea = arr[3 * j + 2];
        r.lnA0 = arr0[3 * j]; r.b0 = arr0[3 * j + 1]; r.Ea0 = arr0[3 * j + 2];
        r.alpha = troe[4 * j]; r.T3 = troe[4 * j + 1]; r.T1 = troe[4 * j + 2]; r.T2 = troe[4 * j + 3];
        r.has_T2 = !std::isnan(r.T2);
        for (int e = eff_ptr[j]; e < eff_ptr[j + 1]; ++e) {
            r.eff_sp.push_back(eff_idx[e]);
            r.eff_val.push_back(eff_val[e]);
        }
        for (int k = 0; k < 5; ++k) r.sri[k] = sri[5 * j + k];
        for (int e = plog_ptr[j]; e < plog_ptr[j + 1]; ++e) {
            r.pl_lnp.push_back(std::log(plog[4 * e]));
            r.pl_lnA.push_back(plog[4 * e + 1]);
            r.pl_b.push_back(plog[4 * e + 2]);
            r.pl_Ea.push_back(plog[4 * e + 3]);
        }
    }
    return m;
}

void cgref_mech_destroy(void* h) { delete static_cast<Mech*>(h); }

// Replace the thermodynamics by a c_p polynomial of degree n_p (Section 2.1,
// eq. specific_heat_polynomial; Appendix C.1): coef[ns][n_p + 3] holds a_0..a_np
// of c_p/R (molar) and the h/R and s/R constants. 0, or -1 for n_p outside [0, 15].
int cgref_mech_set_thermo(void* h, int np, const double* coef) {
    if (np < 0 || np > 15) return -1;
    Mech& m = *static_cast<Mech*>(h);
    set_thermo(m, np, coef, np + 3);
    return 0;
}

// Mass-specific thermo per species at one temperature: cp, h, u, s, g, cv.
void cgref_thermo(const void* h, double T, double* cp, double* hh, double* u, double* s, double* g,
                  double* cv) {
    const Mech& m = *static_cast<const Mech*>(h);
    double lnT = std::log(T);
    for (int i = 0; i < m.ns; ++i) {
        cp[i] = cp_i(m, i, T); hh[i] = h_i(m, i, T); u[i] = u_i(m, i, T);
        s[i] = s_i(m, i, T, lnT); g[i] = g_i(m, i, T, lnT); cv[i] = cv_i(m, i, T);
    }
}

// Forward/reverse rate constants and rates of progress of one state.
void cgref_rates(const void* h, double T, const double* C, double* kf, double* kr, double* q) {
    const Mech& m = *static_cast<const Mech*>(h);
    progress_rates(m, T, C, kf, kr, q);
}

// S(y) for N cells, y cell-major [N][ns+1].
void cgref_source(const void* h, int reactor, long N, const double* y, double* S) {
    const Mech& m = *static_cast<const Mech*>(h);
    const int n = m.ns + 1;
    for (long c = 0; c < N; ++c) source(m, reactor, y + c * n, S + c * n);
}

// S(y) with complex state (for complex-step differentiation).
void cgref_source_complex(const void* h, int reactor, const double* y_re, const double* y_im,
                          double* S_re, double* S_im) {
    const Mech& m = *static_cast<const Mech*>(h);
    const int n = m.ns + 1;
    std::vector<cplx> y(n), S(n);
    for (int i = 0; i < n; ++i) y[i] = cplx(y_re[i], y_im[i]);
    source(m, reactor, y.data(), S.data());
    for (int i = 0; i < n; ++i) { S_re[i] = S[i].real(); S_im[i] = S[i].imag(); }
}

// J(y) for N cells, J cell-major [N][n][n] row-major.
void cgref_jacobian(const void* h, int reactor, long N, const double* y, double* J) {
    const Mech& m = *static_cast<const Mech*>(h);
    const int n = m.ns + 1;
    for (long c = 0; c < N; ++c) jacobian(m, reactor, y + c * n, J + c * n * n);
}

// Solve A x = b with LU and partial pivoting; A, b overwritten (x in b). 0 if singular.
// GMRES of Section 3.4 on one dense system (row-major A, b in, x out).
int cgref_gmres(int n, const double* A, double* b, int prec, int m, int maxit, double tol, int* iters) {
    return gmres(n, A, b, prec, m, maxit, tol, iters) ? 1 : 0;
}

int cgref_lu_solve(int n, double* A, double* b) {
    std::vector<int> piv(n);
    if (!lu_factor(n, A, piv.data())) return 0;
    lu_solve(n, A, piv.data(), b);
    return 1;
}

// Temperature from mass-specific energy (u for CONV, h otherwise) and Y.
void cgref_temperature(const void* h, int reactor, long N, const double* e, const double* Y,
                       const double* T0, int iters, double* T) {
    const Mech& m = *static_cast<const Mech*>(h);
    for (long c = 0; c < N; ++c) T[c] = recover_T(m, reactor, e[c], Y + c * m.ns, T0[c], iters);
}

namespace {
void unpack(const int* iopt, const double* dopt, const double* tab, Opts& o, Tableau& tb);
}  // namespace

// Integrate N cells over dt. y in/out cell-major [N][ns+1] = (T, C).
// status[N]; stats[N][4] = accepted steps, rejected/failed attempts, Newton
// iterations, LU factorisations.
void cgref_integrate(const void* h, const int* iopt, const double* dopt, const double* tab,
                     long N, double* y, int* status, int* stats, int nthreads) {
    const Mech& m = *static_cast<const Mech*>(h);
    Opts o;
    Tableau tb;
    unpack(iopt, dopt, tab, o, tb);
    const int n = m.ns + 1;
    parallel_for(N, nthreads, [&](long c) {
        Cell cell(m, o);
        std::vector<double> yc(y + c * n, y + (c + 1) * n);
        int s = cell.integrate(tb, yc);
        if (s == ST_OK && !finite_vec(yc)) s = ST_NONFINITE;
        std::copy(yc.begin(), yc.end(), y + c * n);
        status[c] = s;
        stats[4 * c + 0] = cell.st.steps;
        stats[4 * c + 1] = cell.st.rejects;
        stats[4 * c + 2] = cell.st.newton;
        stats[4 * c + 3] = cell.st.lu;
    });
}

namespace {

void unpack(const int* iopt, const double* dopt, const double* tab, Opts& o, Tableau& tb) {
    o.method = iopt[0]; o.reactor = iopt[1]; o.adaptive = iopt[2]; o.nsub = iopt[3];
    o.max_newton = iopt[4]; o.max_steps = iopt[5]; o.max_halvings = iopt[6]; o.err_filter = iopt[7];
    o.dt = dopt[0]; o.rtol = dopt[1]; o.atol = dopt[2]; o.newton_tol = dopt[3];
    o.h0 = dopt[4]; o.hmin = dopt[5]; o.neg_tol = dopt[6];
    o.linear_solver = iopt[8]; o.prec = iopt[9]; o.gmres_m = iopt[10]; o.gmres_maxit = iopt[11];
    o.gmres_tol = dopt[7];
    tb.s = (int)tab[0];
    tb.err_order = (int)tab[1];
    for (int i = 0; i < 5; ++i) {
        for (int j = 0; j < 5; ++j) tb.A[i][j] = tab[2 + 5 * i + j];
        tb.b[i] = tab[27 + i];
        tb.bhat[i] = tab[32 + i];
    }
}

}  // namespace

// Integrate and return the accepted step sizes (hs[N][cap], hn[N]); a cell
// with more than cap accepted steps gets hn = -1.
void cgref_integrate_hist(const void* h, const int* iopt, const double* dopt, const double* tab, long N,
                          double* y, int* status, double* hs, int* hn, int cap, int nthreads) {
    const Mech& m = *static_cast<const Mech*>(h);
    Opts o;
    Tableau tb;
    unpack(iopt, dopt, tab, o, tb);
    const int n = m.ns + 1;
    parallel_for(N, nthreads, [&](long c) {
        Cell cell(m, o);
        cell.record = true;
        std::vector<double> yc(y + c * n, y + (c + 1) * n);
        status[c] = cell.integrate(tb, yc);
        std::copy(yc.begin(), yc.end(), y + c * n);
        hn[c] = (int)cell.hist.size() <= cap ? (int)cell.hist.size() : -1;
        for (size_t k = 0; k < cell.hist.size() && (int)k < cap; ++k) hs[c * cap + k] = cell.hist[k].h;
    });
}

// Steps of the given sizes from y (in/out).
void cgref_replay(const void* h, const int* iopt, const double* dopt, const double* tab, long N, double* y,
                  const double* hs, const int* hn, int cap, int* status, int nthreads) {
    const Mech& m = *static_cast<const Mech*>(h);
    Opts o;
    Tableau tb;
    unpack(iopt, dopt, tab, o, tb);
    const int n = m.ns + 1;
    parallel_for(N, nthreads, [&](long c) {
        Cell cell(m, o);
        std::vector<double> yc(y + c * n, y + (c + 1) * n);
        status[c] = cell.replay(tb, yc, hs + c * cap, hn[c]);
        std::copy(yc.begin(), yc.end(), y + c * n);
    });
}

// Discrete adjoint: integrates y0 (recording the accepted steps), then
// sweeps back with lam = dL/dy_end. Out: dL/dy_0 (dy0[N][n]) and
// dL/dtheta per cell (grad[N][3 nr], (ln A, b, Ea) of each reaction).
void cgref_adjoint(const void* h, const int* iopt, const double* dopt, const double* tab, long N,
                   const double* y0, const double* lam_end, double* dy0, double* grad, int* status,
                   int nthreads) {
    const Mech& m = *static_cast<const Mech*>(h);
    Opts o;
    Tableau tb;
    unpack(iopt, dopt, tab, o, tb);
    const int n = m.ns + 1;
    parallel_for(N, nthreads, [&](long c) {
        Cell cell(m, o);
        cell.record = true;
        std::vector<double> yc(y0 + c * n, y0 + (c + 1) * n);
        int s = cell.integrate(tb, yc);
        std::vector<double> lam(lam_end + c * n, lam_end + (c + 1) * n), g(3 * m.nr, 0.0);
        if (s == ST_OK && !cell.adjoint(tb, lam, g)) s = ST_NEWTON_FAIL;
        status[c] = s;
        std::copy(lam.begin(), lam.end(), dy0 + c * n);
        std::copy(g.begin(), g.end(), grad + c * 3 * m.nr);
    });
}

// Forward sensitivity of y_end to dy0 and to one parameter (pj, pk).
void cgref_tangent(const void* h, const int* iopt, const double* dopt, const double* tab, long N,
                   const double* y0, const double* dy0, int pj, int pk, double* dyend, int* status,
                   int nthreads) {
    const Mech& m = *static_cast<const Mech*>(h);
    Opts o;
    Tableau tb;
    unpack(iopt, dopt, tab, o, tb);
    const int n = m.ns + 1;
    parallel_for(N, nthreads, [&](long c) {
        Cell cell(m, o);
        cell.record = true;
        std::vector<double> yc(y0 + c * n, y0 + (c + 1) * n);
        int s = cell.integrate(tb, yc);
        std::vector<double> dy(dy0 + c * n, dy0 + (c + 1) * n);
        if (s == ST_OK && !cell.tangent(tb, dy, pj, pk)) s = ST_NEWTON_FAIL;
        status[c] = s;
        std::copy(dy.begin(), dy.end(), dyend + c * n);
    });
}

}  // extern "C"
