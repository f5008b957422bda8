// C-ABI of chemgb (declared in include/chemgb.h): mechanism upload and the
// host-side preparation of the kernels (reaction ordering, thermo table,
// assembly schedules, shared-memory layout, Butcher tableaux).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "chemgb.h"
#include "chemgb_testing.h"
#include "chem_internal.h"

using cg::DevMech;
using cg::IntParams;
using cg::Layout;

namespace {

thread_local std::string g_err;

// An NVTX range named after the entry point around each call (seen by
// profilers such as Nsight Systems and ncu --nvtx; header-only NVTX v3,
// nothing is recorded when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#define CG_RANGE(name) NvtxRange cg_nvtx_range_(name)

cg_status fail(cg_status code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

cg_status cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? CG_ENOMEM : CG_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

const double kR = 8314.46261815324;
const double kPref = 101325.0;
const size_t kMaxSmemPerBlock = 227 * 1024;
const int kMaxThermoDegree = 15;   // c_p polynomials of degree 0..15 (Appendix C.1 goes to 15)

// One term of an assembly schedule: out[dst] += fac * in[src].
struct Term {
    int dst, src;
    double fac;
    long order;   // accumulation order within one destination
};

struct Schedule {
    int len = 0;   // terms per lane
    std::vector<int> dst, src;
    std::vector<double> fac;
};

// Lane-owned schedule: terms are grouped by destination (in their `order`
// within a destination), destinations are dealt to the lanes longest first
// onto the least-loaded lane, and each lane's terms are laid out at
// [t * lanes + lane]; every term carries its destination, flagged
// cg::kSchedFirst on the first and cg::kSchedLast on the last term of its run.
Schedule make_schedule(std::vector<Term> terms, int lanes_n) {
    std::stable_sort(terms.begin(), terms.end(), [](const Term& a, const Term& b) {
        return a.dst != b.dst ? a.dst < b.dst : a.order < b.order;
    });
    struct Run { int dst; size_t b, e; };
    std::vector<Run> runs;
    for (size_t i = 0; i < terms.size();) {
        size_t j = i;
        while (j < terms.size() && terms[j].dst == terms[i].dst) ++j;
        runs.push_back({terms[i].dst, i, j});
        i = j;
    }
    std::vector<Run> by_len = runs;
    std::stable_sort(by_len.begin(), by_len.end(),
                     [](const Run& a, const Run& b) { return a.e - a.b > b.e - b.b; });
    std::vector<std::vector<Run>> lanes(lanes_n);
    std::vector<size_t> load(lanes_n, 0);
    for (const Run& r : by_len) {
        int best = 0;
        for (int l = 1; l < lanes_n; ++l)
            if (load[l] < load[best]) best = l;
        lanes[best].push_back(r);
        load[best] += r.e - r.b;
    }
    Schedule s;
    s.len = (int)*std::max_element(load.begin(), load.end());
    const size_t slots = (size_t)std::max(1, s.len) * lanes_n;
    s.dst.assign(slots, 0);
    s.src.assign(slots, 0);
    s.fac.assign(slots, 0.0);
    for (int l = 0; l < lanes_n; ++l) {
        std::sort(lanes[l].begin(), lanes[l].end(), [](const Run& a, const Run& b) { return a.dst < b.dst; });
        size_t t = 0;
        for (const Run& r : lanes[l])
            for (size_t i = r.b; i < r.e; ++i, ++t) {
                const size_t k = t * lanes_n + l;
                s.src[k] = terms[i].src;
                s.fac[k] = terms[i].fac;
                s.dst[k] = r.dst | (i == r.b ? cg::kSchedFirst : 0) | (i + 1 == r.e ? cg::kSchedLast : 0);
            }
    }
    return s;
}

// Place one cell's arrays: hottest first into shared memory (at most
// smem_limit bytes per cell), the rest into the cell's global scratch slot.
// mat_bytes: 8 for the FP64 Newton matrix, 4 for the FP32 one; adjoint:
// add the arrays of the backward sweep (size 0 otherwise). sizes_out and
// order_out (A_COUNT entries each, may be NULL) receive the placed size of
// every array and the priority order.
Layout make_layout(int ns, int nr, int mat_bytes, size_t smem_limit, bool adjoint = false, int gmres_m = 0,
                   int* sizes_out = nullptr, int* order_out = nullptr) {
    using namespace cg;
    const int n = ns + 1;
    Layout L;
    L.ld = (n % 2) ? n : n + 1;   // odd stride: fewer bank conflicts on column walks
    int size[A_COUNT];
    size[A_G] = (n * L.ld * mat_bytes + 7) / 8;
    size[A_RD] = 9 * nr;
    size[A_SP] = 4 * ns;
    size[A_V] = ns;
    for (int a : {A_YN, A_Y, A_BASE, A_S, A_S0, A_F, A_ERR, A_Y1, A_COLA, A_COLB, A_RINV}) size[a] = n;
    size[A_GAM] = 5 * n;
    size[A_PIV] = (n + 1) / 2;
    size[A_RED] = 24;
    size[A_XF] = adjoint ? nr : 0;
    size[A_GRAD] = adjoint ? 3 * nr : 0;
    for (int a : {A_LAM, A_LAMN, A_NU, A_RHS}) size[a] = adjoint ? n : 0;
    size[A_ACC] = adjoint ? 5 * n : 0;
    size[A_SEG] = adjoint ? kSegSteps * (n + 1) : 0;
    size[A_KV] = gmres_m ? (gmres_m + 1) * (n | 1) : 0;
    size[A_KH] = gmres_m ? (gmres_m + 1) * gmres_m + 2 * gmres_m + 2 * (gmres_m + 1) : 0;
    const int order[A_COUNT] = {A_RED, A_PIV, A_G, A_RINV, A_YN, A_Y, A_F, A_S, A_BASE,
                                A_S0, A_ERR, A_Y1, A_COLA, A_COLB, A_SP, A_V, A_GAM, A_KH, A_KV,
                                A_NU, A_RHS, A_LAM, A_LAMN, A_ACC, A_XF, A_RD, A_GRAD, A_SEG};
    // 1 KiB of the block's shared memory stays free for the kernels' static variables
    const long budget = (long)((smem_limit > 2048 ? smem_limit - 1024 : 1024) / sizeof(double));
    int so = 0, go = 0;
    L.gmask = 0;
    bool spill = false;
    for (int k = 0; k < A_COUNT; ++k) {
        const int a = order[k];
#ifdef CG_DEBUG
        L.size[a] = (size[a] + 1) & ~1;
        const int sz = L.size[a] + (size[a] ? kGuard : 0);   // guard words after each array
#else
        const int sz = (size[a] + 1) & ~1;   // 16-byte aligned arrays
#endif
        if (a == A_RED || (!spill && so + sz <= budget)) {
            L.off[a] = so;
            so += sz;
        } else {
            spill = true;   // keep the priority order: once one array spills, the rest follow
            L.off[a] = go;
            go += sz;
            L.gmask |= 1u << a;
        }
        if (sizes_out) sizes_out[a] = sz;
        if (order_out) order_out[k] = a;
    }
    L.stotal = so;
    L.gtotal = go;
    return L;
}

// ---------------------------------------------------------------------------
// Butcher tableaux (Appendix A), in stage-derivative form.

struct Tab {
    int s = 1, err_order = 0, start_zero = 0;
    double A[5][5] = {}, b[5] = {}, bh[5] = {};
};

typedef long double ld_t;

// order conditions up to order 4 of a 5-stage method with b = last row of A
void sdirk4_residual(const ld_t x[9], ld_t res[9]) {
    const ld_t g = (ld_t)4 / 15;
    ld_t A[5][5] = {{g, 0, 0, 0, 0},
                    {(ld_t)1 / 2, g, 0, 0, 0},
                    {x[0], x[1], g, 0, 0},
                    {x[2], x[3], x[4], g, 0},
                    {x[5], x[6], x[7], x[8], g}};
    ld_t c[5], Ac[5], Ac2[5], AAc[5];
    for (int i = 0; i < 5; ++i) {
        c[i] = 0;
        for (int j = 0; j < 5; ++j) c[i] += A[i][j];
    }
    for (int i = 0; i < 5; ++i) {
        Ac[i] = Ac2[i] = 0;
        for (int j = 0; j < 5; ++j) { Ac[i] += A[i][j] * c[j]; Ac2[i] += A[i][j] * c[j] * c[j]; }
    }
    for (int i = 0; i < 5; ++i) {
        AAc[i] = 0;
        for (int j = 0; j < 5; ++j) AAc[i] += A[i][j] * Ac[j];
    }
    const ld_t* b = A[4];
    ld_t s1 = 0, s2 = 0, s3 = 0, s4 = 0, s5 = 0, s6 = 0, s7 = 0, s8 = 0;
    for (int i = 0; i < 5; ++i) {
        s1 += b[i];
        s2 += b[i] * c[i];
        s3 += b[i] * c[i] * c[i];
        s4 += b[i] * Ac[i];
        s5 += b[i] * c[i] * c[i] * c[i];
        s6 += b[i] * c[i] * Ac[i];
        s7 += b[i] * Ac2[i];
        s8 += b[i] * AAc[i];
    }
    res[0] = s1 - 1;
    res[1] = s2 - (ld_t)1 / 2;
    res[2] = s3 - (ld_t)1 / 3;
    res[3] = s4 - (ld_t)1 / 6;
    res[4] = s5 - (ld_t)1 / 4;
    res[5] = s6 - (ld_t)1 / 8;
    res[6] = s7 - (ld_t)1 / 12;
    res[7] = s8 - (ld_t)1 / 24;
    res[8] = x[0] + x[1] - (ld_t)3 / 10;   // c3 = 17/30 from the printed row sums
}

bool gauss_solve(int n, ld_t* M, ld_t* r) {   // M n x n row-major, r rhs -> solution
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i < n; ++i)
            if (fabsl(M[i * n + k]) > fabsl(M[p * n + k])) p = i;
        if (M[p * n + k] == 0) return false;
        if (p != k) {
            for (int j = 0; j < n; ++j) std::swap(M[k * n + j], M[p * n + j]);
            std::swap(r[k], r[p]);
        }
        for (int i = k + 1; i < n; ++i) {
            const ld_t f = M[i * n + k] / M[k * n + k];
            for (int j = k; j < n; ++j) M[i * n + j] -= f * M[k * n + j];
            r[i] -= f * r[k];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        for (int j = i + 1; j < n; ++j) r[i] -= M[i * n + j] * r[j];
        r[i] /= M[i * n + i];
    }
    return true;
}

// SDIRK-4 of Appendix A.2: gamma = 4/15, a21 = 1/2, printed to seven digits
// (a52 not printed; the scheme is stiffly accurate, so a52 = b2). The full
// precision coefficients solve the order-4 conditions near the printed values.
bool make_sdirk4(Tab& t) {
    ld_t x[9] = {0.3541539L, -0.05415395L, 0.08515494L, -0.06484332L, 0.07915325L,
                 2.100115L, -0.7677800L, 2.399816L, -2.998818L};
    for (int it = 0; it < 60; ++it) {
        ld_t r[9], Jm[81];
        sdirk4_residual(x, r);
        ld_t rmax = 0;
        for (int i = 0; i < 9; ++i) rmax = std::max(rmax, fabsl(r[i]));
        if (rmax < 1e-18L) break;
        for (int k = 0; k < 9; ++k) {
            ld_t xp[9], xm[9], rp[9], rm[9];
            std::copy(x, x + 9, xp);
            std::copy(x, x + 9, xm);
            const ld_t hstep = 1e-7L;
            xp[k] += hstep;
            xm[k] -= hstep;
            sdirk4_residual(xp, rp);
            sdirk4_residual(xm, rm);
            for (int i = 0; i < 9; ++i) Jm[i * 9 + k] = (rp[i] - rm[i]) / (2 * hstep);
        }
        for (int i = 0; i < 9; ++i) r[i] = -r[i];
        if (!gauss_solve(9, Jm, r)) return false;
        for (int i = 0; i < 9; ++i) x[i] += r[i];
    }
    ld_t r[9];
    sdirk4_residual(x, r);
    for (int i = 0; i < 9; ++i)
        if (fabsl(r[i]) > 1e-15L) return false;
    const ld_t g = (ld_t)4 / 15;
    ld_t A[5][5] = {{g, 0, 0, 0, 0},
                    {(ld_t)1 / 2, g, 0, 0, 0},
                    {x[0], x[1], g, 0, 0},
                    {x[2], x[3], x[4], g, 0},
                    {x[5], x[6], x[7], x[8], g}};
    // embedded third-order weights on stages 1-4
    ld_t c[5], Ac[5];
    for (int i = 0; i < 5; ++i) {
        c[i] = 0;
        for (int j = 0; j < 5; ++j) c[i] += A[i][j];
    }
    for (int i = 0; i < 5; ++i) {
        Ac[i] = 0;
        for (int j = 0; j < 5; ++j) Ac[i] += A[i][j] * c[j];
    }
    ld_t M[16], rhs[4] = {1, (ld_t)1 / 2, (ld_t)1 / 3, (ld_t)1 / 6};
    for (int j = 0; j < 4; ++j) {
        M[0 * 4 + j] = 1;
        M[1 * 4 + j] = c[j];
        M[2 * 4 + j] = c[j] * c[j];
        M[3 * 4 + j] = Ac[j];
    }
    if (!gauss_solve(4, M, rhs)) return false;
    t.s = 5;
    t.err_order = 3;
    t.start_zero = 0;
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) t.A[i][j] = (double)A[i][j];
    for (int j = 0; j < 5; ++j) {
        t.b[j] = (double)A[4][j];
        t.bh[j] = j < 4 ? (double)rhs[j] : 0.0;
    }
    return true;
}

bool make_tableau(int method, Tab& t) {
    t = Tab();
    if (method == CG_BE || method == CG_YASS) {   // YASS: one backward-Euler Newton iteration
        t.s = 1; t.A[0][0] = 1.0; t.b[0] = 1.0; t.err_order = 0; t.start_zero = 1;
        return true;
    }
    if (method == CG_ROS2) {   // Appendix A.3: gamma, alpha, beta in A, m1, m2 in b
        const double g = 1.0 + std::sqrt(2.0) / 2.0;
        t.s = 2; t.A[0][0] = g; t.A[1][0] = 1.0 / g; t.A[1][1] = -2.0 / g;
        t.b[0] = 3.0 / (2.0 * g); t.b[1] = 1.0 / (2.0 * g);
        t.bh[0] = t.b[0] - 0.5 / g; t.bh[1] = t.b[1] - 0.5 / g;   // embedded: y_n + Gamma_1 / gamma
        t.err_order = 1;
        return true;
    }
    if (method == CG_SDIRK2) {
        const double g = 1.0 - std::sqrt(2.0) / 2.0;
        t.s = 2; t.A[0][0] = g; t.A[1][0] = 1.0 - g; t.A[1][1] = g;
        t.b[0] = 1.0 - g; t.b[1] = g; t.bh[0] = 1.0; t.bh[1] = 0.0; t.err_order = 1;
        return true;
    }
    if (method == CG_SDIRK4) {
        static Tab cached;
        static bool ok = make_sdirk4(cached);
        t = cached;
        return ok;
    }
    return false;
}

template <class T> cg_status upload(std::vector<void*>& allocs, const std::vector<T>& h, const T** out) {
    void* d = nullptr;
    const size_t bytes = std::max<size_t>(1, h.size()) * sizeof(T);
    cudaError_t e = cudaMalloc(&d, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (mechanism)");
    allocs.push_back(d);
    if (!h.empty()) {
        e = cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy (mechanism)");
    }
    *out = static_cast<const T*>(d);
    return CG_OK;
}

}  // namespace

struct cg_mech {
    DevMech dm;
    Layout L;     // FP64 Newton matrix
    Layout L32;   // FP32 Newton matrix (mixed precision)
    Layout LA;    // adjoint sweep (FP64 Newton matrix plus the adjoint arrays)
    int ns = 0, nr = 0;
    std::vector<int> perm;             // internal reaction index -> caller's index
    std::vector<int> itype;            // reaction types, internal order
    std::vector<double> arr, arr0;     // caller's Arrhenius triples (caller's order)
    const int* dperm = nullptr;        // perm on the device
    int tpb = 1;                       // teams per block (team = dm.team threads)
    size_t smem_limit = 0;             // shared memory per cell before arrays spill to scratch
    std::vector<void*> allocs;         // mechanism data
    std::vector<void*> sched_allocs;   // schedules (rebuilt when the team size changes)
    std::vector<Term> wterms, vterms, jterms;
    // device workspace of cg_integrate_host
    int64_t cap = 0;
    double *wT = nullptr, *wY = nullptr, *wP = nullptr;
    int32_t *wStatus = nullptr, *wStats = nullptr;
    cudaStream_t hstream = nullptr;
};

namespace {

// Default launch shape: one warp per cell for small mechanisms (several
// cells per block), two warps per cell from 24 unknowns on, so that every SM
// sub-partition holds two instruction streams, and four warps above 96
// unknowns, with the working set in L2 (below): at 161 unknowns four such
// cells per SM run 1.4 times the rate of one eight-warp cell holding its
// Newton matrix in shared memory (measured, FP64 and FP32 matrices).
int default_team(int n) { return n <= 24 ? 32 : (n <= 96 ? 64 : 128); }

// Default shared memory per cell: everything, unless the per-reaction block
// (rates of progress and their partial derivatives, 9 nr doubles, read by
// the assembly schedules) is what keeps the cells per SM low; then it goes
// to the L2-resident scratch slot and the rest stays in shared memory
// (measured at 53 species / 325 reactions: 6 cells per SM instead of 4,
// 1.29 times the rate).
size_t default_smem_limit(int ns, int nr) {
    const int n = ns + 1, ld = (n % 2) ? n : n + 1;
    // a Newton matrix too large for two cells per SM: the whole working set
    // goes to the L2 slot (the layout keeps the priority order, so nothing
    // after the matrix stays in shared memory either)
    if ((size_t)n * ld * sizeof(double) > kMaxSmemPerBlock / 2) return 64 * 1024;
    // two-warp cells: eight per SM (the register cap allows eight) when the
    // Newton matrix and the arrays placed before it fit in 28 KiB; what does
    // not fit follows the per-reaction block into L2 (53 species: 33,381
    // cells/s against 31,007 at six cells per SM, measured)
    if (default_team(n) == 64) {
        const size_t eighth = 28 * 1024;
        if (!((make_layout(ns, nr, 8, eighth).gmask >> cg::A_G) & 1u)) return eighth;
    }
    const Layout full = make_layout(ns, nr, 8, kMaxSmemPerBlock);
    const size_t rd = 9 * (size_t)nr * sizeof(double);
    const size_t per_cell = (size_t)full.stotal * sizeof(double);
    if ((full.gmask >> cg::A_RD) & 1u || rd < 8 * 1024 || per_cell < 40 * 1024) return kMaxSmemPerBlock;
    return per_cell - rd + 1024;   // the layout keeps 1 KiB of the limit free
}


// Default panel width of the LU: unblocked for small matrices (the
// rank-one loop packs the trailing block into whole warps, the tiles leave
// lanes idle at the ragged edges), panels of 16 above (161 unknowns with the
// matrix in L2: 1.26 times the unblocked rate, fewer L2 accesses per
// multiply-add).
int default_lu_nb(int n) { return n >= 96 ? 16 : 0; }

int default_tpb(int team, const Layout& L) {
    if (team > 32) return 1;
    const size_t per = (size_t)L.stotal * sizeof(double);
    if (per > 24 * 1024) return 1;
    int w = 4;
    while (w > 1 && (size_t)w * per > kMaxSmemPerBlock) --w;
    return w;
}

template <class T> cg_status upload_sched(cg_mech* m, const std::vector<T>& h, const T** out) {
    return upload(m->sched_allocs, h, out);
}

// Reaction chunks of the rates loop for teams of `team` threads: runs of at
// most 32 consecutive reactions (internal order, sorted by type) of one kind
// (plain, falloff, PLOG), so that no warp runs two branches;
// chunks are dealt to the team's warps by estimated cost (a falloff chunk
// about three plain ones), longest first onto the least-loaded warp.
void make_rate_chunks(const std::vector<int>& itype, int team, std::vector<int>& ptr, std::vector<int>& first,
                      std::vector<int>& len) {
    const int nw = team / 32, nr = (int)itype.size();
    struct Chunk { int first, len; double cost; };
    std::vector<Chunk> all;
    // kind 0: elementary and third-body, 1: falloff (Lindemann, Troe, SRI), 2: PLOG
    auto kind = [](int t) { return t == CG_RXN_PLOG ? 2 : (t >= CG_RXN_LINDEMANN ? 1 : 0); };
    for (int j = 0; j < nr;) {
        const int kd = kind(itype[j]);
        int k = j;
        while (k < nr && k - j < 32 && kind(itype[k]) == kd) ++k;
        all.push_back({j, k - j, kd == 0 ? 1.0 : 3.0});
        j = k;
    }
    std::vector<Chunk> order = all;
    std::stable_sort(order.begin(), order.end(), [](const Chunk& a, const Chunk& b) { return a.cost > b.cost; });
    std::vector<std::vector<Chunk>> per(nw);
    std::vector<double> load(nw, 0.0);
    for (const Chunk& c : order) {
        int best = 0;
        for (int w = 1; w < nw; ++w)
            if (load[w] < load[best]) best = w;
        per[best].push_back(c);
        load[best] += c.cost;
    }
    ptr.assign(1, 0);
    first.clear();
    len.clear();
    for (int w = 0; w < nw; ++w) {
        std::sort(per[w].begin(), per[w].end(), [](const Chunk& a, const Chunk& b) { return a.first < b.first; });
        for (const Chunk& c : per[w]) {
            first.push_back(c.first);
            len.push_back(c.len);
        }
        ptr.push_back((int)first.size());
    }
}

cg_status build_schedules(cg_mech* m, int team) {
    for (void* p : m->sched_allocs) cudaFree(p);
    m->sched_allocs.clear();
    const Schedule ws = make_schedule(m->wterms, team), vs = make_schedule(m->vterms, team),
                   js = make_schedule(m->jterms, team);
    std::vector<int> rc_ptr, rc_first, rc_len;
    make_rate_chunks(m->itype, team, rc_ptr, rc_first, rc_len);
    DevMech& dm = m->dm;
    cg_status st;
    if ((st = upload_sched(m, ws.dst, &dm.w_dst)) || (st = upload_sched(m, ws.src, &dm.w_src)) ||
        (st = upload_sched(m, ws.fac, &dm.w_fac)) || (st = upload_sched(m, vs.dst, &dm.v_dst)) ||
        (st = upload_sched(m, vs.src, &dm.v_src)) || (st = upload_sched(m, vs.fac, &dm.v_fac)) ||
        (st = upload_sched(m, js.dst, &dm.j_dst)) || (st = upload_sched(m, js.src, &dm.j_src)) ||
        (st = upload_sched(m, js.fac, &dm.j_fac)) || (st = upload_sched(m, rc_ptr, &dm.rc_ptr)) ||
        (st = upload_sched(m, rc_first, &dm.rc_first)) || (st = upload_sched(m, rc_len, &dm.rc_len)))
        return st;
    dm.w_len = ws.len;
    dm.v_len = vs.len;
    dm.j_len = js.len;
    dm.team = team;
    return CG_OK;
}

// Layout of one cell for the options: the mechanism's own for the LU, one
// with the Krylov arrays for GMRES.
Layout task_layout(const cg_mech* m, const IntParams& P) {
    if (P.linear_solver == 0) return P.precision ? m->L32 : m->L;
    return make_layout(m->ns, m->nr, P.precision ? 4 : 8, m->smem_limit, false, P.gmres_m);
}

cg::Task make_task(const cg_mech* m, const IntParams& P, int64_t N, int64_t first, double* T, double* Y,
                   const double* p, int32_t* status, int32_t* stats) {
    cg::Task t;
    t.M = m->dm;
    t.L = task_layout(m, P);
    t.N = N;
    t.first = first;
    t.T = T;
    t.Y = Y;
    t.p = p;
    t.status = status;
    t.stats = stats;
    t.ckpt = nullptr;
    t.ckpt_n = nullptr;
    t.ckpt_cap = 0;
    return t;
}

cg_status validate(const cg_mech_desc* d) {
    if (!d) return fail(CG_EINVAL, "desc is NULL");
    const int ns = d->n_species, nr = d->n_reactions;
    if (ns < 1 || nr < 0) return fail(CG_EINVAL, "n_species must be >= 1 and n_reactions >= 0");
    if (!d->W || !d->nasa7) return fail(CG_EINVAL, "W and nasa7 are required");
    for (int i = 0; i < ns; ++i) {
        if (!(d->W[i] > 0.0) || !std::isfinite(d->W[i])) return fail(CG_EINVAL, "W[%d] must be positive", i);
        for (int k = 0; k < 7; ++k)
            if (!std::isfinite(d->nasa7[7 * i + k])) return fail(CG_EINVAL, "nasa7[%d][%d] not finite", i, k);
    }
    if (nr == 0) return CG_OK;
    if (!d->rxn_type || !d->reversible || !d->rf_idx || !d->rf_nu || !d->rr_idx || !d->rr_nu ||
        !d->arr || !d->arr0 || !d->troe || !d->eff_ptr)
        return fail(CG_EINVAL, "reaction arrays are required when n_reactions > 0");
    if (d->eff_ptr[0] != 0) return fail(CG_EINVAL, "eff_ptr[0] must be 0");
    if (d->plog_ptr && d->plog_ptr[0] != 0) return fail(CG_EINVAL, "plog_ptr[0] must be 0");
    if (d->plog_ptr)
        for (int j = 0; j < nr; ++j)
            if (d->plog_ptr[j + 1] < d->plog_ptr[j]) return fail(CG_EINVAL, "plog_ptr must be non-decreasing");
    for (int j = 0; j < nr; ++j) {
        const int t = d->rxn_type[j];
        if (t < CG_RXN_ELEMENTARY || t > CG_RXN_PLOG) return fail(CG_EINVAL, "reaction %d: bad type %d", j, t);
        int nf = 0, nb = 0;
        for (int s = 0; s < 3; ++s) {
            const int a = d->rf_idx[3 * j + s], b = d->rr_idx[3 * j + s];
            const int na = d->rf_nu[3 * j + s], nbv = d->rr_nu[3 * j + s];
            if (a < -1 || a >= ns || b < -1 || b >= ns)
                return fail(CG_EINVAL, "reaction %d: species index out of range", j);
            if ((a >= 0) != (na > 0) || (b >= 0) != (nbv > 0) || na < 0 || nbv < 0 || na > 8 || nbv > 8)
                return fail(CG_EINVAL, "reaction %d: coefficients must be 1..8 on used slots, 0 on empty", j);
            for (int s2 = 0; s2 < s; ++s2) {
                if (a >= 0 && d->rf_idx[3 * j + s2] == a) return fail(CG_EINVAL, "reaction %d: repeated reactant", j);
                if (b >= 0 && d->rr_idx[3 * j + s2] == b) return fail(CG_EINVAL, "reaction %d: repeated product", j);
            }
            nf += a >= 0;
            nb += b >= 0;
        }
        if (nf == 0 || nb == 0) return fail(CG_EINVAL, "reaction %d: needs reactants and products", j);
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(d->arr[3 * j + k])) return fail(CG_EINVAL, "reaction %d: arr not finite", j);
        if (t == CG_RXN_LINDEMANN || t == CG_RXN_TROE || t == CG_RXN_SRI)
            for (int k = 0; k < 3; ++k)
                if (!std::isfinite(d->arr0[3 * j + k])) return fail(CG_EINVAL, "reaction %d: arr0 not finite", j);
        if (t == CG_RXN_SRI) {
            if (!d->sri) return fail(CG_EINVAL, "reaction %d is SRI but sri is NULL", j);
            const double* q = d->sri + 5 * j;
            for (int k = 0; k < 5; ++k)
                if (!std::isfinite(q[k])) return fail(CG_EINVAL, "reaction %d: SRI parameters not finite", j);
            if (!(q[0] >= 0.0) || !(q[2] > 0.0) || !(q[3] > 0.0))
                return fail(CG_EINVAL, "reaction %d: SRI needs a >= 0, c > 0, d > 0", j);
        }
        const int p0 = d->plog_ptr ? d->plog_ptr[j] : 0, p1 = d->plog_ptr ? d->plog_ptr[j + 1] : 0;
        if (t == CG_RXN_PLOG) {
            if (!d->plog_ptr || !d->plog) return fail(CG_EINVAL, "reaction %d is PLOG but plog is NULL", j);
            if (p1 <= p0) return fail(CG_EINVAL, "reaction %d: PLOG needs at least one rate expression", j);
            for (int e = p0; e < p1; ++e) {
                const double* q = d->plog + 4 * e;
                if (!(q[0] > 0.0) || !std::isfinite(q[0]) || !std::isfinite(q[1]) || !std::isfinite(q[2]) ||
                    !std::isfinite(q[3]))
                    return fail(CG_EINVAL, "reaction %d: PLOG entry %d invalid", j, e - p0);
                if (e > p0 && q[0] < q[-4]) return fail(CG_EINVAL, "reaction %d: PLOG pressures must not decrease", j);
            }
        } else if (p1 != p0) {
            return fail(CG_EINVAL, "reaction %d: only PLOG reactions take PLOG entries", j);
        }
        if (t == CG_RXN_TROE) {
            const double* tr = d->troe + 4 * j;
            if (!std::isfinite(tr[0]) || !(tr[1] != 0.0) || !(tr[2] != 0.0) || !std::isfinite(tr[1]) ||
                !std::isfinite(tr[2]) || std::isinf(tr[3]))
                return fail(CG_EINVAL, "reaction %d: Troe parameters invalid", j);
        }
        const int e0 = d->eff_ptr[j], e1 = d->eff_ptr[j + 1];
        if (e1 < e0) return fail(CG_EINVAL, "eff_ptr must be non-decreasing (reaction %d)", j);
        if ((t == CG_RXN_ELEMENTARY || t == CG_RXN_PLOG) && e1 != e0)
            return fail(CG_EINVAL, "reaction %d: elementary and PLOG reactions take no efficiencies", j);
        for (int e = e0; e < e1; ++e) {
            if (!d->eff_idx || !d->eff_val) return fail(CG_EINVAL, "eff_idx/eff_val required");
            if (d->eff_idx[e] < 0 || d->eff_idx[e] >= ns)
                return fail(CG_EINVAL, "reaction %d: efficiency species out of range", j);
            if (!std::isfinite(d->eff_val[e])) return fail(CG_EINVAL, "reaction %d: efficiency not finite", j);
        }
    }
    return CG_OK;
}

}  // namespace

extern "C" {

const char* cg_last_error(void) { return g_err.c_str(); }

cg_status cgx_exp_check(const cg_mech* m, int64_t n, const double* x, double* y_tab, double* y_lib,
                        void* stream) {
    if (!m || n < 0 || (n > 0 && (!x || !y_tab || !y_lib))) return fail(CG_EINVAL, "bad arguments");
    cudaError_t e = cg::launch_exp_check(m->dm, n, x, y_tab, y_lib, (cudaStream_t)stream);
    return e == cudaSuccess ? CG_OK : cuda_fail(e, "exp check launch");
}

cg_status cgx_debug_flags(const cg_mech* m, uint64_t* arrays, int64_t* first_cell) {
    if (!m || !arrays || !first_cell) return fail(CG_EINVAL, "bad arguments");
#ifdef CG_DEBUG
    unsigned long long h[2] = {0ull, 0ull};
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(h, m->dm.dbg, sizeof h, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(m->dm.dbg, 0, sizeof h);
    if (e != cudaSuccess) return cuda_fail(e, "debug flags");
    *arrays = h[0];
    *first_cell = (int64_t)h[1] - 1;
    return CG_OK;
#else
    *arrays = 0;
    *first_cell = -1;
    return fail(CG_EUNSUPPORTED, "not a debug build (build with debug=True)");
#endif
}

cg_status cgx_rcp_check(int64_t n, const double* x, double* y, void* stream) {
    if (n < 0 || (n > 0 && (!x || !y))) return fail(CG_EINVAL, "bad arguments");
    cudaError_t e = cg::launch_rcp_check(n, x, y, (cudaStream_t)stream);
    return e == cudaSuccess ? CG_OK : cuda_fail(e, "reciprocal check launch");
}

// ---------------------------------------------------------------------------
// Test hooks on the host-side planners (no device work).

cg_status cgx_schedule(int64_t n_terms, const int* dst, const int* src, const double* fac, const int64_t* order,
                       int lanes, int* len, int* sdst, int* sflags, int* ssrc, double* sfac, int64_t capacity) {
    if (n_terms < 0 || lanes < 1 || lanes > 1024 || !len || (n_terms > 0 && (!dst || !src || !fac || !order)))
        return fail(CG_EINVAL, "bad arguments");
    std::vector<Term> terms((size_t)n_terms);
    for (int64_t i = 0; i < n_terms; ++i) {
        if (dst[i] < 0 || dst[i] > cg::kSchedIndex) return fail(CG_EINVAL, "destination %d out of range", dst[i]);
        terms[(size_t)i] = {dst[i], src[i], fac[i], (long)order[i]};
    }
    const Schedule s = make_schedule(terms, lanes);
    *len = s.len;
    if (!sdst && !sflags && !ssrc && !sfac) return CG_OK;
    const int64_t slots = (int64_t)s.len * lanes;
    if (!sdst || !sflags || !ssrc || !sfac) return fail(CG_EINVAL, "output arrays: all or none");
    if (capacity < slots) return fail(CG_ECAPACITY, "the schedule has %lld slots", (long long)slots);
    for (int64_t k = 0; k < slots; ++k) {
        const int d = s.dst[(size_t)k];
        sdst[k] = d & cg::kSchedIndex;
        sflags[k] = ((d & cg::kSchedFirst) ? 1 : 0) | ((d & cg::kSchedLast) ? 2 : 0);
        ssrc[k] = s.src[(size_t)k];
        sfac[k] = s.fac[(size_t)k];
    }
    return CG_OK;
}

cg_status cgx_rate_chunks(int nr, const int* rxn_type, int team, int* n_chunks, int* warp_ptr, int* first,
                          int* len, int capacity) {
    if (nr < 0 || (nr > 0 && !rxn_type) || !n_chunks || !warp_ptr ||
        (team != 32 && team != 64 && team != 128 && team != 256))
        return fail(CG_EINVAL, "bad arguments");
    std::vector<int> itype(rxn_type, rxn_type + nr), ptr, f, l;
    make_rate_chunks(itype, team, ptr, f, l);
    *n_chunks = (int)f.size();
    for (size_t w = 0; w < ptr.size(); ++w) warp_ptr[w] = ptr[w];
    if (!first && !len) return CG_OK;
    if (!first || !len) return fail(CG_EINVAL, "output arrays: both or none");
    if (capacity < (int)f.size()) return fail(CG_ECAPACITY, "%zu chunks", f.size());
    for (size_t c = 0; c < f.size(); ++c) {
        first[c] = f[c];
        len[c] = l[c];
    }
    return CG_OK;
}

cg_status cgx_layout(int ns, int nr, int mat_bytes, int64_t smem_limit, int adjoint, int gmres_m, int* ld,
                     int* n_arrays, int* offset, int* size, int* in_global, int* priority, int* smem_doubles,
                     int* global_doubles) {
    if (ns < 1 || nr < 0 || (mat_bytes != 4 && mat_bytes != 8) || smem_limit < 0 || gmres_m < 0 || !ld ||
        !n_arrays || !offset || !size || !in_global || !priority || !smem_doubles || !global_doubles)
        return fail(CG_EINVAL, "bad arguments");
    const Layout L = make_layout(ns, nr, mat_bytes, (size_t)smem_limit, adjoint != 0, gmres_m, size, priority);
    *ld = L.ld;
    *n_arrays = cg::A_COUNT;
    for (int a = 0; a < cg::A_COUNT; ++a) {
        offset[a] = L.off[a];
        in_global[a] = (L.gmask >> a) & 1u;
    }
    *smem_doubles = L.stotal;
    *global_doubles = L.gtotal;
    return CG_OK;
}

cg_status cgx_tableau(int method, int* s, double* A, double* b, double* bh, int* err_order) {
    if (!s || !A || !b || !bh || !err_order) return fail(CG_EINVAL, "bad arguments");
    Tab t;
    if (!make_tableau(method, t)) return fail(CG_EINVAL, "no tableau for method %d", method);
    *s = t.s;
    *err_order = t.err_order;
    for (int i = 0; i < 5; ++i) {
        b[i] = t.b[i];
        bh[i] = t.bh[i];
        for (int j = 0; j < 5; ++j) A[5 * i + j] = t.A[i][j];
    }
    return CG_OK;
}

void cg_mech_destroy(cg_mech* m) {
    if (!m) return;
    for (void* p : m->allocs) cudaFree(p);
    for (void* p : m->sched_allocs) cudaFree(p);
    cudaFree(m->wT);
    cudaFree(m->wY);
    cudaFree(m->wP);
    cudaFree(m->wStatus);
    cudaFree(m->wStats);
    if (m->hstream) cudaStreamDestroy(m->hstream);
    delete m;
}

int cg_mech_n_species(const cg_mech* m) { return m ? m->ns : -1; }
int cg_mech_n_reactions(const cg_mech* m) { return m ? m->nr : -1; }

cg_status cg_mech_set_launch(cg_mech* m, int team, int teams_per_block) {
    if (!m) return fail(CG_EINVAL, "mech is NULL");
    if (team != 32 && team != 64 && team != 128 && team != 256)
        return fail(CG_EINVAL, "team must be 32, 64, 128 or 256 threads");
    if (teams_per_block < 1 || (team > 32 && teams_per_block != 1) || team * teams_per_block > 1024)
        return fail(CG_EINVAL, "teams_per_block must be 1 for teams above one warp, and blocks <= 1024 threads");
    if ((size_t)teams_per_block * m->L.stotal * sizeof(double) > kMaxSmemPerBlock)
        return fail(CG_ECAPACITY, "%d cells per block need more than %zu bytes of shared memory",
                    teams_per_block, kMaxSmemPerBlock);
    if (team != m->dm.team) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
        cg_status st = build_schedules(m, team);
        if (st != CG_OK) return st;
    }
    m->tpb = teams_per_block;
    return CG_OK;
}

cg_status cg_mech_set_smem_limit(cg_mech* m, int64_t bytes) {
    if (!m) return fail(CG_EINVAL, "mech is NULL");
    if (bytes < 1024 || bytes > (int64_t)kMaxSmemPerBlock)
        return fail(CG_EINVAL, "limit must be 1 KiB .. %zu bytes", kMaxSmemPerBlock);
    const cg::Layout L = make_layout(m->ns, m->nr, 8, (size_t)bytes);
    const cg::Layout L32 = make_layout(m->ns, m->nr, 4, (size_t)bytes);
    if ((size_t)m->tpb * L.stotal * sizeof(double) > kMaxSmemPerBlock) m->tpb = 1;
    m->L = L;
    m->L32 = L32;
    m->LA = make_layout(m->ns, m->nr, 8, (size_t)bytes, true);
    m->smem_limit = (size_t)bytes;
    return CG_OK;
}

cg_status cg_mech_set_lu_panel(cg_mech* m, int nb) {
    if (!m) return fail(CG_EINVAL, "mech is NULL");
    if (nb < 0 || nb > 64) return fail(CG_EINVAL, "panel width must be 0 (unblocked) .. 64");
    m->dm.lu_nb = nb;
    return CG_OK;
}

int cg_mech_get_lu_panel(const cg_mech* m) { return m ? m->dm.lu_nb : -1; }

int cg_mech_get_launch(const cg_mech* m, int* team, int* teams_per_block) {
    if (!m) return -1;
    if (team) *team = m->dm.team;
    if (teams_per_block) *teams_per_block = m->tpb;
    return 0;
}

cg_status cg_mech_create(const cg_mech_desc* d, cg_mech** out) {
    CG_RANGE("cg_mech_create");
    if (!out) return fail(CG_EINVAL, "out is NULL");
    *out = nullptr;
    cg_status st = validate(d);
    if (st != CG_OK) return st;
    const int ns = d->n_species, nr = d->n_reactions, n = ns + 1;
    if (n > 1024) return fail(CG_ECAPACITY, "at most 1023 species are supported (got %d)", ns);
    const size_t smem_limit = default_smem_limit(ns, nr);
    const Layout L = make_layout(ns, nr, 8, smem_limit);

    // internal reaction order: by type, stable
    std::vector<int> perm(nr);
    for (int j = 0; j < nr; ++j) perm[j] = j;
    std::stable_sort(perm.begin(), perm.end(),
                     [&](int a, int b) { return d->rxn_type[a] < d->rxn_type[b]; });

    // room for the largest degree, so that cg_mech_set_thermo never moves the table
    std::vector<double> th((size_t)cg::th_rows(kMaxThermoDegree) * ns, 0.0), W(ns), invW(ns);
    for (int i = 0; i < ns; ++i) {
        const double* a = d->nasa7 + 7 * i;
        auto T = [&](int r) -> double& { return th[(size_t)r * ns + i]; };
        T(cg::TH_A1) = a[0]; T(cg::TH_A2) = a[1]; T(cg::TH_A3) = a[2]; T(cg::TH_A4) = a[3]; T(cg::TH_A5) = a[4];
        T(cg::TH_H2) = a[1] / 2; T(cg::TH_H3) = a[2] / 3; T(cg::TH_H4) = a[3] / 4; T(cg::TH_H5) = a[4] / 5;
        T(cg::TH_A6) = a[5];
        T(cg::TH_S3) = a[2] / 2; T(cg::TH_S4) = a[3] / 3; T(cg::TH_S5) = a[4] / 4;
        T(cg::TH_A7) = a[6];
        T(cg::TH_D3) = 2 * a[2]; T(cg::TH_D4) = 3 * a[3]; T(cg::TH_D5) = 4 * a[4];
        W[i] = d->W[i];
        invW[i] = 1.0 / d->W[i];
    }

    std::vector<int> rtype(nr), rev(nr), sumnu(nr), sidx(6 * (size_t)nr, -1), snu(6 * (size_t)nr, 0),
        hasT2(nr, 0), eff_ptr(nr + 1, 0), eff_idx;
    std::vector<double> lnA(nr), beta(nr), Ta(nr), dlnA0(nr, 0.0), dbeta0(nr, 0.0), dTa0(nr, 0.0),
        talpha(nr, 0.0), tiT3(nr, 0.0), tiT1(nr, 0.0), tT2(nr, 0.0), eff_am1, snud(6 * (size_t)nr, 0.0),
        sumnud(nr, 0.0), sri(5 * (size_t)nr, 0.0), pl_lnp, pl_lnA, pl_b, pl_Ta;
    std::vector<int> pl_lev(nr + 1, 0), pl_rate;
    std::vector<Term> wterms, vterms, jterms;
    std::vector<double> nu(ns);
    for (int jj = 0; jj < nr; ++jj) {
        const int j = perm[jj];
        rtype[jj] = d->rxn_type[j];
        rev[jj] = d->reversible[j] ? 1 : 0;
        int sn = 0;
        std::fill(nu.begin(), nu.end(), 0.0);
        for (int s = 0; s < 3; ++s) {
            const int a = d->rf_idx[3 * j + s], b = d->rr_idx[3 * j + s];
            sidx[(size_t)s * nr + jj] = a;
            snu[(size_t)s * nr + jj] = a >= 0 ? d->rf_nu[3 * j + s] : 0;
            sidx[(size_t)(3 + s) * nr + jj] = b;
            snu[(size_t)(3 + s) * nr + jj] = b >= 0 ? d->rr_nu[3 * j + s] : 0;
            if (a >= 0) { sn -= d->rf_nu[3 * j + s]; nu[a] -= d->rf_nu[3 * j + s]; }
            if (b >= 0) { sn += d->rr_nu[3 * j + s]; nu[b] += d->rr_nu[3 * j + s]; }
        }
        sumnu[jj] = sn;
        sumnud[jj] = sn;
        for (int s = 0; s < 6; ++s) snud[(size_t)s * nr + jj] = snu[(size_t)s * nr + jj];
        lnA[jj] = d->arr[3 * j];
        beta[jj] = d->arr[3 * j + 1];
        Ta[jj] = d->arr[3 * j + 2] / kR;
        const bool fall = rtype[jj] == CG_RXN_LINDEMANN || rtype[jj] == CG_RXN_TROE || rtype[jj] == CG_RXN_SRI;
        if (rtype[jj] == CG_RXN_SRI) {
            const double* q = d->sri + 5 * j;
            sri[0 * (size_t)nr + jj] = q[0];
            sri[1 * (size_t)nr + jj] = q[1];
            sri[2 * (size_t)nr + jj] = 1.0 / q[2];
            sri[3 * (size_t)nr + jj] = std::log(q[3]);
            sri[4 * (size_t)nr + jj] = q[4];
        }
        if (rtype[jj] == CG_RXN_PLOG) {   // levels of equal pressure, each with its rates
            for (int e = d->plog_ptr[j]; e < d->plog_ptr[j + 1]; ++e) {
                const double* q = d->plog + 4 * e;
                if (e == d->plog_ptr[j] || q[0] != q[-4]) {
                    pl_lnp.push_back(std::log(q[0]));
                    pl_rate.push_back((int)pl_lnA.size());
                }
                pl_lnA.push_back(q[1]);
                pl_b.push_back(q[2]);
                pl_Ta.push_back(q[3] / kR);
            }
        }
        pl_lev[jj + 1] = (int)pl_lnp.size();
        if (fall) {
            dlnA0[jj] = d->arr0[3 * j] - d->arr[3 * j];
            dbeta0[jj] = d->arr0[3 * j + 1] - d->arr[3 * j + 1];
            dTa0[jj] = (d->arr0[3 * j + 2] - d->arr[3 * j + 2]) / kR;
        }
        if (rtype[jj] == CG_RXN_TROE) {
            const double* tr = d->troe + 4 * j;
            talpha[jj] = tr[0];
            tiT3[jj] = 1.0 / tr[1];
            tiT1[jj] = 1.0 / tr[2];
            hasT2[jj] = std::isnan(tr[3]) ? 0 : 1;
            tT2[jj] = hasT2[jj] ? tr[3] : 0.0;
        }
        std::vector<std::pair<int, double>> effs;
        for (int e = d->eff_ptr[j]; e < d->eff_ptr[j + 1]; ++e) {
            eff_idx.push_back(d->eff_idx[e]);
            eff_am1.push_back(d->eff_val[e] - 1.0);
            effs.push_back({d->eff_idx[e], d->eff_val[e] - 1.0});
        }
        eff_ptr[jj + 1] = (int)eff_idx.size();

        // schedule terms of this reaction, in a fixed order per destination
        const bool press = rtype[jj] != CG_RXN_ELEMENTARY;
        for (int i = 0; i < ns; ++i) {
            if (nu[i] == 0.0) continue;
            const long base_order = (long)jj * 64;
            wterms.push_back({1 + i, 0 * nr + jj, nu[i], base_order});
            if (press) vterms.push_back({i, 2 * nr + jj, nu[i], base_order});
            const int row = (1 + i) * L.ld;
            jterms.push_back({row + 0, 1 * nr + jj, nu[i], base_order});
            for (int s = 0; s < 6; ++s) {
                const int sp = sidx[(size_t)s * nr + jj];
                if (sp >= 0) jterms.push_back({row + 1 + sp, (3 + s) * nr + jj, nu[i], base_order + 1 + s});
            }
            if (press)
                for (size_t e = 0; e < effs.size(); ++e)
                    jterms.push_back({row + 1 + effs[e].first, 2 * nr + jj, nu[i] * effs[e].second,
                                      base_order + 8 + (long)e});
        }
    }

    cg_mech* m = new cg_mech();
    m->ns = ns;
    m->nr = nr;
    m->L = L;
    m->L32 = make_layout(ns, nr, 4, smem_limit);
    m->LA = make_layout(ns, nr, 8, smem_limit, true);
    m->smem_limit = smem_limit;
    m->perm = perm;
    m->itype = rtype;
    m->arr.assign(d->arr, d->arr + 3 * (size_t)nr);
    m->arr0.assign(d->arr0 ? d->arr0 : d->arr, (d->arr0 ? d->arr0 : d->arr) + 3 * (size_t)nr);
    DevMech& dm = m->dm;
    dm.ns = ns;
    dm.nr = nr;
    dm.n = n;
    dm.ln_pref_R = std::log(kPref / kR);
    dm.th_np = 4;
    dm.lu_nb = default_lu_nb(n);
    dm.slots = 2;
    for (int jj = 0; jj < nr; ++jj)
        if (sidx[(size_t)2 * nr + jj] >= 0 || sidx[(size_t)5 * nr + jj] >= 0) dm.slots = 3;
#define UP(vec, field)                                           \
    if ((st = upload(m->allocs, vec, &dm.field)) != CG_OK) {     \
        cg_mech_destroy(m);                                      \
        return st;                                               \
    }
    UP(th, th) UP(W, W) UP(invW, invW) UP(rtype, rtype) UP(rev, rev) UP(sumnu, sumnu)
    UP(sidx, sidx) UP(snu, snu) UP(snud, snud) UP(sumnud, sumnud) UP(lnA, lnA) UP(beta, beta) UP(Ta, Ta) UP(dlnA0, dlnA0)
    UP(dbeta0, dbeta0) UP(dTa0, dTa0) UP(talpha, talpha) UP(tiT3, tiT3) UP(tiT1, tiT1)
    UP(tT2, tT2) UP(hasT2, hasT2) UP(eff_ptr, eff_ptr) UP(eff_idx, eff_idx) UP(eff_am1, eff_am1)
    UP(sri, sri)
#undef UP
    pl_rate.push_back((int)pl_lnA.size());
    dm.has_plog = pl_lnp.empty() ? 0 : 1;
#define UP(vec, field)                                           \
    if ((st = upload(m->allocs, vec, &dm.field)) != CG_OK) {     \
        cg_mech_destroy(m);                                      \
        return st;                                               \
    }
    UP(pl_lev, pl_lev) UP(pl_rate, pl_rate) UP(pl_lnp, pl_lnp) UP(pl_lnA, pl_lnA) UP(pl_b, pl_b) UP(pl_Ta, pl_Ta)
#undef UP
    if ((st = upload(m->allocs, perm, &m->dperm)) != CG_OK) {
        cg_mech_destroy(m);
        return st;
    }
#ifdef CG_DEBUG
    {
        const std::vector<unsigned long long> zero(2, 0ull);
        const unsigned long long* dbg = nullptr;
        if ((st = upload(m->allocs, zero, &dbg)) != CG_OK) {
            cg_mech_destroy(m);
            return st;
        }
        dm.dbg = const_cast<unsigned long long*>(dbg);
    }
#endif
    std::vector<double> exp2j(64);   // 2^(j/64), rounded once from extended precision
    for (int j = 0; j < 64; ++j) exp2j[j] = (double)std::exp2((long double)j / 64.0L);
    if ((st = upload(m->allocs, exp2j, &dm.exp2j)) != CG_OK) {
        cg_mech_destroy(m);
        return st;
    }
    m->wterms.swap(wterms);
    m->vterms.swap(vterms);
    m->jterms.swap(jterms);
    const int team = default_team(n);
    if ((st = build_schedules(m, team)) != CG_OK) {
        cg_mech_destroy(m);
        return st;
    }
    m->tpb = default_tpb(team, L);
    *out = m;
    return CG_OK;
}

cg_status cg_eval_rates(const cg_mech* m, int reactor, int64_t N, const double* T, const double* C,
                        double* S, void* stream) {
    CG_RANGE("cg_eval_rates");
    if (!m) return fail(CG_EINVAL, "mech is NULL");
    if (N < 0 || reactor < CG_CONV || reactor > CG_CONP_LITERAL) return fail(CG_EINVAL, "bad N or reactor");
    if (N == 0) return CG_OK;
    if (!T || !C || !S) return fail(CG_EINVAL, "NULL array");
    cudaError_t e = cg::launch_eval_rates(m->dm, m->L, m->tpb, reactor, N, T, C, S,
                                          (cudaStream_t)stream);
    return e == cudaSuccess ? CG_OK : cuda_fail(e, "eval_rates launch");
}

cg_status cg_eval_jacobian(const cg_mech* m, int reactor, int64_t N, const double* T, const double* C,
                           double* J, void* stream) {
    CG_RANGE("cg_eval_jacobian");
    if (!m) return fail(CG_EINVAL, "mech is NULL");
    if (N < 0 || reactor < CG_CONV || reactor > CG_CONP_LITERAL) return fail(CG_EINVAL, "bad N or reactor");
    if (N == 0) return CG_OK;
    if (!T || !C || !J) return fail(CG_EINVAL, "NULL array");
    cudaError_t e = cg::launch_eval_jacobian(m->dm, m->L, m->tpb, reactor, N, T, C, J,
                                             (cudaStream_t)stream);
    return e == cudaSuccess ? CG_OK : cuda_fail(e, "eval_jacobian launch");
}

cg_status cg_temperature_from_energy(const cg_mech* m, int reactor, int64_t N, const double* e,
                                     const double* Y, double* T, int iters, void* stream) {
    CG_RANGE("cg_temperature_from_energy");
    if (!m) return fail(CG_EINVAL, "mech is NULL");
    if (N < 0 || iters < 0 || reactor < CG_CONV || reactor > CG_CONP_LITERAL)
        return fail(CG_EINVAL, "bad N, iters or reactor");
    if (N == 0) return CG_OK;
    if (!e || !Y || !T) return fail(CG_EINVAL, "NULL array");
    cudaError_t err = cg::launch_temperature(m->dm, reactor, N, e, Y, T, iters, (cudaStream_t)stream);
    return err == cudaSuccess ? CG_OK : cuda_fail(err, "temperature launch");
}

void cg_integrate_opts_default(cg_integrate_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->method = CG_SDIRK4;
    o->reactor = CG_CONP;
    o->adaptive = 1;
    o->precision = CG_FP64;
    o->nsub = 1;
    o->max_newton = 7;
    o->max_steps = 100000;
    o->max_halvings = 10;
    o->err_filter = 1;
    o->dt = 1e-6;
    o->rtol = 1e-6;
    o->atol = 1e-12;
    o->newton_tol = 0.03;
    o->h0 = 0.0;
    o->hmin = 1e-20;
    o->neg_tol = 1e-6;
    o->linear_solver = CG_LU;
    o->preconditioner = CG_PC_GAUSS_SEIDEL;
    o->gmres_restart = 30;
    o->gmres_maxit = 200;
    o->gmres_tol = 1e-10;
}

static cg_status make_params(const cg_integrate_opts* o, IntParams& P) {
    if (!o) return fail(CG_EINVAL, "opts is NULL");
    if (o->method < CG_BE || o->method > CG_YASS) return fail(CG_EINVAL, "bad method");
    if (o->precision == CG_FP32LU && (o->method == CG_ROS2 || o->method == CG_YASS))
        return fail(CG_EUNSUPPORTED, "Rosenbrock-2 and YASS take no Newton correction: FP64 factorisation only");
    if (o->reactor < CG_CONV || o->reactor > CG_CONP_LITERAL) return fail(CG_EINVAL, "bad reactor");
    if (o->precision != CG_FP64 && o->precision != CG_FP32LU)
        return fail(CG_EINVAL, "bad precision %d", o->precision);
    if (!(o->dt > 0.0) || !std::isfinite(o->dt)) return fail(CG_EINVAL, "dt must be positive");
    if (o->nsub < 1 || o->max_newton < 1 || o->max_steps < 1 || o->max_halvings < 0 || o->max_halvings > 40)
        return fail(CG_EINVAL, "nsub, max_newton, max_steps >= 1 and 0 <= max_halvings <= 40 required");
    if (!(o->rtol >= 0.0) || !(o->atol >= 0.0) || !(o->rtol + o->atol > 0.0) || !(o->newton_tol > 0.0) ||
        !(o->hmin >= 0.0) || !(o->h0 >= 0.0) || !(o->neg_tol >= 0.0))
        return fail(CG_EINVAL, "tolerances must be non-negative (rtol + atol and newton_tol positive)");
    if (o->linear_solver != CG_LU && o->linear_solver != CG_GMRES) return fail(CG_EINVAL, "bad linear_solver");
    if (o->linear_solver == CG_GMRES &&
        (o->preconditioner < CG_PC_NONE || o->preconditioner > CG_PC_GAUSS_SEIDEL || o->gmres_restart < 1 ||
         o->gmres_restart > 64 || o->gmres_maxit < 1 || !(o->gmres_tol > 0.0)))
        return fail(CG_EINVAL, "GMRES needs a preconditioner 0..2, 1 <= gmres_restart <= 64, gmres_maxit >= 1 "
                               "and gmres_tol > 0");
    Tab t;
    if (!make_tableau(o->method, t)) return fail(CG_EINVAL, "tableau construction failed");
    P.method = o->method;
    P.reactor = o->reactor;
    P.adaptive = (o->adaptive && o->method != CG_BE && o->method != CG_YASS) ? 1 : 0;
    P.nsub = o->nsub;
    P.max_newton = o->method == CG_YASS ? 1 : o->max_newton;
    P.max_steps = o->max_steps;
    P.max_halvings = o->max_halvings;
    P.err_filter = o->err_filter;
    P.precision = o->precision;
    P.dt = o->dt;
    P.rtol = o->rtol;
    P.atol = o->atol;
    P.newton_tol = o->newton_tol;
    P.h0 = o->h0;
    P.hmin = o->hmin;
    P.neg_tol = o->neg_tol;
    P.linear_solver = o->linear_solver;
    P.prec = o->preconditioner;
    P.gmres_m = o->linear_solver == CG_GMRES ? o->gmres_restart : 0;
    P.gmres_maxit = o->gmres_maxit;
    P.gmres_tol = o->gmres_tol;
    P.s = t.s;
    P.err_order = t.err_order;
    P.start_zero = t.start_zero;
    for (int i = 0; i < 5; ++i) {
        for (int j = 0; j < 5; ++j) P.A[i][j] = t.A[i][j];
        P.b[i] = t.b[i];
        P.bh[i] = t.bh[i];
    }
    return CG_OK;
}

cg_status cg_integrate(const cg_mech* m, const cg_integrate_opts* o, int64_t N, double* T, double* Y,
                       const double* p_or_rho, int32_t* cell_status, int32_t* cell_stats,
                       void* stream) {
    CG_RANGE("cg_integrate");
    if (!m) return fail(CG_EINVAL, "mech is NULL");
    IntParams P;
    cg_status st = make_params(o, P);
    if (st != CG_OK) return st;
    if (N < 0) return fail(CG_EINVAL, "N < 0");
    if (N == 0) return CG_OK;
    if (!T || !Y || !p_or_rho) return fail(CG_EINVAL, "NULL array");
    cg::Tasks tasks;
    tasks.count = 1;
    tasks.total = N;
    tasks.t[0] = make_task(m, P, N, 0, T, Y, p_or_rho, cell_status, cell_stats);
    cudaError_t e = cg::launch_integrate(tasks, P, m->dm.team, m->tpb, o->persistent != 0,
                                         (cudaStream_t)stream);
    return e == cudaSuccess ? CG_OK : cuda_fail(e, "integrate launch");
}

cg_status cg_integrate_batch(int n_mech, const cg_mech* const* mechs, const int64_t* N,
                             double* const* T, double* const* Y, const double* const* p_or_rho,
                             int32_t* const* cell_status, int32_t* const* cell_stats,
                             const cg_integrate_opts* o, void* stream) {
    CG_RANGE("cg_integrate_batch");
    if (n_mech < 1 || n_mech > cg::kMaxTasks)
        return fail(CG_EINVAL, "n_mech must be 1..%d", cg::kMaxTasks);
    if (!mechs || !N || !T || !Y || !p_or_rho) return fail(CG_EINVAL, "NULL array");
    IntParams P;
    cg_status st = make_params(o, P);
    if (st != CG_OK) return st;
    cg::Tasks tasks;
    tasks.count = n_mech;
    tasks.total = 0;
    tasks.total_split = 0;
    // the launch's team size is the largest; one-warp mechanisms in a wider
    // launch run split (each warp of a team integrates its own cells)
    int team = 0;
    for (int k = 0; k < n_mech; ++k) {
        if (!mechs[k]) return fail(CG_EINVAL, "mechs[%d] is NULL", k);
        team = std::max(team, mechs[k]->dm.team);
    }
    int tpb = 1 << 30;
    for (int k = 0; k < n_mech; ++k) {
        const cg_mech* m = mechs[k];
        const bool split = m->dm.team < team;
        if (split && m->dm.team != 32)
            return fail(CG_EINVAL, "a batch may mix one-warp mechanisms with one wider team size; mechanism %d has "
                                   "%d threads per cell in a launch of %d (cg_mech_set_launch)", k, m->dm.team, team);
        if (N[k] < 0) return fail(CG_EINVAL, "N[%d] < 0", k);
        if (N[k] > 0 && (!T[k] || !Y[k] || !p_or_rho[k])) return fail(CG_EINVAL, "NULL array for mechanism %d", k);
        int64_t& space = split ? tasks.total_split : tasks.total;
        tasks.t[k] = make_task(m, P, N[k], space, T[k], Y[k], p_or_rho[k],
                               cell_status ? cell_status[k] : nullptr, cell_stats ? cell_stats[k] : nullptr);
        tasks.t[k].split = split ? 1 : 0;
        space += N[k];
        if (!split) tpb = std::min(tpb, m->tpb);
    }
    if (tasks.total + tasks.total_split == 0) return CG_OK;
    cudaError_t e = cg::launch_integrate(tasks, P, team, tpb, true, (cudaStream_t)stream);
    return e == cudaSuccess ? CG_OK : cuda_fail(e, "integrate launch");
}

// Operator-split reaction step of a compressible flow solver.
cg_status cg_react_split(const cg_mech* m, const cg_integrate_opts* o, int64_t N, const double* rho,
                         const double* e, const double* rhoY, double* T, double* R, int iters,
                         int32_t* cell_status, int32_t* cell_stats, void* stream) {
    CG_RANGE("cg_react_split");
    if (!m) return fail(CG_EINVAL, "mech is NULL");
    IntParams P;
    cg_status st = make_params(o, P);
    if (st != CG_OK) return st;
    if (o->reactor != CG_CONV) return fail(CG_EINVAL, "the split reaction step is at constant volume (CG_CONV)");
    if (N < 0 || iters < 0 || iters > 100) return fail(CG_EINVAL, "N >= 0 and 0 <= iters <= 100 required");
    if (N == 0) return CG_OK;
    if (!rho || !e || !rhoY || !T || !R) return fail(CG_EINVAL, "NULL array");
    cg::SplitTask t;
    t.M = m->dm;
    t.L = task_layout(m, P);
    t.N = N;
    t.rho = rho;
    t.e = e;
    t.rhoY = rhoY;
    t.T = T;
    t.R = R;
    t.status = cell_status;
    t.stats = cell_stats;
    t.iters = iters;
    cudaError_t err = cg::launch_react_split(t, P, m->dm.team, m->tpb, (cudaStream_t)stream);
    return err == cudaSuccess ? CG_OK : cuda_fail(err, "react_split launch");
}

// Forward integration that records the checkpoints of the adjoint.
cg_status cg_integrate_ckpt(const cg_mech* m, const cg_integrate_opts* o, int64_t N, double* T, double* Y,
                            const double* p_or_rho, int32_t* cell_status, int32_t* cell_stats, double* ckpt,
                            int32_t* ckpt_n, int ckpt_cap, void* stream) {
    CG_RANGE("cg_integrate_ckpt");
    if (!m) return fail(CG_EINVAL, "mech is NULL");
    IntParams P;
    cg_status st = make_params(o, P);
    if (st != CG_OK) return st;
    if (N < 0 || ckpt_cap < 2) return fail(CG_EINVAL, "N >= 0 and ckpt_cap >= 2 required");
    if (N == 0) return CG_OK;
    if (!T || !Y || !p_or_rho || !ckpt || !ckpt_n) return fail(CG_EINVAL, "NULL array");
    cg::Tasks tasks;
    tasks.count = 1;
    tasks.total = N;
    tasks.t[0] = make_task(m, P, N, 0, T, Y, p_or_rho, cell_status, cell_stats);
    tasks.t[0].ckpt = ckpt;
    tasks.t[0].ckpt_n = ckpt_n;
    tasks.t[0].ckpt_cap = ckpt_cap;
    cudaError_t e = cg::launch_integrate(tasks, P, m->dm.team, m->tpb, o->persistent != 0,
                                         (cudaStream_t)stream);
    return e == cudaSuccess ? CG_OK : cuda_fail(e, "integrate launch (checkpoints)");
}

// Backward sweep of the discrete adjoint over the checkpoints of
// cg_integrate_ckpt.
cg_status cg_integrate_adjoint(const cg_mech* m, const cg_integrate_opts* o, int64_t N, const double* ckpt,
                               const int32_t* ckpt_n, int ckpt_cap, const double* dT_end, const double* dY_end,
                               double* dT0, double* dY0, double* dtheta, double* dtheta_cells,
                               int32_t* cell_status, void* stream) {
    CG_RANGE("cg_integrate_adjoint");
    if (!m) return fail(CG_EINVAL, "mech is NULL");
    IntParams P;
    cg_status st = make_params(o, P);
    if (st != CG_OK) return st;
    if (N < 0 || ckpt_cap < 2) return fail(CG_EINVAL, "N >= 0 and ckpt_cap >= 2 required");
    if (o->method == CG_ROS2 || o->method == CG_YASS)
        return fail(CG_EUNSUPPORTED, "the adjoint covers backward Euler and SDIRK");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (N == 0) {
        if (dtheta && m->nr > 0 &&
            (e = cudaMemsetAsync(dtheta, 0, 3 * (size_t)m->nr * sizeof(double), s)) != cudaSuccess)
            return cuda_fail(e, "cudaMemsetAsync");
        return CG_OK;
    }
    if (!ckpt || !ckpt_n || !dT_end || !dY_end || !dT0 || !dY0) return fail(CG_EINVAL, "NULL array");
    const cg::Layout LA = P.linear_solver ? make_layout(m->ns, m->nr, 8, m->smem_limit, true, P.gmres_m) : m->LA;
    int tpb = m->dm.team > 32 ? 1 : m->tpb;
    while (tpb > 1 && (size_t)tpb * LA.stotal * sizeof(double) > kMaxSmemPerBlock) --tpb;
    if ((size_t)LA.stotal * sizeof(double) > kMaxSmemPerBlock)
        return fail(CG_ECAPACITY, "adjoint arrays need %zu bytes of shared memory per cell",
                    (size_t)LA.stotal * sizeof(double));
    cg::AdjTask t;
    t.M = m->dm;
    t.L = LA;
    t.N = N;
    t.ckpt = ckpt;
    t.ckpt_n = ckpt_n;
    t.ckpt_cap = ckpt_cap;
    t.dT_end = dT_end;
    t.dY_end = dY_end;
    t.dT0 = dT0;
    t.dY0 = dY0;
    t.perm = m->dperm;
    t.grad_cells = dtheta_cells;
    t.status = cell_status;
    void* tmp = nullptr;
    if (!t.grad_cells && m->nr > 0) {   // per-cell gradients in a stream-ordered temporary
        if ((e = cudaMallocAsync(&tmp, 3 * (size_t)m->nr * N * sizeof(double), s)) != cudaSuccess)
            return cuda_fail(e, "cudaMallocAsync (per-cell gradients)");
        t.grad_cells = static_cast<double*>(tmp);
    }
    e = cg::launch_adjoint(t, P, m->dm.team, tpb, dtheta, s);
    cudaError_t e2 = tmp ? cudaFreeAsync(tmp, s) : cudaSuccess;
    if (e != cudaSuccess) return cuda_fail(e, "adjoint launch");
    return e2 == cudaSuccess ? CG_OK : cuda_fail(e2, "cudaFreeAsync");
}

cg_status cg_mech_set_arrhenius(cg_mech* m, const double* arr) {
    CG_RANGE("cg_mech_set_arrhenius");
    if (!m) return fail(CG_EINVAL, "mech is NULL");
    const int nr = m->nr;
    if (nr == 0) return CG_OK;
    if (!arr) return fail(CG_EINVAL, "arr is NULL");
    for (int k = 0; k < 3 * nr; ++k)
        if (!std::isfinite(arr[k])) return fail(CG_EINVAL, "arr[%d] not finite", k);
    std::vector<double> lnA(nr), beta(nr), Ta(nr), dlnA0(nr, 0.0), dbeta0(nr, 0.0), dTa0(nr, 0.0);
    const std::vector<int>& types = m->itype;
    for (int jj = 0; jj < nr; ++jj) {
        const int j = m->perm[jj];
        lnA[jj] = arr[3 * j];
        beta[jj] = arr[3 * j + 1];
        Ta[jj] = arr[3 * j + 2] / kR;
        if (types[jj] == CG_RXN_LINDEMANN || types[jj] == CG_RXN_TROE || types[jj] == CG_RXN_SRI) {   // k_0 kept
            dlnA0[jj] = m->arr0[3 * j] - arr[3 * j];
            dbeta0[jj] = m->arr0[3 * j + 1] - arr[3 * j + 1];
            dTa0[jj] = (m->arr0[3 * j + 2] - arr[3 * j + 2]) / kR;
        }
    }
    const size_t b = nr * sizeof(double);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    if ((e = cudaMemcpy(const_cast<double*>(m->dm.lnA), lnA.data(), b, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(const_cast<double*>(m->dm.beta), beta.data(), b, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(const_cast<double*>(m->dm.Ta), Ta.data(), b, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(const_cast<double*>(m->dm.dlnA0), dlnA0.data(), b, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(const_cast<double*>(m->dm.dbeta0), dbeta0.data(), b, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(const_cast<double*>(m->dm.dTa0), dTa0.data(), b, cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpy (Arrhenius parameters)");
    m->arr.assign(arr, arr + 3 * (size_t)nr);
    return CG_OK;
}

namespace {

// The device thermo table of a c_p polynomial of degree np (layout of
// cg::th_rows); returns the table's degree P = max(np, 4), since degrees
// below 4 are the NASA-7 form with zero upper coefficients.
cg_status thermo_table(int ns, int np, const double* coef, int* P_out, std::vector<double>& th) {
    if (np < 0 || np > kMaxThermoDegree) return fail(CG_EINVAL, "degree %d outside [0, %d]", np, kMaxThermoDegree);
    if (ns > 0 && !coef) return fail(CG_EINVAL, "coef is NULL");
    for (int k = 0; k < ns * (np + 3); ++k)
        if (!std::isfinite(coef[k])) return fail(CG_EINVAL, "coef[%d] not finite", k);
    const int P = std::max(np, 4);
    th.assign((size_t)cg::th_rows(P) * ns, 0.0);
    for (int i = 0; i < ns; ++i) {
        const double* c = coef + (size_t)i * (np + 3);
        auto a = [&](int k) { return k <= np ? c[k] : 0.0; };
        auto T = [&](int r) -> double& { return th[(size_t)r * ns + i]; };
        for (int k = 0; k <= P; ++k) T(k) = a(k);
        for (int k = 1; k <= P; ++k) T(P + k) = a(k) / (k + 1);
        T(2 * P + 1) = c[np + 1];
        for (int k = 2; k <= P; ++k) T(2 * P + k) = a(k) / k;
        T(3 * P + 1) = c[np + 2];
        for (int k = 2; k <= P; ++k) T(3 * P + k) = k * a(k);
    }
    *P_out = P;
    return CG_OK;
}

}  // namespace

cg_status cgx_thermo_table(int ns, int np, const double* coef, int* P, double* table, int64_t capacity) {
    if (ns < 1 || !P) return fail(CG_EINVAL, "bad arguments");
    std::vector<double> th;
    cg_status st = thermo_table(ns, np, coef, P, th);
    if (st != CG_OK || !table) return st;
    if (capacity < (int64_t)th.size()) return fail(CG_ECAPACITY, "the table has %zu entries", th.size());
    std::copy(th.begin(), th.end(), table);
    return CG_OK;
}

cg_status cg_mech_set_thermo(cg_mech* m, int np, const double* coef) {
    CG_RANGE("cg_mech_set_thermo");
    if (!m) return fail(CG_EINVAL, "mech is NULL");
    std::vector<double> th;
    int P = 4;
    cg_status st = thermo_table(m->ns, np, coef, &P, th);
    if (st != CG_OK) return st;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    if ((e = cudaMemcpy(const_cast<double*>(m->dm.th), th.data(), th.size() * sizeof(double),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpy (thermo table)");
    m->dm.th_np = P;
    return CG_OK;
}

cg_status cg_integrate_host(const cg_mech* mc, const cg_integrate_opts* o, int64_t N, double* T,
                            double* Y, const double* p_or_rho, int32_t* cell_status,
                            int32_t* cell_stats) {
    CG_RANGE("cg_integrate_host");
    if (!mc) return fail(CG_EINVAL, "mech is NULL");
    cg_mech* m = const_cast<cg_mech*>(mc);
    IntParams P;
    cg_status st = make_params(o, P);
    if (st != CG_OK) return st;
    if (N < 0) return fail(CG_EINVAL, "N < 0");
    if (N == 0) return CG_OK;
    if (!T || !Y || !p_or_rho) return fail(CG_EINVAL, "NULL array");
    cudaError_t e;
    if (!m->hstream && (e = cudaStreamCreateWithFlags(&m->hstream, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamCreate");
    if (N > m->cap) {
        cudaFree(m->wT); cudaFree(m->wY); cudaFree(m->wP); cudaFree(m->wStatus); cudaFree(m->wStats);
        m->wT = m->wY = m->wP = nullptr;
        m->wStatus = m->wStats = nullptr;
        m->cap = 0;
        if ((e = cudaMalloc(&m->wT, N * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc(&m->wY, N * m->ns * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc(&m->wP, N * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc(&m->wStatus, N * sizeof(int32_t))) != cudaSuccess ||
            (e = cudaMalloc(&m->wStats, 4 * N * sizeof(int32_t))) != cudaSuccess)
            return cuda_fail(e, "cudaMalloc (host-call workspace)");
        m->cap = N;
    }
    cudaStream_t s = m->hstream;
    if ((e = cudaMemcpyAsync(m->wT, T, N * sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(m->wY, Y, N * m->ns * sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(m->wP, p_or_rho, N * sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync H2D");
    cg::Tasks tasks;
    tasks.count = 1;
    tasks.total = N;
    tasks.t[0] = make_task(m, P, N, 0, m->wT, m->wY, m->wP, m->wStatus, m->wStats);
    if ((e = cg::launch_integrate(tasks, P, m->dm.team, m->tpb, o->persistent != 0, s)) != cudaSuccess)
        return cuda_fail(e, "integrate launch");
    if ((e = cudaMemcpyAsync(T, m->wT, N * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(Y, m->wY, N * m->ns * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync D2H");
    if (cell_status &&
        (e = cudaMemcpyAsync(cell_status, m->wStatus, N * sizeof(int32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync D2H");
    if (cell_stats &&
        (e = cudaMemcpyAsync(cell_stats, m->wStats, 4 * N * sizeof(int32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync D2H");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return CG_OK;
}

// Autotuner: time cg_integrate on a sample of cells for every launch shape
// (threads per cell, cells per block, shared-memory limit) that fits, keep
// the fastest. The sample is integrated from a fresh copy of its inputs for
// each timing; the caller's arrays are not modified.
cg_status cg_autotune(cg_mech* m, const cg_integrate_opts* o, int64_t N, const double* T, const double* Y,
                      const double* p_or_rho, const char* cache_json, void* stream, double* best_ms) {
    CG_RANGE("cg_autotune");
    if (!m) return fail(CG_EINVAL, "mech is NULL");
    IntParams P;
    cg_status st = make_params(o, P);
    if (st != CG_OK) return st;
    if (N <= 0 || !T || !Y || !p_or_rho) return fail(CG_EINVAL, "a non-empty sample is required");
    if (cache_json) {   // reuse a previous result for the same mechanism size and options
        FILE* f = fopen(cache_json, "r");
        if (f) {
            int ns = -1, nr = -1, prec = -1, method = -1, team = 0, tpb = 0, nb = -1;
            long long lim = 0;
            double ms = 0;
            const int got = fscanf(f, "{\"ns\": %d, \"nr\": %d, \"precision\": %d, \"method\": %d, \"team\": %d, "
                                      "\"teams_per_block\": %d, \"smem_limit\": %lld, \"lu_panel\": %d, \"ms\": %lf}",
                                   &ns, &nr, &prec, &method, &team, &tpb, &lim, &nb, &ms);
            fclose(f);
            if (got == 9 && ns == m->ns && nr == m->nr && prec == o->precision && method == o->method) {
                if ((st = cg_mech_set_smem_limit(m, lim)) != CG_OK) return st;
                if ((st = cg_mech_set_launch(m, team, tpb)) != CG_OK) return st;
                if ((st = cg_mech_set_lu_panel(m, nb)) != CG_OK) return st;
                if (best_ms) *best_ms = ms;
                return CG_OK;
            }
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    double *wT = nullptr, *wY = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e;
    const size_t yb = (size_t)N * m->ns * sizeof(double);
    if ((e = cudaMalloc(&wT, N * sizeof(double))) != cudaSuccess || (e = cudaMalloc(&wY, yb)) != cudaSuccess ||
        (e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaFree(wT);
        cudaFree(wY);
        return cuda_fail(e, "autotune workspace");
    }
    const int old_team = m->dm.team, old_tpb = m->tpb, old_nb = m->dm.lu_nb;
    const int64_t old_lim = (int64_t)m->smem_limit;
    struct Shape { int team, tpb; int64_t lim; int nb; };
    std::vector<Shape> shapes;
    std::vector<int64_t> lims = {(int64_t)kMaxSmemPerBlock, (int64_t)kMaxSmemPerBlock / 2, (int64_t)48 * 1024};
    const int64_t def_lim = (int64_t)default_smem_limit(m->ns, m->nr);
    if (std::find(lims.begin(), lims.end(), def_lim) == lims.end()) lims.push_back(def_lim);
    // panel widths of the LU (identical results): only where the matrix is
    // large enough for panels to matter
    std::vector<int> panels = {0};
    if (m->ns + 1 >= 48 && P.linear_solver == 0) panels.push_back(16);
    for (int64_t lim : lims)
        for (int team : {32, 64, 128, 256})
            for (int tpb : {1, 2, 4})
                for (int nb : panels)
                    if (team == 32 || tpb == 1) shapes.push_back({team, tpb, lim, nb});
    Shape best = {old_team, old_tpb, old_lim, old_nb};
    float best_t = -1.0f;
    for (const Shape& sh : shapes) {
        if (cg_mech_set_smem_limit(m, sh.lim) != CG_OK || cg_mech_set_launch(m, sh.team, sh.tpb) != CG_OK ||
            cg_mech_set_lu_panel(m, sh.nb) != CG_OK)
            continue;
        float t_ms = 0.0f;
        bool ok = true;
        for (int rep = 0; rep < 2 && ok; ++rep) {   // first run warms up, second is timed
            ok = cudaMemcpyAsync(wT, T, N * sizeof(double), cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
                 cudaMemcpyAsync(wY, Y, yb, cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
                 cudaEventRecord(e0, s) == cudaSuccess &&
                 cg_integrate(m, o, N, wT, wY, p_or_rho, nullptr, nullptr, stream) == CG_OK &&
                 cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                 cudaEventElapsedTime(&t_ms, e0, e1) == cudaSuccess;
        }
        if (ok && (best_t < 0.0f || t_ms < best_t)) {
            best_t = t_ms;
            best = sh;
        }
    }
    cudaFree(wT);
    cudaFree(wY);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if ((st = cg_mech_set_smem_limit(m, best.lim)) != CG_OK) return st;
    if ((st = cg_mech_set_launch(m, best.team, best.tpb)) != CG_OK) return st;
    if ((st = cg_mech_set_lu_panel(m, best.nb)) != CG_OK) return st;
    if (best_t < 0.0f) return fail(CG_ECUDA, "no launch shape ran: %s", g_err.c_str());
    if (best_ms) *best_ms = best_t;
    if (cache_json) {
        FILE* f = fopen(cache_json, "w");
        if (f) {
            fprintf(f, "{\"ns\": %d, \"nr\": %d, \"precision\": %d, \"method\": %d, \"team\": %d, "
                       "\"teams_per_block\": %d, \"smem_limit\": %lld, \"lu_panel\": %d, \"ms\": %.6f}\n",
                    m->ns, m->nr, o->precision, o->method, best.team, best.tpb, (long long)best.lim, best.nb, best_t);
            fclose(f);
        }
    }
    return CG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Integration without any allocation, for callers that cannot allocate
// device memory while they run (for example a host code whose own memory
// manager owns the device heap, or a solver that must not enter the
// allocator inside its time step). The per-team scratch slots and the work
// counter live in one fixed array of this file's device module. CUDA loads
// a module (and so allocates the array, on that device) when it is first
// used there, or when the library loads if module loading is eager: the
// first cg_integrate_noalloc call on a device (an N = 0 call is enough)
// does it, and that call belongs in the caller's set-up, before it takes
// over the device heap and before any stream capture.

namespace {

constexpr size_t kNoAllocBytes = 32u << 20;                      // 32 MiB
constexpr int64_t kNoAllocDoubles = (int64_t)(kNoAllocBytes / sizeof(double));
constexpr int64_t kNoAllocCounterDoubles = 32;                  // first 256 bytes: the work counter

static __device__ __align__(256) double g_noalloc[kNoAllocDoubles];

// Device address of the array on the current device. The host-side name
// g_noalloc is not a device address; the lookup is repeated on every call
// (cheap once the module is loaded), so a device reset or a new context
// never leaves a stale pointer.
cg_status noalloc_array(double** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress (no-alloc scratch)");
    *out = static_cast<double*>(p);
    return CG_OK;
}

// Scratch an integration launch of these tasks needs from the fixed array:
// one slot per team of every resident block, at least one block's worth.
cg_status noalloc_plan(const cg::Tasks& tasks, int team, int tpb, int64_t* need_doubles) {
    const int64_t per_block = cg::integrate_slot_doubles(tasks, team) * cg::integrate_tpb(tasks, team, tpb);
    const int64_t avail = kNoAllocDoubles - kNoAllocCounterDoubles;
    if (need_doubles) *need_doubles = per_block;
    if (per_block > avail)
        return fail(CG_ECAPACITY,
                    "one block of this mechanism needs %lld bytes of scratch; cg_integrate_noalloc has %lld "
                    "(raise cg_mech_set_smem_limit or use cg_integrate)",
                    (long long)(per_block * (int64_t)sizeof(double)), (long long)(avail * (int64_t)sizeof(double)));
    return CG_OK;
}

}  // namespace

extern "C" cg_status cgx_noalloc_plan(int ns, int nr, int mat_bytes, int64_t smem_limit, int gmres_m, int team,
                                      int teams_per_block, int64_t* scratch_bytes) {
    if (ns < 1 || nr < 0 || (mat_bytes != 4 && mat_bytes != 8) || smem_limit < 1024 || gmres_m < 0 ||
        (team != 32 && team != 64 && team != 128 && team != 256) || teams_per_block < 1)
        return fail(CG_EINVAL, "bad arguments");
    cg::Tasks tasks;
    tasks.count = 1;
    tasks.total = 1;
    tasks.t[0].L = make_layout(ns, nr, mat_bytes, (size_t)smem_limit, false, gmres_m);
    int64_t need = 0;
    const cg_status st = noalloc_plan(tasks, team, teams_per_block, &need);
    if (scratch_bytes) *scratch_bytes = need * (int64_t)sizeof(double);
    return st;
}

extern "C" cg_status cg_integrate_noalloc(const cg_mech* m, const cg_integrate_opts* o, int64_t N,
                                          double* T, double* Y, const double* p_or_rho,
                                          int32_t* cell_status, int32_t* cell_stats, void* stream) {
    if (!m) return fail(CG_EINVAL, "mech is NULL");
    IntParams P;
    cg_status st = make_params(o, P);
    if (st != CG_OK) return st;
    if (N < 0) return fail(CG_EINVAL, "N < 0");
    double* base = nullptr;   // also on N = 0: the set-up call that loads the array
    if ((st = noalloc_array(&base)) != CG_OK) return st;
    if (N == 0) return CG_OK;
    if (!T || !Y || !p_or_rho) return fail(CG_EINVAL, "NULL array");
    cg::Tasks tasks;
    tasks.count = 1;
    tasks.total = N;
    tasks.t[0] = make_task(m, P, N, 0, T, Y, p_or_rho, cell_status, cell_stats);
    if ((st = noalloc_plan(tasks, m->dm.team, m->tpb, nullptr)) != CG_OK) return st;
    unsigned long long* counter = reinterpret_cast<unsigned long long*>(base);
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync (work counter)");
    e = cg::launch_integrate_on(tasks, P, m->dm.team, m->tpb, base + kNoAllocCounterDoubles,
                                kNoAllocDoubles - kNoAllocCounterDoubles, counter, (cudaStream_t)stream);
    return e == cudaSuccess ? CG_OK : cuda_fail(e, "integrate launch (no-alloc)");
}
