// Host-side internals shared by the C-ABI layer and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "chem_device.cuh"

namespace cg {

// One mechanism's share of an integration launch: cells [first, first + N)
// of the launch's cell index space are cells [0, N) of these arrays.
struct Task {
    DevMech M;
    Layout L;
    int64_t N, first;
    // split (a one-warp mechanism in a launch of wider teams): its cells are
    // integrated by single warps, each with its own slice of the team's
    // shared memory and scratch slot, and numbered in the launch's second
    // index space (first counts there)
    int split = 0;
    double* T;
    double* Y;
    const double* p;
    int32_t* status;
    int32_t* stats;
    // optional checkpoints of the accepted steps (adjoint): cell c's step k
    // is ckpt[(c * ckpt_cap + k) * (n + 1) + i] = (y_k, h_k); entry
    // ckpt_n[c] holds the final state and the initial density rho_0;
    // ckpt_n[c] = -1 when the cell failed; when its S steps do not fit,
    // ckpt_n[c] = -(S + 2) and the last entry holds the final state
    double* ckpt;
    int32_t* ckpt_n;
    int ckpt_cap;
};

// One adjoint launch: cells integrated by a checkpointing forward call.
struct AdjTask {
    DevMech M;
    Layout L;
    int64_t N;
    const double* p;           // pressure (CONP) or density (CONV)
    const double* ckpt;
    const int32_t* ckpt_n;
    int ckpt_cap;
    const double* dT_end;      // dL/dT at the end        [N]
    const double* dY_end;      // dL/dY_k at the end      [ns][N]
    double* dT0;               // out: dL/dT0             [N]
    double* dY0;               // out: dL/dY0_k           [ns][N]
    const int* perm;           // internal reaction index -> caller's index
    double* grad_cells;        // out: dL/dtheta per cell [nr][3][N], caller's reaction order
    int32_t* status;           // out
};

// One operator-split call of a flow solver (Section 5.5): conserved
// variables in, temperature and the species source out.
struct SplitTask {
    DevMech M;
    Layout L;
    int64_t N;
    const double* rho;    // density                    [N]
    const double* e;      // mass-specific internal energy u [N]
    const double* rhoY;   // species densities rho Y_i  [ns][N]
    double* T;            // in: first guess, out: temperature after dt [N]
    double* R;            // out: W_i (C_i^{n+1} - C_i^n) / dt   [ns][N]
    int32_t* status;
    int32_t* stats;
    int iters;            // Newton iterations of the temperature recovery
};

constexpr int kMaxTasks = 4;

struct Tasks {
    Task t[kMaxTasks];
    int count;
    int64_t total;         // cells of the tasks run by whole teams
    int64_t total_split = 0;   // cells of the split tasks (0: none)
};

cudaError_t launch_eval_rates(const DevMech& M, const Layout& L, int tpb, int reactor, int64_t N,
                              const double* T, const double* C, double* S, cudaStream_t st);
cudaError_t launch_eval_jacobian(const DevMech& M, const Layout& L, int tpb, int reactor, int64_t N,
                                 const double* T, const double* C, double* J, cudaStream_t st);
cudaError_t launch_temperature(const DevMech& M, int reactor, int64_t N, const double* e,
                               const double* Y, double* T, int iters, cudaStream_t st);
cudaError_t launch_exp_check(const DevMech& M, int64_t n, const double* x, double* y_tab, double* y_lib,
                             cudaStream_t st);
cudaError_t launch_rcp_check(int64_t n, const double* x, double* y, cudaStream_t st);
// All tasks share one team size; `persistent` selects the resident grid with
// the work counter (always used when a cell needs global scratch).
cudaError_t launch_integrate(const Tasks& tasks, const IntParams& P, int team, int tpb, bool persistent,
                             cudaStream_t st);
// Persistent launch on caller-provided scratch (scratch_doubles doubles) and
// a work counter that is zero on the stream when the kernel starts.
// cudaErrorMemoryAllocation: not even one team's slot fits in the scratch.
cudaError_t launch_integrate_on(const Tasks& tasks, const IntParams& P, int team, int tpb, double* scratch,
                                int64_t scratch_doubles, unsigned long long* counter, cudaStream_t st);
// Global scratch of one team's slot (doubles) and the teams per block an
// integration launch of `team` threads per cell actually uses (the requested
// count, lowered until the block's shared memory fits in 227 KB).
// A team of `team` threads holds one cell of a whole-team task or team/32
// cells of a split task at a time.
int64_t integrate_slot_doubles(const Tasks& tasks, int team);
int integrate_tpb(const Tasks& tasks, int team, int tpb);
// Shared-memory stride (doubles) of one team's slice: the largest of the tasks.
int integrate_sstride(const Tasks& tasks, int team);
// Operator-split reaction step (persistent launch, `team` threads per cell).
cudaError_t launch_react_split(const SplitTask& t, const IntParams& P, int team, int tpb, cudaStream_t st);
// Backward sweep of the discrete adjoint over the cells of t (persistent
// launch with `team` threads per cell), then, with dtheta != nullptr, the
// fixed-order sum of the per-cell parameter gradients into dtheta[nr][3].
cudaError_t launch_adjoint(const AdjTask& t, const IntParams& P, int team, int tpb, double* dtheta,
                           cudaStream_t st);

// The launchers of one team size TEAM (threads per cell) and Newton-matrix
// type MT, explicitly instantiated in instances.cu (one object per
// combination); the dispatchers above select among them.
template <int TEAM>
cudaError_t launch_eval_team(bool jacobian, const DevMech& M, const Layout& L, int tpb, int reactor, int64_t N,
                             const double* T, const double* C, double* out, cudaStream_t st);
template <int TEAM, class MT>
cudaError_t launch_integrate_team(const Tasks& tasks, const IntParams& P, int tpb, bool persistent,
                                  cudaStream_t st);
template <int TEAM, class MT>
cudaError_t launch_integrate_on_team(const Tasks& tasks, const IntParams& P, int tpb, double* scratch,
                                     int64_t scratch_doubles, unsigned long long* counter, cudaStream_t st);
template <int TEAM, class MT>
cudaError_t launch_split_team(const SplitTask& t, const IntParams& P, int tpb, cudaStream_t st);
template <int TEAM, class MT>
cudaError_t launch_adjoint_team(const AdjTask& t, const IntParams& P, int tpb, cudaStream_t st);

}  // namespace cg
