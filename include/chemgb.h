/*
 * chemgb -- batched stiff chemistry integration on one GPU (C ABI).
 *
 * The library integrates the chemical source term of a reacting-flow solver
 * cell by cell under operator splitting, following ChemGen (arXiv 2510.10005):
 * the state of a cell is y = (T, C_1..C_ns) (Section 3, eq.
 * extracted_problem-1), its right-hand side S(y) = (omega_T, dC/dt) is built
 * from NASA-7 thermodynamics (Section 2.1, Table 1), Gibbs-based equilibrium
 * constants and Arrhenius, third-body, Lindemann / Troe / SRI falloff and
 * PLOG rates (Section 2.2), and a cell is advanced over dt with backward
 * Euler + Newton (Section 3.2), an SDIRK scheme in stage-derivative form
 * (Appendix A.1, A.2), second-order Rosenbrock (Appendix A.3) or YASS
 * (Appendix A.4), each linear system (I - gamma h J) delta = -f taking the
 * analytical Jacobian J (Section 3.2) and a dense LU with partial pivoting
 * or restarted, preconditioned GMRES (Section 3.4). cg_react_split is the
 * operator-split call of a compressible flow solver (Section 5.5), and
 * cg_integrate_ckpt / cg_integrate_adjoint differentiate the integration.
 *
 * Conventions shared by every entry point:
 *   - Units are SI-kmol: C in kmol/m^3, T in K, p in Pa, rho in kg/m^3,
 *     W in kg/kmol, Ea in J/kmol, R = 8314.46261815324 J/(kmol K),
 *     p_ref = 101325 Pa.
 *   - Per-cell arrays are caller-owned DEVICE pointers laid out
 *     structure-of-arrays: component k of cell c is at [k * N + c].
 *     (cg_integrate_host is the one exception: host pointers.)
 *   - Work is enqueued on the CUDA stream `stream` (a cudaStream_t; NULL is
 *     the legacy default stream) and returns before it completes, except
 *     where a function says it synchronises.
 *   - Return values: CG_OK, or an error code for invalid arguments, resource
 *     or CUDA failures; cg_last_error() then describes the failure (per
 *     calling thread). Numerical failures of individual cells are reported in
 *     the per-cell status array, never as a process abort.
 *   - A cg_mech changes only through the cg_mech_set_* calls; other calls
 *     with the same mechanism may run concurrently on different streams.
 */
#ifndef CHEMGB_H
#define CHEMGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cg_mech cg_mech;

typedef enum {
    CG_OK = 0,
    CG_EINVAL = 1,        /* invalid argument or mechanism data            */
    CG_ENOMEM = 2,        /* device or host allocation failed              */
    CG_ECUDA = 3,         /* a CUDA runtime call failed                    */
    CG_ECAPACITY = 4,     /* a size exceeds what the library supports      */
    CG_EUNSUPPORTED = 5   /* option combination not implemented           */
} cg_status;

/* per-cell status written by cg_integrate */
enum {
    CG_CELL_OK = 0,
    CG_CELL_NEWTON_FAIL = 1,      /* Newton failed at the deepest halving   */
    CG_CELL_STEP_TOO_SMALL = 2,   /* adaptive step fell below hmin          */
    CG_CELL_MAX_STEPS = 3,        /* more than max_steps step attempts      */
    CG_CELL_NONFINITE = 4,        /* input state not finite                 */
    CG_CELL_NO_RECORD = 5         /* adjoint: the forward pass failed on this
                                     cell, so it left no usable record */
};

/* reaction types (Section 2.2): elementary, third-body, falloff with
 * Lindemann, Troe or SRI broadening (Section 2.2.3), pressure-dependent
 * Arrhenius "PLOG" (Section 2.2.4; the pressure is the cell's own
 * R T sum C) */
enum { CG_RXN_ELEMENTARY = 0, CG_RXN_THREE_BODY = 1, CG_RXN_LINDEMANN = 2, CG_RXN_TROE = 3,
       CG_RXN_SRI = 4, CG_RXN_PLOG = 5 };

/* reactor forms: constant volume (Section 3, eq. temperature_source);
 * constant pressure with the dilution of the cell's volume (the reading of
 * Appendix B that keeps p = R T sum C fixed); Appendix B as printed
 * (enthalpy form of omega_T, dC/dt = omega). */
enum { CG_CONV = 0, CG_CONP = 1, CG_CONP_LITERAL = 2 };

/* integrators: backward Euler (Section 3.2), SDIRK-2 (Appendix A.1),
 * SDIRK-4 (Appendix A.2), second-order Rosenbrock (Appendix A.3: one
 * Jacobian and one factorisation per step, FATODE's Ros2 coefficients; the
 * printed extra -S(y_n) of its second stage, which would make the scheme
 * inconsistent, is not taken; embedded first-order error for adaptive
 * steps), YASS (Appendix A.4: one backward-Euler Newton iteration per step;
 * a step whose decrement has WRMS norm above alpha = opts->newton_tol is
 * halved, at most max_halvings times; fixed steps only) */
enum { CG_BE = 0, CG_SDIRK2 = 1, CG_SDIRK4 = 2, CG_ROS2 = 3, CG_YASS = 4 };

/* arithmetic of the Newton matrix factorisation */
enum { CG_FP64 = 0, CG_FP32LU = 1 };

/* linear solver of the Newton systems (Section 3.4): the dense LU with
 * partial pivoting, or restarted GMRES with left preconditioning (x0 = 0,
 * Givens rotations, converged when the preconditioned residual is at most
 * gmres_tol times that of x = 0); preconditioners: none, Jacobi (the
 * diagonal), Gauss-Seidel (the lower triangle with the diagonal). A GMRES
 * solve that does not converge within gmres_maxit iterations fails the step
 * like a singular matrix. */
enum { CG_LU = 0, CG_GMRES = 1 };
enum { CG_PC_NONE = 0, CG_PC_JACOBI = 1, CG_PC_GAUSS_SEIDEL = 2 };

/*
 * Mechanism description (host arrays, copied by cg_mech_create; the caller
 * keeps ownership). Reactions are written sum nu^f_i A_i <=> sum nu^r_i A_i
 * with at most three distinct species on each side.
 *   W[ns]           molecular masses
 *   nasa7[ns*7]     a1..a5 (c_p/R polynomial), a6 (h/R constant), a7 (s/R
 *                   constant); one range used at every temperature. This
 *                   is the n_p = 4 case of eq. specific_heat_polynomial;
 *                   cg_mech_set_thermo takes other degrees.
 *   rxn_type[nr]    CG_RXN_*
 *   reversible[nr]  0 or 1; reverse rate k_f / K_c (eq. reverse_rate)
 *   rf_idx/rf_nu[nr*3]  reactant species and integer coefficients (-1 / 0 pad)
 *   rr_idx/rr_nu[nr*3]  product species and coefficients
 *   arr[nr*3]       ln A, b, Ea of k = A T^b exp(-Ea/(R T)) (k_inf of falloff)
 *   arr0[nr*3]      ln A0, b0, Ea0 of the low-pressure limit (falloff only)
 *   troe[nr*4]      alpha, T3, T1, T2 of eq. f_and_fcent; T2 = NaN: absent
 *   eff_ptr[nr+1], eff_idx[], eff_val[]  CSR of third-body efficiencies
 *                   that differ from 1 (eq. TB_optimization); none for
 *                   elementary and PLOG reactions
 *   sri[nr*5]       a, b (K), c (K), d, e of SRI falloff (a >= 0, c > 0,
 *                   d > 0); may be NULL when no reaction is CG_RXN_SRI
 *   plog_ptr[nr+1], plog[K*4]  CSR of the PLOG rate expressions of each
 *                   reaction: p (Pa), ln A, b, Ea, in non-decreasing p;
 *                   expressions at the same p add (eq. plog_rate); only
 *                   CG_RXN_PLOG reactions have entries (at least one); may
 *                   be NULL when no reaction is CG_RXN_PLOG. arr is unused
 *                   for PLOG reactions.
 */
typedef struct {
    int n_species, n_reactions;
    const double *W, *nasa7;
    const int *rxn_type, *reversible;
    const int *rf_idx, *rf_nu, *rr_idx, *rr_nu;
    const double *arr, *arr0, *troe;
    const int *eff_ptr, *eff_idx;
    const double *eff_val;
    const double *sri;
    const int *plog_ptr;
    const double *plog;
} cg_mech_desc;

/* Validate the description (index ranges, coefficients, sizes), build the
 * device copy and the assembly schedules of omega and J. Allocates device
 * memory owned by the mechanism. Errors: CG_EINVAL (bad data; message names
 * the first offending entry), CG_ECAPACITY (more species or reactions than
 * one warp's shared memory holds), CG_ENOMEM, CG_ECUDA. */
cg_status cg_mech_create(const cg_mech_desc *desc, cg_mech **out);
/* Free a mechanism (NULL is ignored). No call using it may be in flight. */
void cg_mech_destroy(cg_mech *mech);
int cg_mech_n_species(const cg_mech *mech);
int cg_mech_n_reactions(const cg_mech *mech);

/* Launch shape of every kernel that uses this mechanism: `team` threads
 * (32, 64, 128 or 256) cooperate on one cell and `teams_per_block` cells
 * share a block (must be 1 when team > 32). The default is one warp per cell
 * up to 24 unknowns, two warps per cell up to 96 and four above. Changing
 * the team size
 * rebuilds the assembly schedules (synchronises the device); no call using
 * the mechanism may run concurrently. Results do not depend on the shape
 * beyond the summation order of team-wide reductions. Errors: CG_EINVAL
 * (bad shape), CG_ECAPACITY (shared memory), CG_ENOMEM, CG_ECUDA. This is
 * a launch-tuning hook, not part of the method of the paper. */
cg_status cg_mech_set_launch(cg_mech *mech, int team, int teams_per_block);
/* Shared memory a cell may use (bytes, 1 KiB .. 227 KiB). A cell's arrays
 * are placed hottest first (Newton matrix, state vectors, thermo, stage
 * derivatives, per-reaction data); those beyond the limit go to a per-team
 * slot of global scratch that the library allocates stream-ordered for each
 * launch (mechanisms whose Newton matrix alone nears the limit, such as 160
 * species in FP64, always spill). A lower limit trades L2 traffic for more
 * cells per SM. Default: 64 KiB when the FP64 Newton matrix alone exceeds
 * half of 227 KiB (160 species), which puts the whole working set in the
 * L2 slot so that four cells share an SM; 28 KiB for two-warp cells whose
 * Newton matrix fits in it (eight cells per SM; 53 species); otherwise
 * 227 KiB, except when the per-reaction block (9 nr doubles) is at least
 * 8 KiB of a per-cell total of 40 KiB or more, which then goes to L2. This
 * call sets one limit for both matrix types. Same
 * concurrency rule as cg_mech_set_launch. Launch tuning, not part of the
 * paper's method. */
cg_status cg_mech_set_smem_limit(cg_mech *mech, int64_t bytes);

/* Current launch shape; returns 0, or -1 for a NULL mechanism. */
int cg_mech_get_launch(const cg_mech *mech, int *team, int *teams_per_block);

/* Panel width of the dense LU with partial pivoting of the Newton matrix
 * (Section 3.4; the direct solver whose O(n^3) cost the paper names):
 * 0 factors column by column with a rank-one update of the whole trailing
 * block after each; nb = 1..64 factors panels of nb columns and then
 * updates the trailing block once per panel from register tiles (a
 * right-looking blocked LU). Both apply the same fused multiply-adds to
 * every element in the same order, so the factors, the pivots and every
 * result are identical to the last bit; only the memory traffic and the
 * number of synchronisations differ. Default: 0 below 96 unknowns, 16
 * above. Same concurrency rule as cg_mech_set_launch. Errors: CG_EINVAL.
 * cg_mech_get_lu_panel returns the width, or -1 for a NULL mechanism. */
cg_status cg_mech_set_lu_panel(cg_mech *mech, int nb);
int cg_mech_get_lu_panel(const cg_mech *mech);

/* Source term S(y) = (omega_T, dC_1/dt .. dC_ns/dt) for N cells
 * (Section 2.2, eqs. chemical-reaction-rate-of-progress, temperature_source;
 * Appendix B). T[N], C[ns*N] in; S[(ns+1)*N] out, row 0 = omega_T. */
cg_status cg_eval_rates(const cg_mech *mech, int reactor, int64_t N, const double *T,
                        const double *C, double *S, void *stream);

/* Analytical Jacobian J = dS/dy (Section 3.2, eq.
 * derivative_matrices_temp_evol, T and C independent) for N cells.
 * T[N], C[ns*N] in; J[N*n*n] out, n = ns+1, one row-major n x n block per
 * cell (cell-major, the one non-SoA output), row/column 0 = T. */
cg_status cg_eval_jacobian(const cg_mech *mech, int reactor, int64_t N, const double *T,
                           const double *C, double *J, void *stream);

/* Temperature from the mass-specific energy e (u for CG_CONV, h otherwise)
 * and mass fractions Y[ns*N] by `iters` Newton iterations on
 * sum_i Y_i e_i(T) = e (Section 2.1, eqs. temperature-nonlinear ..
 * netwon_iteration_temperature; the paper uses 5). T[N] holds the initial
 * guess on entry and the result on exit. */
cg_status cg_temperature_from_energy(const cg_mech *mech, int reactor, int64_t N,
                                     const double *e, const double *Y, double *T, int iters,
                                     void *stream);

/* Integration options (fill with cg_integrate_opts_default, then adjust). */
typedef struct {
    int method;        /* CG_BE, CG_SDIRK2, CG_SDIRK4, CG_ROS2, CG_YASS               */
    int reactor;       /* CG_CONV, CG_CONP, CG_CONP_LITERAL                           */
    int adaptive;      /* 1: error-controlled steps (SDIRK, Rosenbrock); 0: nsub fixed steps */
    int precision;     /* CG_FP64, or CG_FP32LU (BE and SDIRK): Newton matrix assembled and factored
                          in FP32, residual, solves and updates in FP64 (an inexact
                          Newton whose converged result meets the same tolerances)  */
    int nsub;          /* fixed mode: number of equal steps over dt                   */
    int max_newton;    /* Newton iterations per stage                                 */
    int max_steps;     /* adaptive: step attempts before CG_CELL_MAX_STEPS            */
    int max_halvings;  /* fixed mode: depth of step halving after a failed step       */
    int err_filter;    /* adaptive: filter the error estimate by (I - gamma h J)^-1   */
    int persistent;    /* 1: resident grid whose teams take cells from a shared work
                          counter (work stealing; also used when a cell's arrays
                          spill to global scratch, when one-warp mechanisms run
                          split, and when the cells need more than one wave of
                          blocks); 0: one launch slot per cell otherwise          */
    double dt;         /* integration interval, s                                     */
    double rtol, atol; /* weights w_i = atol + rtol max(|y_n,i|, |y_i|)               */
    double newton_tol; /* Newton converged when WRMS(change of stage state) <= this;
                          YASS: the decrement bound alpha                          */
    double h0;         /* adaptive: first step (0: dt)                                */
    double hmin;       /* adaptive: smallest step                                     */
    double neg_tol;    /* a step is rejected when some C_i < -neg_tol * sum C         */
    int linear_solver; /* CG_LU (default) or CG_GMRES                                 */
    int preconditioner;/* GMRES: CG_PC_NONE, CG_PC_JACOBI, CG_PC_GAUSS_SEIDEL         */
    int gmres_restart; /* GMRES: Krylov dimension before a restart, 1..64             */
    int gmres_maxit;   /* GMRES: iterations per linear solve                          */
    double gmres_tol;  /* GMRES: relative tolerance of the preconditioned residual    */
} cg_integrate_opts;

void cg_integrate_opts_default(cg_integrate_opts *opts);

/* Autotuner: integrates a caller-given sample of cells (device arrays as in
 * cg_integrate; not modified: each timing runs on a copy) once per launch
 * shape -- threads per cell {32, 64, 128, 256}, cells per block {1, 2, 4}
 * for one-warp teams, shared-memory limit {227, 113, 48} KiB and the
 * mechanism's default, LU panel width {0, 16} from 48 unknowns on (LU
 * only) -- and applies the fastest to the mechanism (cg_mech_set_launch,
 * cg_mech_set_smem_limit, cg_mech_set_lu_panel).
 * Synchronises `stream`; allocates two sample-sized work arrays for its
 * duration. With cache_json != NULL, a file written by an earlier call for
 * a mechanism of the same size and the same method and precision is applied
 * without timing, otherwise the result is written there. *best_ms (may be
 * NULL) receives the sample's time with the chosen shape. Launch tuning, not
 * part of the paper's method. */
cg_status cg_autotune(cg_mech *mech, const cg_integrate_opts *opts, int64_t N, const double *T,
                      const double *Y, const double *p_or_rho, const char *cache_json, void *stream,
                      double *best_ms);

/* Integrate N cells over opts->dt (cell_stats[3*N + c] counts LU
 * factorisations, or GMRES iterations with CG_GMRES).
 *   T[N], Y[ns*N]   in: initial temperature and mass fractions;
 *                   out: final ones (overwritten in place)
 *   p_or_rho[N]     pressure (CG_CONP, CG_CONP_LITERAL: C = rho Y / W with
 *                   rho = p / (R T sum Y/W)) or density (CG_CONV)
 *   cell_status[N]  CG_CELL_* per cell (may be NULL)
 *   cell_stats[4*N] per cell: accepted steps, rejected or failed attempts,
 *                   Newton iterations, LU factorisations (SoA; may be NULL)
 * The work of a cell never depends on another cell. */
cg_status cg_integrate(const cg_mech *mech, const cg_integrate_opts *opts, int64_t N, double *T,
                       double *Y, const double *p_or_rho, int32_t *cell_status,
                       int32_t *cell_stats, void *stream);

/* Integrate the cells of up to 4 mechanisms in ONE persistent launch: the
 * cells of all mechanisms form one index space (mechanism 0 first) from
 * which resident teams take cells through a shared work counter, so cheap
 * and expensive cells of either mechanism balance across the GPU. Array
 * k-th entries are those of cg_integrate for mechanism k (cell_status and
 * cell_stats may be NULL, or hold NULL entries). The launch takes the
 * largest team size of the mechanisms (cg_mech_set_launch); mechanisms of
 * one-warp teams in a wider launch run split: once the other mechanisms'
 * cells are taken, every warp of a team claims their cells on its own from
 * a second counter and integrates them with one warp per cell, as
 * cg_integrate would (the same results to the last bit). Other team sizes
 * must all be equal (CG_EINVAL otherwise). The same options apply to all.
 * Allocates its work counter and any global scratch stream-ordered
 * (cudaMallocAsync) and releases them on the same stream. */
cg_status cg_integrate_batch(int n_mech, const cg_mech *const *mechs, const int64_t *N,
                             double *const *T, double *const *Y, const double *const *p_or_rho,
                             int32_t *const *cell_status, int32_t *const *cell_stats,
                             const cg_integrate_opts *opts, void *stream);

/*
 * Operator-split reaction step of a compressible flow solver (Section 5.5,
 * eq. openfom_fvm): per cell, from the conserved variables the flow solver
 * holds -- rho[N] (kg/m^3), the mass-specific internal energy e[N] (u, J/kg,
 * chemical plus sensible, NASA-7 reference) and rhoY[ns*N] (kg/m^3, SoA) --
 * recovers T by `iters` Newton iterations on sum_i Y_i u_i(T) = e from the
 * guess in T (Section 2.1; the paper uses 5), integrates the concentrations
 * C_i = rho Y_i / W_i at constant volume over opts->dt (Section 3, eq.
 * temperature_source; opts->reactor must be CG_CONV) and writes the
 * temperature after the step to T and the species source
 *   R[i*N + c] = W_i (C_i^{n+1} - C_i^n) / dt   (kg/m^3/s; sum_i R_i = 0)
 * that the flow solver adds to its species equations. Cells whose input is
 * not finite (or whose recovered T is not positive) get status
 * CG_CELL_NONFINITE, R = 0 and T unchanged. cell_status, cell_stats as
 * cg_integrate. Device arrays; allocates only the stream-ordered work
 * counter and scratch of a persistent launch. Errors: as cg_integrate, and
 * CG_EINVAL for another reactor or iters outside 0..100.
 */
cg_status cg_react_split(const cg_mech *mech, const cg_integrate_opts *opts, int64_t N, const double *rho,
                         const double *e, const double *rhoY, double *T, double *R, int iters,
                         int32_t *cell_status, int32_t *cell_stats, void *stream);

/*
 * Discrete adjoint (reverse-mode gradients of a loss of the final states).
 * The paper builds ChemGen for use in differentiable solvers (Section 1); the
 * derivative here is that of the integrators of Section 3.2 and Appendix A on
 * their converged stage equations, with the accepted steps (y_n, h_n) frozen
 * to those of the forward pass (Newton iterations and step-size decisions
 * are not differentiated). Parameters theta are (ln A, b, Ea) of every
 * reaction (k_inf for falloff reactions; k_0 held fixed).
 *
 * cg_integrate_ckpt: cg_integrate that also records, per cell c, the state
 * y = (T, C) at the start of every accepted step and the step size:
 *   ckpt[(c * ckpt_cap + k) * (ns + 2) + i], i <= ns: y_k,  i = ns + 1: h_k;
 *   record ckpt_n[c] holds the final state and the initial density.
 *   ckpt[N * ckpt_cap * (ns + 2)] and ckpt_n[N] are caller-owned device
 *   arrays; ckpt_n[c] = -1 when the cell failed (its adjoint then reports
 *   CG_CELL_NO_RECORD). A cell whose S accepted steps need more than
 *   ckpt_cap - 1 records gets ckpt_n[c] = -(S + 2): record 0 keeps its
 *   initial state and record ckpt_cap - 1 its final state and density, and
 *   the adjoint recomputes the steps from record 0 in segments of 32 (a
 *   second level of checkpointing in its own scratch: the replay runs the
 *   forward arithmetic again, so the gradients are identical to those from
 *   a full record, at the cost of about S^2 / 64 extra steps).
 *   ckpt_cap >= 2. Other arguments and results as cg_integrate.
 *
 * cg_integrate_adjoint: from dL/dT_end[N] and dL/dY_end[ns*N] (SoA, device),
 * computes dL/dT0[N], dL/dY0[ns*N] (through C = rho Y / W, with rho fixed at
 * constant volume or rho = p / (R T0 sum Y/W) otherwise) and
 *   dtheta[nr*3]              sum over cells of dL/d(ln A, b, Ea), in the
 *                             caller's reaction order (may be NULL)
 *   dtheta_cells[nr*3*N]      per-cell gradients, entry (3 j + k) * N + c
 *                             (may be NULL: then a stream-ordered temporary)
 *   cell_status[N]            CG_CELL_OK, CG_CELL_NO_RECORD, or
 *                             CG_CELL_NEWTON_FAIL (may be NULL)
 * Cells that do not end CG_CELL_OK contribute zeros. `opts` must be those of
 * the forward call (the stages are recomputed with them, bit for bit). The
 * sum over cells is in a fixed order: results do not depend on the launch
 * shape or on timing. FP64 transposed solves whatever opts->precision.
 * Errors: as cg_integrate; CG_ECAPACITY when one cell's adjoint arrays do not
 * fit in shared memory.
 */
cg_status cg_integrate_ckpt(const cg_mech *mech, const cg_integrate_opts *opts, int64_t N, double *T,
                            double *Y, const double *p_or_rho, int32_t *cell_status, int32_t *cell_stats,
                            double *ckpt, int32_t *ckpt_n, int ckpt_cap, void *stream);
cg_status cg_integrate_adjoint(const cg_mech *mech, const cg_integrate_opts *opts, int64_t N,
                               const double *ckpt, const int32_t *ckpt_n, int ckpt_cap,
                               const double *dT_end, const double *dY_end, double *dT0, double *dY0,
                               double *dtheta, double *dtheta_cells, int32_t *cell_status, void *stream);

/* Replace ln A, b, Ea of every reaction (host arr[nr*3], the caller's order
 * and units of cg_mech_desc.arr; the low-pressure limits of falloff
 * reactions stay as created). Synchronises the device; no call using the
 * mechanism may be in flight. For parameter fitting with the adjoint.
 * Errors: CG_EINVAL (NULL or non-finite entries), CG_ECUDA. */
cg_status cg_mech_set_arrhenius(cg_mech *mech, const double *arr);

/* Replace the thermodynamics by a c_p polynomial of degree np in [0, 15]
 * (Section 2.1, eq. specific_heat_polynomial; Appendix C.1 refits NASA data
 * to np = 7 and 15). coef[ns * (np + 3)] (host) holds per species a_0..a_np
 * of c_p/R = sum_k a_k T^k (molar) followed by the h/R and s/R constants, so
 * that h/R = sum_k a_k T^(k+1)/(k+1) + a_(np+1) and s/R = a_0 ln T +
 * sum_(k>=1) a_k T^k / k + a_(np+2); np = 4 is the nasa7 row. Synchronises
 * the device; the table keeps its address, but the degree reaches kernels
 * by value, so a CUDA graph captured earlier must be captured again.
 * Errors: CG_EINVAL (NULL arguments, np out of range, non-finite entries),
 * CG_ECUDA. */
cg_status cg_mech_set_thermo(cg_mech *mech, int np, const double *coef);

/* Same as cg_integrate with HOST arrays: copies the inputs to device memory
 * owned by the mechanism (grown on demand, freed with it), integrates,
 * copies the results back and synchronises before returning. Not safe for
 * concurrent calls on the same mechanism. */
cg_status cg_integrate_host(const cg_mech *mech, const cg_integrate_opts *opts, int64_t N,
                            double *T, double *Y, const double *p_or_rho, int32_t *cell_status,
                            int32_t *cell_stats);

/* cg_integrate for callers that cannot allocate device memory while they
 * run: a host code whose own memory manager owns the device heap, or a
 * solver that must not enter an allocator inside its time step. The paper
 * has no counterpart; this is a deployment variant of cg_integrate with the
 * same arguments and results. It always uses the persistent work-stealing
 * launch, and calls no cudaMalloc, cudaFree or other allocating routine:
 * the per-team scratch slots and the work counter live in one fixed 32 MiB
 * device array inside the library.
 *   - CUDA allocates that array on a device when it loads the library's
 *     module there: at the first cg_integrate_noalloc call on the device
 *     (under lazy module loading, the default), or when the library loads
 *     (eager loading). Make one call per device during set-up, with the
 *     device current, before taking over the device heap and before any
 *     stream capture; a call with N = 0 is enough. The array is then held
 *     until the process exits.
 *   - Each call looks up the array's device address (cudaGetSymbolAddress)
 *     on the current device, so a device reset between calls is harmless.
 *   - All calls share the array and it keeps the last call's contents; each
 *     call clears the work counter on its stream. Calls whose work overlaps
 *     on the GPU (other streams, other threads) race on the array: serialise
 *     them.
 *   - Errors: as cg_integrate, and CG_ECAPACITY when one block of cells
 *     needs more scratch than the array holds (the message gives both
 *     sizes; a lower cg_mech_set_smem_limit never helps, since it moves
 *     arrays from shared memory into the scratch). */
cg_status cg_integrate_noalloc(const cg_mech *mech, const cg_integrate_opts *opts, int64_t N, double *T,
                               double *Y, const double *p_or_rho, int32_t *cell_status,
                               int32_t *cell_stats, void *stream);

/* Message of the last failing call on this thread ("" if none). */
const char *cg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CHEMGB_H */
