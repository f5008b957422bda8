/*
 * chemgb test hooks (C ABI). Not part of the method: entry points that let
 * the tests check device functions of the library against CUDA's own, and
 * the host-side planners of the kernels (assembly schedules, reaction
 * chunks, per-cell memory layout) without a GPU.
 */
#ifndef CHEMGB_TESTING_H
#define CHEMGB_TESTING_H

#include <stdint.h>

#include "chemgb.h"

#ifdef __cplusplus
extern "C" {
#endif

/* For n arguments x (device array), writes the library's table-driven
 * exponential (Tang's method, used by the rate evaluation of Section 2.2)
 * to y_tab and CUDA's exp to y_lib (device arrays of n doubles), on
 * `stream`. Errors: CG_EINVAL (NULL mechanism or arrays, n < 0), CG_ECUDA. */
cg_status cgx_exp_check(const cg_mech *mech, int64_t n, const double *x, double *y_tab, double *y_lib,
                        void *stream);

/* For n arguments x (device array), writes the library's reciprocal (two
 * Newton-Raphson steps from the hardware's single-precision approximation,
 * used for the LU pivots of Section 3.4; division outside the
 * single-precision exponent range) to y (device array of n doubles), on
 * `stream`. Errors: CG_EINVAL (n < 0, NULL arrays), CG_ECUDA. */
cg_status cgx_rcp_check(int64_t n, const double *x, double *y, void *stream);

/* The thread-owned assembly schedule the kernels walk to form sparse sums
 * out[dst] += fac * in[src] (the production rates omega_i = sum_j nu_ij q_j
 * of Section 2.2 and the Jacobian entries of Section 3.2). Host only.
 * Input: n_terms terms (dst, src, fac, order); terms of one destination are
 * summed in increasing `order`. dst must lie in [0, 2^29 - 1].
 * Output: *len = terms per lane. If the four arrays are non-NULL (all or
 * none), slot t of lane l, at [t * lanes + l] for t < *len, receives the
 * destination, flags (bit 0: the first term of the destination's run,
 * bit 1: its last), source and factor; padding slots after a lane's last
 * run hold 0, 0, 0, 0.0. capacity: the arrays' length, at least
 * *len * lanes. Errors: CG_EINVAL (bad counts, NULL input arrays, a
 * destination out of range), CG_ECAPACITY (capacity too small). */
cg_status cgx_schedule(int64_t n_terms, const int *dst, const int *src, const double *fac, const int64_t *order,
                       int lanes, int *len, int *sdst, int *sflags, int *ssrc, double *sfac, int64_t capacity);

/* The reaction chunks of the rate loop for teams of `team` threads (32, 64,
 * 128 or 256): runs of at most 32 consecutive reactions of one kind
 * (elementary and third-body; falloff; PLOG; rxn_type[nr] holds the
 * CG_RXN_* codes in the library's internal order) dealt to the team's warps.
 * Host only. Writes *n_chunks and warp_ptr[team / 32 + 1] (warp w takes
 * chunks warp_ptr[w] .. warp_ptr[w + 1] - 1); if first and len are non-NULL
 * (both or neither, `capacity` entries), chunk c covers reactions first[c]
 * .. first[c] + len[c] - 1. Errors: CG_EINVAL, CG_ECAPACITY. */
cg_status cgx_rate_chunks(int nr, const int *rxn_type, int team, int *n_chunks, int *warp_ptr, int *first,
                          int *len, int capacity);

/* The per-cell memory layout for ns species and nr reactions: which arrays
 * of a cell's working set go to shared memory (at most smem_limit bytes per
 * cell, 1 KiB of it kept free) and which to the cell's global scratch slot.
 * mat_bytes: 8 (FP64 Newton matrix) or 4 (FP32); adjoint: non-zero adds the
 * backward sweep's arrays; gmres_m: the GMRES restart length, 0 for the LU.
 * Host only. Writes *ld (row stride of the Newton matrix), *n_arrays (at
 * most 32) and, per array a, offset[a] and size[a] in doubles within its
 * space and in_global[a] (0 shared, 1 global); priority[k] is the array
 * placed k-th (shared memory is filled in this order until one does not
 * fit; it and all later ones go to global scratch, except the reduction
 * scratch, which is always shared); *smem_doubles and *global_doubles are
 * the totals. Arrays of 32 ints. Errors: CG_EINVAL. */
cg_status cgx_layout(int ns, int nr, int mat_bytes, int64_t smem_limit, int adjoint, int gmres_m, int *ld,
                     int *n_arrays, int *offset, int *size, int *in_global, int *priority, int *smem_doubles,
                     int *global_doubles);

/* The per-species thermo table that cg_mech_set_thermo(mech, np, coef)
 * uploads for ns species (Section 2.1, eq. specific_heat_polynomial), in
 * the kernels' layout: table[r * ns + i] for rows r < 4 P + 1, where
 * P = max(np, 4) is written to *P; rows a_k (k = 0..P), a_k/(k+1) at
 * P + k (k >= 1), the h/R constant at 2 P + 1, a_k/k at 2 P + k (k >= 2),
 * the s/R constant at 3 P + 1, k a_k at 3 P + k (k >= 2), with a_k = 0
 * above np. Host only. table may be NULL (only *P is written); otherwise
 * `capacity` entries, at least (4 P + 1) ns. Errors: CG_EINVAL (as
 * cg_mech_set_thermo, ns < 1), CG_ECAPACITY. */
cg_status cgx_thermo_table(int ns, int np, const double *coef, int *P, double *table, int64_t capacity);

/* The Butcher tableau the kernels use for `method` (CG_BE, CG_SDIRK2,
 * CG_SDIRK4; Appendix A.1, A.2, in stage-derivative form): *s stages,
 * A[5*5] row-major, b[5], the embedded weights bh[5] and the embedded
 * order *err_order (0: none). SDIRK-4's coefficients are the full-precision
 * root of its order conditions near the printed values. Host only.
 * Errors: CG_EINVAL (NULL arrays, a method without a tableau). */
cg_status cgx_tableau(int method, int *s, double *A, double *b, double *bh, int *err_order);

/* Debug build only (compiled with CG_DEBUG: one-warp teams, two guard
 * words after every array of a cell's working memory, every array poisoned
 * with NaN -- zero for the pivot and reduction integers -- before each cell
 * of cg_integrate, the guards checked after it). Synchronises the device,
 * then writes the arrays whose guards changed since the last call (bit a:
 * the library's array number a) to *arrays and the first such cell to
 * *first_cell (-1: none), and clears both. Errors: CG_EINVAL, CG_ECUDA;
 * CG_EUNSUPPORTED in the normal build. */
cg_status cgx_debug_flags(const cg_mech *mech, uint64_t *arrays, int64_t *first_cell);

/* The scratch cg_integrate_noalloc would need for a mechanism of ns
 * species and nr reactions: the per-cell layout for mat_bytes (8 FP64, 4
 * FP32 Newton matrix), smem_limit bytes of shared memory per cell and
 * gmres_m (0: LU), times the teams per block the launch would use (team
 * threads per cell; teams_per_block lowered while the block's shared memory
 * exceeds 227 KB; 1 for teams above a warp). Host only. *scratch_bytes
 * receives that need. Returns CG_ECAPACITY, with the message
 * cg_integrate_noalloc gives, when it exceeds the library's fixed array.
 * Errors: CG_EINVAL. */
cg_status cgx_noalloc_plan(int ns, int nr, int mat_bytes, int64_t smem_limit, int gmres_m, int team,
                           int teams_per_block, int64_t *scratch_bytes);

#ifdef __cplusplus
}
#endif

#endif /* CHEMGB_TESTING_H */
