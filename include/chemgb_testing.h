/*
 * chemgb test hooks (C ABI). Not part of the method: entry points that let
 * the tests check device functions of the library against CUDA's own.
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

#ifdef __cplusplus
}
#endif

#endif /* CHEMGB_TESTING_H */
