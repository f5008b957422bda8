// Host-side internals shared by the C-ABI layer and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "chem_device.cuh"

namespace cg {

cudaError_t launch_eval_rates(const DevMech& M, const Layout& L, int wpb, int reactor, int64_t N,
                              const double* T, const double* C, double* S, cudaStream_t st);
cudaError_t launch_eval_jacobian(const DevMech& M, const Layout& L, int wpb, int reactor, int64_t N,
                                 const double* T, const double* C, double* J, cudaStream_t st);
cudaError_t launch_temperature(const DevMech& M, int reactor, int64_t N, const double* e,
                               const double* Y, double* T, int iters, cudaStream_t st);
cudaError_t launch_integrate(const DevMech& M, const Layout& L, const IntParams& P, int wpb,
                             int64_t N, double* T, double* Y, const double* p_or_rho,
                             int32_t* status, int32_t* stats, cudaStream_t st);

}  // namespace cg
