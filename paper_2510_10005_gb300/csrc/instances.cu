// Explicit instantiation of the integration, operator-split and adjoint
// kernels for one team size CG_TEAM and one Newton-matrix type CG_MT
// (double: FP64, float: FP32 mixed precision), and of the rate and Jacobian
// kernels with the FP64 ones. The build compiles this file once per
// combination (paper_2510_10005_gb300/build.py), in parallel.
#include "adjoint.cuh"
#include "integrate.cuh"
#include "split.cuh"

#if !defined(CG_TEAM) || !defined(CG_MT) || !defined(CG_MT_F64)
#error "compile with -DCG_TEAM=32|64|128|256 -DCG_MT=double|float -DCG_MT_F64=1|0"
#endif

namespace cg {

template cudaError_t launch_integrate_team<CG_TEAM, CG_MT>(const Tasks&, const IntParams&, int, bool, cudaStream_t);
template cudaError_t launch_integrate_on_team<CG_TEAM, CG_MT>(const Tasks&, const IntParams&, int, double*, int64_t,
                                                              unsigned long long*, cudaStream_t);
template cudaError_t launch_split_team<CG_TEAM, CG_MT>(const SplitTask&, const IntParams&, int, cudaStream_t);
template cudaError_t launch_adjoint_team<CG_TEAM, CG_MT>(const AdjTask&, const IntParams&, int, cudaStream_t);
#if CG_MT_F64
template cudaError_t launch_eval_team<CG_TEAM>(bool, const DevMech&, const Layout&, int, int, int64_t, const double*,
                                               const double*, double*, cudaStream_t);
#endif

}  // namespace cg
