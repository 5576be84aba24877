// FP64 vectors, native FP64 arithmetic. A CW_PREC_F64_NATIVE operator stores its metric (or its
// trilinear-map coefficients) as IEEE doubles: the plain FP64 operator, the speed baseline and the
// operator of the solver's outer residual. The same arithmetic on a CW_PREC_F64 operator reads that
// operator's (hi, lo) float-pair metric, widened to double exactly on load.
#include "cw_launch.cuh"
namespace cw {
cudaError_t apply_launch_f64n(const Op &op, const void *x, void *y, cudaStream_t s, int *xfuse)
{
    if (op.prec == CW_PREC_F64_NATIVE) return launch_degree<ArF64, double, double, false, double>(op, x, y, s, xfuse);
    return launch_degree<ArF64, double, df64s, false, df64s>(op, x, y, s, xfuse);
}
}  // namespace cw
