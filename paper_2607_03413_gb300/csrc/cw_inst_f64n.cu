// FP64 vectors, native FP64 arithmetic (CW_PREC_F64_NATIVE): the speed baseline. The metric is the
// (hi, lo) float-pair form shared with CW_PREC_F64, widened to double exactly on load.
#include "cw_launch.cuh"
namespace cw {
cudaError_t apply_launch_f64n(const Op &op, const void *x, void *y, cudaStream_t s, int *xfuse)
{
    return launch_degree<ArF64, double, df64s, false>(op, x, y, s, xfuse);
}
}  // namespace cw
