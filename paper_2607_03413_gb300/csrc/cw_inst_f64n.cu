// FP64 storage, native FP64 arithmetic (CW_PREC_F64_NATIVE): the speed baseline.
#include "cw_launch.cuh"
namespace cw {
cudaError_t apply_launch_f64n(const Op &op, const void *x, void *y, cudaStream_t s)
{
    return launch_degree<ArF64, double, double, false>(op, x, y, s);
}
}  // namespace cw
