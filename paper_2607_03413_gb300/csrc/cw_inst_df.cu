// FP64 storage, double-float arithmetic (CW_PREC_F64).
#include "cw_launch.cuh"
namespace cw {
cudaError_t apply_launch_df(const Op &op, const void *x, void *y, cudaStream_t s)
{
    return launch_degree<ArDF, double, double>(op, x, y, s);
}
}  // namespace cw
