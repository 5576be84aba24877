// FP64 storage, double-float arithmetic (CW_PREC_F64).
#include "cw_launch.cuh"
namespace cw {
cudaError_t apply_launch_df(const Op &op, const void *x, void *y, cudaStream_t s, int *xfuse)
{
    return launch_degree<ArDF, double, df64s>(op, x, y, s, xfuse);
}
cudaError_t apply_dot_launch_df(const Op &op, const void *x, void *y, double *part, int64_t *nb, cudaStream_t s)
{
    return launch_dot_degree<ArDF, double, df64s>(op, x, y, part, nb, s);
}
}  // namespace cw
