// Fused multigrid smoothing sweep on curved cells, FP64 vectors, double-float arithmetic (CW_PREC_F64).
#include "cw_launch.cuh"
namespace cw {
cudaError_t mg_smooth_launch_df(const Op &op, void *u, const void *b, const void *dhat, cudaStream_t s, int *xfuse)
{
    return launch_smooth_degree<ArDF, double, df64s>(op, u, b, dhat, s, xfuse);
}
}  // namespace cw
