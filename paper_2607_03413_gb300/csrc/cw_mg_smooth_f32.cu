// Fused multigrid smoothing sweep on curved cells, FP32 vectors, metric and arithmetic (CW_PREC_F32).
#include "cw_launch.cuh"
namespace cw {
cudaError_t mg_smooth_launch_f32(const Op &op, void *u, const void *b, const void *dhat, cudaStream_t s, int *xfuse)
{
    return launch_smooth_degree<ArF32, float, float>(op, u, b, dhat, s, xfuse);
}
}  // namespace cw
