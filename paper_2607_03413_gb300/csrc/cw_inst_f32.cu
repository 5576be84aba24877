// FP32 vectors, FP32 metric, FP32 arithmetic (CW_PREC_F32), plus the FP32-arithmetic dispatch.
#include "cw_launch.cuh"
namespace cw {
cudaError_t apply_launch_f32g16(const Op &op, const void *x, void *y, cudaStream_t s, int *xfuse);
cudaError_t apply_launch_bf16(const Op &op, const void *x, void *y, cudaStream_t s, int *xfuse);
cudaError_t apply_launch_f32(const Op &op, const void *x, void *y, cudaStream_t s, int *xfuse)
{
    switch (op.prec) {
    case CW_PREC_F32: return launch_degree<ArF32, float, float>(op, x, y, s, xfuse);
    case CW_PREC_F32_BF16G: return apply_launch_f32g16(op, x, y, s, xfuse);
    default: return apply_launch_bf16(op, x, y, s, xfuse);
    }
}
cudaError_t apply_dot_launch_f32(const Op &op, const void *x, void *y, double *part, int64_t *nb, cudaStream_t s)
{
    return launch_dot_degree<ArF32, float, float>(op, x, y, part, nb, s);
}
}  // namespace cw
