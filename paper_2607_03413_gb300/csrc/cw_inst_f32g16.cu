// FP32 vectors, BF16 metric, FP32 arithmetic (CW_PREC_F32_BF16G).
#include <cuda_bf16.h>

#include "cw_launch.cuh"
namespace cw {
cudaError_t apply_launch_f32g16(const Op &op, const void *x, void *y, cudaStream_t s, int *xfuse)
{
    return launch_degree<ArF32, float, __nv_bfloat16>(op, x, y, s, xfuse);
}
cudaError_t apply_dot_launch_f32g16(const Op &op, const void *x, void *y, double *part, int64_t *nb, cudaStream_t s)
{
    return launch_dot_degree<ArF32, float, __nv_bfloat16>(op, x, y, part, nb, s);
}
}  // namespace cw
