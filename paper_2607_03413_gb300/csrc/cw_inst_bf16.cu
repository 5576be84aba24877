// BF16 vectors, BF16 metric, FP32 arithmetic (CW_PREC_BF16).
#include <cuda_bf16.h>

#include "cw_launch.cuh"
namespace cw {
cudaError_t apply_launch_bf16(const Op &op, const void *x, void *y, cudaStream_t s, int *xfuse)
{
    return launch_degree<ArF32, __nv_bfloat16, __nv_bfloat16>(op, x, y, s, xfuse);
}
}  // namespace cw
