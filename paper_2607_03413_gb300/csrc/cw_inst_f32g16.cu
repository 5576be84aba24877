// FP32 vectors, BF16 metric, FP32 arithmetic (CW_PREC_F32_BF16G).
#include <cuda_bf16.h>

#include "cw_launch.cuh"
namespace cw {
cudaError_t apply_launch_f32g16(const Op &op, const void *x, void *y, cudaStream_t s)
{
    return launch_degree<ArF32, float, __nv_bfloat16>(op, x, y, s);
}
}  // namespace cw
