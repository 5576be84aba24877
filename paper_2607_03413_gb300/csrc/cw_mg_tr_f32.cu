// Multigrid transfers, FP32 vectors and arithmetic (CW_PREC_F32).
#include "cw_launch.cuh"
#include "cw_mg.cuh"
namespace cw {
cudaError_t mg_prolong_launch_f32(const Op &fine, const Op &coarse, const void *uc, void *uf, bool add, cudaStream_t s)
{
    (void)fine;
    return prolong_degree<ArF32, float>(coarse, uc, uf, add, s);
}
cudaError_t mg_restrict_launch_f32(const Op &fine, const Op &coarse, const void *bf, const void *vf, void *bc,
                                  cudaStream_t s)
{
    (void)fine;
    return restrict_degree<ArF32, float>(coarse, bf, vf, bc, s);
}
}  // namespace cw
