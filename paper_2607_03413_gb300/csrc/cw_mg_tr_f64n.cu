// Multigrid transfers, FP64 vectors, native FP64 arithmetic (CW_PREC_F64_NATIVE).
#include "cw_launch.cuh"
#include "cw_mg.cuh"
namespace cw {
cudaError_t mg_prolong_launch_f64n(const Op &fine, const Op &coarse, const void *uc, void *uf, bool add, cudaStream_t s)
{
    (void)fine;
    return prolong_degree<ArF64, double>(coarse, uc, uf, add, s);
}
cudaError_t mg_restrict_launch_f64n(const Op &fine, const Op &coarse, const void *bf, const void *vf, void *bc,
                                  cudaStream_t s)
{
    (void)fine;
    return restrict_degree<ArF64, double>(coarse, bf, vf, bc, s);
}
}  // namespace cw
