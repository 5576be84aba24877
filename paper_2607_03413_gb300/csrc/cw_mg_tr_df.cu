// Multigrid transfers, FP64 vectors, double-float arithmetic (CW_PREC_F64).
#include "cw_launch.cuh"
#include "cw_mg.cuh"
namespace cw {
cudaError_t mg_prolong_launch_df(const Op &fine, const Op &coarse, const void *uc, void *uf, bool add, cudaStream_t s)
{
    (void)fine;
    return prolong_degree<ArDF, double>(coarse, uc, uf, add, s);
}
cudaError_t mg_restrict_launch_df(const Op &fine, const Op &coarse, const void *bf, const void *vf, void *bc,
                                  cudaStream_t s)
{
    (void)fine;
    return restrict_degree<ArDF, double>(coarse, bf, vf, bc, s);
}
}  // namespace cw
