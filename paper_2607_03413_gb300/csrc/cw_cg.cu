// cw_cg.cu -- cell-wise Jacobi-preconditioned CG (placeholder until the solver lands).
#include "cw_internal.h"
using namespace cw;
namespace cw {
void cg_release(Op *op) { (void)op; }
}  // namespace cw
extern "C" cw_status cw_cg_solve(cw_op, const double *, double *, double, int, int, cw_cg_stats *, void *)
{
    return fail(CW_ERR_UNSUPPORTED, "cw_cg_solve: not built yet");
}
