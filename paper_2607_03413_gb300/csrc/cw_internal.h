// cw_internal.h -- host-side structures shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/cwfem.h"

namespace cw {

// Host-side NVTX range around an entry point or a solver phase: a profiler's timeline (and ncu's
// --nvtx filters) sees "cwfem:<name>". Header-only NVTX: with no tool attached a push or a pop is a
// call through a null-checked pointer.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

// Cells per CTA of the curved kernels: the default; the tuner's alternative is half of it. FP32
// arithmetic (FP32 and BF16 storage; bound by shared-memory traffic) takes more cells at n = 2, 3, 6,
// 7 (fewer barriers and bulk copies per value: 17-22 % faster at n = 3, 30 % for BF16 at n = 7);
// double-float and FP64 tiles (bound by registers and the FP32 pipes) keep the smaller ones.
__host__ __device__ constexpr int tile_cells(int n, bool f32)
{
    return n == 2 ? (f32 ? 64 : 32) : n == 3 ? (f32 ? 32 : 16) : n == 4 ? 8 : n == 5 ? 8
           : n == 6 ? (f32 ? 8 : 4) : n == 7 ? (f32 ? 8 : 4) : 2;
}

// whether a precision computes in FP32 arithmetic (its kernels use the FP32 tile sizes)
__host__ __device__ inline bool prec_f32_arith(int prec)
{
    return prec == CW_PREC_F32 || prec == CW_PREC_F32_BF16G || prec == CW_PREC_BF16;
}


constexpr int kMaxDegree = 7;
// cells per mesh direction: the DSS launches put one direction on the grid's y extent (<= 65535)
constexpr int kMaxCellsPerDir = 65535;
constexpr int kMaxN = kMaxDegree + 1;

// 1D tables of one degree, in double (built from long-double rules by cw_tables.cpp)
struct Tables1D {
    int p = 0, n = 0;
    double gll[kMaxN];          // Gauss-Lobatto nodes on [0,1]
    double xq[kMaxN], wq[kMaxN];  // Gauss points and weights on [0,1]
    double B[kMaxN][kMaxN];     // B[q][m] = l_m(xq)
    double Bd[kMaxN][kMaxN];    // Bd[q][m] = l_m'(xq)
    double D[kMaxN][kMaxN];     // collocation derivative on the Gauss points
    double M1[kMaxN][kMaxN];    // 1D mass matrix of the GLL basis
    double K1[kMaxN][kMaxN];    // 1D stiffness matrix of the GLL basis
    double P0[kMaxN][kMaxN];    // P_b[i][a] = l_a((gll_i + b)/2): parent basis at the nodes of child b
    double P1[kMaxN][kMaxN];
};
void build_tables(int p, Tables1D &t);

struct Mesh {
    int nx = 0, ny = 0, nz = 0;
    double *d_verts = nullptr;
    std::vector<double> h_verts;
    bool cartesian = false;
    int64_t ncells() const { return (int64_t)nx * ny * nz; }
};

struct CgScratch;

struct Op {
    Mesh *mesh = nullptr;
    int p = 0, n = 0, kind = 0, geom = 0, prec = 0, bc = 0;
    int64_t E = 0, L = 0, NG = 0;
    Tables1D tab;
    void *d_geo = nullptr;  // metric [E][ncomp][n^3] in the metric type (CW_PREC_F64: df64s pairs; CW_PREC_F64_NATIVE:
                            // doubles), or affine [E][4] doubles
    int64_t geo_bytes = 0;
    double *d_dinv = nullptr;  // cell-wise masked inverse diagonal (solver), lazily
    CgScratch *cg = nullptr;
    Op *inner = nullptr;   // reduced-precision twin used by iterative refinement
    Op *native = nullptr;  // IEEE FP64 twin (CW_PREC_F64_NATIVE, metric as doubles): the solver's outer residual
    // host-buffer apply (cw_apply_host): device staging vectors, streams and events, lazily
    void *h_dx = nullptr, *h_dy = nullptr;
    cudaStream_t h_st[3] = {nullptr, nullptr, nullptr};
    static constexpr int kNominalSlabs = 16;  // equal slabs: 32 measured slower than 16
    static constexpr int kMaxSlabs = 32;      // with the ramped first and last slabs
    cudaEvent_t h_ev[2][kMaxSlabs] = {};
    cudaEvent_t h_done = nullptr;
    unsigned *d_status = nullptr;  // device status word: kDevStatusTimeout when a bounded wait expired
    uint32_t dbg_tma_extra = 0;    // fault injection for tests: extra bytes armed on the staged input tile
    int cpb = 0;          // apply kernel variant: cells per CTA (0 = default for the degree)
    int stage = 1;        // apply kernel variant: TMA staging of the input and metric tiles
    int64_t owned_bytes = 0;
};

// bumped whenever an operator's kernel choice or fault-injection setting changes: CUDA graphs captured
// before (the solvers' iteration graphs bake kernels and their arguments in) are re-captured
uint64_t op_generation();
void op_generation_bump();

size_t vec_elem_size(int prec);
bool metric_is_f64(int prec);

// launchers implemented in the instantiation units
// xfuse != nullptr asks the curved-cell kernel to apply the DSS x pass inside each tile; *xfuse
// receives the tile size in cells (0: nothing fused, e.g. Cartesian cells)
cudaError_t apply_launch_df(const Op &op, const void *x, void *y, cudaStream_t s, int *xfuse = nullptr);
cudaError_t apply_launch_f64n(const Op &op, const void *x, void *y, cudaStream_t s, int *xfuse = nullptr);
cudaError_t apply_launch_f32(const Op &op, const void *x, void *y, cudaStream_t s, int *xfuse = nullptr);

// y = A x plus the per-CTA partials of <x, y> (curved cells, default tile and staging; for
// CW_PREC_F64, CW_PREC_F32 and CW_PREC_F32_BF16G); *nb = number of partials
cudaError_t apply_dot_launch_df(const Op &op, const void *x, void *y, double *part, int64_t *nb, cudaStream_t s);
cudaError_t apply_dot_launch_f32(const Op &op, const void *x, void *y, double *part, int64_t *nb, cudaStream_t s);
cudaError_t apply_dot_launch_f32g16(const Op &op, const void *x, void *y, double *part, int64_t *nb, cudaStream_t s);

// dispatch to the right unit
cudaError_t apply_local(const Op &op, const void *x, void *y, cudaStream_t s, int *xfuse = nullptr);
// xtile > 0: the x pass skips the interfaces inside tiles of xtile consecutive cells (already summed)
cudaError_t dss_launch(const Op &op, void *v, int flags, cudaStream_t s, int xtile = 0);
// out of place: dst = S src (flags CW_DSS_SUM) or S_bar src (CW_DSS_AVERAGE); the x pass is fused
// with the copy
cudaError_t dss_from(const Op &op, const void *src, void *dst, int flags, cudaStream_t s);
// dst = S (r - a q) with a = *active ? *alpha : 0 (device scalars): the CG residual update fused into
// the DSS (r is left unchanged unless the vector exceeds 32-bit line indexing, where it is updated
// in place first). FP32 or FP64 vectors. x_only: only the x pass (the caller completes the y and z
// sums; needs L < 2^31, else cudaErrorInvalidValue).
cudaError_t dss_from_axpy(const Op &op, void *r, const void *q, const double *alpha, const int *active, void *dst,
                          cudaStream_t s, bool x_only = false);

// solver scratch release (cw_cg.cu)
void cg_release(Op *op);

// element matrices A[e][i][j] (FP64, E * (p+1)^6 doubles) of every cell of the operator's mesh
cudaError_t element_matrices_launch(const Op &op, double *A, cudaStream_t s);

// ---- multigrid (cw_mg.cu, transfers in cw_mg_tr_*.cu)
// uf = P uc (add: uf += P uc) between the coarse level `coarse` and its refinement `fine`
cudaError_t mg_prolong_launch(const Op &fine, const Op &coarse, const void *uc, void *uf, bool add, cudaStream_t s);
// bc = R (bf - vf) (vf may be NULL: bc = R bf)
cudaError_t mg_restrict_launch(const Op &fine, const Op &coarse, const void *bf, const void *vf, void *bc,
                               cudaStream_t s);
cudaError_t mg_prolong_launch_df(const Op &fine, const Op &coarse, const void *uc, void *uf, bool add, cudaStream_t s);
cudaError_t mg_restrict_launch_df(const Op &fine, const Op &coarse, const void *bf, const void *vf, void *bc,
                                  cudaStream_t s);
cudaError_t mg_prolong_launch_f32(const Op &fine, const Op &coarse, const void *uc, void *uf, bool add, cudaStream_t s);
cudaError_t mg_restrict_launch_f32(const Op &fine, const Op &coarse, const void *bf, const void *vf, void *bc,
                                   cudaStream_t s);
cudaError_t mg_prolong_launch_f64n(const Op &fine, const Op &coarse, const void *uc, void *uf, bool add, cudaStream_t s);
cudaError_t mg_restrict_launch_f64n(const Op &fine, const Op &coarse, const void *bf, const void *vf, void *bc,
                                    cudaStream_t s);
// one fused smoothing sweep on curved cells (metric stored or recomputed), in place on u: the operator
// epilogue forms u + D_hat (b - A u) and averages the x-interfaces inside each tile of *xfuse cells
cudaError_t mg_smooth_launch_df(const Op &op, void *u, const void *b, const void *dhat, cudaStream_t s, int *xfuse);
cudaError_t mg_smooth_launch_f32(const Op &op, void *u, const void *b, const void *dhat, cudaStream_t s, int *xfuse);
// the averaging DSS (every pass halves its pair sums, so no separate division by the valence) with the
// x pass restricted to the interfaces between tiles of xtile cells (0: all)
cudaError_t dss_average_launch(const Op &op, void *v, cudaStream_t s, int xtile);
struct MgHier;
// u = MG(b): one V-cycle on the finest level from a zero initial guess (enqueue only)
cudaError_t mg_vcycle_zero(MgHier &h, const void *b, void *u, cudaStream_t s);
const Op &mg_top_op(const MgHier &h);
// op_status_take over the hierarchy's level operators
cw_status mg_status_take(MgHier &h, cudaStream_t s);
uint64_t mg_id(const MgHier &h);

// device status words: CW_ERR_TIMEOUT (and the word cleared) if a bounded wait of the operator's
// kernels expired since the last check, else CW_OK; reads the word on stream s (synchronising it)
cw_status op_status_take(Op *op, cudaStream_t s, const char *where);

// error reporting (thread-local message)
void set_error(const std::string &msg);
cw_status fail(cw_status st, const std::string &msg);
cw_status cuda_fail(cudaError_t e, const char *where);

}  // namespace cw

#define CW_CUDA_TRY(expr)                                              \
    do {                                                               \
        cudaError_t e_ = (expr);                                       \
        if (e_ != cudaSuccess) return ::cw::cuda_fail(e_, #expr);      \
    } while (0)
