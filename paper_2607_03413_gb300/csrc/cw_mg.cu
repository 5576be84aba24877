// cw_mg.cu -- geometric multigrid V-cycle on cell-wise data over a uniform mesh hierarchy.
//
// Algorithm mg_vcycle (Sec. 3) with the pieces of Sec. 5:
//  - smoother: the fused damped-Jacobi sweep of Algorithm smoother_fused, u <- S_bar(u + D_hat (b - A u))
//    with D_hat = omega K_cell D_cell^-1 (valence K_cell baked in at set-up, Eq. (valence_baking);
//    zeros on Dirichlet DoFs, "Constraints baked into the diagonal"); S_bar is the averaging DSS of
//    Eq. (averaging_dss);
//  - zero initial guess: the first pre-smoothing sweep of a level entered with u = 0 skips the
//    operator (A 0 = 0: u = D_hat b);
//  - fused residual restriction: R (b - A u) with the difference formed in the restriction's load;
//  - transfers: Algorithms prolongation and restriction (cw_mg.cuh, per arithmetic in cw_mg_tr_*.cu);
//  - coarse solve A_0^-1: the interior block of the level-0 matrix A_CG, assembled in FP64 from
//    explicit element matrices and inverted once on the host (Cholesky); at run time
//    u_0 = G (A_int^-1 (G^T b_0)|_int), one dense matrix-vector product.
// Every launch is enqueued on the caller's stream with no host synchronisation, so a cycle can be
// captured into a CUDA graph (the preconditioned CG in cw_cg.cu does so).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "cw_internal.h"

namespace cw {

// largest number of interior DoFs of the coarsest level (dense inverse: 128 MB at the limit)
constexpr int64_t kMgMaxCoarse = 4096;

// ------------------------------------------------------------------------------ kernels ----
#define CW_MG_LOOP(i, n) \
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// D_hat = omega * valence / d on interior DoFs, 0 on the Dirichlet boundary (d: assembled diagonal)
template <class VS>
__global__ void k_make_dhat(const double *__restrict__ d, VS *__restrict__ dhat, int nx, int ny, int nz, int p,
                            int64_t L, double omega)
{
    const int n = p + 1, n3 = n * n * n;
    CW_MG_LOOP(t, L)
    {
        const int64_t e = t / n3;
        const int loc = (int)(t - e * n3), i = loc % n, j = (loc / n) % n, k = loc / (n * n);
        const int64_t cx = e % nx, cy = (e / nx) % ny, cz = e / ((int64_t)nx * ny);
        const bool bnd = (cx == 0 && i == 0) || (cx == nx - 1 && i == p) || (cy == 0 && j == 0) ||
                         (cy == ny - 1 && j == p) || (cz == 0 && k == 0) || (cz == nz - 1 && k == p);
        int kap = 1;
        if ((i == 0 && cx > 0) || (i == p && cx < nx - 1)) kap *= 2;
        if ((j == 0 && cy > 0) || (j == p && cy < ny - 1)) kap *= 2;
        if ((k == 0 && cz > 0) || (k == p && cz < nz - 1)) kap *= 2;
        dhat[t] = bnd ? VS(0) : static_cast<VS>(omega * kap / d[t]);
    }
}

// u <- u + D_hat (b - v): the per-copy update of Algorithm smoother_fused (before S_bar)
template <class VS>
__global__ void k_jacobi(VS *__restrict__ u, const VS *__restrict__ b, const VS *__restrict__ v,
                         const VS *__restrict__ dhat, int64_t n)
{
    CW_MG_LOOP(i, n) u[i] = u[i] + dhat[i] * (b[i] - v[i]);
}

// u <- D_hat b (the same update from u = 0)
template <class VS>
__global__ void k_jacobi_zero(VS *__restrict__ u, const VS *__restrict__ b, const VS *__restrict__ dhat, int64_t n)
{
    CW_MG_LOOP(i, n) u[i] = dhat[i] * b[i];
}

// xg[i] = w[rep[i]]: one copy of every interior DoF of the assembled coarse right-hand side
template <class VS>
__global__ void k_coarse_pick(const VS *__restrict__ w, const int *__restrict__ rep, double *__restrict__ xg, int ni)
{
    CW_MG_LOOP(i, ni) xg[i] = static_cast<double>(w[rep[i]]);
}

// y = A x for a dense row-major n x n FP64 matrix: one warp per row
__global__ void k_dense_matvec(const double *__restrict__ A, const double *__restrict__ x, double *__restrict__ y,
                               int n)
{
    const int lane = threadIdx.x & 31;
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= n) return;
    const double *a = A + row * n;
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s = fma(a[j], x[j], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = s;
}

// u[t] = y[gi[t]] for interior copies, 0 on the boundary (the gather G of the coarse solution)
template <class VS>
__global__ void k_coarse_put(const double *__restrict__ y, const int *__restrict__ gi, VS *__restrict__ u, int64_t L)
{
    CW_MG_LOOP(t, L)
    {
        const int g = gi[t];
        u[t] = g >= 0 ? static_cast<VS>(y[g]) : VS(0);
    }
}

// ------------------------------------------------------------------------------ hierarchy ----
struct MgLevel {
    Op *op = nullptr;     // the caller's operator of the level (not owned)
    void *dhat = nullptr;  // omega K_cell D_cell^-1, masked, in the level's vector type
    void *b = nullptr, *u = nullptr, *v = nullptr;  // right-hand side, iterate, operator output
};

struct MgHier {
    std::vector<MgLevel> lv;
    int nu1 = 2, nu2 = 2;
    double omega = 0.7;
    int prec = CW_PREC_F64;
    size_t es = 8;  // vector element size
    uint64_t id = 0;
    // coarse solve
    int ni0 = 0;
    double *ainv = nullptr, *xg = nullptr, *yg = nullptr;
    int *rep = nullptr, *gi = nullptr;
    void *w0 = nullptr;
    int64_t bytes = 0;
};

const Op &mg_top_op(const MgHier &h) { return *h.lv.back().op; }
cw_status mg_status_take(MgHier &h, cudaStream_t s)
{
    for (MgLevel &L : h.lv) {
        cw_status st = op_status_take(L.op, s, "multigrid cycle");
        if (st != CW_OK) return st;
    }
    return CW_OK;
}
uint64_t mg_id(const MgHier &h) { return h.id; }

static unsigned vgrid(int64_t n) { return (unsigned)std::min<int64_t>(1216, std::max<int64_t>(1, (n + 255) / 256)); }

static cudaError_t prolong(const MgHier &h, int l, const void *uc, void *uf, bool add, cudaStream_t s)
{
    const Op &f = *h.lv[l].op, &c = *h.lv[l - 1].op;
    switch (h.prec) {
    case CW_PREC_F64: return mg_prolong_launch_df(f, c, uc, uf, add, s);
    case CW_PREC_F64_NATIVE: return mg_prolong_launch_f64n(f, c, uc, uf, add, s);
    default: return mg_prolong_launch_f32(f, c, uc, uf, add, s);
    }
}

static cudaError_t restrict_(const MgHier &h, int l, const void *bf, const void *vf, void *bc, cudaStream_t s)
{
    const Op &f = *h.lv[l].op, &c = *h.lv[l - 1].op;
    switch (h.prec) {
    case CW_PREC_F64: return mg_restrict_launch_df(f, c, bf, vf, bc, s);
    case CW_PREC_F64_NATIVE: return mg_restrict_launch_f64n(f, c, bf, vf, bc, s);
    default: return mg_restrict_launch_f32(f, c, bf, vf, bc, s);
    }
}

// Whether a sweep can run as one operator launch with the Jacobi update and the in-tile x averages in
// its epilogue (curved cells in double-float or FP32 arithmetic; the x pass between tiles then indexes
// its interfaces with 32 bits)
static bool fused_sweep(const MgHier &h, const Op &op)
{
    return (h.prec == CW_PREC_F64 || h.prec == CW_PREC_F32) && op.geom != CW_GEOM_AFFINE &&
           op.E * (int64_t)(op.n * op.n) < ((int64_t)1 << 32);
}

// `sweeps` sweeps of Algorithm smoother_fused: u <- S_bar (u + D_hat (b - A u)). The first sweep from
// u = 0 (zero) is u = S_bar D_hat b. A fused sweep is one operator launch whose epilogue applies the
// update and the x averages inside its tiles, then the x pass between tiles and the y and z passes of
// the averaging DSS; otherwise operator, update kernel and the three averaging passes.
template <class VS>
static cudaError_t smooth_t(const MgHier &h, int l, const VS *b, VS *u, int sweeps, bool zero, cudaStream_t s)
{
    const MgLevel &L = h.lv[l];
    const Op &op = *L.op;
    const VS *dh = static_cast<const VS *>(L.dhat);
    VS *v = static_cast<VS *>(L.v);
    const bool fused = fused_sweep(h, op);
    for (int k = 0; k < sweeps; ++k) {
        cudaError_t e;
        int xtile = 0;
        if (zero && k == 0) {
            k_jacobi_zero<VS><<<vgrid(op.L), 256, 0, s>>>(u, b, dh, op.L);
        } else if (fused) {
            e = h.prec == CW_PREC_F64 ? mg_smooth_launch_df(op, u, b, dh, s, &xtile)
                                      : mg_smooth_launch_f32(op, u, b, dh, s, &xtile);
            if (e != cudaSuccess) return e;
        } else {
            if ((e = apply_local(op, u, v, s)) != cudaSuccess) return e;
            k_jacobi<VS><<<vgrid(op.L), 256, 0, s>>>(u, b, v, dh, op.L);
        }
        if ((e = dss_average_launch(op, u, s, xtile)) != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

static cudaError_t smooth(const MgHier &h, int l, const void *b, void *u, int sweeps, bool zero, cudaStream_t s)
{
    if (h.es == 8) return smooth_t(h, l, static_cast<const double *>(b), static_cast<double *>(u), sweeps, zero, s);
    return smooth_t(h, l, static_cast<const float *>(b), static_cast<float *>(u), sweeps, zero, s);
}

template <class VS>
static cudaError_t coarse_t(const MgHier &h, const VS *b, VS *u, cudaStream_t s)
{
    const Op &op = *h.lv[0].op;
    cudaError_t e = dss_from(op, b, h.w0, CW_DSS_SUM, s);  // G G^T b: every copy holds the assembled value
    if (e != cudaSuccess) return e;
    k_coarse_pick<VS><<<vgrid(h.ni0), 256, 0, s>>>(static_cast<const VS *>(h.w0), h.rep, h.xg, h.ni0);
    k_dense_matvec<<<(unsigned)((h.ni0 * 32 + 255) / 256), 256, 0, s>>>(h.ainv, h.xg, h.yg, h.ni0);
    k_coarse_put<VS><<<vgrid(op.L), 256, 0, s>>>(h.yg, h.gi, u, op.L);
    return cudaGetLastError();
}

static cudaError_t coarse_solve(const MgHier &h, const void *b, void *u, cudaStream_t s)
{
    if (h.es == 8) return coarse_t(h, static_cast<const double *>(b), static_cast<double *>(u), s);
    return coarse_t(h, static_cast<const float *>(b), static_cast<float *>(u), s);
}

// Algorithm mg_vcycle on level l: u <- MG(b, u); zero: u enters as 0 (its content is ignored)
static cudaError_t vcycle(const MgHier &h, int l, const void *b, void *u, bool zero, cudaStream_t s)
{
    if (l == 0) return coarse_solve(h, b, u, s);
    const MgLevel &L = h.lv[l], &C = h.lv[l - 1];
    const Op &op = *L.op;
    cudaError_t e;
    if ((e = smooth(h, l, b, u, h.nu1, zero, s)) != cudaSuccess) return e;
    if (zero && h.nu1 == 0) {  // u = 0: the residual is b itself
        if ((e = cudaMemsetAsync(u, 0, op.L * h.es, s)) != cudaSuccess) return e;
        if ((e = restrict_(h, l, b, nullptr, C.b, s)) != cudaSuccess) return e;
    } else {
        if ((e = apply_local(op, u, L.v, s)) != cudaSuccess) return e;
        if ((e = restrict_(h, l, b, L.v, C.b, s)) != cudaSuccess) return e;  // R (b - A u)
    }
    if ((e = vcycle(h, l - 1, C.b, C.u, true, s)) != cudaSuccess) return e;  // e_{l-1} from 0
    if ((e = prolong(h, l, C.u, u, true, s)) != cudaSuccess) return e;      // u += P e
    return smooth(h, l, b, u, h.nu2, false, s);
}

cudaError_t mg_vcycle_zero(MgHier &h, const void *b, void *u, cudaStream_t s)
{
    return vcycle(h, (int)h.lv.size() - 1, b, u, true, s);
}

static void free_hier(MgHier *h)
{
    for (MgLevel &L : h->lv) {
        cudaFree(L.dhat);
        cudaFree(L.b);
        cudaFree(L.u);
        cudaFree(L.v);
    }
    cudaFree(h->ainv);
    cudaFree(h->xg);
    cudaFree(h->yg);
    cudaFree(h->rep);
    cudaFree(h->gi);
    cudaFree(h->w0);
    delete h;
}

// f(i) for i in [0, n) on up to 16 host threads (contiguous chunks)
template <class F>
static void host_parallel_for(int n, F f)
{
    const int nt = std::max(1, std::min<int>({16, (int)std::thread::hardware_concurrency(), n / 8}));
    if (nt == 1) {
        for (int i = 0; i < n; ++i) f(i);
        return;
    }
    std::atomic<int> next{0};
    auto work = [&]() {
        for (int i; (i = next.fetch_add(1)) < n;) f(i);
    };
    std::vector<std::thread> th;
    try {
        for (int t = 1; t < nt; ++t) th.emplace_back(work);
    } catch (...) {  // no more threads: the ones started and this one share the indices
    }
    work();
    for (auto &t : th) t.join();
}

// In-place inverse of a symmetric positive definite row-major n x n matrix through its Cholesky
// factor A = L L^T (blocked by columns: each panel of kNb columns is factored, then the trailing
// lower triangle is updated row by row on the host threads), then W^T = L^-T by forward substitution
// of the columns of L^-1 (independent, on the threads; stored as rows, so every inner loop reads
// memory contiguously) and A^-1 = W^T W as dot products of rows of W^T. Returns false if a pivot is
// not positive.
static bool spd_inverse(std::vector<double> &A, int n)
{
    constexpr int kNb = 48;
    std::vector<double> Lm(A);  // lower triangle: A, then L
    auto row = [&](int i) { return &Lm[(size_t)i * n]; };
    for (int kb = 0; kb < n; kb += kNb) {
        const int ke = std::min(n, kb + kNb);
        // panel: columns kb..ke-1 (earlier panels are already subtracted from them)
        for (int j = kb; j < ke; ++j) {
            double *lj = row(j);
            double d = lj[j];
            for (int k = kb; k < j; ++k) d -= lj[k] * lj[k];
            if (!(d > 0.0)) return false;
            d = std::sqrt(d);
            lj[j] = d;
            for (int i = j + 1; i < n; ++i) {
                double *li = row(i);
                double s = li[j];
                for (int k = kb; k < j; ++k) s -= li[k] * lj[k];
                li[j] = s / d;
            }
        }
        // trailing update: A[i][j] -= sum_{k in panel} L[i][k] L[j][k] for ke <= j <= i
        host_parallel_for(n - ke, [&](int r) {
            const int i = ke + r;
            double *li = row(i);
            for (int j = ke; j <= i; ++j) {
                const double *lj = row(j);
                double s = 0.0;
                for (int k = kb; k < ke; ++k) s += li[k] * lj[k];
                li[j] -= s;
            }
        });
    }
    // Wt row j = column j of L^-1: solve L x = e_j (x_i = 0 for i < j)
    std::vector<double> Wt((size_t)n * n, 0.0);
    host_parallel_for(n, [&](int j) {
        double *x = &Wt[(size_t)j * n];
        for (int i = j; i < n; ++i) {
            const double *li = row(i);
            double s = (i == j) ? 1.0 : 0.0;
            for (int k = j; k < i; ++k) s -= li[k] * x[k];
            x[i] = s / li[i];
        }
    });
    // (A^-1)_ij = sum_{k >= max(i, j)} W_ki W_kj = <Wt row i, Wt row j> over k >= i (j <= i)
    host_parallel_for(n, [&](int i) {
        const double *wi = &Wt[(size_t)i * n];
        for (int j = 0; j <= i; ++j) {
            const double *wj = &Wt[(size_t)j * n];
            double s = 0.0;
            for (int k = i; k < n; ++k) s += wi[k] * wj[k];
            A[(size_t)i * n + j] = s;
        }
    });
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j) A[(size_t)j * n + i] = A[(size_t)i * n + j];
    return true;
}

// level-0 set-up: assemble the interior block of A_CG from the element matrices, invert it, and
// build the copy <-> interior-DoF maps
static cw_status coarse_setup(MgHier &h)
{
    const Op &op = *h.lv[0].op;
    const Mesh &m = *op.mesh;
    const int p = op.p, n = op.n, n3 = n * n * n;
    const int64_t gx = (int64_t)m.nx * p + 1, gy = (int64_t)m.ny * p + 1, gz = (int64_t)m.nz * p + 1;
    const int64_t ni = (gx - 2) * (gy - 2) * (gz - 2);
    if (ni < 1) return fail(CW_ERR_ARG, "cw_mg_create: the coarsest level has no interior DoF");
    if (ni > kMgMaxCoarse)
        return fail(CW_ERR_UNSUPPORTED, "cw_mg_create: the coarsest level has " + std::to_string(ni) +
                                            " interior DoFs, more than the dense coarse solve's limit of " +
                                            std::to_string(kMgMaxCoarse));
    h.ni0 = (int)ni;
    std::vector<int> gi(op.L), rep(ni, -1);
    for (int64_t e = 0; e < op.E; ++e) {
        const int64_t cx = e % m.nx, cy = (e / m.nx) % m.ny, cz = e / ((int64_t)m.nx * m.ny);
        for (int loc = 0; loc < n3; ++loc) {
            const int64_t X = cx * p + loc % n, Y = cy * p + (loc / n) % n, Z = cz * p + loc / (n * n);
            const bool in = X > 0 && X < gx - 1 && Y > 0 && Y < gy - 1 && Z > 0 && Z < gz - 1;
            const int64_t t = e * n3 + loc;
            const int g = in ? (int)((X - 1) + (gx - 2) * ((Y - 1) + (gy - 2) * (Z - 1))) : -1;
            gi[t] = g;
            if (g >= 0 && rep[g] < 0) rep[g] = (int)t;
        }
    }
    // element matrices on the device (FP64, from the vertices), assembled here
    double *dA = nullptr;
    const size_t abytes = (size_t)op.E * n3 * n3 * sizeof(double);
    CW_CUDA_TRY(cudaMalloc(&dA, abytes));
    std::vector<double> Ae;
    try {
        Ae.resize((size_t)op.E * n3 * n3);
    } catch (const std::bad_alloc &) {
        cudaFree(dA);
        return fail(CW_ERR_OOM, "cw_mg_create: host allocation failed");
    }
    cudaError_t e = element_matrices_launch(op, dA, 0);
    if (e == cudaSuccess) e = cudaMemcpy(Ae.data(), dA, abytes, cudaMemcpyDeviceToHost);
    cudaFree(dA);
    if (e != cudaSuccess) return cuda_fail(e, "cw_mg_create: coarse element matrices");
    std::vector<double> A;
    try {  // the dense interior block and the inverse's work arrays (up to 134 MB each)
        A.assign((size_t)ni * ni, 0.0);
        for (int64_t c = 0; c < op.E; ++c)
            for (int i = 0; i < n3; ++i) {
                const int gi_ = gi[c * n3 + i];
                if (gi_ < 0) continue;
                for (int j = 0; j < n3; ++j) {
                    const int gj = gi[c * n3 + j];
                    if (gj >= 0) A[(size_t)gi_ * ni + gj] += Ae[((size_t)c * n3 + i) * n3 + j];
                }
            }
        if (!spd_inverse(A, (int)ni))
            return fail(CW_ERR_ARG, "cw_mg_create: the coarse matrix is not positive definite");
    } catch (const std::bad_alloc &) {
        return fail(CW_ERR_OOM, "cw_mg_create: host allocation failed (coarse matrix)");
    }
    CW_CUDA_TRY(cudaMalloc(&h.ainv, A.size() * sizeof(double)));
    CW_CUDA_TRY(cudaMalloc(&h.xg, ni * sizeof(double)));
    CW_CUDA_TRY(cudaMalloc(&h.yg, ni * sizeof(double)));
    CW_CUDA_TRY(cudaMalloc(&h.rep, ni * sizeof(int)));
    CW_CUDA_TRY(cudaMalloc(&h.gi, op.L * sizeof(int)));
    CW_CUDA_TRY(cudaMalloc(&h.w0, op.L * h.es));
    CW_CUDA_TRY(cudaMemcpy(h.ainv, A.data(), A.size() * sizeof(double), cudaMemcpyHostToDevice));
    CW_CUDA_TRY(cudaMemcpy(h.rep, rep.data(), ni * sizeof(int), cudaMemcpyHostToDevice));
    CW_CUDA_TRY(cudaMemcpy(h.gi, gi.data(), op.L * sizeof(int), cudaMemcpyHostToDevice));
    h.bytes += (int64_t)(A.size() + 2 * ni) * 8 + ni * 4 + op.L * 4 + op.L * (int64_t)h.es;
    return CW_OK;
}

static std::atomic<uint64_t> g_mg_ids{1};

}  // namespace cw

using namespace cw;

extern "C" {

cw_status cw_mg_create(const cw_op *levels, int nlevels, int nu1, int nu2, double omega, cw_mg *out)
{
    cw::Range nvtx_range("cwfem:cw_mg_create");
    if (!out) return fail(CW_ERR_ARG, "cw_mg_create: out is NULL");
    *out = nullptr;
    if (!levels || nlevels < 1 || nlevels > 16) return fail(CW_ERR_ARG, "cw_mg_create: need 1..16 levels");
    if (nu1 < 0 || nu2 < 0 || nu1 > 64 || nu2 > 64) return fail(CW_ERR_ARG, "cw_mg_create: nu1, nu2 in 0..64");
    if (!(omega > 0.0) || !(omega < 2.0)) return fail(CW_ERR_ARG, "cw_mg_create: omega must be in (0, 2)");
    const Op *o0 = reinterpret_cast<const Op *>(levels[0]);
    if (!o0) return fail(CW_ERR_ARG, "cw_mg_create: NULL level operator");
    for (int l = 0; l < nlevels; ++l) {
        const Op *o = reinterpret_cast<const Op *>(levels[l]);
        if (!o) return fail(CW_ERR_ARG, "cw_mg_create: NULL level operator");
        if (o->p != o0->p || o->kind != o0->kind || o->prec != o0->prec)
            return fail(CW_ERR_ARG, "cw_mg_create: levels differ in degree, kind or precision");
        if (o->prec != CW_PREC_F64 && o->prec != CW_PREC_F64_NATIVE && o->prec != CW_PREC_F32)
            return fail(CW_ERR_ARG, "cw_mg_create: precision must be CW_PREC_F64, CW_PREC_F64_NATIVE or CW_PREC_F32");
        if (o->bc != CW_BC_DIRICHLET0) return fail(CW_ERR_ARG, "cw_mg_create: levels must use CW_BC_DIRICHLET0");
        if (l > 0) {
            const Mesh &c = *reinterpret_cast<const Op *>(levels[l - 1])->mesh, &f = *o->mesh;
            if (f.nx != 2 * c.nx || f.ny != 2 * c.ny || f.nz != 2 * c.nz)
                return fail(CW_ERR_ARG, "cw_mg_create: level l+1 must have twice the cells of level l per direction");
            // nested meshes: the coarse vertices are the even-indexed fine vertices
            bool nested = true;
            for (int64_t vz = 0; vz <= c.nz && nested; ++vz)
                for (int64_t vy = 0; vy <= c.ny && nested; ++vy)
                    for (int64_t vx = 0; vx <= c.nx && nested; ++vx) {
                        const double *a = &c.h_verts[((vz * (c.ny + 1) + vy) * (c.nx + 1) + vx) * 3];
                        const double *b =
                            &f.h_verts[((2 * vz * (f.ny + 1) + 2 * vy) * (f.nx + 1) + 2 * vx) * 3];
                        nested = a[0] == b[0] && a[1] == b[1] && a[2] == b[2];
                    }
            if (!nested) return fail(CW_ERR_ARG, "cw_mg_create: level meshes are not nested (vertex mismatch)");
        }
    }
    MgHier *h = new (std::nothrow) MgHier;
    if (!h) return fail(CW_ERR_OOM, "cw_mg_create: host allocation failed");
    h->nu1 = nu1;
    h->nu2 = nu2;
    h->omega = omega;
    h->prec = o0->prec;
    h->es = vec_elem_size(o0->prec);
    h->id = g_mg_ids.fetch_add(1);
    h->lv.resize(nlevels);
    auto bail = [&](cw_status st) {
        free_hier(h);
        return st;
    };
    double *d = nullptr;
    for (int l = 0; l < nlevels; ++l) {
        MgLevel &L = h->lv[l];
        L.op = reinterpret_cast<Op *>(levels[l]);
        const int64_t Ll = L.op->L;
        cudaError_t e = cudaMalloc(&L.dhat, Ll * h->es);
        if (e == cudaSuccess) e = cudaMalloc(&L.v, Ll * h->es);
        if (e == cudaSuccess && l < nlevels - 1) e = cudaMalloc(&L.b, Ll * h->es);
        if (e == cudaSuccess && l < nlevels - 1) e = cudaMalloc(&L.u, Ll * h->es);
        if (e == cudaSuccess) e = cudaMalloc(&d, Ll * sizeof(double));
        if (e != cudaSuccess) {
            cudaFree(d);
            return bail(cuda_fail(e, "cw_mg_create"));
        }
        h->bytes += Ll * (int64_t)h->es * (2 + 2 * (l < nlevels - 1));
        cw_status st = cw_diagonal(levels[l], d, nullptr);
        if (st != CW_OK) {
            cudaFree(d);
            return bail(st);
        }
        const Mesh &m = *L.op->mesh;
        if (h->es == 8)
            k_make_dhat<double><<<vgrid(Ll), 256>>>(d, static_cast<double *>(L.dhat), m.nx, m.ny, m.nz, L.op->p, Ll,
                                                    omega);
        else
            k_make_dhat<float><<<vgrid(Ll), 256>>>(d, static_cast<float *>(L.dhat), m.nx, m.ny, m.nz, L.op->p, Ll,
                                                   omega);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        cudaFree(d);
        d = nullptr;
        if (e != cudaSuccess) return bail(cuda_fail(e, "cw_mg_create: inverse diagonal"));
    }
    cw_status st = coarse_setup(*h);
    if (st != CW_OK) return bail(st);
    *out = reinterpret_cast<cw_mg>(h);
    return CW_OK;
}

cw_status cw_mg_destroy(cw_mg mh)
{
    MgHier *h = reinterpret_cast<MgHier *>(mh);
    if (!h) return fail(CW_ERR_ARG, "cw_mg_destroy: NULL");
    cudaDeviceSynchronize();  // a cycle in flight may still read the hierarchy's buffers
    free_hier(h);
    return CW_OK;
}

int64_t cw_mg_device_bytes(cw_mg mh)
{
    MgHier *h = reinterpret_cast<MgHier *>(mh);
    return h ? h->bytes : -1;
}

cw_status cw_mg_vcycle(cw_mg mh, const void *b, void *u, int zero_guess, void *stream)
{
    cw::Range nvtx_range("cwfem:cw_mg_vcycle");
    MgHier *h = reinterpret_cast<MgHier *>(mh);
    if (!h || !b || !u) return fail(CW_ERR_ARG, "cw_mg_vcycle: NULL argument");
    if (b == u) return fail(CW_ERR_ARG, "cw_mg_vcycle: b and u must not alias");
    CW_CUDA_TRY(vcycle(*h, (int)h->lv.size() - 1, b, u, zero_guess != 0, static_cast<cudaStream_t>(stream)));
    return CW_OK;
}

cw_status cw_mg_prolong(cw_mg mh, int level, const void *uc, void *uf, void *stream)
{
    MgHier *h = reinterpret_cast<MgHier *>(mh);
    if (!h || !uc || !uf) return fail(CW_ERR_ARG, "cw_mg_prolong: NULL argument");
    if (level < 1 || level >= (int)h->lv.size()) return fail(CW_ERR_ARG, "cw_mg_prolong: level must be in 1..nlevels-1");
    CW_CUDA_TRY(prolong(*h, level, uc, uf, false, static_cast<cudaStream_t>(stream)));
    return CW_OK;
}

cw_status cw_mg_restrict(cw_mg mh, int level, const void *rf, void *rc, void *stream)
{
    MgHier *h = reinterpret_cast<MgHier *>(mh);
    if (!h || !rf || !rc) return fail(CW_ERR_ARG, "cw_mg_restrict: NULL argument");
    if (level < 1 || level >= (int)h->lv.size())
        return fail(CW_ERR_ARG, "cw_mg_restrict: level must be in 1..nlevels-1");
    CW_CUDA_TRY(restrict_(*h, level, rf, nullptr, rc, static_cast<cudaStream_t>(stream)));
    return CW_OK;
}

cw_status cw_mg_smooth(cw_mg mh, int level, const void *b, void *u, int sweeps, void *stream)
{
    MgHier *h = reinterpret_cast<MgHier *>(mh);
    if (!h || !b || !u) return fail(CW_ERR_ARG, "cw_mg_smooth: NULL argument");
    if (level < 0 || level >= (int)h->lv.size()) return fail(CW_ERR_ARG, "cw_mg_smooth: bad level");
    if (sweeps < 0) return fail(CW_ERR_ARG, "cw_mg_smooth: sweeps must be >= 0");
    if (b == u) return fail(CW_ERR_ARG, "cw_mg_smooth: b and u must not alias");
    CW_CUDA_TRY(smooth(*h, level, b, u, sweeps, false, static_cast<cudaStream_t>(stream)));
    return CW_OK;
}

cw_status cw_mg_coarse_solve(cw_mg mh, const void *b, void *u, void *stream)
{
    MgHier *h = reinterpret_cast<MgHier *>(mh);
    if (!h || !b || !u) return fail(CW_ERR_ARG, "cw_mg_coarse_solve: NULL argument");
    if (b == u) return fail(CW_ERR_ARG, "cw_mg_coarse_solve: b and u must not alias");
    CW_CUDA_TRY(coarse_solve(*h, b, u, static_cast<cudaStream_t>(stream)));
    return CW_OK;
}

}  // extern "C"
