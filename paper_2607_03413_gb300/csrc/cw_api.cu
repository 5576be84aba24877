// cw_api.cu -- C ABI of the cell-wise FEM library: meshes, operators, gather, DSS, diagonal,
// load vector. The sum-factorised apply kernels live in cw_apply.cuh and are instantiated in
// the cw_inst_*.cu units; the solver is in cw_cg.cu.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "cw_apply.cuh"
#include "cw_index.cuh"
#include "cw_internal.h"
#include "cw_launch.cuh"

namespace cw {

// ------------------------------------------------------------------------------- errors ----
static thread_local std::string g_last_error;
void set_error(const std::string &msg) { g_last_error = msg; }
cw_status fail(cw_status st, const std::string &msg)
{
    set_error(msg);
    return st;
}
cw_status cuda_fail(cudaError_t e, const char *where)
{
    set_error(std::string(where) + ": " + cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();  // not sticky: clear it, or the next launch check would report it again
        return CW_ERR_OOM;
    }
    return CW_ERR_CUDA;
}

static std::atomic<uint64_t> g_op_generation{0};
uint64_t op_generation() { return g_op_generation.load(); }
void op_generation_bump() { g_op_generation.fetch_add(1); }

size_t vec_elem_size(int prec)
{
    switch (prec) {
    case CW_PREC_F64:
    case CW_PREC_F64_NATIVE: return 8;
    case CW_PREC_F32:
    case CW_PREC_F32_BF16G: return 4;
    case CW_PREC_BF16: return 2;
    }
    return 0;
}
static size_t metric_elem_size(int prec)
{
    switch (prec) {
    case CW_PREC_F64:
    case CW_PREC_F64_NATIVE: return 8;
    case CW_PREC_F32: return 4;
    case CW_PREC_F32_BF16G:
    case CW_PREC_BF16: return 2;
    }
    return 0;
}
bool metric_is_f64(int prec) { return prec == CW_PREC_F64 || prec == CW_PREC_F64_NATIVE; }

// --------------------------------------------------------------------- device helpers ----
struct Rule1D {
    double xq[kMaxN], wq[kMaxN];
    double B[kMaxN][kMaxN], Bd[kMaxN][kMaxN];
};

static Rule1D make_rule(const Tables1D &t)
{
    Rule1D r;
    std::memset(&r, 0, sizeof r);
    for (int q = 0; q < t.n; ++q) {
        r.xq[q] = t.xq[q];
        r.wq[q] = t.wq[q];
        for (int m = 0; m < t.n; ++m) {
            r.B[q][m] = t.B[q][m];
            r.Bd[q][m] = t.Bd[q][m];
        }
    }
    return r;
}

// trilinear map of cell e at reference point xi: Jacobian J[r][s] = d x_r / d xi_s and the point
__device__ void cell_jacobian(const double *__restrict__ V, int nx, int ny, int64_t e, double xi0, double xi1,
                              double xi2, double J[3][3], double X[3])
{
    const int64_t cx = e % nx, cy = (e / nx) % ny, cz = e / ((int64_t)nx * ny);
    for (int a = 0; a < 3; ++a) {
        X[a] = 0.0;
        J[a][0] = J[a][1] = J[a][2] = 0.0;
    }
    const double xi[3] = {xi0, xi1, xi2};
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        const int b0 = v & 1, b1 = (v >> 1) & 1, b2 = (v >> 2) & 1;
        const int64_t vid = ((cz + b2) * (ny + 1) + (cy + b1)) * (int64_t)(nx + 1) + (cx + b0);
        const double f0 = b0 ? xi[0] : 1.0 - xi[0], f1 = b1 ? xi[1] : 1.0 - xi[1], f2 = b2 ? xi[2] : 1.0 - xi[2];
        const double d0 = b0 ? 1.0 : -1.0, d1 = b1 ? 1.0 : -1.0, d2 = b2 ? 1.0 : -1.0;
        const double N0 = f0 * f1 * f2, g0 = d0 * f1 * f2, g1 = f0 * d1 * f2, g2 = f0 * f1 * d2;
        for (int a = 0; a < 3; ++a) {
            const double c = V[vid * 3 + a];
            X[a] += c * N0;
            J[a][0] += c * g0;
            J[a][1] += c * g1;
            J[a][2] += c * g2;
        }
    }
}

// metric of one quadrature point: (xx, yy, zz, xy, xz, yz) of w detJ J^-1 J^-T and w detJ
__device__ void qp_metric(const double J[3][3], double w, double out[7], double *det_out)
{
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    // inverse: Ji[s][r] with J^-1 = adj(J)/det, adj(J)[s][r] = cofactor(r, s)
    double Ji[3][3];
    Ji[0][0] = c00 / det;
    Ji[1][0] = c01 / det;
    Ji[2][0] = c02 / det;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    const double s = w * det;
    // G = s * Ji Ji^T (Ji = J^-1, rows indexed by reference direction)
    auto g = [&](int a, int b) { return s * (Ji[a][0] * Ji[b][0] + Ji[a][1] * Ji[b][1] + Ji[a][2] * Ji[b][2]); };
    out[0] = g(0, 0);
    out[1] = g(1, 1);
    out[2] = g(2, 2);
    out[3] = g(0, 1);
    out[4] = g(0, 2);
    out[5] = g(1, 2);
    out[6] = s;
    *det_out = det;
}

template <class GS>
__device__ __forceinline__ void store_g(GS *p, double v);
template <>
__device__ __forceinline__ void store_g<double>(double *p, double v) { *p = v; }
template <>
__device__ __forceinline__ void store_g<float>(float *p, double v) { *p = static_cast<float>(v); }
template <>
__device__ __forceinline__ void store_g<__nv_bfloat16>(__nv_bfloat16 *p, double v) { *p = __double2bfloat16(v); }
// FP64 metric: rounded float pair hi + lo (hi = fl32(v), lo = fl32(v - hi); ~48 significant bits)
template <>
__device__ __forceinline__ void store_g<df64s>(df64s *p, double v)
{
    const float hi = __double2float_rn(v);
    *p = df64s{hi, __double2float_rn(v - static_cast<double>(hi))};
}

// one thread per (cell, quadrature point); comps selected by kind
template <class GS>
__global__ void metric_kernel(const double *__restrict__ V, int nx, int ny, int64_t E, int n, int kind, Rule1D rule,
                              GS *__restrict__ geo, int *__restrict__ bad)
{
    const int n3 = n * n * n, nc = metric_ncomp(kind);
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= E * n3) return;
    const int64_t e = t / n3;
    const int q = (int)(t - e * n3), a = q % n, b = (q / n) % n, c = q / (n * n);
    double J[3][3], X[3], m[7], det;
    cell_jacobian(V, nx, ny, e, rule.xq[a], rule.xq[b], rule.xq[c], J, X);
    qp_metric(J, rule.wq[a] * rule.wq[b] * rule.wq[c], m, &det);
    if (!(det > 0.0)) atomicOr(bad, 1);
    GS *g = geo + e * (int64_t)nc * n3 + q;
    if (kind & 1)
        for (int k = 0; k < 6; ++k) store_g(g + k * n3, m[k]);
    if (kind & 2) store_g(g + (nc - 1) * n3, m[6]);
}

// det J > 0 at every quadrature point (recomputed geometry stores no per-point data)
__global__ void detj_check_kernel(const double *__restrict__ V, int nx, int ny, int64_t E, int n, Rule1D rule,
                                  int *__restrict__ bad)
{
    const int n3 = n * n * n;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= E * n3) return;
    const int64_t e = t / n3;
    const int q = (int)(t - e * n3), a = q % n, b = (q / n) % n, c = q / (n * n);
    double J[3][3], X[3], m[7], det;
    cell_jacobian(V, nx, ny, e, rule.xq[a], rule.xq[b], rule.xq[c], J, X);
    qp_metric(J, 1.0, m, &det);
    if (!(det > 0.0)) atomicOr(bad, 1);
}

// coefficients a1..a7 of the trilinear map of each cell from its 8 vertices X_{ijk} (i, j, k the
// x, y, z bits): a1 = X100 - X000, a2 = X010 - X000, a3 = X001 - X000, a4 = X110 - X100 - X010 + X000,
// a5 = X101 - X100 - X001 + X000, a6 = X011 - X010 - X001 + X000,
// a7 = X111 - X110 - X101 - X011 + X100 + X010 + X001 - X000; formed in FP64, stored rounded
template <class GS>
__global__ void trilinear_coef_kernel(const double *__restrict__ V, int nx, int ny, int64_t E, GS *__restrict__ coef)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const int64_t cx = e % nx, cy = (e / nx) % ny, cz = e / ((int64_t)nx * ny);
    GS *o = coef + e * kTriCoef;
    for (int d = 0; d < 3; ++d) {
        double X[2][2][2];
        for (int v = 0; v < 8; ++v) {
            const int b0 = v & 1, b1 = (v >> 1) & 1, b2 = (v >> 2) & 1;
            const int64_t vid = ((cz + b2) * (ny + 1) + (cy + b1)) * (int64_t)(nx + 1) + (cx + b0);
            X[b0][b1][b2] = V[vid * 3 + d];
        }
        const double a[7] = {
            X[1][0][0] - X[0][0][0],
            X[0][1][0] - X[0][0][0],
            X[0][0][1] - X[0][0][0],
            X[1][1][0] - X[1][0][0] - X[0][1][0] + X[0][0][0],
            X[1][0][1] - X[1][0][0] - X[0][0][1] + X[0][0][0],
            X[0][1][1] - X[0][1][0] - X[0][0][1] + X[0][0][0],
            X[1][1][1] - X[1][1][0] - X[1][0][1] - X[0][1][1] + X[1][0][0] + X[0][1][0] + X[0][0][1] - X[0][0][0]};
        for (int i = 0; i < 7; ++i) store_g(o + 3 * i + d, a[i]);
    }
}

// Cartesian per-cell scalars (a_x, a_y, a_z, a_m), masked by the operator kind
__global__ void affine_kernel(const double *__restrict__ V, int nx, int ny, int64_t E, int kind, double *__restrict__ geo)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const int64_t cx = e % nx, cy = (e / nx) % ny, cz = e / ((int64_t)nx * ny);
    const int64_t v0 = (cz * (ny + 1) + cy) * (int64_t)(nx + 1) + cx;
    const double hx = V[(v0 + 1) * 3 + 0] - V[v0 * 3 + 0];
    const double hy = V[(v0 + (nx + 1)) * 3 + 1] - V[v0 * 3 + 1];
    const double hz = V[(v0 + (int64_t)(nx + 1) * (ny + 1)) * 3 + 2] - V[v0 * 3 + 2];
    const bool k = kind & 1, m = kind & 2;
    geo[e * 4 + 0] = k ? hy * hz / hx : 0.0;
    geo[e * 4 + 1] = k ? hx * hz / hy : 0.0;
    geo[e * 4 + 2] = k ? hx * hy / hz : 0.0;
    geo[e * 4 + 3] = m ? hx * hy * hz : 0.0;
}

template <class VS>
__device__ __forceinline__ void store_v(VS *p, double v);
template <>
__device__ __forceinline__ void store_v<double>(double *p, double v) { *p = v; }
template <>
__device__ __forceinline__ void store_v<float>(float *p, double v) { *p = static_cast<float>(v); }
template <>
__device__ __forceinline__ void store_v<__nv_bfloat16>(__nv_bfloat16 *p, double v) { *p = __double2bfloat16(v); }

template <class VS>
__global__ void gather_kernel(const double *__restrict__ ug, VS *__restrict__ x, int nx, int ny, int p, int64_t L)
{
    const int n = p + 1, n3 = n * n * n;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L) return;
    const int64_t e = t / n3;
    const int loc = (int)(t - e * n3), i = loc % n, j = (loc / n) % n, k = loc / (n * n);
    const int64_t cx = e % nx, cy = (e / nx) % ny, cz = e / ((int64_t)nx * ny);
    const int64_t gx = (int64_t)nx * p + 1, gy = (int64_t)ny * p + 1;
    store_v(x + t, ug[(cx * p + i) + gx * ((cy * p + j) + gy * (cz * p + k))]);
}

// ------------------------------------------------------------------------------- DSS ----
// v * s with s a power of two (exact): valence scaling and the halving of the averaging passes
template <class VS>
struct MulOp {
    static __device__ __forceinline__ VS mul(VS a, double s) { return static_cast<VS>(a * s); }
};
template <>
struct MulOp<float> {
    static __device__ __forceinline__ float mul(float a, double s) { return a * static_cast<float>(s); }
};
template <>
struct MulOp<__nv_bfloat16> {
    static __device__ __forceinline__ __nv_bfloat16 mul(__nv_bfloat16 a, double s)
    {
        return __float2bfloat16_rn(__bfloat162float(a) * static_cast<float>(s));
    }
};

// One pass of Algorithm struct_dss along axis `ax`: for every interior interface normal to ax
// between cells K_L and K_R = K_L + stride, s = v[K_L, face = p] + v[K_R, face = 0] is written to
// both copies. One thread per (interface, face node); no atomics; exchange partners at static
// offsets.

// grid: x covers (face node, first in-face cell coordinate, interface coordinate along ax),
// y the remaining cell coordinate. All index arithmetic is 32-bit.
// HALF: the averaging variant (S_bar): both copies receive (left + right) / 2, so that after the three
// passes every copy holds the sum over the DoF's kappa copies divided by kappa (halving is exact; the
// result equals the summing passes followed by the division by the valence, bit for bit).
template <class VS, bool HALF = false>
__global__ void dss_axis_kernel(VS *__restrict__ v, int nx, int ny, int nz, int p, int ax, uint32_t nx_thr,
                                FastDiv fd_n2, FastDiv fd_e0)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nx_thr) return;
    const int n = p + 1, n2 = n * n, n3 = n2 * n;
    // x index: f + n2 * (c_a + e0 * c_ax) with (c_a, c_ax) the in-face coordinate and the
    // interface coordinate, e0 the extent of c_a
    const uint32_t q = fd_n2.div(t);
    const uint32_t f = t - q * static_cast<uint32_t>(n2);
    const uint32_t c_ax = fd_e0.div(q);
    const uint32_t c_a = q - c_ax * fd_e0.d;
    const uint32_t c_b = blockIdx.y;
    const uint32_t fa = f % n, fb = f / n;  // n <= 8: cheap
    uint32_t cx, cy, cz;
    if (ax == 0) {
        cx = c_ax;
        cy = c_a;
        cz = c_b;
    } else if (ax == 1) {
        cx = c_a;
        cy = c_ax;
        cz = c_b;
    } else {
        cx = c_a;
        cy = c_b;
        cz = c_ax;
    }
    const int64_t KL = cx + (int64_t)nx * (cy + (int64_t)ny * cz);
    const int64_t stride = (ax == 0) ? 1 : (ax == 1 ? nx : (int64_t)nx * ny);
    const int64_t KR = KL + stride;
    int il, ir;
    if (ax == 0) {
        il = p + n * fa + n2 * fb;
        ir = n * fa + n2 * fb;
    } else if (ax == 1) {
        il = fa + n * p + n2 * fb;
        ir = fa + n2 * fb;
    } else {
        il = fa + n * fb + n2 * p;
        ir = fa + n * fb;
    }
    VS *pl = v + KL * n3 + il, *pr = v + KR * n3 + ir;
    VS s = AddOp<VS>::add(*pl, *pr);
    if constexpr (HALF) s = MulOp<VS>::mul(s, 0.5);
    *pl = s;
    *pr = s;
    (void)nz;
}

// The x pass of Algorithm struct_dss restricted to the interfaces between tiles of `xtile`
// consecutive cells (K_L = (b+1) xtile - 1 with K_L + 1 < E and K_L not the last cell of its x-row);
// the interfaces inside tiles were summed by the operator kernel. One thread per (interface, face node).
template <class VS, bool HALF = false>
__global__ void dss_xtile_kernel(VS *__restrict__ v, int nx, int p, int xtile, int64_t E, uint32_t nthr,
                                 FastDiv fd_n2)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nthr) return;
    const int n = p + 1, n2 = n * n, n3 = n2 * n;
    const uint32_t b = fd_n2.div(t);
    const uint32_t f = t - b * static_cast<uint32_t>(n2);
    const int64_t KL = (int64_t)(b + 1) * xtile - 1;
    if (KL + 1 >= E || KL % nx == nx - 1) return;
    const uint32_t fa = f % n, fb = f / n;
    VS *pl = v + KL * n3 + p + n * fa + n2 * fb, *pr = v + (KL + 1) * n3 + n * fa + n2 * fb;
    VS sum = AddOp<VS>::add(*pl, *pr);
    if constexpr (HALF) sum = MulOp<VS>::mul(sum, 0.5);
    *pl = sum;
    *pr = sum;
}


// dst = src with the x pass of Algorithm struct_dss applied: an entry on an interior x-face adds its
// partner copy in the neighbouring cell, every other entry is copied (out of place, so the read of
// a partner never sees an updated value). Replaces a copy and an in-place x pass with one pass.
template <class VS, bool HALF = false>
__global__ void dss_x_from_kernel(const VS *__restrict__ src, VS *__restrict__ dst, int nx, int p, uint32_t nlines,
                                  FastDiv fd_n2, FastDiv fd_nx)
{
    // one thread per x-line (n consecutive entries of a cell); only its two end entries have partners
    const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nlines) return;
    const int n = p + 1;
    const uint32_t n3 = fd_n2.d * n;
    const uint32_t c = fd_n2.div(l);
    const uint32_t cx = c - fd_nx.div(c) * static_cast<uint32_t>(nx);
    const int64_t b = static_cast<int64_t>(l) * n;
    VS v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
        if (i < n) v[i] = src[b + i];
    if (cx > 0) {
        v[0] = AddOp<VS>::add(src[b - n3 + p], v[0]);
        if constexpr (HALF) v[0] = MulOp<VS>::mul(v[0], 0.5);
    }
    if (cx + 1 < static_cast<uint32_t>(nx)) {
        v[p] = AddOp<VS>::add(v[p], src[b + n3]);
        if constexpr (HALF) v[p] = MulOp<VS>::mul(v[p], 0.5);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
        if (i < n) dst[b + i] = v[i];
}

// r - a q with one rounding, written once so that every use (own line, partner copy) gives the same value
template <class VS>
__device__ __forceinline__ VS resid_update(VS r, VS q, VS a) { return fma(-a, q, r); }
template <>
__device__ __forceinline__ float resid_update<float>(float r, float q, float a) { return fmaf(-a, q, r); }

// dst = x pass of (r - a q), a = *active ? *alpha : 0: the CG residual update r <- r - alpha A p fused
// into the first pass of the DSS that follows it (the updated residual itself is only needed as S r).
template <class VS>
__global__ void dss_x_axpy_kernel(const VS *__restrict__ r, const VS *__restrict__ q,
                                  const double *__restrict__ alpha, const int *__restrict__ active,
                                  VS *__restrict__ dst, int nx, int p, uint32_t nlines, FastDiv fd_n2, FastDiv fd_nx)
{
    const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nlines) return;
    const VS a = *active ? static_cast<VS>(*alpha) : VS(0);
    const int n = p + 1;
    const uint32_t n3 = fd_n2.d * n;
    const uint32_t c = fd_n2.div(l);
    const uint32_t cx = c - fd_nx.div(c) * static_cast<uint32_t>(nx);
    const int64_t b = static_cast<int64_t>(l) * n;
    VS v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
        if (i < n) v[i] = resid_update(r[b + i], q[b + i], a);
    if (cx > 0) v[0] = AddOp<VS>::add(resid_update(r[b - n3 + p], q[b - n3 + p], a), v[0]);
    if (cx + 1 < static_cast<uint32_t>(nx)) v[p] = AddOp<VS>::add(v[p], resid_update(r[b + n3], q[b + n3], a));
#pragma unroll
    for (int i = 0; i < 8; ++i)
        if (i < n) dst[b + i] = v[i];
}

// r <- r - a q (a as above), the unfused form for vectors beyond 32-bit line indexing
template <class VS>
__global__ void resid_update_kernel(VS *__restrict__ r, const VS *__restrict__ q, const double *__restrict__ alpha,
                                    const int *__restrict__ active, int64_t L)
{
    const VS a = *active ? static_cast<VS>(*alpha) : VS(0);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = resid_update(r[i], q[i], a);
}

template <class VS>
static cudaError_t dss_typed(const Op &op, VS *v, int flags, cudaStream_t s, int first_axis = 0, int end_axis = 3,
                             int xtile = 0);

// dst = S src (or S_bar src), src unchanged; src and dst must not overlap
template <class VS>
static cudaError_t dss_from_typed(const Op &op, const VS *src, VS *dst, int flags, cudaStream_t s)
{
    const Mesh &m = *op.mesh;
    if (op.L >= (int64_t)1 << 31) {  // 32-bit index path not applicable: copy, then all passes
        cudaError_t e = cudaMemcpyAsync(dst, src, op.L * sizeof(VS), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
        return dss_typed(op, dst, flags, s, 0);
    }
    const uint32_t nlines = (uint32_t)(op.L / op.n);
    if (flags == CW_DSS_AVERAGE)
        dss_x_from_kernel<VS, true><<<(nlines + 255) / 256, 256, 0, s>>>(src, dst, m.nx, op.p, nlines,
                                                                         FastDiv::make(op.n * op.n), FastDiv::make(m.nx));
    else
        dss_x_from_kernel<VS, false><<<(nlines + 255) / 256, 256, 0, s>>>(src, dst, m.nx, op.p, nlines,
                                                                          FastDiv::make(op.n * op.n), FastDiv::make(m.nx));
    return dss_typed(op, dst, flags, s, 1);
}

template <class VS>
static cudaError_t dss_from_axpy_typed(const Op &op, VS *r, const VS *q, const double *alpha, const int *active,
                                       VS *dst, bool x_only, cudaStream_t s)
{
    if (op.L >= (int64_t)1 << 31) {
        if (x_only) return cudaErrorInvalidValue;
        resid_update_kernel<VS><<<1216, 256, 0, s>>>(r, q, alpha, active, op.L);
        return dss_from_typed(op, static_cast<const VS *>(r), dst, CW_DSS_SUM, s);
    }
    const uint32_t nlines = (uint32_t)(op.L / op.n);
    dss_x_axpy_kernel<VS><<<(nlines + 255) / 256, 256, 0, s>>>(r, q, alpha, active, dst, op.mesh->nx, op.p, nlines,
                                                                 FastDiv::make(op.n * op.n), FastDiv::make(op.mesh->nx));
    if (x_only) return cudaGetLastError();
    return dss_typed(op, dst, CW_DSS_SUM, s, 1);
}

cudaError_t dss_from_axpy(const Op &op, void *r, const void *q, const double *alpha, const int *active, void *dst,
                          cudaStream_t s, bool x_only)
{
    switch (vec_elem_size(op.prec)) {
    case 8:
        return dss_from_axpy_typed(op, static_cast<double *>(r), static_cast<const double *>(q), alpha, active,
                                   static_cast<double *>(dst), x_only, s);
    case 4:
        return dss_from_axpy_typed(op, static_cast<float *>(r), static_cast<const float *>(q), alpha, active,
                                   static_cast<float *>(dst), x_only, s);
    default: return cudaErrorInvalidValue;  // the solver keeps FP32 or FP64 vectors
    }
}

cudaError_t dss_from(const Op &op, const void *src, void *dst, int flags, cudaStream_t s)
{
    switch (vec_elem_size(op.prec)) {
    case 8: return dss_from_typed(op, static_cast<const double *>(src), static_cast<double *>(dst), flags, s);
    case 4: return dss_from_typed(op, static_cast<const float *>(src), static_cast<float *>(dst), flags, s);
    default:
        return dss_from_typed(op, static_cast<const __nv_bfloat16 *>(src), static_cast<__nv_bfloat16 *>(dst), flags, s);
    }
}

cudaError_t dss_from_f64(const Op &op, const double *src, double *dst, int flags, cudaStream_t s)
{
    return dss_from_typed(op, src, dst, flags, s);
}

template <class VS>
static cudaError_t dss_typed(const Op &op, VS *v, int flags, cudaStream_t s, int first_axis, int end_axis, int xtile)
{
    const Mesh &m = *op.mesh;
    const int dims[3] = {m.nx, m.ny, m.nz};
    const int n2 = op.n * op.n;
    for (int ax = first_axis; ax < end_axis; ++ax) {
        if (dims[ax] < 2) continue;
        // in-face coordinates: a = lower of the two other axes (x-index part), b = the other (grid y)
        const int a = (ax == 0) ? 1 : 0, b = (ax == 2) ? 1 : 2;
        const uint32_t e0 = dims[a];
        const uint32_t nthr = (uint32_t)n2 * e0 * (uint32_t)(dims[ax] - 1);
        const int bs = 256;
        dim3 grid((nthr + bs - 1) / bs, dims[b]);
        const bool half = flags == CW_DSS_AVERAGE;  // averaging passes: (left + right) / 2 to both copies
        if (ax == 0 && xtile > 1) {  // only the x-interfaces between tiles are left
            const int64_t nb = (op.E / xtile) * n2;  // interface K_L = (b+1) xtile - 1, b < E/xtile
            if (nb >= ((int64_t)1 << 32)) return cudaErrorInvalidValue;  // callers fuse only below this
            if (nb > 0) {
                const unsigned g = (unsigned)((nb + bs - 1) / bs);
                if (half)
                    dss_xtile_kernel<VS, true><<<g, bs, 0, s>>>(v, m.nx, op.p, xtile, op.E, (uint32_t)nb, FastDiv::make(n2));
                else
                    dss_xtile_kernel<VS, false><<<g, bs, 0, s>>>(v, m.nx, op.p, xtile, op.E, (uint32_t)nb, FastDiv::make(n2));
            }
            continue;
        }
        if (half)
            dss_axis_kernel<VS, true><<<grid, bs, 0, s>>>(v, m.nx, m.ny, m.nz, op.p, ax, nthr, FastDiv::make(n2),
                                                          FastDiv::make(e0));
        else
            dss_axis_kernel<VS, false><<<grid, bs, 0, s>>>(v, m.nx, m.ny, m.nz, op.p, ax, nthr, FastDiv::make(n2),
                                                           FastDiv::make(e0));
    }
    return cudaGetLastError();
}

cudaError_t dss_average_launch(const Op &op, void *v, cudaStream_t s, int xtile)
{
    switch (vec_elem_size(op.prec)) {
    case 8: return dss_typed(op, static_cast<double *>(v), CW_DSS_AVERAGE, s, 0, 3, xtile);
    case 4: return dss_typed(op, static_cast<float *>(v), CW_DSS_AVERAGE, s, 0, 3, xtile);
    default: return dss_typed(op, static_cast<__nv_bfloat16 *>(v), CW_DSS_AVERAGE, s, 0, 3, xtile);
    }
}

cudaError_t dss_launch(const Op &op, void *v, int flags, cudaStream_t s, int xtile)
{
    switch (vec_elem_size(op.prec)) {
    case 8: return dss_typed(op, static_cast<double *>(v), flags, s, 0, 3, xtile);
    case 4: return dss_typed(op, static_cast<float *>(v), flags, s, 0, 3, xtile);
    default: return dss_typed(op, static_cast<__nv_bfloat16 *>(v), flags, s, 0, 3, xtile);
    }
}

// sum passes of the axes [ax0, ax1) only (no averaging); used on slab views of the mesh
static cudaError_t dss_axes(const Op &op, void *v, int ax0, int ax1, cudaStream_t s, int xtile = 0)
{
    switch (vec_elem_size(op.prec)) {
    case 8: return dss_typed(op, static_cast<double *>(v), CW_DSS_SUM, s, ax0, ax1, xtile);
    case 4: return dss_typed(op, static_cast<float *>(v), CW_DSS_SUM, s, ax0, ax1, xtile);
    default: return dss_typed(op, static_cast<__nv_bfloat16 *>(v), CW_DSS_SUM, s, ax0, ax1, xtile);
    }
}

cudaError_t apply_local(const Op &op, const void *x, void *y, cudaStream_t s, int *xfuse)
{
    switch (op.prec) {
    case CW_PREC_F64: return apply_launch_df(op, x, y, s, xfuse);
    case CW_PREC_F64_NATIVE: return apply_launch_f64n(op, x, y, s, xfuse);
    default: return apply_launch_f32(op, x, y, s, xfuse);
    }
}

// ----------------------------------------------------------- diagonal and load vector ----
// One CTA per cell (at least n^3 threads): the metric of all quadrature points is computed from the
// vertices in FP64 into shared memory, then
//   diag_i = sum_q (grad phi_i)^T G_q (grad phi_i) + c_q phi_i^2
// with grad phi_i(q) = (Bd[a][i1] B[b][i2] B[c][i3], B Bd B, B B Bd) (q = (a, b, c)). Every term is
// separable: G_de(q) grad_d phi_i grad_e phi_i = G_de(q) prod_k W_k[q_k][i_k] with the 1D factor
// W_k = X_dk X_ek (X_dk = Bd if k = d, else B; B B for the mass term), so each of the seven metric
// components is contracted with its three 1D factors in turn (sum factorisation: 3 n^4 instead of
// n^6 products per component and cell); off-diagonal components count twice.
__device__ __forceinline__ double diag_factor(const Rule1D &rule, int k, int d, int e, int q, int i)
{
    const double xd = (k == d) ? rule.Bd[q][i] : rule.B[q][i];
    const double xe = (k == e) ? rule.Bd[q][i] : rule.B[q][i];
    return xd * xe;
}
__global__ void diag_kernel(const double *__restrict__ V, int nx, int ny, int n, int kind, Rule1D rule,
                            double *__restrict__ d)
{
    extern __shared__ double sm[];  // [7][n^3] metric, then two [n^3] work buffers
    const int n2 = n * n, n3 = n2 * n;
    const int64_t e = blockIdx.x;
    for (int q = threadIdx.x; q < n3; q += blockDim.x) {
        const int a = q % n, b = (q / n) % n, c = q / (n * n);
        double J[3][3], X[3], m[7], det;
        cell_jacobian(V, nx, ny, e, rule.xq[a], rule.xq[b], rule.xq[c], J, X);
        qp_metric(J, rule.wq[a] * rule.wq[b] * rule.wq[c], m, &det);
        for (int k = 0; k < 7; ++k) sm[k * n3 + q] = m[k];
    }
    double *w0 = sm + 7 * n3, *w1 = w0 + n3;
    const int t = threadIdx.x;  // the launch gives at least n^3 threads: one entry i = t each
    const int t1 = t % n, t2 = (t / n) % n, t3 = t / n2;
    double acc = 0.0;
    for (int comp = 0; comp < 7; ++comp) {
        if (comp < 6 ? !(kind & 1) : !(kind & 2)) continue;  // kind-uniform
        // components (xx, yy, zz, xy, xz, yz, mass): derivative directions (dd, de); -1: none
        const int dd = comp < 3 ? comp : (comp < 5 ? 0 : (comp == 5 ? 1 : -1));
        const int de = comp < 3 ? comp : (comp == 3 ? 1 : (comp < 6 ? 2 : -1));
        __syncthreads();  // the metric is in place; the previous component's buffers are read
        if (t < n3) {  // along x: (q1, q2, q3) -> (i1, q2, q3)
            double s = 0.0;
            for (int q = 0; q < n; ++q) s += diag_factor(rule, 0, dd, de, q, t1) * sm[comp * n3 + q + n * (t2 + n * t3)];
            w0[t] = s;
        }
        __syncthreads();
        if (t < n3) {  // along y: (i1, q2, q3) -> (i1, i2, q3)
            double s = 0.0;
            for (int q = 0; q < n; ++q) s += diag_factor(rule, 1, dd, de, q, t2) * w0[t1 + n * (q + n * t3)];
            w1[t] = s;
        }
        __syncthreads();
        if (t < n3) {  // along z: (i1, i2, q3) -> (i1, i2, i3)
            double s = 0.0;
            for (int q = 0; q < n; ++q) s += diag_factor(rule, 2, dd, de, q, t3) * w1[t1 + n * (t2 + n * q)];
            acc += (comp >= 3 && comp < 6) ? 2.0 * s : s;
        }
    }
    if (t < n3) d[e * n3 + t] = acc;
}

// Element matrices of the cells, A[e][i][j] = sum_q (grad phi_i)^T G_q (grad phi_j) + c_q phi_i phi_j
// (FP64, metric from the vertices as in the diagonal): grid (E, ceil(n^6 / blockDim)), one thread per
// (i, j). Used to assemble the small coarsest level of a multigrid hierarchy.
__global__ void elem_matrix_kernel(const double *__restrict__ V, int nx, int ny, int n, int kind, Rule1D rule,
                                   double *__restrict__ A)
{
    extern __shared__ double sm[];  // [7][n^3]
    const int n3 = n * n * n;
    const int64_t e = blockIdx.x;
    for (int q = threadIdx.x; q < n3; q += blockDim.x) {
        const int a = q % n, b = (q / n) % n, c = q / (n * n);
        double J[3][3], X[3], m[7], det;
        cell_jacobian(V, nx, ny, e, rule.xq[a], rule.xq[b], rule.xq[c], J, X);
        qp_metric(J, rule.wq[a] * rule.wq[b] * rule.wq[c], m, &det);
        for (int k = 0; k < 7; ++k) sm[k * n3 + q] = m[k];
    }
    __syncthreads();
    const int64_t pair = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    if (pair >= (int64_t)n3 * n3) return;
    const int i = (int)(pair / n3), j = (int)(pair - (int64_t)i * n3);
    const int i1 = i % n, i2 = (i / n) % n, i3 = i / (n * n);
    const int j1 = j % n, j2 = (j / n) % n, j3 = j / (n * n);
    double s = 0.0;
    for (int q = 0; q < n3; ++q) {
        const int a = q % n, b = (q / n) % n, c = q / (n * n);
        const double Bi1 = rule.B[a][i1], Bi2 = rule.B[b][i2], Bi3 = rule.B[c][i3];
        const double Bj1 = rule.B[a][j1], Bj2 = rule.B[b][j2], Bj3 = rule.B[c][j3];
        if (kind & 1) {
            const double gi[3] = {rule.Bd[a][i1] * Bi2 * Bi3, Bi1 * rule.Bd[b][i2] * Bi3, Bi1 * Bi2 * rule.Bd[c][i3]};
            const double gj[3] = {rule.Bd[a][j1] * Bj2 * Bj3, Bj1 * rule.Bd[b][j2] * Bj3, Bj1 * Bj2 * rule.Bd[c][j3]};
            const double G[3][3] = {{sm[0 * n3 + q], sm[3 * n3 + q], sm[4 * n3 + q]},
                                    {sm[3 * n3 + q], sm[1 * n3 + q], sm[5 * n3 + q]},
                                    {sm[4 * n3 + q], sm[5 * n3 + q], sm[2 * n3 + q]}};
            for (int r = 0; r < 3; ++r)
                for (int t = 0; t < 3; ++t) s += gi[r] * G[r][t] * gj[t];
        }
        if (kind & 2) s += sm[6 * n3 + q] * (Bi1 * Bi2 * Bi3) * (Bj1 * Bj2 * Bj3);
    }
    A[e * (int64_t)n3 * n3 + pair] = s;
}

cudaError_t element_matrices_launch(const Op &op, double *A, cudaStream_t s)
{
    const int n3 = op.n * op.n * op.n;
    const Rule1D rule = make_rule(op.tab);
    const int bs = 256;
    dim3 grid((unsigned)op.E, (unsigned)(((int64_t)n3 * n3 + bs - 1) / bs));
    elem_matrix_kernel<<<grid, bs, 7 * n3 * sizeof(double), s>>>(op.mesh->d_verts, op.mesh->nx, op.mesh->ny, op.n,
                                                                  op.kind, rule, A);
    return cudaGetLastError();
}

__device__ __forceinline__ void exact_rhs(int which, const double X[3], double *f)
{
    if (which == 0) {
        const double pi = 3.141592653589793238462643383279502884;
        *f = 3.0 * pi * pi * sin(pi * X[0]) * sin(pi * X[1]) * sin(pi * X[2]);
    } else {
        const double bx = X[0] * (1 - X[0]), by = X[1] * (1 - X[1]), bz = X[2] * (1 - X[2]);
        *f = 2.0 * (by * bz + bx * bz + bx * by);
    }
}

__global__ void load_kernel(const double *__restrict__ V, int nx, int ny, int n, int which, Rule1D rule,
                            double *__restrict__ b)
{
    extern __shared__ double sm[];  // [n^3] : w detJ f at the quadrature points
    const int n3 = n * n * n;
    const int64_t e = blockIdx.x;
    for (int q = threadIdx.x; q < n3; q += blockDim.x) {
        const int a = q % n, bb = (q / n) % n, c = q / (n * n);
        double J[3][3], X[3], m[7], det, f;
        cell_jacobian(V, nx, ny, e, rule.xq[a], rule.xq[bb], rule.xq[c], J, X);
        qp_metric(J, rule.wq[a] * rule.wq[bb] * rule.wq[c], m, &det);
        exact_rhs(which, X, &f);
        sm[q] = m[6] * f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n3; i += blockDim.x) {
        const int i1 = i % n, i2 = (i / n) % n, i3 = i / (n * n);
        double s = 0.0;
        for (int q = 0; q < n3; ++q) {
            const int a = q % n, bb = (q / n) % n, c = q / (n * n);
            s += sm[q] * rule.B[a][i1] * rule.B[bb][i2] * rule.B[c][i3];
        }
        b[e * n3 + i] = s;
    }
}

}  // namespace cw

using namespace cw;

// =================================================================================== C ABI ====
extern "C" {

const char *cw_status_string(cw_status s)
{
    switch (s) {
    case CW_OK: return "CW_OK";
    case CW_ERR_ARG: return "CW_ERR_ARG";
    case CW_ERR_OOM: return "CW_ERR_OOM";
    case CW_ERR_CUDA: return "CW_ERR_CUDA";
    case CW_ERR_NOT_CONVERGED: return "CW_ERR_NOT_CONVERGED";
    case CW_ERR_BREAKDOWN: return "CW_ERR_BREAKDOWN";
    case CW_ERR_TIMEOUT: return "CW_ERR_TIMEOUT";
    case CW_ERR_UNSUPPORTED: return "CW_ERR_UNSUPPORTED";
    }
    return "CW_ERR_UNKNOWN";
}

const char *cw_last_error(void) { return g_last_error.c_str(); }

cw_status cw_mesh_create(int nx, int ny, int nz, const double *verts_host, cw_mesh *out)
{
    if (!out) return fail(CW_ERR_ARG, "cw_mesh_create: out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || !verts_host) return fail(CW_ERR_ARG, "cw_mesh_create: bad sizes or NULL vertices");
    if (nx > kMaxCellsPerDir || ny > kMaxCellsPerDir || nz > kMaxCellsPerDir)
        return fail(CW_ERR_ARG, "cw_mesh_create: more than 65535 cells in one direction");
    const int64_t nv = ((int64_t)nx + 1) * ((int64_t)ny + 1) * ((int64_t)nz + 1);
    if ((int64_t)nx * ny * nz > (int64_t)1 << 31) return fail(CW_ERR_ARG, "cw_mesh_create: more than 2^31 cells");
    Mesh *m = new (std::nothrow) Mesh;
    if (!m) return fail(CW_ERR_OOM, "cw_mesh_create: host allocation failed");
    m->nx = nx;
    m->ny = ny;
    m->nz = nz;
    try {
        m->h_verts.assign(verts_host, verts_host + nv * 3);
    } catch (const std::bad_alloc &) {
        delete m;
        return fail(CW_ERR_OOM, "cw_mesh_create: host allocation failed");
    }
    // Cartesian test: x depends on vx only, y on vy only, z on vz only
    bool cart = true;
    for (int64_t vz = 0; vz <= nz && cart; ++vz)
        for (int64_t vy = 0; vy <= ny && cart; ++vy)
            for (int64_t vx = 0; vx <= nx && cart; ++vx) {
                const double *c = &m->h_verts[((vz * (ny + 1) + vy) * (nx + 1) + vx) * 3];
                cart = c[0] == m->h_verts[vx * 3 + 0] && c[1] == m->h_verts[(vy * (nx + 1)) * 3 + 1] &&
                       c[2] == m->h_verts[(vz * (ny + 1) * (nx + 1)) * 3 + 2];
            }
    m->cartesian = cart;
    cudaError_t e = cudaMalloc(&m->d_verts, nv * 3 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(m->d_verts, verts_host, nv * 3 * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(m->d_verts);
        delete m;
        return cuda_fail(e, "cw_mesh_create");
    }
    *out = reinterpret_cast<cw_mesh>(m);
    return CW_OK;
}

cw_status cw_mesh_create_box(int nx, int ny, int nz, double perturb, const int *freq, const double *direction,
                             cw_mesh *out)
{
    if (!out) return fail(CW_ERR_ARG, "cw_mesh_create_box: out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return fail(CW_ERR_ARG, "cw_mesh_create_box: sizes must be >= 1");
    if (nx > kMaxCellsPerDir || ny > kMaxCellsPerDir || nz > kMaxCellsPerDir)
        return fail(CW_ERR_ARG, "cw_mesh_create_box: more than 65535 cells in one direction");
    if ((int64_t)nx * ny * nz > (int64_t)1 << 31) return fail(CW_ERR_ARG, "cw_mesh_create_box: more than 2^31 cells");
    if (!std::isfinite(perturb)) return fail(CW_ERR_ARG, "cw_mesh_create_box: non-finite perturbation");
    const int f[3] = {freq ? freq[0] : 1, freq ? freq[1] : 1, freq ? freq[2] : 1};
    double d[3] = {1.0, 1.0, 1.0};
    if (direction) d[0] = direction[0], d[1] = direction[1], d[2] = direction[2];
    const double dn = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (!(dn > 0.0) || !std::isfinite(dn)) return fail(CW_ERR_ARG, "cw_mesh_create_box: zero or non-finite direction");
    for (double &c : d) c /= dn;
    const double h = 1.0 / std::max(nx, std::max(ny, nz));
    const double pi = 3.14159265358979323846;
    std::vector<double> v;
    try {
        v.resize((size_t)(nx + 1) * (ny + 1) * (nz + 1) * 3);
    } catch (const std::bad_alloc &) {
        return fail(CW_ERR_OOM, "cw_mesh_create_box: host allocation failed");
    }
    for (int vz = 0; vz <= nz; ++vz)
        for (int vy = 0; vy <= ny; ++vy)
            for (int vx = 0; vx <= nx; ++vx) {
                double *c = &v[(((size_t)vz * (ny + 1) + vy) * (nx + 1) + vx) * 3];
                const double X = vx / (double)nx, Y = vy / (double)ny, Z = vz / (double)nz;
                c[0] = X;
                c[1] = Y;
                c[2] = Z;
                if (perturb != 0.0) {
                    const double sv = std::sin(2.0 * pi * f[0] * X) * std::sin(2.0 * pi * f[1] * Y) *
                                      std::sin(2.0 * pi * f[2] * Z);
                    for (int a = 0; a < 3; ++a) c[a] += perturb * h * sv * d[a];
                    // the boundary stays the unit cube exactly
                    if (vx == 0) c[0] = 0.0;
                    if (vx == nx) c[0] = 1.0;
                    if (vy == 0) c[1] = 0.0;
                    if (vy == ny) c[1] = 1.0;
                    if (vz == 0) c[2] = 0.0;
                    if (vz == nz) c[2] = 1.0;
                }
            }
    return cw_mesh_create(nx, ny, nz, v.data(), out);
}

cw_status cw_rules_1d(int degree, double *gll_nodes, double *gauss_points, double *gauss_weights)
{
    if (degree < 1 || degree > kMaxDegree) return fail(CW_ERR_ARG, "cw_rules_1d: degree must be in 1..7");
    Tables1D t;
    build_tables(degree, t);
    for (int i = 0; i < t.n; ++i) {
        if (gll_nodes) gll_nodes[i] = t.gll[i];
        if (gauss_points) gauss_points[i] = t.xq[i];
        if (gauss_weights) gauss_weights[i] = t.wq[i];
    }
    return CW_OK;
}

cw_status cw_basis_1d(int degree, double *B, double *Bd, double *D, double *M1, double *K1)
{
    if (degree < 1 || degree > kMaxDegree) return fail(CW_ERR_ARG, "cw_basis_1d: degree must be in 1..7");
    Tables1D t;
    build_tables(degree, t);
    for (int r = 0; r < t.n; ++r)
        for (int c = 0; c < t.n; ++c) {
            const int o = r * t.n + c;
            if (B) B[o] = t.B[r][c];
            if (Bd) Bd[o] = t.Bd[r][c];
            if (D) D[o] = t.D[r][c];
            if (M1) M1[o] = t.M1[r][c];
            if (K1) K1[o] = t.K1[r][c];
        }
    return CW_OK;
}

cw_status cw_mesh_refine_vertices(int nx, int ny, int nz, const double *verts, double *out)
{
    if (!verts || !out) return fail(CW_ERR_ARG, "cw_mesh_refine_vertices: NULL pointer");
    if (nx < 1 || ny < 1 || nz < 1 || 2 * (int64_t)nx > kMaxCellsPerDir || 2 * (int64_t)ny > kMaxCellsPerDir ||
        2 * (int64_t)nz > kMaxCellsPerDir || 8 * (int64_t)nx * ny * nz > (int64_t)1 << 31)
        return fail(CW_ERR_ARG, "cw_mesh_refine_vertices: sizes outside the mesh limits after refinement");
    // the parent cell's trilinear map at the half points is separable: along each axis in turn keep
    // the vertex rows and insert the midpoint of every pair of neighbours
    int64_t dims[3] = {(int64_t)nx + 1, (int64_t)ny + 1, (int64_t)nz + 1};
    std::vector<double> a, b;
    try {
        a.assign(verts, verts + dims[0] * dims[1] * dims[2] * 3);
    } catch (const std::bad_alloc &) {
        return fail(CW_ERR_OOM, "cw_mesh_refine_vertices: host allocation failed");
    }
    for (int ax = 0; ax < 3; ++ax) {
        int64_t nd[3] = {dims[0], dims[1], dims[2]};
        nd[ax] = 2 * dims[ax] - 1;
        try {
            b.resize((size_t)(nd[0] * nd[1] * nd[2] * 3));
        } catch (const std::bad_alloc &) {
            return fail(CW_ERR_OOM, "cw_mesh_refine_vertices: host allocation failed");
        }
        for (int64_t z = 0; z < nd[2]; ++z)
            for (int64_t y = 0; y < nd[1]; ++y)
                for (int64_t x = 0; x < nd[0]; ++x) {
                    int64_t s[3] = {x, y, z};
                    const int64_t o = s[ax];
                    s[ax] = o / 2;
                    const double *lo = &a[((s[2] * dims[1] + s[1]) * dims[0] + s[0]) * 3];
                    double *d = &b[((z * nd[1] + y) * nd[0] + x) * 3];
                    if (o % 2 == 0) {
                        for (int c = 0; c < 3; ++c) d[c] = lo[c];
                    } else {
                        s[ax] = o / 2 + 1;
                        const double *hi = &a[((s[2] * dims[1] + s[1]) * dims[0] + s[0]) * 3];
                        for (int c = 0; c < 3; ++c) d[c] = 0.5 * (lo[c] + hi[c]);
                    }
                }
        a.swap(b);
        dims[ax] = nd[ax];
    }
    std::memcpy(out, a.data(), a.size() * sizeof(double));
    return CW_OK;
}

cw_status cw_mesh_destroy(cw_mesh mh)
{
    Mesh *m = reinterpret_cast<Mesh *>(mh);
    if (!m) return fail(CW_ERR_ARG, "cw_mesh_destroy: NULL");
    cudaFree(m->d_verts);
    delete m;
    return CW_OK;
}

cw_status cw_op_create(cw_mesh mh, int degree, int kind, int geom, int prec, int bc, cw_op *out)
{
    cw::Range nvtx_range("cwfem:cw_op_create");
    if (!out) return fail(CW_ERR_ARG, "cw_op_create: out is NULL");
    *out = nullptr;
    Mesh *m = reinterpret_cast<Mesh *>(mh);
    if (!m) return fail(CW_ERR_ARG, "cw_op_create: NULL mesh");
    if (degree < 1 || degree > kMaxDegree) return fail(CW_ERR_ARG, "cw_op_create: degree must be in 1..7");
    if (kind < 1 || kind > 3) return fail(CW_ERR_ARG, "cw_op_create: bad kind");
    if (geom != CW_GEOM_AFFINE && geom != CW_GEOM_METRIC && geom != CW_GEOM_RECOMPUTE)
        return fail(CW_ERR_ARG, "cw_op_create: bad geometry mode");
    if (prec < CW_PREC_F64 || prec > CW_PREC_BF16) return fail(CW_ERR_ARG, "cw_op_create: bad precision");
    if (bc != CW_BC_NONE && bc != CW_BC_DIRICHLET0) return fail(CW_ERR_ARG, "cw_op_create: bad bc");
    if (geom == CW_GEOM_AFFINE && !m->cartesian)
        return fail(CW_ERR_ARG, "cw_op_create: CW_GEOM_AFFINE needs a Cartesian (axis-aligned) mesh");
    {  // the DSS axis passes index one plane of face nodes with 32 bits
        const int64_t n2 = (int64_t)(degree + 1) * (degree + 1);
        const int64_t plane[3] = {n2 * m->ny * (m->nx - 1), n2 * m->nx * (m->ny - 1), n2 * m->nx * (m->nz - 1)};
        for (int64_t c : plane)
            if (c >= ((int64_t)1 << 32))
                return fail(CW_ERR_UNSUPPORTED, "cw_op_create: a DSS plane holds 2^32 or more face-node pairs");
    }
    Op *op = new Op;
    op->mesh = m;
    op->p = degree;
    op->n = degree + 1;
    op->kind = kind;
    op->geom = geom;
    op->prec = prec;
    op->bc = bc;
    op->E = m->ncells();
    const int n3 = op->n * op->n * op->n;
    op->L = op->E * n3;
    op->NG = ((int64_t)m->nx * degree + 1) * ((int64_t)m->ny * degree + 1) * ((int64_t)m->nz * degree + 1);
    build_tables(degree, op->tab);
    const Rule1D rule = make_rule(op->tab);
    cudaError_t e;
    int *d_bad = nullptr;
    if (geom == CW_GEOM_METRIC) {
        const int nc = metric_ncomp(kind);
        op->geo_bytes = op->E * nc * n3 * (int64_t)metric_elem_size(prec);
        e = cudaMalloc(&op->d_geo, op->geo_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&d_bad, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(d_bad, 0, sizeof(int));
        if (e == cudaSuccess) {
            const int64_t nthr = op->E * n3;
            const unsigned blocks = (unsigned)((nthr + 255) / 256);
            if (prec == CW_PREC_F64)  // float pairs for the double-float arithmetic
                metric_kernel<df64s><<<blocks, 256>>>(m->d_verts, m->nx, m->ny, op->E, op->n, kind, rule,
                                                      static_cast<df64s *>(op->d_geo), d_bad);
            else if (prec == CW_PREC_F64_NATIVE)  // IEEE doubles
                metric_kernel<double><<<blocks, 256>>>(m->d_verts, m->nx, m->ny, op->E, op->n, kind, rule,
                                                       static_cast<double *>(op->d_geo), d_bad);
            else if (prec == CW_PREC_F32)
                metric_kernel<float><<<blocks, 256>>>(m->d_verts, m->nx, m->ny, op->E, op->n, kind, rule,
                                                      static_cast<float *>(op->d_geo), d_bad);
            else
                metric_kernel<__nv_bfloat16><<<blocks, 256>>>(m->d_verts, m->nx, m->ny, op->E, op->n, kind, rule,
                                                              static_cast<__nv_bfloat16 *>(op->d_geo), d_bad);
            e = cudaGetLastError();
        }
        int bad = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost);
        cudaFree(d_bad);
        if (e == cudaSuccess && bad) {
            cudaFree(op->d_geo);
            delete op;
            return fail(CW_ERR_ARG, "cw_op_create: non-positive Jacobian determinant at a quadrature point");
        }
    } else if (geom == CW_GEOM_RECOMPUTE) {
        const bool f64 = metric_is_f64(prec);
        op->geo_bytes = op->E * kTriCoef * (int64_t)(f64 ? sizeof(double) : sizeof(float));
        e = cudaMalloc(&op->d_geo, op->geo_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&d_bad, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(d_bad, 0, sizeof(int));
        if (e == cudaSuccess) {
            const int64_t nthr = op->E * n3;
            detj_check_kernel<<<(unsigned)((nthr + 255) / 256), 256>>>(m->d_verts, m->nx, m->ny, op->E, op->n, rule,
                                                                        d_bad);
            const unsigned cb = (unsigned)((op->E + 255) / 256);
            if (prec == CW_PREC_F64)
                trilinear_coef_kernel<df64s><<<cb, 256>>>(m->d_verts, m->nx, m->ny, op->E, static_cast<df64s *>(op->d_geo));
            else if (prec == CW_PREC_F64_NATIVE)
                trilinear_coef_kernel<double><<<cb, 256>>>(m->d_verts, m->nx, m->ny, op->E, static_cast<double *>(op->d_geo));
            else
                trilinear_coef_kernel<float><<<cb, 256>>>(m->d_verts, m->nx, m->ny, op->E, static_cast<float *>(op->d_geo));
            e = cudaGetLastError();
        }
        int bad = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost);
        cudaFree(d_bad);
        if (e == cudaSuccess && bad) {
            cudaFree(op->d_geo);
            delete op;
            return fail(CW_ERR_ARG, "cw_op_create: non-positive Jacobian determinant at a quadrature point");
        }
    } else {
        op->geo_bytes = op->E * 4 * (int64_t)sizeof(double);
        e = cudaMalloc(&op->d_geo, op->geo_bytes);
        if (e == cudaSuccess) {
            affine_kernel<<<(unsigned)((op->E + 255) / 256), 256>>>(m->d_verts, m->nx, m->ny, op->E, kind,
                                                                     static_cast<double *>(op->d_geo));
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        cudaFree(op->d_geo);
        delete op;
        return cuda_fail(e, "cw_op_create");
    }
    e = cudaMalloc(&op->d_status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(op->d_status, 0, sizeof(unsigned));
    if (e != cudaSuccess) {
        cudaFree(op->d_status);
        cudaFree(op->d_geo);
        delete op;
        return cuda_fail(e, "cw_op_create");
    }
    op->owned_bytes = op->geo_bytes + (int64_t)sizeof(unsigned);
    *out = reinterpret_cast<cw_op>(op);
    return CW_OK;
}

cw_status cw_op_destroy(cw_op oh)
{
    Op *op = reinterpret_cast<Op *>(oh);
    if (!op) return fail(CW_ERR_ARG, "cw_op_destroy: NULL");
    cg_release(op);
    if (op->inner) cw_op_destroy(reinterpret_cast<cw_op>(op->inner));
    if (op->native) cw_op_destroy(reinterpret_cast<cw_op>(op->native));
    cudaFree(op->h_dx);
    cudaFree(op->h_dy);
    for (int i = 0; i < 3; ++i)
        if (op->h_st[i]) cudaStreamDestroy(op->h_st[i]);
    for (int a = 0; a < 2; ++a)
        for (int k = 0; k < Op::kMaxSlabs; ++k)
            if (op->h_ev[a][k]) cudaEventDestroy(op->h_ev[a][k]);
    if (op->h_done) cudaEventDestroy(op->h_done);
    cudaFree(op->d_geo);
    cudaFree(op->d_dinv);
    cudaFree(op->d_status);
    delete op;
    return CW_OK;
}

int64_t cw_op_cellwise_len(cw_op oh)
{
    Op *op = reinterpret_cast<Op *>(oh);
    return op ? op->L : -1;
}
int64_t cw_op_global_len(cw_op oh)
{
    Op *op = reinterpret_cast<Op *>(oh);
    return op ? op->NG : -1;
}
int64_t cw_op_device_bytes(cw_op oh)
{
    Op *op = reinterpret_cast<Op *>(oh);
    if (!op) return -1;
    return op->owned_bytes + (op->inner ? op->inner->owned_bytes : 0) + (op->native ? op->native->owned_bytes : 0);
}

cw_status cw_gather(cw_op oh, const double *ug, void *x, void *stream)
{
    Op *op = reinterpret_cast<Op *>(oh);
    if (!op || !ug || !x) return fail(CW_ERR_ARG, "cw_gather: NULL argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const unsigned blocks = (unsigned)((op->L + 255) / 256);
    const Mesh &m = *op->mesh;
    switch (vec_elem_size(op->prec)) {
    case 8: gather_kernel<double><<<blocks, 256, 0, s>>>(ug, static_cast<double *>(x), m.nx, m.ny, op->p, op->L); break;
    case 4: gather_kernel<float><<<blocks, 256, 0, s>>>(ug, static_cast<float *>(x), m.nx, m.ny, op->p, op->L); break;
    default:
        gather_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(ug, static_cast<__nv_bfloat16 *>(x), m.nx, m.ny, op->p, op->L);
    }
    CW_CUDA_TRY(cudaGetLastError());
    return CW_OK;
}

cw_status cw_apply(cw_op oh, const void *x, void *y, int flags, void *stream)
{
    cw::Range nvtx_range("cwfem:cw_apply");
    Op *op = reinterpret_cast<Op *>(oh);
    if (!op || !x || !y) return fail(CW_ERR_ARG, "cw_apply: NULL argument");
    if (flags != CW_APPLY_LOCAL && flags != CW_APPLY_ASSEMBLE) return fail(CW_ERR_ARG, "cw_apply: bad flags");
    if (x == y) return fail(CW_ERR_ARG, "cw_apply: x and y must not alias");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (flags == CW_APPLY_LOCAL) {
        CW_CUDA_TRY(apply_local(*op, x, y, s));
        return CW_OK;
    }
    // the operator kernel sums the x-interfaces inside its tiles; the DSS does the rest
    int xtile = 0;
    const bool fuse = op->E * (int64_t)(op->n * op->n) < ((int64_t)1 << 32);
    CW_CUDA_TRY(apply_local(*op, x, y, s, fuse ? &xtile : nullptr));
    CW_CUDA_TRY(dss_launch(*op, y, CW_DSS_SUM, s, xtile));
    return CW_OK;
}

cw_status cw_dss(cw_op oh, void *v, int flags, void *stream)
{
    Op *op = reinterpret_cast<Op *>(oh);
    if (!op || !v) return fail(CW_ERR_ARG, "cw_dss: NULL argument");
    if (flags != CW_DSS_SUM && flags != CW_DSS_AVERAGE) return fail(CW_ERR_ARG, "cw_dss: bad flags");
    CW_CUDA_TRY(dss_launch(*op, v, flags, static_cast<cudaStream_t>(stream)));
    return CW_OK;
}

cw_status cw_diagonal(cw_op oh, double *d, void *stream)
{
    cw::Range nvtx_range("cwfem:cw_diagonal");
    Op *op = reinterpret_cast<Op *>(oh);
    if (!op || !d) return fail(CW_ERR_ARG, "cw_diagonal: NULL argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n3 = op->n * op->n * op->n;
    const Rule1D rule = make_rule(op->tab);
    diag_kernel<<<(unsigned)op->E, n3 < 128 ? 128 : n3, 9 * n3 * sizeof(double), s>>>(
        op->mesh->d_verts, op->mesh->nx, op->mesh->ny, op->n, op->kind, rule, d);
    CW_CUDA_TRY(cudaGetLastError());
    CW_CUDA_TRY(dss_typed(*op, d, CW_DSS_SUM, s));
    return CW_OK;
}

cw_status cw_load_vector(cw_op oh, int which, double *b, void *stream)
{
    Op *op = reinterpret_cast<Op *>(oh);
    if (!op || !b) return fail(CW_ERR_ARG, "cw_load_vector: NULL argument");
    if (which != 0 && which != 1) return fail(CW_ERR_ARG, "cw_load_vector: which must be 0 or 1");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n3 = op->n * op->n * op->n;
    const Rule1D rule = make_rule(op->tab);
    load_kernel<<<(unsigned)op->E, n3 < 128 ? 128 : (n3 > 512 ? 512 : n3), n3 * sizeof(double), s>>>(
        op->mesh->d_verts, op->mesh->nx, op->mesh->ny, op->n, which, rule, b);
    CW_CUDA_TRY(cudaGetLastError());
    return CW_OK;
}

}  // extern "C"

namespace cw {
cw_status op_status_take(Op *op, cudaStream_t s, const char *where)
{
    if (!op || !op->d_status) return CW_OK;
    unsigned w = 0;
    CW_CUDA_TRY(cudaMemcpyAsync(&w, op->d_status, sizeof w, cudaMemcpyDeviceToHost, s));
    CW_CUDA_TRY(cudaStreamSynchronize(s));
    if (w == 0) return CW_OK;
    CW_CUDA_TRY(cudaMemsetAsync(op->d_status, 0, sizeof(unsigned), s));
    CW_CUDA_TRY(cudaStreamSynchronize(s));
    return fail(CW_ERR_TIMEOUT, std::string(where) +
                                    ": a bounded wait for a staged tile expired (the tile was left without output)");
}
}  // namespace cw

extern "C" {

cw_status cw_op_check(cw_op oh, void *stream)
{
    Op *op = reinterpret_cast<Op *>(oh);
    if (!op) return fail(CW_ERR_ARG, "cw_op_check: NULL handle");
    return op_status_take(op, static_cast<cudaStream_t>(stream), "cw_op_check");
}

cw_status cw_op_inject_stall(cw_op oh, int on)
{
    Op *op = reinterpret_cast<Op *>(oh);
    if (!op) return fail(CW_ERR_ARG, "cw_op_inject_stall: NULL handle");
    op->dbg_tma_extra = on ? 16u : 0u;
    op_generation_bump();
    return CW_OK;
}

cw_status cw_op_set_variant(cw_op oh, int cells_per_cta, int stage)
{
    Op *op = reinterpret_cast<Op *>(oh);
    if (!op) return fail(CW_ERR_ARG, "cw_op_set_variant: NULL handle");
    int ch[2];
    cpb_choices(op->p, op->prec, ch);
    if (cells_per_cta != 0 && cells_per_cta != ch[0] && cells_per_cta != ch[1])
        return fail(CW_ERR_ARG, "cw_op_set_variant: cells_per_cta must be 0 or one of cw_op_get_variant's choices");
    if (stage < 0 || stage > 2) return fail(CW_ERR_ARG, "cw_op_set_variant: stage must be 0, 1 or 2");
    if (op->prec == CW_PREC_F64_NATIVE && (cells_per_cta != 0 || stage != 0))
        return fail(CW_ERR_UNSUPPORTED, "cw_op_set_variant: CW_PREC_F64_NATIVE has only the default variant");
    if (op->geom == CW_GEOM_RECOMPUTE && cells_per_cta != 0 && cells_per_cta != ch[0])
        return fail(CW_ERR_UNSUPPORTED, "cw_op_set_variant: CW_GEOM_RECOMPUTE uses the default cells per CTA");
    op->cpb = cells_per_cta == ch[0] ? 0 : cells_per_cta;
    op->stage = stage;
    op_generation_bump();
    return CW_OK;
}

cw_status cw_op_get_variant(cw_op oh, int *cells_per_cta, int *stage, int *choices2)
{
    Op *op = reinterpret_cast<Op *>(oh);
    if (!op) return fail(CW_ERR_ARG, "cw_op_get_variant: NULL handle");
    int ch[2];
    cpb_choices(op->p, op->prec, ch);
    if (cells_per_cta) *cells_per_cta = op->cpb == 0 ? ch[0] : op->cpb;
    if (stage) *stage = op->stage;
    if (choices2) {
        choices2[0] = ch[0];
        choices2[1] = ch[1];
    }
    return CW_OK;
}

cw_status cw_op_autotune(cw_op oh, const void *x, void *y, int reps, void *stream, float *best_ms)
{
    cw::Range nvtx_range("cwfem:cw_op_autotune");
    Op *op = reinterpret_cast<Op *>(oh);
    if (!op || !x || !y || x == y) return fail(CW_ERR_ARG, "cw_op_autotune: NULL or aliasing argument");
    if (reps < 1) return fail(CW_ERR_ARG, "cw_op_autotune: reps must be >= 1");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (op->prec == CW_PREC_F64_NATIVE) {
        op->cpb = 0;
        op->stage = 0;
        if (best_ms) *best_ms = -1.0f;
        return CW_OK;
    }
    int ch[2];
    cpb_choices(op->p, op->prec, ch);
    cudaEvent_t e0, e1;
    CW_CUDA_TRY(cudaEventCreate(&e0));
    if (const cudaError_t ee = cudaEventCreate(&e1); ee != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ee, "cw_op_autotune");
    }
    float best = 1e30f;
    int bc = 0, bs = op->stage;
    // curved: both tile sizes x three staging modes; recomputed geometry: default tile, direct or
    // TMA-staged input; Cartesian: both tile sizes
    const int nstage = op->geom == CW_GEOM_METRIC ? 3 : (op->geom == CW_GEOM_RECOMPUTE ? 2 : 1);
    const int ncpb = op->geom == CW_GEOM_RECOMPUTE ? 1 : 2;
    for (int ci = 0; ci < ncpb; ++ci)
        for (int st = 0; st < nstage; ++st) {
            op->cpb = ci == 0 ? 0 : ch[1];
            op->stage = st;
            if (apply_local(*op, x, y, s) != cudaSuccess) {  // variant not launchable (smem)
                cudaGetLastError();
                continue;
            }
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps; ++r) apply_local(*op, x, y, s);
            cudaEventRecord(e1, s);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return cuda_fail(e, "cw_op_autotune");
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= reps;
            if (ms < best) {
                best = ms;
                bc = op->cpb;
                bs = st;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    op->cpb = bc;
    op->stage = bs;
    op_generation_bump();
    if (best_ms) *best_ms = best;
    return op_status_take(op, s, "cw_op_autotune");
}

}  // extern "C"

extern "C" {

// Apply with host input and output. The cells are split into slabs of whole z-layers: the
// host-to-device copy of slab k overlaps the work of slab k-1. The nominal slab has P = nz / 16
// layers (rounded up); the first and the last slabs ramp through 1, 2, 4, ... < P layers, so that the
// pipeline starts on a small copy and ends on a small apply and copy (with equal slabs the link ran
// one direction only for about one slab time at each end). For CW_APPLY_LOCAL slab k is copied
// back as soon as its apply is done. For CW_APPLY_ASSEMBLE each slab runs its apply, its x and y DSS
// passes and the z pass of its interior interfaces, then the z pass of the interface with slab k-1;
// the DSS cascade couples slabs only through that interface, so slab k-1 is then final and its
// copy back overlaps the work on slab k.
cw_status cw_apply_host(cw_op oh, const void *x_host, void *y_host, int flags, void *stream)
{
    cw::Range nvtx_range("cwfem:cw_apply_host");
    Op *op = reinterpret_cast<Op *>(oh);
    if (!op || !x_host || !y_host) return fail(CW_ERR_ARG, "cw_apply_host: NULL argument");
    if (flags != CW_APPLY_LOCAL && flags != CW_APPLY_ASSEMBLE) return fail(CW_ERR_ARG, "cw_apply_host: bad flags");
    if (x_host == y_host) return fail(CW_ERR_ARG, "cw_apply_host: x and y must not alias");
    const size_t es = vec_elem_size(op->prec);
    const int64_t n3 = (int64_t)op->n * op->n * op->n;
    if (!op->h_dx) {
        CW_CUDA_TRY(cudaMalloc(&op->h_dx, op->L * es));
        CW_CUDA_TRY(cudaMalloc(&op->h_dy, op->L * es));
        for (int i = 0; i < 3; ++i) CW_CUDA_TRY(cudaStreamCreateWithFlags(&op->h_st[i], cudaStreamNonBlocking));
        for (int a = 0; a < 2; ++a)
            for (int k = 0; k < Op::kMaxSlabs; ++k)
                CW_CUDA_TRY(cudaEventCreateWithFlags(&op->h_ev[a][k], cudaEventDisableTiming));
        CW_CUDA_TRY(cudaEventCreateWithFlags(&op->h_done, cudaEventDisableTiming));
        op->owned_bytes += 2 * op->L * (int64_t)es;
    }
    cudaStream_t us = static_cast<cudaStream_t>(stream);
    cudaStream_t sin = op->h_st[0], scomp = op->h_st[1], sout = op->h_st[2];
    CW_CUDA_TRY(cudaEventRecord(op->h_done, us));  // order after the caller's stream
    for (int i = 0; i < 3; ++i) CW_CUDA_TRY(cudaStreamWaitEvent(op->h_st[i], op->h_done, 0));
    const Mesh &m = *op->mesh;
    const int64_t plane = (int64_t)m.nx * m.ny;  // cells per z-layer
    // slab plan: first z-layer of every slab, and an end marker
    std::vector<int> zs;
    {
        const int P = std::max(1, (m.nz + Op::kNominalSlabs - 1) / Op::kNominalSlabs);
        std::vector<int> ramp;
        int rs = 0;
        for (int r = 1; r < P; r *= 2) ramp.push_back(r), rs += r;
        if (2 * rs + P > m.nz) ramp.clear(), rs = 0;  // too few layers to ramp
        int z = 0;
        for (int r : ramp) zs.push_back(z), z += r;
        const int zend = m.nz - rs;
        for (; z < zend; z += P) zs.push_back(z);
        z = zend;
        for (auto it = ramp.rbegin(); it != ramp.rend(); ++it) zs.push_back(z), z += *it;
        if ((int)zs.size() > Op::kMaxSlabs) {  // cannot happen for kMaxSlabs >= 16 + 2 log2(P); keep it safe
            zs.clear();
            for (z = 0; z < m.nz; z += P) zs.push_back(z);
        }
        zs.push_back(m.nz);
    }
    const int nslab = (int)zs.size() - 1;
    const size_t gbytes_per_cell = op->geo_bytes / op->E;
    unsigned char *dx = static_cast<unsigned char *>(op->h_dx), *dy = static_cast<unsigned char *>(op->h_dy);
    const unsigned char *hx = static_cast<const unsigned char *>(x_host);
    unsigned char *hy = static_cast<unsigned char *>(y_host);
    // a view of the operator on z-layers [z0, z0 + nzv)
    std::vector<Mesh> views(nslab + 1);
    // slab views share the operator's device data; the host copy of the vertices is not carried
    // (copying it per slab made the host, not the GPU, the bottleneck of this entry point)
    auto shallow = [&](int nzv) {
        Mesh v;
        v.nx = m.nx;
        v.ny = m.ny;
        v.nz = nzv;
        v.d_verts = m.d_verts;
        v.cartesian = m.cartesian;
        return v;
    };
    auto view = [&](int vi, int z0, int nzv, Op &o) {
        views[vi] = shallow(nzv);
        o = *op;
        o.mesh = &views[vi];
        o.E = plane * nzv;
        o.L = o.E * n3;
        o.d_geo = static_cast<unsigned char *>(op->d_geo) + z0 * plane * gbytes_per_cell;
    };
    auto slab_bytes = [&](int k, size_t &off, size_t &bytes) {
        const int64_t z0 = zs[k], nz = zs[k + 1] - zs[k];
        off = (size_t)(z0 * plane * n3) * es;
        bytes = (size_t)(nz * plane * n3) * es;
    };
    Mesh bview = shallow(2);  // two-layer view across a slab interface
    for (int k = 0; k < nslab; ++k) {
        size_t off, bytes;
        slab_bytes(k, off, bytes);
        const int z0 = zs[k], nzk = zs[k + 1] - zs[k];
        CW_CUDA_TRY(cudaMemcpyAsync(dx + off, hx + off, bytes, cudaMemcpyHostToDevice, sin));
        CW_CUDA_TRY(cudaEventRecord(op->h_ev[0][k], sin));
        CW_CUDA_TRY(cudaStreamWaitEvent(scomp, op->h_ev[0][k], 0));
        Op part;
        view(k, z0, nzk, part);
        int xtile = 0;  // x-interfaces inside the operator's tiles are summed by its kernel
        const bool fuse = flags == CW_APPLY_ASSEMBLE && part.E * (int64_t)(n3 / op->n) < ((int64_t)1 << 32);
        CW_CUDA_TRY(apply_local(part, dx + off, dy + off, scomp, fuse ? &xtile : nullptr));
        if (flags == CW_APPLY_ASSEMBLE) {
            CW_CUDA_TRY(dss_axes(part, dy + off, 0, 3, scomp, xtile));  // x, y and interior z interfaces
            if (k > 0) {
                Op bop = *op;
                bop.mesh = &bview;
                bop.E = plane * 2;
                bop.L = bop.E * n3;
                const size_t boff = (size_t)((int64_t)(z0 - 1) * plane * n3) * es;
                CW_CUDA_TRY(dss_axes(bop, dy + boff, 2, 3, scomp));  // the interface with slab k-1
            }
        }
        CW_CUDA_TRY(cudaEventRecord(op->h_ev[1][k], scomp));
        const int ready = (flags == CW_APPLY_ASSEMBLE) ? k - 1 : k;  // slab that is final now
        if (ready >= 0) {
            size_t roff, rbytes;
            slab_bytes(ready, roff, rbytes);
            CW_CUDA_TRY(cudaStreamWaitEvent(sout, op->h_ev[1][k], 0));
            CW_CUDA_TRY(cudaMemcpyAsync(hy + roff, dy + roff, rbytes, cudaMemcpyDeviceToHost, sout));
        }
    }
    if (flags == CW_APPLY_ASSEMBLE) {  // the last slab
        size_t roff, rbytes;
        slab_bytes(nslab - 1, roff, rbytes);
        CW_CUDA_TRY(cudaStreamWaitEvent(sout, op->h_ev[1][nslab - 1], 0));
        CW_CUDA_TRY(cudaMemcpyAsync(hy + roff, dy + roff, rbytes, cudaMemcpyDeviceToHost, sout));
    }
    CW_CUDA_TRY(cudaEventRecord(op->h_done, sout));
    CW_CUDA_TRY(cudaStreamWaitEvent(us, op->h_done, 0));
    return CW_OK;
}

}  // extern "C"
