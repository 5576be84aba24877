// cw_cg.cu -- Jacobi-preconditioned conjugate gradients on cell-wise data, and FP64 iterative
// refinement around a reduced-precision inner CG.
//
// Primal-dual CG (Sec. 4.4; Sec. 2.1, Eq. (pairing_global)): iterate u and search direction p are
// continuous primal vectors, the residual r = b - A u is an unassembled dual vector. Every inner
// product pairs one dual with one primal vector, so it needs no assembly. The preconditioner is
// z = D_cell^-1 S r (Sec. 4.1, Eq. (jacobi_recap)) with the Dirichlet rows zeroed in the stored
// inverse diagonal (Sec. 5, "Constraints baked into the diagonal"), which also keeps u and p zero
// on the boundary. With a consistent preconditioner the iterates equal those of Jacobi-PCG on the
// assembled interior system, iteration by iteration.
//
// Convergence: ||m G^T r|| / ||m G^T b|| <= rtol, evaluated cell-wise as <m S r, r> (m = interior
// mask), since <S r, r> = ||G^T r||^2.
//
// Device-side control: every scalar (rho, <p,q>, alpha, beta, residual) lives in device memory;
// one small kernel per reduction turns block partials into the scalars and raises a `done` flag
// on convergence, breakdown or maxit, after which the update kernels leave u untouched. The host
// replays a CUDA graph of `kBatch` iterations and reads the flag once per replay.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <type_traits>

#include "cw_arith.cuh"
#include "cw_index.cuh"
#include "cw_internal.h"

namespace cw {

constexpr int kRedBlocks = 1216;  // 152 SMs x 8
constexpr int kRedThreads = 256;
constexpr int kBatch = 16;

// device scalar slots
enum : int { S_RHO = 0, S_PQ, S_ALPHA, S_BETA, S_RES0, S_RES, S_RHO_NEW, S_TOL2, S_ENERGY, S_NSCAL = 16 };
// device flag slots
// F_ACTIVE: the current iteration started before convergence (set at its <p,Ap> stage); its
// direction update p = z + beta p runs even if the iteration converges, so that a later segment
// can continue from a consistent (r, p) pair
// F_BLOCKS: arrival counter of the fused reductions (last block finalises, then resets it)
enum : int { F_DONE = 0, F_ITER, F_STATUS, F_MAXIT, F_ACTIVE, F_BLOCKS = 7, F_NFLAG = 8 };
enum : int { ST_RUNNING = 0, ST_CONVERGED = 1, ST_BREAKDOWN = 2, ST_MAXIT = 3 };

struct CgLevel {  // vectors of one precision level
    void *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr, *dinv = nullptr;
    cudaGraphExec_t graph = nullptr;  // kBatch iterations; kernel arguments baked in
    const void *graph_u = nullptr;    // iterate pointer the graph was captured with
    const Op *graph_op = nullptr;     // operator the graph was captured with
    int graph_ak = -1;                // operator evaluation the graph was captured with
    uint64_t graph_gen = 0;           // operator generation (kernel choices) at capture
};

struct CgScratch {
    CgLevel lv64, lv32;      // FP64 inner level / FP32 inner level
    double *rout = nullptr;  // outer FP64 residual b - A u
    double *q64b = nullptr;  // FP64 apply output / work in outer steps
    double *d64 = nullptr;   // FP64 inner correction
    float *d32 = nullptr;    // FP32 inner correction
    double *partials = nullptr;
    double *dotpart = nullptr;  // one <p, Ap> partial per apply CTA (at most one per cell)
    double *scal = nullptr;
    int *flags = nullptr;
    uint8_t *kappa = nullptr;  // valence of every cell-wise entry (1, 2, 4 or 8)
    double *h_scal = nullptr;
    int *h_flags = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int64_t bytes = 0;
    // multigrid-preconditioned CG: FP32 copies of the cycle's input and output (FP32 hierarchy) and
    // the graph of one iteration, keyed by the hierarchy, the correction vector and the operator
    float *r32 = nullptr, *z32 = nullptr;
    cudaGraphExec_t mg_graph = nullptr;
    uint64_t mg_graph_id = 0;
    const void *mg_graph_d = nullptr;
    const Op *mg_graph_op = nullptr;
    uint64_t mg_graph_gen = 0;
};

// ---------------------------------------------------------------------------- kernels ----
template <class V>
__device__ __forceinline__ df64 as_df(V v);
template <>
__device__ __forceinline__ df64 as_df<double>(double v) { return split_f64(v); }
template <>
__device__ __forceinline__ df64 as_df<float>(float v) { return df64{v, 0.0f}; }

// block-level sum of a double into partial slot (blockIdx.x) of `out`
__device__ __forceinline__ void block_sum_store(double v, double *out)
{
    __shared__ double sh[kRedThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < kRedThreads / 32 ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) out[blockIdx.x] = v;
    }
    __syncthreads();
}

// 16-byte chunks of a vector (float4 / double2 loads and stores); every vector here is the start
// of a cudaMalloc allocation, so chunk k at element k*W is 16-byte aligned; the last n % W
// elements are handled one by one
template <class V>
struct __align__(16) Chunk {
    static constexpr int W = 16 / sizeof(V);
    V v[W];
};
template <class V>
__device__ __forceinline__ Chunk<V> ldc(const V *p, int64_t k)
{
    return reinterpret_cast<const Chunk<V> *>(p)[k];
}
template <class V>
__device__ __forceinline__ void stc(V *p, int64_t k, const Chunk<V> &c)
{
    reinterpret_cast<Chunk<V> *>(p)[k] = c;
}

#define CW_GRID_LOOP(i, n)                                                                          \
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// partial <a, b> with double-float accumulation (products exact in the FP32-pair format)
template <class V>
__global__ void __launch_bounds__(kRedThreads) k_dot(const V *__restrict__ a, const V *__restrict__ b, int64_t n,
                                                     double *__restrict__ part)
{
    constexpr int W = Chunk<V>::W;
    df64 acc{0.0f, 0.0f};
    CW_GRID_LOOP(k, n / W)
    {
        const Chunk<V> ca = ldc(a, k), cb = ldc(b, k);
#pragma unroll
        for (int l = 0; l < W; ++l) df_mad(acc, as_df(ca.v[l]), as_df(cb.v[l]));
    }
    for (int64_t i = n / W * W + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        df_mad(acc, as_df(a[i]), as_df(b[i]));
    block_sum_store(df_to_double(acc), part);
}

// valence (number of cells sharing the DoF) of cell-wise entry t
__device__ __host__ __forceinline__ int entry_valence(int64_t t, int nx, int ny, int nz, int p)
{
    const int n = p + 1, n3 = n * n * n;
    const int64_t e = t / n3;
    const int loc = (int)(t - e * n3), i = loc % n, j = (loc / n) % n, k = loc / (n * n);
    const int64_t cx = e % nx, cy = (e / nx) % ny, cz = e / ((int64_t)nx * ny);
    int v = 1;
    if ((i == 0 && cx > 0) || (i == p && cx < nx - 1)) v *= 2;
    if ((j == 0 && cy > 0) || (j == p && cy < ny - 1)) v *= 2;
    if ((k == 0 && cz > 0) || (k == p && cz < nz - 1)) v *= 2;
    return v;
}

// Given w = S r: z = dinv * w (in place on w), r <- w / kappa (the averaged dual S_bar r, which has
// the same assembly G^T r, so every later use of r is unchanged, but each copy now carries 1/kappa
// of the assembled value instead of a partial integral with cancellation), and partials
// <r, z> and <m w, r> (m = dinv != 0) = ||m G^T r||^2.
template <class V>
__device__ __forceinline__ void precond_one(V &r, V &w, V d, uint8_t kap, df64 &a1, df64 &a2)
{
    const V wi = w;
    const V zi = d * wi;
    // kappa is 1, 2, 4 or 8: multiplying by its reciprocal is exact and bit-identical to dividing,
    // and keeps the FP64 divide sequence (dozens of slow-pipe FP64 operations) out of the pass
    const V ri = wi * V(kap == 1 ? 1.0f : (kap == 2 ? 0.5f : (kap == 4 ? 0.25f : 0.125f)));
    w = zi;
    r = ri;
    df_mad(a1, as_df(ri), as_df(zi));
    if (d != V(0)) df_mad(a2, as_df(wi), as_df(ri));
}

template <class V>
__global__ void __launch_bounds__(kRedThreads) k_precond(V *__restrict__ r, V *__restrict__ w,
                                                         const V *__restrict__ dinv, int64_t n,
                                                         const uint8_t *__restrict__ kappa,
                                                         double *__restrict__ part, const int *__restrict__ flags)
{
    if (flags[F_DONE]) return;
    constexpr int W = Chunk<V>::W;
    df64 a1{0.0f, 0.0f}, a2{0.0f, 0.0f};
    CW_GRID_LOOP(k, n / W)
    {
        Chunk<V> cr, cw = ldc(w, k);  // r is written only
        const Chunk<V> cd = ldc(dinv, k);
#pragma unroll
        for (int l = 0; l < W; ++l) precond_one(cr.v[l], cw.v[l], cd.v[l], kappa[k * W + l], a1, a2);
        stc(r, k, cr);
        stc(w, k, cw);
    }
    for (int64_t i = n / W * W + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        precond_one(r[i], w[i], dinv[i], kappa[i], a1, a2);
    block_sum_store(df_to_double(a1), part);
    block_sum_store(df_to_double(a2), part + gridDim.x);
}

// u += alpha p (iteration active), then p = z + beta p (and not broken down): the iterate update
// of the iteration joined to the direction update, one pass over p
template <class V, class U>
__global__ void k_pupdate_u(U *__restrict__ u, V *__restrict__ p, const V *__restrict__ z, int64_t n,
                            const double *__restrict__ scal, const int *__restrict__ flags)
{
    static_assert(sizeof(U) == sizeof(V), "iterate and vectors share one type");
    if (!flags[F_ACTIVE]) return;
    const bool dir = flags[F_STATUS] != ST_BREAKDOWN;
    const V a = static_cast<V>(scal[S_ALPHA]), beta = static_cast<V>(scal[S_BETA]);
    constexpr int W = Chunk<V>::W;
    CW_GRID_LOOP(k, n / W)
    {
        Chunk<V> cu = ldc(reinterpret_cast<const V *>(u), k), cp = ldc(p, k);
#pragma unroll
        for (int l = 0; l < W; ++l) cu.v[l] = cu.v[l] + a * cp.v[l];
        stc(reinterpret_cast<V *>(u), k, cu);
        if (dir) {
            const Chunk<V> cz = ldc(z, k);
#pragma unroll
            for (int l = 0; l < W; ++l) cp.v[l] = cz.v[l] + beta * cp.v[l];
            stc(p, k, cp);
        }
    }
    for (int64_t i = n / W * W + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const V pi = p[i];
        u[i] = u[i] + a * pi;
        if (dir) p[i] = z[i] + beta * pi;
    }
}

template <class D, class S>
__global__ void k_copy(D *__restrict__ dst, const S *__restrict__ src, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = static_cast<D>(src[i]);
}

// dst = a - b (FP64 residual of the outer refinement step)
__global__ void k_sub(double *__restrict__ dst, const double *__restrict__ a, const double *__restrict__ b, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = a[i] - b[i];
}

__global__ void k_add_correction_f64(double *__restrict__ u, const double *__restrict__ d, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        u[i] += d[i];
}

// u += d (FP64 iterate, reduced-precision correction)
__global__ void k_add_correction(double *__restrict__ u, const float *__restrict__ d, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        u[i] += static_cast<double>(d[i]);
}

__global__ void k_make_kappa(uint8_t *__restrict__ kappa, int nx, int ny, int nz, int p, int64_t L)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < L; t += (int64_t)gridDim.x * blockDim.x)
        kappa[t] = static_cast<uint8_t>(entry_valence(t, nx, ny, nz, p));
}

// masked inverse diagonal: 0 on DoFs of the block boundary (homogeneous Dirichlet), 1/d elsewhere
template <class V>
__global__ void k_make_dinv(const double *__restrict__ d, V *__restrict__ dinv, int nx, int ny, int nz, int p,
                            int64_t L, int dirichlet)
{
    const int n = p + 1, n3 = n * n * n;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < L; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = t / n3;
        const int loc = (int)(t - e * n3), i = loc % n, j = (loc / n) % n, k = loc / (n * n);
        const int64_t cx = e % nx, cy = (e / nx) % ny, cz = e / ((int64_t)nx * ny);
        const bool bnd = (cx == 0 && i == 0) || (cx == nx - 1 && i == p) || (cy == 0 && j == 0) ||
                         (cy == ny - 1 && j == p) || (cz == 0 && k == 0) || (cz == nz - 1 && k == p);
        dinv[t] = (dirichlet && bnd) ? V(0) : static_cast<V>(1.0 / d[t]);
    }
}

__device__ __forceinline__ double sum_partials(const double *part, int nb)
{
    __shared__ double sh[kRedThreads];
    // four independent accumulators keep four loads in flight per thread (nb reaches ~1e4 for the
    // per-CTA partials of the operator epilogue)
    const int bd = blockDim.x;
    double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
    int i = threadIdx.x;
    for (; i + 3 * bd < nb; i += 4 * bd) {
        v0 += part[i];
        v1 += part[i + bd];
        v2 += part[i + 2 * bd];
        v3 += part[i + 3 * bd];
    }
    for (; i < nb; i += bd) v0 += part[i];
    sh[threadIdx.x] = (v0 + v1) + (v2 + v3);
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

enum : int { STAGE_INIT = 0, STAGE_PQ = 1, STAGE_RHO = 2, STAGE_RES = 3, STAGE_ENERGY = 4 };

// turns block partials into scalars and runs the CG scalar logic for one stage (one block)
__device__ __forceinline__ void finalize_body(const double *__restrict__ part, int nb, double *__restrict__ scal,
                                              int *__restrict__ flags, int stage)
{
    if (stage == STAGE_PQ && flags[F_DONE]) {  // an iteration after convergence: a no-op
        if (threadIdx.x == 0) flags[F_ACTIVE] = 0;
        return;
    }
    if (stage == STAGE_RHO && !flags[F_ACTIVE]) return;
    const double s0 = sum_partials(part, nb);
    const double s1 = (stage == STAGE_INIT || stage == STAGE_RHO || stage == STAGE_RES) ? sum_partials(part + nb, nb) : 0.0;
    if (threadIdx.x != 0) return;
    if (stage == STAGE_INIT) {
        scal[S_RHO] = s0;
        scal[S_RES0] = s1;
        scal[S_RES] = s1;
        flags[F_ITER] = 0;
        flags[F_STATUS] = ST_RUNNING;
        flags[F_DONE] = 0;
        if (!(s1 > 0.0)) {  // zero right-hand side: u = 0 is the solution
            flags[F_STATUS] = ST_CONVERGED;
            flags[F_DONE] = 1;
        }
    } else if (stage == STAGE_PQ) {
        if (!(s0 > 0.0) || !isfinite(s0)) {
            flags[F_STATUS] = ST_BREAKDOWN;
            flags[F_DONE] = 1;
            flags[F_ACTIVE] = 0;
            return;
        }
        flags[F_ACTIVE] = 1;
        scal[S_PQ] = s0;
        scal[S_ALPHA] = scal[S_RHO] / s0;
    } else if (stage == STAGE_RHO) {
        const double rho_new = s0;
        scal[S_RES] = s1;
        flags[F_ITER] += 1;
        if (!isfinite(rho_new) || !isfinite(s1)) {
            flags[F_STATUS] = ST_BREAKDOWN;
            flags[F_DONE] = 1;
            return;
        }
        if (s1 <= scal[S_TOL2] * scal[S_RES0]) {
            flags[F_STATUS] = ST_CONVERGED;
            flags[F_DONE] = 1;
        } else if (flags[F_ITER] >= flags[F_MAXIT]) {
            flags[F_STATUS] = ST_MAXIT;
            flags[F_DONE] = 1;
        }
        scal[S_BETA] = rho_new / scal[S_RHO];
        scal[S_RHO] = rho_new;
    } else if (stage == STAGE_RES) {
        scal[S_RES] = s1;
    } else {
        scal[S_ENERGY] = s0;
    }
}

__global__ void __launch_bounds__(kRedThreads) k_finalize(const double *__restrict__ part, int nb,
                                                          double *__restrict__ scal, int *__restrict__ flags,
                                                          int stage)
{
    finalize_body(part, nb, scal, flags, stage);
}

// called by every block after block_sum_store: the last block to arrive (threadfence reduction)
// sums all partials and runs the stage logic, so no separate finalize launch is needed
__device__ __forceinline__ void last_block_finalize(const double *__restrict__ part, double *__restrict__ scal,
                                                    int *__restrict__ flags, int stage)
{
    __shared__ int s_last;
    __threadfence();
    if (threadIdx.x == 0)
        s_last = (atomicAdd(reinterpret_cast<unsigned *>(flags + F_BLOCKS), 1u) == gridDim.x - 1) ? 1 : 0;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    finalize_body(part, gridDim.x, scal, flags, stage);
    if (threadIdx.x == 0) flags[F_BLOCKS] = 0;
}

// sums nb partials (one per operator CTA) into this grid's block partials, then the last block
// runs the stage logic
__global__ void __launch_bounds__(kRedThreads) k_sum_fin(const double *__restrict__ in, int64_t nb,
                                                         double *__restrict__ part, double *__restrict__ scal,
                                                         int *__restrict__ flags, int stage)
{
    double v = 0.0;
    CW_GRID_LOOP(i, nb) v += in[i];
    block_sum_store(v, part);
    last_block_finalize(part, scal, flags, stage);
}

template <class V>
__global__ void __launch_bounds__(kRedThreads) k_dot_fin(const V *__restrict__ a, const V *__restrict__ b, int64_t n,
                                                         double *__restrict__ part, double *__restrict__ scal,
                                                         int *__restrict__ flags, int stage)
{
    constexpr int W = Chunk<V>::W;
    df64 acc{0.0f, 0.0f};
    CW_GRID_LOOP(k, n / W)
    {
        const Chunk<V> ca = ldc(a, k), cb = ldc(b, k);
#pragma unroll
        for (int l = 0; l < W; ++l) df_mad(acc, as_df(ca.v[l]), as_df(cb.v[l]));
    }
    for (int64_t i = n / W * W + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        df_mad(acc, as_df(a[i]), as_df(b[i]));
    block_sum_store(df_to_double(acc), part);
    last_block_finalize(part, scal, flags, stage);
}

template <class V>
__global__ void __launch_bounds__(kRedThreads) k_precond_fin(V *__restrict__ r, V *__restrict__ w,
                                                             const V *__restrict__ dinv, int64_t n,
                                                             const uint8_t *__restrict__ kappa,
                                                             double *__restrict__ part, double *__restrict__ scal,
                                                             int *__restrict__ flags, int stage)
{
    if (stage == STAGE_RHO && flags[F_DONE]) return;  // an iteration after convergence
    constexpr int W = Chunk<V>::W;
    df64 a1{0.0f, 0.0f}, a2{0.0f, 0.0f};
    CW_GRID_LOOP(k, n / W)
    {
        Chunk<V> cr, cw = ldc(w, k);  // r is written only
        const Chunk<V> cd = ldc(dinv, k);
#pragma unroll
        for (int l = 0; l < W; ++l) precond_one(cr.v[l], cw.v[l], cd.v[l], kappa[k * W + l], a1, a2);
        stc(r, k, cr);
        stc(w, k, cw);
    }
    for (int64_t i = n / W * W + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        precond_one(r[i], w[i], dinv[i], kappa[i], a1, a2);
    block_sum_store(df_to_double(a1), part);
    block_sum_store(df_to_double(a2), part + gridDim.x);
    last_block_finalize(part, scal, flags, stage);
}

// Line access of the fused kernel below: N consecutive values; one 16-byte access for N = 4 floats
// (every line start there is 16-byte aligned: lines are 16 bytes apart and the partner offsets are
// multiples of 4 floats).
template <int N, class V>
struct LineIO {
    static __device__ __forceinline__ void ld(const V *p, V (&v)[N])
    {
#pragma unroll
        for (int m = 0; m < N; ++m) v[m] = p[m];
    }
    static __device__ __forceinline__ void st(V *p, const V (&v)[N])
    {
#pragma unroll
        for (int m = 0; m < N; ++m) p[m] = v[m];
    }
};
template <>
struct LineIO<4, float> {
    static __device__ __forceinline__ void ld(const float *p, float (&v)[4])
    {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
    }
    static __device__ __forceinline__ void st(float *p, const float (&v)[4])
    {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};

// The y and z passes of the DSS fused with the preconditioner: w holds S_x r' (x pass done, from
// dss_from_axpy); every x-line gathers its y-partner, z-partner and yz-partner lines and sums them in
// the passes' order ((own + y) + (z + zy), each copy the same tree, so all copies agree and the result
// equals the in-place passes bit for bit); then z_out = D^-1 s, r = s / kappa and the partials of
// <r, z> and <m s, r> as k_precond_fin. Out of place (w is only read). One thread per x-line,
// 32-bit line indexing (nlines < 2^31).
template <int N, class V>
__global__ void __launch_bounds__(kRedThreads) k_precond_yz_fin(
    const V *__restrict__ w, V *__restrict__ r, V *__restrict__ zo, const V *__restrict__ dinv,
    uint32_t nlines, int nx, int ny, int nz, FastDiv fd_nx, FastDiv fd_ny,
    double *__restrict__ part, double *__restrict__ scal, int *__restrict__ flags, int stage)
{
    if (stage == STAGE_RHO && flags[F_DONE]) return;  // an iteration after convergence
    constexpr int P = N - 1, N2 = N * N, N3 = N2 * N;
    using IO = LineIO<N, V>;
    const int sx = nx * N3, sxy = nx * ny * N3;  // < L < 2^31
    df64 a1{0.0f, 0.0f}, a2{0.0f, 0.0f};
    for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < nlines; l += gridDim.x * blockDim.x) {
        const uint32_t e = l / N2;
        const int rl = static_cast<int>(l - e * N2), j = rl % N, k = rl / N;
        const uint32_t q = fd_nx.div(e), cz = fd_ny.div(q);
        const int cy = static_cast<int>(q - cz * static_cast<uint32_t>(ny));
        const int cx = static_cast<int>(e - q * static_cast<uint32_t>(nx));
        const int oy = (j == 0 && cy > 0) ? -(sx - P * N) : ((j == P && cy < ny - 1) ? (sx - P * N) : 0);
        const int oz = (k == 0 && cz > 0) ? -(sxy - P * N2) : ((k == P && (int)cz < nz - 1) ? (sxy - P * N2) : 0);
        // valences of the line's entries from the same neighbour tests (no valence array read)
        const int kyz = (oy ? 2 : 1) * (oz ? 2 : 1);
        const int k0 = kyz * (cx > 0 ? 2 : 1), kp = kyz * (cx < nx - 1 ? 2 : 1);
        const V *b = w + static_cast<size_t>(l) * N;
        V sv[N], t[N];
        IO::ld(b, sv);
        if (oy) {
            IO::ld(b + oy, t);
#pragma unroll
            for (int m = 0; m < N; ++m) sv[m] = sv[m] + t[m];
        }
        if (oz) {
            V c[N];
            IO::ld(b + oz, c);
            if (oy) {
                IO::ld(b + oz + oy, t);
#pragma unroll
                for (int m = 0; m < N; ++m) c[m] = c[m] + t[m];
            }
#pragma unroll
            for (int m = 0; m < N; ++m) sv[m] = sv[m] + c[m];
        }
        const size_t o = static_cast<size_t>(l) * N;
        V dv[N], rv[N];
        IO::ld(dinv + o, dv);
#pragma unroll
        for (int m = 0; m < N; ++m)
            precond_one(rv[m], sv[m], dv[m], static_cast<uint8_t>(m == 0 ? k0 : (m == P ? kp : kyz)), a1, a2);
        IO::st(r + o, rv);
        IO::st(zo + o, sv);
    }
    block_sum_store(df_to_double(a1), part);
    block_sum_store(df_to_double(a2), part + gridDim.x);
    last_block_finalize(part, scal, flags, stage);
}

template <class V>
static cudaError_t launch_precond_yz(const Op &op, const V *w, V *r, V *zo, const V *dinv, double *part,
                                     double *scal, int *flags, int stage, cudaStream_t s)
{
    const Mesh &m = *op.mesh;
    const uint32_t nl = static_cast<uint32_t>(op.L / op.n);
    const FastDiv fx = FastDiv::make(m.nx), fy = FastDiv::make(m.ny);
#define CW_PYZ(NN)                                                                                     \
    k_precond_yz_fin<NN, V><<<res_grid(k_precond_yz_fin<NN, V>, kRedThreads), kRedThreads, 0, s>>>( \
        w, r, zo, dinv, nl, m.nx, m.ny, m.nz, fx, fy, \
                                                              part, scal, flags, stage)
    switch (op.n) {
    case 2: CW_PYZ(2); break;
    case 3: CW_PYZ(3); break;
    case 4: CW_PYZ(4); break;
    case 5: CW_PYZ(5); break;
    case 6: CW_PYZ(6); break;
    case 7: CW_PYZ(7); break;
    case 8: CW_PYZ(8); break;
    default: return cudaErrorInvalidValue;
    }
#undef CW_PYZ
    return cudaGetLastError();
}

// --------------------------------------------------------------------------- host side ----
static unsigned vec_grid() { return kRedBlocks; }

// Grid of a grid-stride kernel whose reduction (if any) takes its partial count from gridDim.x: whole
// waves of the blocks that are resident at once on this device, at most kRedBlocks. A fixed grid that
// is not a multiple of that runs its last blocks as a partial wave at a fraction of the occupancy (40
// registers leave 6 of 8 blocks of 256 threads per SM resident: 912 of 1216 blocks, then 304).
template <class K>
static unsigned res_grid(K kernel, int threads)
{
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, int>, unsigned> cache;  // (kernel, threads, device)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return kRedBlocks;
    const std::tuple<const void *, int, int> key(reinterpret_cast<const void *>(kernel), threads, dev);
    std::lock_guard<std::mutex> g(mu);
    const auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return kRedBlocks;
    }
    const int wave = per_sm * sms;
    const unsigned grid = (unsigned)(wave >= kRedBlocks ? kRedBlocks : wave * (kRedBlocks / wave));
    cache[key] = grid;
    return grid;
}

// CWFEM_DEBUG=1 in the environment prints the outer refinement loop of cw_cg_solve to stderr
static bool debug_trace()
{
    static const bool on = [] {
        const char *e = std::getenv("CWFEM_DEBUG");
        return e && e[0] && e[0] != '0';
    }();
    return on;
}

// which operator evaluation an inner level uses
enum ApplyKind : int { AK_DF = 0, AK_NATIVE = 1, AK_OP = 2 };

static cudaError_t apply_by_kind(const Op &op, int ak, const void *x, void *y, cudaStream_t s)
{
    if (ak == AK_NATIVE) return apply_launch_f64n(op, x, y, s);  // the op's own FP64 metric, native arithmetic
    return apply_local(op, x, y, s);
}

// whether q = A p can carry the <p, q> partials in its epilogue (curved cells, default tile and
// TMA staging, double-float or FP32 arithmetic)
static bool apply_dot_ok(const Op &op, int ak)
{
    if (ak == AK_NATIVE) return false;
    // curved stored metric: the TMA-staged default; recomputed metric: its default (input staged)
    if (op.geom == CW_GEOM_METRIC ? op.stage != 1 : op.geom != CW_GEOM_RECOMPUTE) return false;
    if (op.cpb != 0 && op.cpb != tile_cells(op.n, prec_f32_arith(op.prec))) return false;  // not the default tile
    return op.prec == CW_PREC_F64 || op.prec == CW_PREC_F32 || op.prec == CW_PREC_F32_BF16G;
}

static cudaError_t apply_dot_by_kind(const Op &op, const void *x, void *y, double *part, int64_t *nb, cudaStream_t s)
{
    switch (op.prec) {
    case CW_PREC_F64: return apply_dot_launch_df(op, x, y, part, nb, s);
    case CW_PREC_F32: return apply_dot_launch_f32(op, x, y, part, nb, s);
    default: return apply_dot_launch_f32g16(op, x, y, part, nb, s);
    }
}

template <class V>
static cudaError_t alloc_level(CgLevel &lv, int64_t L, int64_t &bytes)
{
    void **ptrs[5] = {&lv.r, &lv.p, &lv.q, &lv.z, &lv.dinv};
    for (void **pp : ptrs) {
        cudaError_t e = cudaMalloc(pp, L * sizeof(V));
        if (e != cudaSuccess) return e;
        bytes += L * sizeof(V);
    }
    return cudaSuccess;
}

static void free_level(CgLevel &lv)
{
    cudaFree(lv.r);
    cudaFree(lv.p);
    cudaFree(lv.q);
    cudaFree(lv.z);
    cudaFree(lv.dinv);
    if (lv.graph) cudaGraphExecDestroy(lv.graph);
    lv = CgLevel();
}

void cg_release(Op *op)
{
    CgScratch *c = op->cg;
    if (!c) return;
    free_level(c->lv64);
    free_level(c->lv32);
    cudaFree(c->rout);
    cudaFree(c->q64b);
    cudaFree(c->d64);
    cudaFree(c->d32);
    cudaFree(c->partials);
    cudaFree(c->dotpart);
    cudaFree(c->scal);
    cudaFree(c->flags);
    cudaFree(c->kappa);
    cudaFree(c->r32);
    cudaFree(c->z32);
    if (c->mg_graph) cudaGraphExecDestroy(c->mg_graph);
    cudaFreeHost(c->h_scal);
    cudaFreeHost(c->h_flags);
    if (c->stream) cudaStreamDestroy(c->stream);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    delete c;
    op->cg = nullptr;
}

// q = A p and the <p, q> stage (alpha = rho / <p, q>, breakdown test)
template <class V>
static cudaError_t apply_pq(const Op &aop, int ak, const V *p, V *q, CgScratch &c, cudaStream_t s)
{
    cudaError_t e;
    if (c.dotpart && apply_dot_ok(aop, ak)) {  // <p, q> from the apply epilogue
        int64_t nb = 0;
        if ((e = apply_dot_by_kind(aop, p, q, c.dotpart, &nb, s)) != cudaSuccess) return e;
        const unsigned g = (unsigned)std::min<int64_t>(kRedBlocks, (nb + kRedThreads - 1) / kRedThreads);
        k_sum_fin<<<g, kRedThreads, 0, s>>>(c.dotpart, nb, c.partials, c.scal, c.flags, STAGE_PQ);
    } else {
        if ((e = apply_by_kind(aop, ak, p, q, s)) != cudaSuccess) return e;
        k_dot_fin<V><<<res_grid(k_dot_fin<V>, kRedThreads), kRedThreads, 0, s>>>(p, q, aop.L, c.partials, c.scal, c.flags, STAGE_PQ);
    }
    return cudaGetLastError();
}

// one CG iteration on level `lv` of operator `aop` with vector type V, iterate U* u
template <class V, class U>
static cudaError_t cg_iteration(const Op &aop, int ak, CgLevel &lv, U *u, CgScratch &c, cudaStream_t s)
{
    const int64_t L = aop.L;
    V *r = static_cast<V *>(lv.r), *p = static_cast<V *>(lv.p), *q = static_cast<V *>(lv.q),
      *z = static_cast<V *>(lv.z), *dinv = static_cast<V *>(lv.dinv);
    cudaError_t e;
    if ((e = apply_pq<V>(aop, ak, p, q, c, s)) != cudaSuccess) return e;
    if constexpr (std::is_same<V, float>::value) {
        if (L < ((int64_t)1 << 31)) {
            // FP32 level: z = S_x(r - alpha q), then the y and z sums gathered inside the
            // preconditioner pass, which writes the preconditioned residual into q (free once the x
            // pass has read it)
            e = dss_from_axpy(aop, r, q, c.scal + S_ALPHA, c.flags + F_ACTIVE, z, s, true);
            if (e != cudaSuccess) return e;
            e = launch_precond_yz<V>(aop, z, r, q, dinv, c.partials, c.scal, c.flags, STAGE_RHO, s);
            if (e != cudaSuccess) return e;
            k_pupdate_u<V, U><<<res_grid(k_pupdate_u<V, U>, 256), 256, 0, s>>>(u, p, q, L, c.scal, c.flags);
            return cudaGetLastError();
        }
    }
    // z = S (r - alpha q): the residual update rides on the DSS's first pass
    if ((e = dss_from_axpy(aop, r, q, c.scal + S_ALPHA, c.flags + F_ACTIVE, z, s)) != cudaSuccess) return e;
    k_precond_fin<V><<<res_grid(k_precond_fin<V>, kRedThreads), kRedThreads, 0, s>>>(r, z, dinv, L, c.kappa, c.partials, c.scal, c.flags,
                                                        STAGE_RHO);
    k_pupdate_u<V, U><<<res_grid(k_pupdate_u<V, U>, 256), 256, 0, s>>>(u, p, z, L, c.scal, c.flags);
    return cudaGetLastError();
}

// CG on A u = rhs for level lv (rhs already in lv.r), u zeroed here. Returns the final status.
// keep_p: continue with the search direction of the previous run (residual replacement / reliable
// update: the new rhs is the accurate residual of the same problem, so the Krylov direction stays
// useful); otherwise p starts as the preconditioned residual.
template <class V, class U>
static cw_status cg_run(const Op &aop, int ak, CgLevel &lv, U *u, CgScratch &c, double rtol, int maxit, int *iters,
                        bool keep_p = false, double *rec_reduction = nullptr)
{
    cudaStream_t s = c.stream;
    const int64_t L = aop.L;
    V *r = static_cast<V *>(lv.r), *p = static_cast<V *>(lv.p), *z = static_cast<V *>(lv.z),
      *dinv = static_cast<V *>(lv.dinv);
    CW_CUDA_TRY(cudaMemsetAsync(u, 0, L * sizeof(U), s));
    c.h_scal[0] = rtol * rtol;
    c.h_flags[0] = 0;
    c.h_flags[1] = maxit;
    CW_CUDA_TRY(cudaMemcpyAsync(c.scal + S_TOL2, c.h_scal, sizeof(double), cudaMemcpyHostToDevice, s));
    CW_CUDA_TRY(cudaMemcpyAsync(c.flags + F_DONE, &c.h_flags[0], sizeof(int), cudaMemcpyHostToDevice, s));
    CW_CUDA_TRY(cudaMemcpyAsync(c.flags + F_MAXIT, &c.h_flags[1], sizeof(int), cudaMemcpyHostToDevice, s));
    // z = D^-1 S r, r <- S_bar r, rho = <r, z>, res0 = <m S r, r>, p = z
    CW_CUDA_TRY(dss_from(aop, r, z, CW_DSS_SUM, s));
    k_precond_fin<V><<<res_grid(k_precond_fin<V>, kRedThreads), kRedThreads, 0, s>>>(r, z, dinv, L, c.kappa, c.partials, c.scal, c.flags,
                                                        STAGE_INIT);
    if (!keep_p) CW_CUDA_TRY(cudaMemcpyAsync(p, z, L * sizeof(V), cudaMemcpyDeviceToDevice, s));
    CW_CUDA_TRY(cudaGetLastError());
    // one eager iteration (first-use initialisation of the kernels), then graph batches
    CW_CUDA_TRY((cg_iteration<V, U>(aop, ak, lv, u, c, s)));
    if (lv.graph && (lv.graph_u != u || lv.graph_op != &aop || lv.graph_ak != ak || lv.graph_gen != op_generation())) {
        cudaGraphExecDestroy(lv.graph);
        lv.graph = nullptr;
    }
    if (!lv.graph) {
        cudaGraph_t g;
        CW_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        for (int b = 0; b < kBatch && e == cudaSuccess; ++b) e = cg_iteration<V, U>(aop, ak, lv, u, c, s);
        cudaError_t e2 = cudaStreamEndCapture(s, &g);
        if (e != cudaSuccess) return cuda_fail(e, "cg capture");
        if (e2 != cudaSuccess) return cuda_fail(e2, "cg capture end");
        e = cudaGraphInstantiate(&lv.graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "cg graph instantiate");
        lv.graph_u = u;
        lv.graph_op = &aop;
        lv.graph_ak = ak;
        lv.graph_gen = op_generation();
    }
    for (;;) {
        CW_CUDA_TRY(cudaMemcpyAsync(c.h_flags, c.flags, F_NFLAG * sizeof(int), cudaMemcpyDeviceToHost, s));
        CW_CUDA_TRY(cudaStreamSynchronize(s));
        if (c.h_flags[F_DONE]) break;
        CW_CUDA_TRY(cudaGraphLaunch(lv.graph, s));
    }
    *iters = c.h_flags[F_ITER];
    if (rec_reduction) {  // recursive residual reduction of this run: sqrt(res / res0)
        CW_CUDA_TRY(cudaMemcpyAsync(c.h_scal, c.scal, S_NSCAL * sizeof(double), cudaMemcpyDeviceToHost, s));
        CW_CUDA_TRY(cudaStreamSynchronize(s));
        *rec_reduction = c.h_scal[S_RES0] > 0.0 ? std::sqrt(c.h_scal[S_RES] / c.h_scal[S_RES0]) : 0.0;
    }
    switch (c.h_flags[F_STATUS]) {
    case ST_CONVERGED: return CW_OK;
    case ST_BREAKDOWN: return fail(CW_ERR_BREAKDOWN, "cw_cg_solve: breakdown (<p,Ap> <= 0 or non-finite)");
    default: return fail(CW_ERR_NOT_CONVERGED, "cw_cg_solve: maxit reached");
    }
}

// ------------------------------------------------------- multigrid-preconditioned CG ----
// Given w = S r: r <- w / kappa (the averaged residual S_bar r: same assembly G^T r, every copy small;
// the V-cycle reads its input only through G^T, so it sees the same right-hand side), and, for an
// FP32 hierarchy, its FP32 copy (the cycle's input). Skipped after convergence (r is then already
// averaged and unchanged).
template <bool F32>
__global__ void __launch_bounds__(256) k_mg_average(double *__restrict__ r, const double *__restrict__ w,
                                                    const uint8_t *__restrict__ kappa, float *__restrict__ r32,
                                                    int64_t n, const int *__restrict__ flags)
{
    if (flags[F_DONE]) return;
    CW_GRID_LOOP(i, n)
    {
        const uint8_t k = kappa[i];
        const double ri = w[i] * (k == 1 ? 1.0 : (k == 2 ? 0.5 : (k == 4 ? 0.25 : 0.125)));  // exact
        r[i] = ri;
        if constexpr (F32) r32[i] = static_cast<float>(ri);
    }
}

// Partials of rho = <r, z> and of <m w, r> = ||m G^T r||^2 (m = dinv != 0), then the stage logic
// (STAGE_INIT or STAGE_RHO); with an FP32 cycle the output z32 is widened into z first.
template <bool F32>
__global__ void __launch_bounds__(kRedThreads) k_mg_dots_fin(const double *__restrict__ r, double *__restrict__ z,
                                                             const float *__restrict__ z32,
                                                             const double *__restrict__ w,
                                                             const double *__restrict__ dinv, int64_t n,
                                                             double *__restrict__ part, double *__restrict__ scal,
                                                             int *__restrict__ flags, int stage)
{
    if (stage == STAGE_RHO && flags[F_DONE]) return;  // an iteration after convergence
    df64 a1{0.0f, 0.0f}, a2{0.0f, 0.0f};
    CW_GRID_LOOP(i, n)
    {
        double zi;
        if constexpr (F32) {
            zi = static_cast<double>(z32[i]);
            z[i] = zi;
        } else {
            zi = z[i];
        }
        const double ri = r[i];
        df_mad(a1, split_f64(ri), split_f64(zi));
        if (dinv[i] != 0.0) df_mad(a2, split_f64(w[i]), split_f64(ri));
    }
    block_sum_store(df_to_double(a1), part);
    block_sum_store(df_to_double(a2), part + gridDim.x);
    last_block_finalize(part, scal, flags, stage);
}

// one iteration: q = A p, alpha; w = S (r - alpha q); r = w / kappa; z = MG(r); rho, residual, beta;
// d += alpha p, p = z + beta p
static cudaError_t mgcg_iteration(const Op &aop, MgHier &h, CgLevel &lv, double *d, CgScratch &c, bool f32,
                                  cudaStream_t s)
{
    const int64_t L = aop.L;
    double *r = static_cast<double *>(lv.r), *p = static_cast<double *>(lv.p), *q = static_cast<double *>(lv.q),
           *z = static_cast<double *>(lv.z), *dinv = static_cast<double *>(lv.dinv), *w = c.q64b;
    cudaError_t e;
    if ((e = apply_pq<double>(aop, AK_DF, p, q, c, s)) != cudaSuccess) return e;
    if ((e = dss_from_axpy(aop, r, q, c.scal + S_ALPHA, c.flags + F_ACTIVE, w, s)) != cudaSuccess) return e;
    if (f32) k_mg_average<true><<<res_grid(k_mg_average<true>, 256), 256, 0, s>>>(r, w, c.kappa, c.r32, L, c.flags);
    else k_mg_average<false><<<res_grid(k_mg_average<false>, 256), 256, 0, s>>>(r, w, c.kappa, nullptr, L, c.flags);
    if ((e = mg_vcycle_zero(h, f32 ? static_cast<void *>(c.r32) : r, f32 ? static_cast<void *>(c.z32) : z, s)) !=
        cudaSuccess)
        return e;
    if (f32)
        k_mg_dots_fin<true><<<res_grid(k_mg_dots_fin<true>, kRedThreads), kRedThreads, 0, s>>>(r, z, c.z32, w, dinv, L, c.partials, c.scal, c.flags,
                                                               STAGE_RHO);
    else
        k_mg_dots_fin<false><<<res_grid(k_mg_dots_fin<false>, kRedThreads), kRedThreads, 0, s>>>(r, z, nullptr, w, dinv, L, c.partials, c.scal,
                                                                c.flags, STAGE_RHO);
    k_pupdate_u<double, double><<<res_grid(k_pupdate_u<double, double>, 256), 256, 0, s>>>(d, p, z, L, c.scal, c.flags);
    return cudaGetLastError();
}

// CG on A d = rhs (rhs in lv.r), d zeroed here, preconditioned by one V-cycle from a zero initial
// guess (Sec. 5), in the primal-dual form of cg_run. One iteration per graph replay; the host reads
// the flags after each.
static cw_status mgcg_run(const Op &aop, MgHier &h, CgLevel &lv, double *d, CgScratch &c, double rtol, int maxit,
                          int *iters, double *rec_reduction)
{
    cudaStream_t s = c.stream;
    const int64_t L = aop.L;
    const bool f32 = mg_top_op(h).prec == CW_PREC_F32;
    double *r = static_cast<double *>(lv.r), *p = static_cast<double *>(lv.p), *z = static_cast<double *>(lv.z),
           *dinv = static_cast<double *>(lv.dinv), *w = c.q64b;
    CW_CUDA_TRY(cudaMemsetAsync(d, 0, L * sizeof(double), s));
    c.h_scal[0] = rtol * rtol;
    c.h_flags[0] = 0;
    c.h_flags[1] = maxit;
    CW_CUDA_TRY(cudaMemcpyAsync(c.scal + S_TOL2, c.h_scal, sizeof(double), cudaMemcpyHostToDevice, s));
    CW_CUDA_TRY(cudaMemcpyAsync(c.flags + F_DONE, &c.h_flags[0], sizeof(int), cudaMemcpyHostToDevice, s));
    CW_CUDA_TRY(cudaMemcpyAsync(c.flags + F_MAXIT, &c.h_flags[1], sizeof(int), cudaMemcpyHostToDevice, s));
    // w = S r; r <- S_bar r; z = MG(r); rho = <r, z>, res0 = <m S r, r>; p = z
    CW_CUDA_TRY(dss_from(aop, r, w, CW_DSS_SUM, s));
    if (f32) k_mg_average<true><<<res_grid(k_mg_average<true>, 256), 256, 0, s>>>(r, w, c.kappa, c.r32, L, c.flags);
    else k_mg_average<false><<<res_grid(k_mg_average<false>, 256), 256, 0, s>>>(r, w, c.kappa, nullptr, L, c.flags);
    CW_CUDA_TRY(mg_vcycle_zero(h, f32 ? static_cast<void *>(c.r32) : r, f32 ? static_cast<void *>(c.z32) : z, s));
    if (f32)
        k_mg_dots_fin<true><<<res_grid(k_mg_dots_fin<true>, kRedThreads), kRedThreads, 0, s>>>(r, z, c.z32, w, dinv, L, c.partials, c.scal, c.flags,
                                                               STAGE_INIT);
    else
        k_mg_dots_fin<false><<<res_grid(k_mg_dots_fin<false>, kRedThreads), kRedThreads, 0, s>>>(r, z, nullptr, w, dinv, L, c.partials, c.scal,
                                                                c.flags, STAGE_INIT);
    CW_CUDA_TRY(cudaMemcpyAsync(p, z, L * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CW_CUDA_TRY(cudaGetLastError());
    CW_CUDA_TRY(mgcg_iteration(aop, h, lv, d, c, f32, s));  // eager: first-use initialisation
    if (c.mg_graph && (c.mg_graph_id != mg_id(h) || c.mg_graph_d != d || c.mg_graph_op != &aop ||
                       c.mg_graph_gen != op_generation())) {
        cudaGraphExecDestroy(c.mg_graph);
        c.mg_graph = nullptr;
    }
    if (!c.mg_graph) {
        cudaGraph_t g;
        CW_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = mgcg_iteration(aop, h, lv, d, c, f32, s);
        cudaError_t e2 = cudaStreamEndCapture(s, &g);
        if (e != cudaSuccess) return cuda_fail(e, "mg-pcg capture");
        if (e2 != cudaSuccess) return cuda_fail(e2, "mg-pcg capture end");
        e = cudaGraphInstantiate(&c.mg_graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "mg-pcg graph instantiate");
        c.mg_graph_id = mg_id(h);
        c.mg_graph_d = d;
        c.mg_graph_op = &aop;
        c.mg_graph_gen = op_generation();
    }
    for (;;) {
        CW_CUDA_TRY(cudaMemcpyAsync(c.h_flags, c.flags, F_NFLAG * sizeof(int), cudaMemcpyDeviceToHost, s));
        CW_CUDA_TRY(cudaStreamSynchronize(s));
        if (c.h_flags[F_DONE]) break;
        CW_CUDA_TRY(cudaGraphLaunch(c.mg_graph, s));
    }
    *iters = c.h_flags[F_ITER];
    CW_CUDA_TRY(cudaMemcpyAsync(c.h_scal, c.scal, S_NSCAL * sizeof(double), cudaMemcpyDeviceToHost, s));
    CW_CUDA_TRY(cudaStreamSynchronize(s));
    *rec_reduction = c.h_scal[S_RES0] > 0.0 ? std::sqrt(c.h_scal[S_RES] / c.h_scal[S_RES0]) : 0.0;
    switch (c.h_flags[F_STATUS]) {
    case ST_CONVERGED: return CW_OK;
    case ST_BREAKDOWN: return fail(CW_ERR_BREAKDOWN, "cw_mg_pcg_solve: breakdown (<p,Ap> <= 0 or non-finite)");
    default: return fail(CW_ERR_NOT_CONVERGED, "cw_mg_pcg_solve: maxit reached");
    }
}

static cw_status ensure_scratch(Op *op, int mode)
{
    CgScratch *c = op->cg;
    const int64_t L = op->L;
    if (!c) {
        c = new CgScratch;
        op->cg = c;
        CW_CUDA_TRY(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        CW_CUDA_TRY(cudaEventCreate(&c->ev0));
        CW_CUDA_TRY(cudaEventCreate(&c->ev1));
        CW_CUDA_TRY(cudaMalloc(&c->partials, 2 * kRedBlocks * sizeof(double)));
        CW_CUDA_TRY(cudaMalloc(&c->dotpart, op->E * sizeof(double)));
        CW_CUDA_TRY(cudaMalloc(&c->scal, S_NSCAL * sizeof(double)));
        CW_CUDA_TRY(cudaMalloc(&c->flags, F_NFLAG * sizeof(int)));
        CW_CUDA_TRY(cudaMemset(c->scal, 0, S_NSCAL * sizeof(double)));
        CW_CUDA_TRY(cudaMemset(c->flags, 0, F_NFLAG * sizeof(int)));
        CW_CUDA_TRY(cudaMallocHost(&c->h_scal, S_NSCAL * sizeof(double)));
        CW_CUDA_TRY(cudaMallocHost(&c->h_flags, F_NFLAG * sizeof(int)));
        CW_CUDA_TRY((alloc_level<double>(c->lv64, L, c->bytes)));
        CW_CUDA_TRY(cudaMalloc(&c->rout, L * sizeof(double)));
        CW_CUDA_TRY(cudaMalloc(&c->q64b, L * sizeof(double)));
        CW_CUDA_TRY(cudaMalloc(&c->kappa, L));
        c->bytes += 2 * L * sizeof(double) + L + 2 * kRedBlocks * sizeof(double) + op->E * sizeof(double);
        k_make_kappa<<<vec_grid(), 256, 0, c->stream>>>(c->kappa, op->mesh->nx, op->mesh->ny, op->mesh->nz, op->p, L);
        // FP64 masked inverse diagonal
        double *d = static_cast<double *>(c->lv64.q);  // borrow q as the diagonal buffer
        cw_status st = cw_diagonal(reinterpret_cast<cw_op>(op), d, c->stream);
        if (st != CW_OK) return st;
        k_make_dinv<double><<<vec_grid(), 256, 0, c->stream>>>(d, static_cast<double *>(c->lv64.dinv), op->mesh->nx,
                                                               op->mesh->ny, op->mesh->nz, op->p, L, 1);
        CW_CUDA_TRY(cudaGetLastError());
        CW_CUDA_TRY(cudaStreamSynchronize(c->stream));
        op->owned_bytes += c->bytes;
    }
    if (!op->native) {  // the IEEE FP64 operator of the outer residual (and of CW_CG_F64_NATIVE)
        cw_op nat;
        cw_status st = cw_op_create(reinterpret_cast<cw_mesh>(op->mesh), op->p, op->kind, op->geom, CW_PREC_F64_NATIVE,
                                    op->bc, &nat);
        if (st != CW_OK) return st;
        op->native = reinterpret_cast<Op *>(nat);
    }
    const bool fp64_inner = (mode == CW_CG_F64 || mode == CW_CG_F64_NATIVE);
    if (fp64_inner && !c->d64) {
        CW_CUDA_TRY(cudaMalloc(&c->d64, L * sizeof(double)));
        op->owned_bytes += L * sizeof(double);
    }
    if (!fp64_inner) {
        const int iprec = (mode == CW_CG_IR_BF16) ? CW_PREC_F32_BF16G : CW_PREC_F32;
        if (op->inner && op->inner->prec != iprec) {  // switch inner metric precision
            cw_op_destroy(reinterpret_cast<cw_op>(op->inner));
            op->inner = nullptr;
            if (c->lv32.graph) {
                cudaGraphExecDestroy(c->lv32.graph);
                c->lv32.graph = nullptr;
            }
        }
        if (!op->inner) {
            cw_op inner;
            cw_status st = cw_op_create(reinterpret_cast<cw_mesh>(op->mesh), op->p, op->kind, op->geom, iprec, op->bc, &inner);
            if (st != CW_OK) return st;
            op->inner = reinterpret_cast<Op *>(inner);
        }
        if (!c->d32) {
            int64_t b = 0;
            CW_CUDA_TRY((alloc_level<float>(c->lv32, L, b)));
            CW_CUDA_TRY(cudaMalloc(&c->d32, L * sizeof(float)));
            b += L * sizeof(float);
            k_copy<float, double><<<vec_grid(), 256, 0, c->stream>>>(static_cast<float *>(c->lv32.dinv),
                                                                     static_cast<const double *>(c->lv64.dinv), L);
            CW_CUDA_TRY(cudaGetLastError());
            CW_CUDA_TRY(cudaStreamSynchronize(c->stream));
            op->owned_bytes += b;
        }
    }
    return CW_OK;
}

// ||m G^T r||^2 = <m S r, r> of an FP64 dual vector r (work buffer w); r is left unchanged
static cw_status residual_norm2(const Op &op, const double *r, double *w, CgScratch &c, double *out)
{
    cudaStream_t s = c.stream;
    const int64_t L = op.L;
    double *rr = static_cast<double *>(c.lv64.r);  // scratch copy: k_precond averages it in place
    CW_CUDA_TRY(dss_from(op, r, w, CW_DSS_SUM, s));
    CW_CUDA_TRY(cudaMemcpyAsync(rr, r, L * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CW_CUDA_TRY(cudaMemsetAsync(c.flags + F_DONE, 0, sizeof(int), s));
    k_precond<double><<<vec_grid(), kRedThreads, 0, s>>>(rr, w, static_cast<double *>(c.lv64.dinv), L, c.kappa,
                                                         c.partials, c.flags);
    k_finalize<<<1, kRedThreads, 0, s>>>(c.partials, kRedBlocks, c.scal, c.flags, STAGE_RES);
    CW_CUDA_TRY(cudaMemcpyAsync(c.h_scal, c.scal + S_RES, sizeof(double), cudaMemcpyDeviceToHost, s));
    CW_CUDA_TRY(cudaStreamSynchronize(s));
    *out = c.h_scal[0];
    return CW_OK;
}

static cw_status energy(const Op &op, const double *r, const double *u, CgScratch &c, double *out)
{
    cudaStream_t s = c.stream;
    k_dot<double><<<vec_grid(), kRedThreads, 0, s>>>(r, u, op.L, c.partials);
    k_finalize<<<1, kRedThreads, 0, s>>>(c.partials, kRedBlocks, c.scal, c.flags, STAGE_ENERGY);
    CW_CUDA_TRY(cudaMemcpyAsync(c.h_scal, c.scal + S_ENERGY, sizeof(double), cudaMemcpyDeviceToHost, s));
    CW_CUDA_TRY(cudaStreamSynchronize(s));
    *out = c.h_scal[0];
    return CW_OK;
}

// S_bar r (averaging DSS, Eq. (averaging_dss)) of the FP64 residual into the inner level's rhs
static cw_status averaged_rhs(const Op &op, const double *r, double *work, void *dst, bool to_f32, cudaStream_t s)
{
    CW_CUDA_TRY(dss_from(op, r, work, CW_DSS_AVERAGE, s));
    if (to_f32)
        k_copy<float, double><<<vec_grid(), 256, 0, s>>>(static_cast<float *>(dst), work, op.L);
    else
        k_copy<double, double><<<vec_grid(), 256, 0, s>>>(static_cast<double *>(dst), work, op.L);
    CW_CUDA_TRY(cudaGetLastError());
    return CW_OK;
}

}  // namespace cw

using namespace cw;

// Every mode runs the same outer loop: r = b - A u with the IEEE FP64 operator (native FP64
// arithmetic on a twin of the operator whose metric is stored as doubles: the accurate residual),
// stop when ||m G^T r|| <= rtol ||m G^T b||, else continue the inner Jacobi-PCG on
// A d = S_bar r and set u += d. The inner solver is FP64 with the double-float operator
// (CW_CG_F64), FP64 with the native operator (CW_CG_F64_NATIVE), or FP32 with the FP32 / BF16-metric
// operator (CW_CG_IR_*). The inner CG is not restarted between segments: each segment replaces the
// recursive residual by the accurate one and keeps the search direction (reliable updates, as in
// mixed-precision Krylov solvers). A segment ends when its recursive residual has dropped by the
// reduction still needed (FP64 inner levels) or by a factor 10 (FP32 inner levels, whose recursive
// residual drifts from the true one as the iteration proceeds).
// The outer refinement loop shared by cw_cg_solve (Jacobi-preconditioned inner CG, mg == nullptr)
// and cw_mg_pcg_solve (V-cycle-preconditioned inner CG in FP64).
static cw_status solve_impl(Op *op, const double *b, double *u, double rtol, int maxit, int mode, MgHier *mg,
                            cw_cg_stats *stats, void *stream, bool warm = false)
{
    cudaStream_t us = static_cast<cudaStream_t>(stream);
    cw_status st = ensure_scratch(op, mode);
    if (st != CW_OK) return st;
    CgScratch &c = *op->cg;
    cudaStream_t s = c.stream;
    // a failed solve first asks the operators' device status words: an expired bounded wait (a tile
    // left without output) explains a breakdown or a non-finite residual and is reported instead
    auto failed = [&](cw_status why) {
        for (Op *o : {op, op->inner, op->native})
            if (op_status_take(o, s, "cw_cg_solve") == CW_ERR_TIMEOUT) return CW_ERR_TIMEOUT;
        if (mg && mg_status_take(*mg, s) == CW_ERR_TIMEOUT) return CW_ERR_TIMEOUT;
        return why;
    };
    const int64_t L = op->L;
    if (mg && mg_top_op(*mg).prec == CW_PREC_F32 && !c.r32) {
        CW_CUDA_TRY(cudaMalloc(&c.r32, L * sizeof(float)));
        CW_CUDA_TRY(cudaMalloc(&c.z32, L * sizeof(float)));
        op->owned_bytes += 2 * L * (int64_t)sizeof(float);
    }
    // order the solve after the caller's stream
    CW_CUDA_TRY(cudaEventRecord(c.ev0, us));
    CW_CUDA_TRY(cudaStreamWaitEvent(s, c.ev0, 0));
    CW_CUDA_TRY(cudaEventRecord(c.ev0, s));
    const bool fp64_inner = (mode == CW_CG_F64 || mode == CW_CG_F64_NATIVE);
    const int ak = mode == CW_CG_F64 ? AK_DF : (mode == CW_CG_F64_NATIVE ? AK_NATIVE : AK_OP);
    const double floor_tol = fp64_inner ? 1e-15 : 0.1;
    double *r = c.rout, *w = c.q64b;
    int iters = 0, outer = 0;
    double res0 = 0.0, res = 0.0;
    k_copy<double, double><<<vec_grid(), 256, 0, s>>>(r, b, L);
    if ((st = residual_norm2(*op, r, w, c, &res0)) != CW_OK) return st;
    if (!std::isfinite(res0)) return fail(CW_ERR_BREAKDOWN, "cw_cg_solve: non-finite right-hand side");
    if (warm && res0 > 0.0) {  // r = b - A u of the caller's iterate, with the IEEE FP64 operator
        CW_CUDA_TRY(apply_launch_f64n(*op->native, u, w, s));
        k_sub<<<vec_grid(), 256, 0, s>>>(r, b, w, L);
        if ((st = residual_norm2(*op, r, w, c, &res)) != CW_OK) return st;
        if (!std::isfinite(res)) return fail(CW_ERR_BREAKDOWN, "cw_cg_solve: non-finite initial residual (warm start)");
    } else {
        CW_CUDA_TRY(cudaMemsetAsync(u, 0, L * sizeof(double), s));
        res = res0;
    }
    st = res0 > 0.0 ? CW_ERR_NOT_CONVERGED : CW_OK;
    bool consistent = false;  // the last segment's true reduction followed its recursive one
    while (res0 > 0.0 && iters < maxit && outer < 200) {
        if (res <= rtol * rtol * res0) {
            st = CW_OK;
            break;
        }
        cw::Range outer_range("cwfem:cg_outer_step");  // inner segment, correction, true residual
        const double need = rtol * std::sqrt(res0 / res);
        const double itol = std::min(0.5, std::max(floor_tol, 0.5 * need));
        int it = 0;
        double rec = 1.0;
        cw_status ist;
        for (int attempt = 0; attempt < 2; ++attempt) {
            // continue the Krylov process only after a consistent segment; restart otherwise or
            // when a continued segment breaks down
            const bool keep = consistent && attempt == 0;
            if (mg) {  // V-cycle-preconditioned CG, restarted at every outer step
                if ((ist = averaged_rhs(*op, r, w, c.lv64.r, false, s)) != CW_OK) return ist;
                ist = mgcg_run(*op, *mg, c.lv64, c.d64, c, itol, maxit - iters, &it, &rec);
            } else if (fp64_inner) {
                if ((ist = averaged_rhs(*op, r, w, c.lv64.r, false, s)) != CW_OK) return ist;
                const Op &iop = (mode == CW_CG_F64_NATIVE) ? *op->native : *op;
                ist = cg_run<double, double>(iop, ak, c.lv64, c.d64, c, itol, maxit - iters, &it, keep, &rec);
            } else {
                if ((ist = averaged_rhs(*op, r, w, c.lv32.r, true, s)) != CW_OK) return ist;
                ist = cg_run<float, float>(*op->inner, AK_OP, c.lv32, c.d32, c, itol, maxit - iters, &it, keep, &rec);
            }
            if (debug_trace())
                std::fprintf(stderr, "[cwfem cg] outer %d: inner status %d, %d iterations (tol %.2e, %s)\n", outer,
                             (int)ist, it, itol, keep ? "continued" : "restarted");
            iters += it;
            if (ist != CW_ERR_BREAKDOWN || !keep || mg) break;
        }
        // breakdown, or a CUDA error of the inner run: the correction may be partly written
        if (ist != CW_OK && ist != CW_ERR_NOT_CONVERGED) return failed(ist);
        if (fp64_inner) k_add_correction_f64<<<vec_grid(), 256, 0, s>>>(u, c.d64, L);
        else k_add_correction<<<vec_grid(), 256, 0, s>>>(u, c.d32, L);
        ++outer;
        // accurate residual with the IEEE FP64 operator (native arithmetic, metric stored as doubles)
        const double res_prev = res;
        CW_CUDA_TRY(apply_launch_f64n(*op->native, u, w, s));
        k_sub<<<vec_grid(), 256, 0, s>>>(r, b, w, L);
        if ((st = residual_norm2(*op, r, w, c, &res)) != CW_OK) return st;
        if (debug_trace()) std::fprintf(stderr, "[cwfem cg] outer %d: true rel residual %.3e\n", outer, std::sqrt(res / res0));
        if (!std::isfinite(res)) return failed(fail(CW_ERR_BREAKDOWN, "cw_cg_solve: non-finite residual"));
        consistent = std::sqrt(res / res_prev) <= 1.25 * rec;
        st = CW_ERR_NOT_CONVERGED;
    }
    if (res <= rtol * rtol * res0) st = CW_OK;
    if (st == CW_ERR_NOT_CONVERGED) set_error("cw_cg_solve: maxit reached before rtol");
    CW_CUDA_TRY(cudaEventRecord(c.ev1, s));
    CW_CUDA_TRY(cudaEventSynchronize(c.ev1));
    float ms = 0.0f;
    CW_CUDA_TRY(cudaEventElapsedTime(&ms, c.ev0, c.ev1));
    double eta = 0.0;
    cw_status s3 = energy(*op, r, u, c, &eta);  // r = b - A u of the returned u
    if (s3 != CW_OK) return s3;
    // an expired bounded wait in any operator kernel of the solve invalidates it
    for (Op *o : {op, op->inner, op->native})
        if ((s3 = op_status_take(o, s, "cw_cg_solve")) != CW_OK) return s3;
    if (mg)
        if ((s3 = mg_status_take(*mg, s)) != CW_OK) return s3;
    CW_CUDA_TRY(cudaEventRecord(c.ev0, s));
    CW_CUDA_TRY(cudaStreamWaitEvent(us, c.ev0, 0));
    if (stats) {
        stats->iterations = iters;
        stats->outer_iterations = outer;
        stats->rel_residual = res0 > 0.0 ? std::sqrt(res / res0) : 0.0;
        stats->energy = eta;
        stats->seconds = ms * 1e-3;
    }
    return st;
}

extern "C" cw_status cw_cg_solve(cw_op oh, const double *b, double *u, double rtol, int maxit, int mode,
                                 cw_cg_stats *stats, void *stream)
{
    cw::Range nvtx_range("cwfem:cw_cg_solve");
    Op *op = reinterpret_cast<Op *>(oh);
    if (!op || !b || !u) return fail(CW_ERR_ARG, "cw_cg_solve: NULL argument");
    if (op->prec != CW_PREC_F64) return fail(CW_ERR_ARG, "cw_cg_solve: the operator must be CW_PREC_F64");
    if (op->bc != CW_BC_DIRICHLET0) return fail(CW_ERR_ARG, "cw_cg_solve: the operator must use CW_BC_DIRICHLET0");
    const bool warm = (mode & CW_CG_WARM_START) != 0;
    mode &= ~CW_CG_WARM_START;
    if (mode < CW_CG_F64 || mode > CW_CG_F64_NATIVE) return fail(CW_ERR_ARG, "cw_cg_solve: bad mode");
    if (!(rtol > 0.0) || maxit < 1) return fail(CW_ERR_ARG, "cw_cg_solve: rtol must be > 0 and maxit >= 1");
    if (b == u) return fail(CW_ERR_ARG, "cw_cg_solve: b and u must not alias");
    return solve_impl(op, b, u, rtol, maxit, mode, nullptr, stats, stream, warm);
}

extern "C" cw_status cw_mg_pcg_solve(cw_mg mh, cw_op oh, const double *b, double *u, double rtol, int maxit,
                                     cw_cg_stats *stats, void *stream)
{
    cw::Range nvtx_range("cwfem:cw_mg_pcg_solve");
    Op *op = reinterpret_cast<Op *>(oh);
    MgHier *mg = reinterpret_cast<MgHier *>(mh);
    if (!mg || !op || !b || !u) return fail(CW_ERR_ARG, "cw_mg_pcg_solve: NULL argument");
    if (op->prec != CW_PREC_F64) return fail(CW_ERR_ARG, "cw_mg_pcg_solve: the operator must be CW_PREC_F64");
    if (op->bc != CW_BC_DIRICHLET0) return fail(CW_ERR_ARG, "cw_mg_pcg_solve: the operator must use CW_BC_DIRICHLET0");
    const Op &top = mg_top_op(*mg);
    if (top.mesh->nx != op->mesh->nx || top.mesh->ny != op->mesh->ny || top.mesh->nz != op->mesh->nz ||
        top.p != op->p || top.kind != op->kind)
        return fail(CW_ERR_ARG, "cw_mg_pcg_solve: the operator and the finest level differ in mesh, degree or kind");
    if (!(rtol > 0.0) || maxit < 1) return fail(CW_ERR_ARG, "cw_mg_pcg_solve: rtol must be > 0 and maxit >= 1");
    if (b == u) return fail(CW_ERR_ARG, "cw_mg_pcg_solve: b and u must not alias");
    return solve_impl(op, b, u, rtol, maxit, CW_CG_F64, mg, stats, stream);
}

// Relative residual ||m G^T (b - A u)|| / ||m G^T b|| of a cell-wise iterate, with A evaluated by the
// IEEE FP64 twin (prec CW_PREC_F64_NATIVE) or by the operator's own double-float arithmetic on its
// float-pair metric (CW_PREC_F64).
extern "C" cw_status cw_cg_residual(cw_op oh, const double *b, const double *u, int prec, double *rel_residual,
                                    void *stream)
{
    Op *op = reinterpret_cast<Op *>(oh);
    if (!op || !b || !u || !rel_residual) return fail(CW_ERR_ARG, "cw_cg_residual: NULL argument");
    if (op->prec != CW_PREC_F64) return fail(CW_ERR_ARG, "cw_cg_residual: the operator must be CW_PREC_F64");
    if (op->bc != CW_BC_DIRICHLET0) return fail(CW_ERR_ARG, "cw_cg_residual: the operator must use CW_BC_DIRICHLET0");
    if (prec != CW_PREC_F64 && prec != CW_PREC_F64_NATIVE)
        return fail(CW_ERR_ARG, "cw_cg_residual: prec must be CW_PREC_F64 or CW_PREC_F64_NATIVE");
    cw_status st = ensure_scratch(op, CW_CG_F64);
    if (st != CW_OK) return st;
    CgScratch &c = *op->cg;
    cudaStream_t s = c.stream;
    CW_CUDA_TRY(cudaEventRecord(c.ev0, static_cast<cudaStream_t>(stream)));
    CW_CUDA_TRY(cudaStreamWaitEvent(s, c.ev0, 0));
    double *r = c.rout, *w = c.q64b;
    double res0 = 0.0, res = 0.0;
    if ((st = residual_norm2(*op, b, w, c, &res0)) != CW_OK) return st;
    if (prec == CW_PREC_F64_NATIVE) CW_CUDA_TRY(apply_launch_f64n(*op->native, u, w, s));
    else CW_CUDA_TRY(apply_local(*op, u, w, s));
    k_sub<<<vec_grid(), 256, 0, s>>>(r, b, w, op->L);
    CW_CUDA_TRY(cudaGetLastError());
    if ((st = residual_norm2(*op, r, w, c, &res)) != CW_OK) return st;
    for (Op *o : {op, op->native})
        if ((st = op_status_take(o, s, "cw_cg_residual")) != CW_OK) return st;
    *rel_residual = res0 > 0.0 ? std::sqrt(res / res0) : 0.0;
    return CW_OK;
}

// ===================================================================== allocation-free solve ====
// cw_cg_solve_noalloc: the same FP64 solve as cw_cg_solve (modes CW_CG_F64 and CW_CG_F64_NATIVE)
// for callers that cannot allocate device memory at solve time -- code running inside a memory
// pool or an allocator callback, a real-time loop, or a host that forbids cudaMalloc after start-up.
// All its scratch lives in one file-scope __device__ array of fixed size, which the module holds on
// every GPU that loads this library until the process exits. Every call uses the same array, so
// calls that overlap on the GPU (two streams, or two threads) race on it.
namespace cw {

constexpr int64_t kNoAllocMaxL = int64_t(1) << 18;  // largest cell-wise length accepted
constexpr size_t kNaVec = size_t(kNoAllocMaxL) * sizeof(double);
// 8 FP64 vectors (rout, w, d, and the inner level r, p, q, z, dinv), the valence bytes, the block
// partials, the device scalars and flags
constexpr size_t kNaBytes = 8 * kNaVec + size_t(kNoAllocMaxL) + 2 * kRedBlocks * sizeof(double) +
                            S_NSCAL * sizeof(double) + F_NFLAG * sizeof(int) + 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// Device address of g_noalloc_scratch in the current device's context. In host code the symbol is
// only a host-side stand-in; its device address comes from cudaGetSymbolAddress, which is resolved
// again on every call: the address belongs to the CUDA context, so a value kept from an earlier call
// could be stale after cudaDeviceReset or under another context on the same device. Once the module
// is loaded on the device this lookup allocates nothing.
static cw_status noalloc_base(unsigned char **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cw_cg_solve_noalloc: cudaGetSymbolAddress");
    *out = static_cast<unsigned char *>(p);
    return CW_OK;
}

// inner CG without graphs: iterations launched eagerly, the flag read every kBatch iterations
static cw_status cg_run_eager(const Op &aop, int ak, CgLevel &lv, double *u, CgScratch &c, double rtol, int maxit,
                              int *iters, cudaStream_t s)
{
    const int64_t L = aop.L;
    double *r = static_cast<double *>(lv.r), *p = static_cast<double *>(lv.p), *z = static_cast<double *>(lv.z),
           *dinv = static_cast<double *>(lv.dinv);
    CW_CUDA_TRY(cudaMemsetAsync(u, 0, L * sizeof(double), s));
    const double tol2 = rtol * rtol;
    const int hf[2] = {0, maxit};
    CW_CUDA_TRY(cudaMemcpyAsync(c.scal + S_TOL2, &tol2, sizeof(double), cudaMemcpyHostToDevice, s));
    CW_CUDA_TRY(cudaMemcpyAsync(c.flags + F_DONE, &hf[0], sizeof(int), cudaMemcpyHostToDevice, s));
    CW_CUDA_TRY(cudaMemcpyAsync(c.flags + F_MAXIT, &hf[1], sizeof(int), cudaMemcpyHostToDevice, s));
    k_copy<double, double><<<vec_grid(), 256, 0, s>>>(z, r, L);
    CW_CUDA_TRY(dss_launch(aop, z, CW_DSS_SUM, s));
    k_precond<double><<<vec_grid(), kRedThreads, 0, s>>>(r, z, dinv, L, c.kappa, c.partials, c.flags);
    k_finalize<<<1, kRedThreads, 0, s>>>(c.partials, kRedBlocks, c.scal, c.flags, STAGE_INIT);
    k_copy<double, double><<<vec_grid(), 256, 0, s>>>(p, z, L);
    CW_CUDA_TRY(cudaGetLastError());
    for (;;) {
        for (int b = 0; b < kBatch; ++b) CW_CUDA_TRY((cg_iteration<double, double>(aop, ak, lv, u, c, s)));
        int hflags[F_NFLAG];
        CW_CUDA_TRY(cudaMemcpyAsync(hflags, c.flags, sizeof hflags, cudaMemcpyDeviceToHost, s));
        CW_CUDA_TRY(cudaStreamSynchronize(s));
        if (hflags[F_DONE]) {
            *iters = hflags[F_ITER];
            if (hflags[F_STATUS] == ST_CONVERGED) return CW_OK;
            if (hflags[F_STATUS] == ST_BREAKDOWN) return fail(CW_ERR_BREAKDOWN, "cw_cg_solve_noalloc: breakdown");
            return fail(CW_ERR_NOT_CONVERGED, "cw_cg_solve_noalloc: maxit reached");
        }
    }
}

}  // namespace cw

extern "C" cw_status cw_cg_solve_noalloc(cw_op oh, const double *b, double *u, double rtol, int maxit, int mode,
                                         cw_cg_stats *stats, void *stream)
{
    cw::Range nvtx_range("cwfem:cw_cg_solve_noalloc");
    Op *op = reinterpret_cast<Op *>(oh);
    if (!op || !b || !u) return fail(CW_ERR_ARG, "cw_cg_solve_noalloc: NULL argument");
    if (op->prec != CW_PREC_F64) return fail(CW_ERR_ARG, "cw_cg_solve_noalloc: the operator must be CW_PREC_F64");
    if (op->bc != CW_BC_DIRICHLET0) return fail(CW_ERR_ARG, "cw_cg_solve_noalloc: the operator must use CW_BC_DIRICHLET0");
    if (mode != CW_CG_F64 && mode != CW_CG_F64_NATIVE)
        return fail(CW_ERR_ARG, "cw_cg_solve_noalloc: only the FP64 modes CW_CG_F64 and CW_CG_F64_NATIVE");
    if (!(rtol > 0.0) || maxit < 1) return fail(CW_ERR_ARG, "cw_cg_solve_noalloc: rtol must be > 0 and maxit >= 1");
    if (b == u) return fail(CW_ERR_ARG, "cw_cg_solve_noalloc: b and u must not alias");
    if (op->L > kNoAllocMaxL)
        return fail(CW_ERR_ARG, "cw_cg_solve_noalloc: cell-wise length " + std::to_string(op->L) +
                                    " exceeds the fixed scratch limit of " + std::to_string(kNoAllocMaxL) + " values");
    const auto t0 = std::chrono::steady_clock::now();
    unsigned char *base = nullptr;
    cw_status st = noalloc_base(&base);
    if (st != CW_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t L = op->L;
    // carve the scratch
    CgScratch c;
    unsigned char *cur = base;
    auto take = [&](size_t bytes) {
        unsigned char *p = cur;
        cur += (bytes + 255) / 256 * 256;
        return static_cast<void *>(p);
    };
    double *r = static_cast<double *>(take(kNaVec));
    double *w = static_cast<double *>(take(kNaVec));
    double *d = static_cast<double *>(take(kNaVec));
    c.lv64.r = take(kNaVec);
    c.lv64.p = take(kNaVec);
    c.lv64.q = take(kNaVec);
    c.lv64.z = take(kNaVec);
    c.lv64.dinv = take(kNaVec);
    c.kappa = static_cast<uint8_t *>(take(kNoAllocMaxL));
    c.partials = static_cast<double *>(take(2 * kRedBlocks * sizeof(double)));
    c.scal = static_cast<double *>(take(S_NSCAL * sizeof(double)));
    c.flags = static_cast<int *>(take(F_NFLAG * sizeof(int)));
    double hscal[S_NSCAL];
    int hflags[F_NFLAG];
    c.h_scal = hscal;
    c.h_flags = hflags;
    c.stream = s;
    // the array keeps the previous call's contents: scalars and flags start from zero, the
    // diagonal, valences and vectors are rebuilt or overwritten below before they are read
    CW_CUDA_TRY(cudaMemsetAsync(c.scal, 0, S_NSCAL * sizeof(double), s));
    CW_CUDA_TRY(cudaMemsetAsync(c.flags, 0, F_NFLAG * sizeof(int), s));
    k_make_kappa<<<vec_grid(), 256, 0, s>>>(c.kappa, op->mesh->nx, op->mesh->ny, op->mesh->nz, op->p, L);
    if ((st = cw_diagonal(oh, static_cast<double *>(c.lv64.q), s)) != CW_OK) return st;
    k_make_dinv<double><<<vec_grid(), 256, 0, s>>>(static_cast<double *>(c.lv64.q), static_cast<double *>(c.lv64.dinv),
                                                   op->mesh->nx, op->mesh->ny, op->mesh->nz, op->p, L, 1);
    CW_CUDA_TRY(cudaGetLastError());
    const int ak = mode == CW_CG_F64 ? AK_DF : AK_NATIVE;
    int iters = 0, outer = 0;
    double res0 = 0.0, res = 0.0;
    CW_CUDA_TRY(cudaMemsetAsync(u, 0, L * sizeof(double), s));
    k_copy<double, double><<<vec_grid(), 256, 0, s>>>(r, b, L);
    if ((st = residual_norm2(*op, r, w, c, &res0)) != CW_OK) return st;
    if (!std::isfinite(res0)) return fail(CW_ERR_BREAKDOWN, "cw_cg_solve_noalloc: non-finite right-hand side");
    res = res0;
    st = res0 > 0.0 ? CW_ERR_NOT_CONVERGED : CW_OK;
    while (res0 > 0.0 && iters < maxit && outer < 50) {
        if (res <= rtol * rtol * res0) {
            st = CW_OK;
            break;
        }
        const double itol = std::min(0.5, std::max(1e-15, 0.5 * rtol * std::sqrt(res0 / res)));
        int it = 0;
        if ((st = averaged_rhs(*op, r, w, c.lv64.r, false, s)) != CW_OK) return st;
        cw_status ist = cg_run_eager(*op, ak, c.lv64, d, c, itol, maxit - iters, &it, s);
        if (ist != CW_OK && ist != CW_ERR_NOT_CONVERGED) return ist;
        k_add_correction_f64<<<vec_grid(), 256, 0, s>>>(u, d, L);
        iters += it;
        ++outer;
        CW_CUDA_TRY(apply_launch_f64n(*op, u, w, s));
        k_sub<<<vec_grid(), 256, 0, s>>>(r, b, w, L);
        if ((st = residual_norm2(*op, r, w, c, &res)) != CW_OK) return st;
        if (!std::isfinite(res)) return fail(CW_ERR_BREAKDOWN, "cw_cg_solve_noalloc: non-finite residual");
        st = CW_ERR_NOT_CONVERGED;
    }
    if (res <= rtol * rtol * res0) st = CW_OK;
    if (st == CW_ERR_NOT_CONVERGED) set_error("cw_cg_solve_noalloc: maxit reached before rtol");
    double eta = 0.0;
    cw_status s3 = energy(*op, r, u, c, &eta);
    if (s3 != CW_OK) return s3;
    if ((s3 = op_status_take(op, s, "cw_cg_solve_noalloc")) != CW_OK) return s3;
    if (stats) {
        stats->iterations = iters;
        stats->outer_iterations = outer;
        stats->rel_residual = res0 > 0.0 ? std::sqrt(res / res0) : 0.0;
        stats->energy = eta;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return st;
}
