// cw_mg.cuh -- kernels of the geometric multigrid V-cycle on cell-wise data (Sec. 3 and Sec. 5).
//
// Levels are uniform refinements: child c = bx + 2 by + 4 bz of coarse cell (cx, cy, cz) is fine
// cell (2cx+bx, 2cy+by, 2cz+bz), every level numbered lexicographically (x fastest). A CTA takes CP
// consecutive coarse cells; the children of one parent with the same (by, bz) are two adjacent fine
// cells, and those of consecutive parents of a row follow each other, so both sides stream in
// contiguous spans without reordering the levels.
//
// Transfers (Algorithms prolongation and restriction): per parent the 3D child operator is the
// Kronecker product P_bz x P_by x P_bx of the 1D matrices P_b[i][a] = l_a((g_i + b)/2), applied
// axis by axis (sum factorisation): prolongation z, then y, then x, fanning 1 -> 2 -> 4 -> 8 blocks;
// restriction the transposes z, y, x, summing the children 8 -> 4 -> 2 -> 1.
// Intermediate blocks live in shared memory.
#pragma once
#include "cw_apply.cuh"

namespace cw {

template <int N, class C>
struct TabTransfer {
    C P[2][N][N];  // P[b][i][a] = l_a((g_i + b) / 2)
};

// coarse cells per CTA of the transfer kernels (threads: 8 N^2 CP for prolongation, 4 N^2 CP for
// restriction)
template <int N>
constexpr int prolong_cp()
{
    return N == 2 ? 8 : N == 3 ? 4 : N == 4 ? 2 : 1;
}
template <int N>
constexpr int restrict_cp()
{
    return N == 2 ? 16 : N == 3 ? 4 : N == 4 ? 4 : N <= 6 ? 2 : 1;
}

__device__ __forceinline__ int64_t child_cell(int64_t e, int nx, int ny, int ch)
{
    const int64_t cx = e % nx, cy = (e / nx) % ny, cz = e / ((int64_t)nx * ny);
    const int bx = ch & 1, by = (ch >> 1) & 1, bz = ch >> 2;
    return (2 * cx + bx) + 2 * (int64_t)nx * ((2 * cy + by) + 2 * (int64_t)ny * (2 * cz + bz));
}

// uf|K_c (+)= (P_bz x P_by x P_bx) uc|K for every child c of the coarse cells of this CTA.
// ADD: add into uf (the V-cycle's u += P e), else overwrite (Algorithm prolongation into a zeroed
// vector). nx, ny: coarse cells per direction. The axes are contracted z, y, x, so that the last phase
// owns whole x-lines of a child: each thread writes N contiguous values, consecutive threads the
// consecutive lines of one child (the Kronecker factors commute).
template <int N, int CP, class Ar, class VS, bool ADD>
__global__ void __launch_bounds__(8 * N * N * CP) prolong_kernel(const VS *__restrict__ uc, VS *__restrict__ uf,
                                                                  int nx, int ny, int64_t ncoarse,
                                                                  TabTransfer<N, typename Ar::C> tab)
{
    using T = typename Ar::T;
    constexpr int N2 = N * N, N3 = N2 * N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *S0 = reinterpret_cast<T *>(smem_raw);  // [CP][N3] coarse values
    T *S1 = S0 + CP * N3;                     // [CP][2][N3] after z (bz)
    T *S2 = S1 + 2 * CP * N3;                 // [CP][4][N3] after y (by + 2 bz)
    const int t = threadIdx.x;
    const int64_t e0 = static_cast<int64_t>(blockIdx.x) * CP;
    const int64_t nval = ncoarse * N3;
    // this thread's fine x-line (last phase): with ADD its old values are loaded first, so that the
    // read overlaps the three contraction phases instead of stalling the store
    const int xc = t / (8 * N2), xr = t - xc * 8 * N2, xch = xr / N2, xjk = xr - xch * N2;
    const int64_t xe = e0 + xc;
    VS *dst = xe < ncoarse ? uf + child_cell(xe, nx, ny, xch) * N3 + xjk * N : nullptr;
    VS old[N];
    if constexpr (ADD) {
#pragma unroll
        for (int i = 0; i < N; ++i) old[i] = dst ? dst[i] : VS(0);
    }
    for (int k = t; k < CP * N3; k += blockDim.x) {
        const int64_t g = e0 * N3 + k;
        S0[k] = g < nval ? Ar::from(ldg_nc(uc + g)) : Ar::zero();
    }
    __syncthreads();
    T in[N], out[N];
    if (t < CP * 2 * N2) {  // z: pencil (i, j) of parent c, child half bz
        const int c = t / (2 * N2), r = t - c * 2 * N2, bz = r / N2, ij = r - bz * N2;
#pragma unroll
        for (int m = 0; m < N; ++m) in[m] = S0[c * N3 + ij + N2 * m];
        contract<N, false, Ar>(tab.P[bz], in, out);
#pragma unroll
        for (int k = 0; k < N; ++k) S1[(c * 2 + bz) * N3 + ij + N2 * k] = out[k];
    }
    __syncthreads();
    if (t < CP * 4 * N2) {  // y: line (i, k) of the quarter q = by + 2 bz
        const int c = t / (4 * N2), r = t - c * 4 * N2, q = r / N2, ik = r - q * N2;
        const int i = ik % N, k = ik / N, by = q & 1, bz = q >> 1;
#pragma unroll
        for (int m = 0; m < N; ++m) in[m] = S1[(c * 2 + bz) * N3 + i + N * m + N2 * k];
        contract<N, false, Ar>(tab.P[by], in, out);
#pragma unroll
        for (int j = 0; j < N; ++j) S2[(c * 4 + q) * N3 + i + N * j + N2 * k] = out[j];
    }
    __syncthreads();
    {  // x: line (j, k) of child ch = bx + 2 by + 4 bz
#pragma unroll
        for (int m = 0; m < N; ++m) in[m] = S2[(xc * 4 + (xch >> 1)) * N3 + xjk * N + m];
        contract<N, false, Ar>(tab.P[xch & 1], in, out);
        if (dst) {
#pragma unroll
            for (int i = 0; i < N; ++i) {
                VS o;
                Ar::to(o, out[i]);
                if constexpr (ADD) dst[i] = old[i] + o;
                else dst[i] = o;
            }
        }
    }
}

// bc|K = sum_c (P_bz x P_by x P_bx)^T (bf - vf)|K_c for the coarse cells of this CTA (Algorithm
// restriction, additive over the children). SUB: the fine residual b - A u is formed from its two
// operands as they are loaded (fused residual restriction, Sec. 5); else vf is not read.
template <int N, int CP, class Ar, class VS, bool SUB>
__global__ void __launch_bounds__(4 * N * N * CP) restrict_kernel(const VS *__restrict__ bf, const VS *__restrict__ vf,
                                                                   VS *__restrict__ bc, int nx, int ny, int64_t ncoarse,
                                                                   TabTransfer<N, typename Ar::C> tab)
{
    using T = typename Ar::T;
    constexpr int N2 = N * N, N3 = N2 * N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *S0 = reinterpret_cast<T *>(smem_raw);  // [CP][8][N3] fine residual of the children
    T *S1 = S0 + 8 * CP * N3;                 // [CP][4][N3] after z (bx + 2 by)
    T *S2 = S1 + 4 * CP * N3;                 // [CP][2][N3] after y (bx)
    const int t = threadIdx.x;
    const int64_t e0 = static_cast<int64_t>(blockIdx.x) * CP;
    // first fine value of each child pair (bx = 0, 1: two adjacent cells) of each parent, -1 past the
    // end; computed once per CTA so that the load loop does no 64-bit index division
    __shared__ int64_t s_base[CP * 4];
    if (t < CP * 4) {
        const int64_t e = e0 + t / 4;
        s_base[t] = e < ncoarse ? child_cell(e, nx, ny, 2 * (t % 4)) * N3 : -1;
    }
    __syncthreads();
    // load: for each parent and child pair one contiguous span of 2 N3 fine values
    for (int k = t; k < CP * 8 * N3; k += blockDim.x) {
        const int q = k / (2 * N3), w = k - q * (2 * N3);  // q = 4 c + pr
        const int64_t base = s_base[q];
        T v = Ar::zero();
        if (base >= 0) {
            v = Ar::from(ldg_nc(bf + base + w));
            if constexpr (SUB) v = Ar::sub(v, Ar::from(ldg_nc(vf + base + w)));
        }
        S0[k] = v;  // k = c 8 N3 + (2 pr + bx) N3 + local
    }
    __syncthreads();
    T in[N], out[N], acc[N];
    if (t < CP * 4 * N2) {  // z: pencil (i, j) of the quarter q = bx + 2 by, both bz
        const int c = t / (4 * N2), r = t - c * 4 * N2, q = r / N2, ij = r - q * N2;
#pragma unroll
        for (int bz = 0; bz < 2; ++bz) {
#pragma unroll
            for (int m = 0; m < N; ++m) in[m] = S0[(c * 8 + q + 4 * bz) * N3 + ij + N2 * m];
            contract<N, true, Ar>(tab.P[bz], in, out);
#pragma unroll
            for (int a = 0; a < N; ++a) acc[a] = bz ? Ar::add(acc[a], out[a]) : out[a];
        }
#pragma unroll
        for (int a = 0; a < N; ++a) S1[(c * 4 + q) * N3 + ij + N2 * a] = acc[a];
    }
    __syncthreads();
    if (t < CP * 2 * N2) {  // y: line (i, cz) of the half bx, both by
        const int c = t / (2 * N2), r = t - c * 2 * N2, bx = r / N2, ik = r - bx * N2;
        const int i = ik % N, k = ik / N;
#pragma unroll
        for (int by = 0; by < 2; ++by) {
#pragma unroll
            for (int m = 0; m < N; ++m) in[m] = S1[(c * 4 + bx + 2 * by) * N3 + i + N * m + N2 * k];
            contract<N, true, Ar>(tab.P[by], in, out);
#pragma unroll
            for (int a = 0; a < N; ++a) acc[a] = by ? Ar::add(acc[a], out[a]) : out[a];
        }
#pragma unroll
        for (int j = 0; j < N; ++j) S2[(c * 2 + bx) * N3 + i + N * j + N2 * k] = acc[j];
    }
    __syncthreads();
    if (t < CP * N2) {  // x: line (j, k) of the parent, both bx
        const int c = t / N2, jk = t - c * N2;
        const int64_t e = e0 + c;
#pragma unroll
        for (int bx = 0; bx < 2; ++bx) {
#pragma unroll
            for (int m = 0; m < N; ++m) in[m] = S2[(c * 2 + bx) * N3 + jk * N + m];
            contract<N, true, Ar>(tab.P[bx], in, out);
#pragma unroll
            for (int a = 0; a < N; ++a) acc[a] = bx ? Ar::add(acc[a], out[a]) : out[a];
        }
        if (e < ncoarse) {
            VS *dst = bc + e * N3 + jk * N;
#pragma unroll
            for (int a = 0; a < N; ++a) Ar::to(dst[a], acc[a]);
        }
    }
}

}  // namespace cw

// ------------------------------------------------------------------------- host launchers ----
// (included by the per-arithmetic units cw_mg_tr_*.cu, after cw_launch.cuh)
namespace cw {

template <int N, class Ar>
TabTransfer<N, typename Ar::C> transfer_tab(const Tables1D &t)
{
    TabTransfer<N, typename Ar::C> tab;
    for (int i = 0; i < N; ++i)
        for (int a = 0; a < N; ++a) {
            tab.P[0][i][a] = MakeC<Ar>::from(t.P0[i][a]);
            tab.P[1][i][a] = MakeC<Ar>::from(t.P1[i][a]);
        }
    return tab;
}

template <int N, class Ar, class VS>
cudaError_t prolong_n(const Op &coarse, const void *uc, void *uf, bool add, cudaStream_t s)
{
    constexpr int CP = prolong_cp<N>();
    const auto tab = transfer_tab<N, Ar>(coarse.tab);
    const size_t smem = 7 * CP * N * N * N * sizeof(typename Ar::T);
    const unsigned grid = (unsigned)((coarse.E + CP - 1) / CP);
    const VS *in = static_cast<const VS *>(uc);
    VS *out = static_cast<VS *>(uf);
    if (add)
        prolong_kernel<N, CP, Ar, VS, true><<<grid, 8 * N * N * CP, smem, s>>>(in, out, coarse.mesh->nx, coarse.mesh->ny,
                                                                              coarse.E, tab);
    else
        prolong_kernel<N, CP, Ar, VS, false><<<grid, 8 * N * N * CP, smem, s>>>(in, out, coarse.mesh->nx,
                                                                               coarse.mesh->ny, coarse.E, tab);
    return cudaGetLastError();
}

template <int N, class Ar, class VS>
cudaError_t restrict_n(const Op &coarse, const void *bf, const void *vf, void *bc, cudaStream_t s)
{
    constexpr int CP = restrict_cp<N>();
    const auto tab = transfer_tab<N, Ar>(coarse.tab);
    const size_t smem = 14 * CP * N * N * N * sizeof(typename Ar::T);
    static size_t opted[kMaxDevices] = {};
    if (cudaError_t e = vf ? ensure_smem(restrict_kernel<N, CP, Ar, VS, true>, smem, opted) : cudaSuccess;
        e != cudaSuccess)
        return e;
    static size_t opted0[kMaxDevices] = {};
    if (cudaError_t e = vf ? cudaSuccess : ensure_smem(restrict_kernel<N, CP, Ar, VS, false>, smem, opted0);
        e != cudaSuccess)
        return e;
    const unsigned grid = (unsigned)((coarse.E + CP - 1) / CP);
    const VS *b = static_cast<const VS *>(bf), *v = static_cast<const VS *>(vf);
    VS *out = static_cast<VS *>(bc);
    if (vf)
        restrict_kernel<N, CP, Ar, VS, true><<<grid, 4 * N * N * CP, smem, s>>>(b, v, out, coarse.mesh->nx,
                                                                                coarse.mesh->ny, coarse.E, tab);
    else
        restrict_kernel<N, CP, Ar, VS, false><<<grid, 4 * N * N * CP, smem, s>>>(b, v, out, coarse.mesh->nx,
                                                                                 coarse.mesh->ny, coarse.E, tab);
    return cudaGetLastError();
}

template <class Ar, class VS>
cudaError_t prolong_degree(const Op &coarse, const void *uc, void *uf, bool add, cudaStream_t s)
{
    switch (coarse.n) {
    case 2: return prolong_n<2, Ar, VS>(coarse, uc, uf, add, s);
    case 3: return prolong_n<3, Ar, VS>(coarse, uc, uf, add, s);
    case 4: return prolong_n<4, Ar, VS>(coarse, uc, uf, add, s);
    case 5: return prolong_n<5, Ar, VS>(coarse, uc, uf, add, s);
    case 6: return prolong_n<6, Ar, VS>(coarse, uc, uf, add, s);
    case 7: return prolong_n<7, Ar, VS>(coarse, uc, uf, add, s);
    case 8: return prolong_n<8, Ar, VS>(coarse, uc, uf, add, s);
    }
    return cudaErrorInvalidValue;
}

template <class Ar, class VS>
cudaError_t restrict_degree(const Op &coarse, const void *bf, const void *vf, void *bc, cudaStream_t s)
{
    switch (coarse.n) {
    case 2: return restrict_n<2, Ar, VS>(coarse, bf, vf, bc, s);
    case 3: return restrict_n<3, Ar, VS>(coarse, bf, vf, bc, s);
    case 4: return restrict_n<4, Ar, VS>(coarse, bf, vf, bc, s);
    case 5: return restrict_n<5, Ar, VS>(coarse, bf, vf, bc, s);
    case 6: return restrict_n<6, Ar, VS>(coarse, bf, vf, bc, s);
    case 7: return restrict_n<7, Ar, VS>(coarse, bf, vf, bc, s);
    case 8: return restrict_n<8, Ar, VS>(coarse, bf, vf, bc, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace cw
