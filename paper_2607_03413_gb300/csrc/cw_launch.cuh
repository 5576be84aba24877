// cw_launch.cuh -- host launchers for the apply kernels: table conversion, tile size per degree,
// shared-memory opt-in, and the (degree, kind, geometry) dispatch used by the cw_inst_*.cu units.
#pragma once
#include <cuda_runtime.h>

#include "cw_apply.cuh"
#include "cw_internal.h"

namespace cw {

template <class Ar>
struct MakeC;
template <>
struct MakeC<ArDF> {
    static df64 from(double v)
    {
        const float h = static_cast<float>(v);
        return df64{h, static_cast<float>(v - static_cast<double>(h))};
    }
};
template <>
struct MakeC<ArF64> {
    static double from(double v) { return v; }
};
template <>
struct MakeC<ArF32> {
    static float from(double v) { return static_cast<float>(v); }
};

// cells per CTA: about 128-200 threads per CTA
template <int N>
constexpr int cells_per_cta()
{
    return N == 2 ? 32 : N == 3 ? 16 : N == 4 ? 8 : N == 5 ? 8 : N == 6 ? 4 : N == 7 ? 4 : 2;
}

template <class K>
static cudaError_t opt_in_smem(K kernel, size_t smem)
{
    if (smem <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int N, class Ar, class VS, class GS, int KIND>
cudaError_t launch_metric(const Op &op, const void *x, void *y, cudaStream_t s)
{
    constexpr int CPB = cells_per_cta<N>();
    TabMetric<N, typename Ar::C> tab;
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
            tab.B[a][b] = MakeC<Ar>::from(op.tab.B[a][b]);
            tab.D[a][b] = MakeC<Ar>::from(op.tab.D[a][b]);
        }
    const size_t smem = 3 * CPB * Lines<N>::CS * sizeof(typename Ar::T);
    auto kern = apply_metric_kernel<N, CPB, Ar, VS, GS, KIND>;
    static cudaError_t attr = opt_in_smem(kern, smem);
    if (attr != cudaSuccess) return attr;
    const unsigned grid = (unsigned)((op.E + CPB - 1) / CPB);
    kern<<<grid, N * N * CPB, smem, s>>>(static_cast<const VS *>(x), static_cast<VS *>(y),
                                         static_cast<const GS *>(op.d_geo), op.E, tab);
    return cudaGetLastError();
}

template <int N, class Ar, class VS, int KIND>
cudaError_t launch_affine(const Op &op, const void *x, void *y, cudaStream_t s)
{
    constexpr int CPB = cells_per_cta<N>();
    TabAffine<N, typename Ar::C> tab;
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
            tab.M[a][b] = MakeC<Ar>::from(op.tab.M1[a][b]);
            tab.K[a][b] = MakeC<Ar>::from(op.tab.K1[a][b]);
        }
    const size_t smem = 2 * CPB * Lines<N>::CS * sizeof(typename Ar::T);
    auto kern = apply_affine_kernel<N, CPB, Ar, VS, KIND>;
    static cudaError_t attr = opt_in_smem(kern, smem);
    if (attr != cudaSuccess) return attr;
    const unsigned grid = (unsigned)((op.E + CPB - 1) / CPB);
    kern<<<grid, N * N * CPB, smem, s>>>(static_cast<const VS *>(x), static_cast<VS *>(y),
                                         static_cast<const double *>(op.d_geo), op.E, tab);
    return cudaGetLastError();
}

template <int N, class Ar, class VS, class GS>
cudaError_t launch_kind(const Op &op, const void *x, void *y, cudaStream_t s)
{
    if (op.geom == CW_GEOM_AFFINE) {
        switch (op.kind) {
        case 1: return launch_affine<N, Ar, VS, 1>(op, x, y, s);
        case 2: return launch_affine<N, Ar, VS, 2>(op, x, y, s);
        default: return launch_affine<N, Ar, VS, 3>(op, x, y, s);
        }
    }
    switch (op.kind) {
    case 1: return launch_metric<N, Ar, VS, GS, 1>(op, x, y, s);
    case 2: return launch_metric<N, Ar, VS, GS, 2>(op, x, y, s);
    default: return launch_metric<N, Ar, VS, GS, 3>(op, x, y, s);
    }
}

template <class Ar, class VS, class GS>
cudaError_t launch_degree(const Op &op, const void *x, void *y, cudaStream_t s)
{
    switch (op.n) {
    case 2: return launch_kind<2, Ar, VS, GS>(op, x, y, s);
    case 3: return launch_kind<3, Ar, VS, GS>(op, x, y, s);
    case 4: return launch_kind<4, Ar, VS, GS>(op, x, y, s);
    case 5: return launch_kind<5, Ar, VS, GS>(op, x, y, s);
    case 6: return launch_kind<6, Ar, VS, GS>(op, x, y, s);
    case 7: return launch_kind<7, Ar, VS, GS>(op, x, y, s);
    case 8: return launch_kind<8, Ar, VS, GS>(op, x, y, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace cw
