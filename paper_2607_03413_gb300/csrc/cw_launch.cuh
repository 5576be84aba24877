// cw_launch.cuh -- host launchers for the apply kernels: table conversion, tile size per degree,
// shared-memory opt-in, and the (degree, tile, staging) dispatch used by the cw_inst_*.cu units.
#pragma once
#include <cuda_runtime.h>

#include <mutex>
#include <type_traits>

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

// lane pair (a, b) of two double-float constants (host side)
inline df64p pair(df64 a, df64 b)
{
    df64p p;
    p.hi.x = a.hi;
    p.hi.y = b.hi;
    p.lo.x = a.lo;
    p.lo.y = b.lo;
    return p;
}

// fills the full and even-odd forms of B and D from the double tables
template <int N, class C, class MK>
void fill_metric_tab(TabMetric<N, C> &t, const Tables1D &tb, MK mk)
{
    double B[N][N], Bt[N][N], D[N][N], Dt[N][N];
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
            B[a][b] = tb.B[a][b];
            Bt[a][b] = tb.B[b][a];
            D[a][b] = tb.D[a][b];
            Dt[a][b] = tb.D[b][a];
            t.B[a][b] = mk(tb.B[a][b]);
            t.D[a][b] = mk(tb.D[a][b]);
        }
    auto eo = [&](EOMat<N, C> &E, const double (&M)[N][N]) {
        constexpr int H = N / 2, NA = (N + 1) / 2;
        for (int a = 0; a < NA; ++a) {
            for (int b = 0; b < (H > 0 ? H : 1); ++b) {
                E.E[a][b] = mk(b < H ? 0.5 * (M[a][b] + M[a][N - 1 - b]) : 0.0);
                E.O[a][b] = mk(b < H ? 0.5 * (M[a][b] - M[a][N - 1 - b]) : 0.0);
            }
            E.Mid[a] = mk((N % 2 == 1) ? M[a][H] : 0.0);
            if constexpr (std::is_same<C, df64>::value) {
                for (int b = 0; b < (H > 0 ? H : 1); ++b) E.P[a][b] = pair(E.E[a][b], E.O[a][b]);
                E.PM[a] = pair(E.Mid[a], df64{0.0f, 0.0f});
            }
            if constexpr (std::is_same<C, float>::value) {
                for (int b = 0; b < (H > 0 ? H : 1); ++b) {
                    E.P[a][b].x = E.E[a][b];
                    E.P[a][b].y = E.O[a][b];
                }
                E.PM[a].x = E.Mid[a];
                E.PM[a].y = 0.0f;
            }
        }
    };
    eo(t.Bf, B);
    eo(t.Bt, Bt);
    eo(t.Df, D);
    eo(t.Dt, Dt);
    for (int a = 0; a < N; ++a) {
        t.xq[a] = mk(tb.xq[a]);
        t.wq[a] = mk(tb.wq[a]);
    }
}

// storage type of the recomputed geometry's coefficients: float pairs for the FP64 arithmetics,
// float for FP32 arithmetic (whatever the vector and metric storage)
template <class Ar>
struct RCStore {
    using type = df64s;
};
template <>
struct RCStore<ArF32> {
    using type = float;
};

// cells per CTA of an arithmetic's curved kernels (tile_cells): the default and the alternative the
// tuner can pick
template <int N, class Ar>
constexpr int cpb_default()
{
    return tile_cells(N, std::is_same<Ar, ArF32>::value);
}
template <int N, class Ar>
constexpr int cpb_alt()
{
    return cpb_default<N, Ar>() / 2;
}

template <class K>
static cudaError_t opt_in_smem(K kernel, size_t smem)
{
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    if (smem <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Dynamic shared-memory opt-in of one kernel instantiation, done once per device and size:
// `opted[dev]` records the largest size opted in on device dev. The lock keeps host threads that
// create or launch operators concurrently from racing on that record.
constexpr int kMaxDevices = 64;
inline std::mutex &smem_opt_mutex()
{
    static std::mutex m;
    return m;
}
template <class K>
static cudaError_t ensure_smem(K kernel, size_t smem, size_t (&opted)[kMaxDevices])
{
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;  // past the per-CTA limit
    if (smem <= 48 * 1024) return cudaSuccess;                     // no opt-in needed
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return opt_in_smem(kernel, smem);
    std::lock_guard<std::mutex> lock(smem_opt_mutex());
    if (smem <= opted[dev]) return cudaSuccess;
    e = opt_in_smem(kernel, smem);
    if (e == cudaSuccess) opted[dev] = smem;
    return e;
}

// The same for persistent kernels, which also need their resident CTAs per SM at that size:
// per_sm[dev] is recomputed whenever a larger size is opted in.
template <class K>
static cudaError_t ensure_smem_occupancy(K kernel, size_t smem, int threads, size_t (&opted)[kMaxDevices],
                                         int (&per_sm)[kMaxDevices], int *out_per_sm)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(smem_opt_mutex());
    if (smem > opted[dev] || per_sm[dev] == 0) {
        e = opt_in_smem(kernel, smem);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[dev], kernel, threads, smem);
        if (e != cudaSuccess) return e;
        if (smem > opted[dev]) opted[dev] = smem;
    }
    *out_per_sm = per_sm[dev];
    return cudaSuccess;
}

// xfuse != nullptr: the kernel also applies the x pass of the DSS inside each tile and *xfuse
// receives the tile size (cells), so the DSS x pass only has the interfaces between tiles left
// the plain or the register-capped instantiation (only the one used is compiled)
template <int N, int CPB, class Ar, class VS, class GS, int STAGE, bool RC>
constexpr auto metric_kernel_ptr()
{
    if constexpr (df_capped<Ar, N, RC>()) return apply_metric_kernel_capped<N, CPB, Ar, VS, GS, STAGE, RC>;
    else return apply_metric_kernel<N, CPB, Ar, VS, GS, STAGE, RC>;
}

template <int N, int CPB, class Ar, class VS, class GS, int STAGE, bool RC = false>
cudaError_t launch_metric(const Op &op, const void *x, void *y, cudaStream_t s, int *xfuse = nullptr)
{
    TabMetric<N, typename Ar::C> tab;
    fill_metric_tab<N>(tab, op.tab, [](double v) { return MakeC<Ar>::from(v); });
    const size_t smem = metric_smem_bytes<N, CPB, typename Ar::T, GS>(metric_ncomp(op.kind), STAGE);
    auto kern = metric_kernel_ptr<N, CPB, Ar, VS, GS, STAGE, RC>();
    static size_t opted[kMaxDevices] = {};  // largest size opted in so far, per device
    if (cudaError_t e = ensure_smem(kern, smem, opted); e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((op.E + CPB - 1) / CPB);
    if (xfuse) *xfuse = CPB;
    kern<<<grid, N * N * CPB, smem, s>>>(static_cast<const VS *>(x), static_cast<VS *>(y),
                                         static_cast<const GS *>(op.d_geo), op.E, op.kind, tab,
                                         xfuse ? op.mesh->nx : 0, op.d_status, op.dbg_tma_extra);
    return cudaGetLastError();
}

// One fused smoothing sweep (smooth_metric_kernel): default tile, input tile staged by TMA and the
// metric prefetched into L2 (stage 2); the x-interfaces inside tiles are averaged, *xfuse receives the
// tile size for the x pass between tiles.
template <int N, class Ar, class VS, class GS, bool RC>
cudaError_t launch_smooth(const Op &op, void *u, const void *b, const void *dhat, cudaStream_t s, int *xfuse)
{
    constexpr int CPB = cpb_default<N, Ar>();
    TabMetric<N, typename Ar::C> tab;
    fill_metric_tab<N>(tab, op.tab, [](double v) { return MakeC<Ar>::from(v); });
    const size_t smem = metric_smem_bytes<N, CPB, typename Ar::T, GS>(metric_ncomp(op.kind), 2);
    auto kern = smooth_metric_kernel<N, CPB, Ar, VS, GS, 2, RC>;
    static size_t opted[kMaxDevices] = {};
    if (cudaError_t e = ensure_smem(kern, smem, opted); e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((op.E + CPB - 1) / CPB);
    *xfuse = CPB;
    kern<<<grid, N * N * CPB, smem, s>>>(static_cast<VS *>(u), static_cast<const VS *>(b),
                                         static_cast<const VS *>(dhat), static_cast<const GS *>(op.d_geo), op.E,
                                         op.kind, tab, op.mesh->nx, op.d_status, op.dbg_tma_extra);
    return cudaGetLastError();
}

template <class Ar, class VS, class GS>
cudaError_t launch_smooth_degree(const Op &op, void *u, const void *b, const void *dhat, cudaStream_t s, int *xfuse)
{
    using GC = typename RCStore<Ar>::type;
    const bool rc = op.geom == CW_GEOM_RECOMPUTE;
#define CW_SM(NN) \
    return rc ? launch_smooth<NN, Ar, VS, GC, true>(op, u, b, dhat, s, xfuse) \
              : launch_smooth<NN, Ar, VS, GS, false>(op, u, b, dhat, s, xfuse)
    switch (op.n) {
    case 2: CW_SM(2);
    case 3: CW_SM(3);
    case 4: CW_SM(4);
    case 5: CW_SM(5);
    case 6: CW_SM(6);
    case 7: CW_SM(7);
    case 8: CW_SM(8);
    }
#undef CW_SM
    return cudaErrorInvalidValue;
}

// y = A x with the CTA partials of <x, y> written to part (default tile size, TMA staging);
// *nblocks receives the number of partials
template <int N, class Ar, class VS, class GS, bool RC = false>
cudaError_t launch_metric_dot(const Op &op, const void *x, void *y, double *part, int64_t *nblocks, cudaStream_t s)
{
    constexpr int CPB = cpb_default<N, Ar>(), ST = RC ? 2 : 1;
    TabMetric<N, typename Ar::C> tab;
    fill_metric_tab<N>(tab, op.tab, [](double v) { return MakeC<Ar>::from(v); });
    const size_t smem = metric_smem_bytes<N, CPB, typename Ar::T, GS>(metric_ncomp(op.kind), ST);
    auto kern = apply_metric_dot_kernel<N, CPB, Ar, VS, GS, ST, RC>;
    static size_t opted[kMaxDevices] = {};  // largest size opted in so far, per device
    if (cudaError_t e = ensure_smem(kern, smem, opted); e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((op.E + CPB - 1) / CPB);
    *nblocks = grid;
    kern<<<grid, N * N * CPB, smem, s>>>(static_cast<const VS *>(x), static_cast<VS *>(y),
                                         static_cast<const GS *>(op.d_geo), op.E, op.kind, tab, part, op.d_status,
                                         op.dbg_tma_extra);
    return cudaGetLastError();
}

template <class Ar, class VS, class GS, bool RC>
cudaError_t launch_dot_degree_rc(const Op &op, const void *x, void *y, double *part, int64_t *nb, cudaStream_t s)
{
    switch (op.n) {
    case 2: return launch_metric_dot<2, Ar, VS, GS, RC>(op, x, y, part, nb, s);
    case 3: return launch_metric_dot<3, Ar, VS, GS, RC>(op, x, y, part, nb, s);
    case 4: return launch_metric_dot<4, Ar, VS, GS, RC>(op, x, y, part, nb, s);
    case 5: return launch_metric_dot<5, Ar, VS, GS, RC>(op, x, y, part, nb, s);
    case 6: return launch_metric_dot<6, Ar, VS, GS, RC>(op, x, y, part, nb, s);
    case 7: return launch_metric_dot<7, Ar, VS, GS, RC>(op, x, y, part, nb, s);
    case 8: return launch_metric_dot<8, Ar, VS, GS, RC>(op, x, y, part, nb, s);
    }
    return cudaErrorInvalidValue;
}

template <class Ar, class VS, class GS>
cudaError_t launch_dot_degree(const Op &op, const void *x, void *y, double *part, int64_t *nb, cudaStream_t s)
{
    if (op.geom == CW_GEOM_RECOMPUTE)
        return launch_dot_degree_rc<Ar, VS, typename RCStore<Ar>::type, true>(op, x, y, part, nb, s);
    return launch_dot_degree_rc<Ar, VS, GS, false>(op, x, y, part, nb, s);
}

template <int N, int CPB, class Ar, class VS>
cudaError_t launch_affine(const Op &op, const void *x, void *y, cudaStream_t s)
{
    TabAffine<N, typename Ar::C> tab;
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
            tab.M[a][b] = MakeC<Ar>::from(op.tab.M1[a][b]);
            tab.K[a][b] = MakeC<Ar>::from(op.tab.K1[a][b]);
        }
    const size_t smem = 2 * CPB * Lines<N>::CS * sizeof(typename Ar::T);
    auto kern = apply_affine_kernel<N, CPB, Ar, VS>;
    static size_t opted[kMaxDevices] = {};  // largest size opted in so far, per device
    if (cudaError_t e = ensure_smem(kern, smem, opted); e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((op.E + CPB - 1) / CPB);
    kern<<<grid, N * N * CPB, smem, s>>>(static_cast<const VS *>(x), static_cast<VS *>(y),
                                         static_cast<const double *>(op.d_geo), op.E, op.kind, tab);
    return cudaGetLastError();
}

// variant selection: op.cpb (0 = default, else cpb_default or cpb_alt), op.stage (0/1); GC is the
// storage type of the recomputed geometry's coefficients
template <int N, class Ar, class VS, class GS, bool ALL_VARIANTS, class GC>
cudaError_t launch_variant(const Op &op, const void *x, void *y, cudaStream_t s, int *xfuse)
{
    constexpr int D = cpb_default<N, Ar>(), A = cpb_alt<N, Ar>();
    if (op.geom == CW_GEOM_AFFINE) {  // no fused DSS work: *xfuse stays 0
        if constexpr (ALL_VARIANTS)
            if (op.cpb == A) return launch_affine<N, A, Ar, VS>(op, x, y, s);
        return launch_affine<N, D, Ar, VS>(op, x, y, s);
    }
    if (op.geom == CW_GEOM_RECOMPUTE) {  // default tile; direct loads or a TMA-staged input tile
        if constexpr (ALL_VARIANTS)
            if (op.stage != 0) return launch_metric<N, D, Ar, VS, GC, 2, true>(op, x, y, s, xfuse);
        return launch_metric<N, D, Ar, VS, GC, 0, true>(op, x, y, s, xfuse);
    }
    if constexpr (ALL_VARIANTS) {
        const bool alt = (op.cpb == A);
        if (op.stage == 1) return alt ? launch_metric<N, A, Ar, VS, GS, 1>(op, x, y, s, xfuse)
                                      : launch_metric<N, D, Ar, VS, GS, 1>(op, x, y, s, xfuse);
        if (op.stage == 2) return alt ? launch_metric<N, A, Ar, VS, GS, 2>(op, x, y, s, xfuse)
                                      : launch_metric<N, D, Ar, VS, GS, 2>(op, x, y, s, xfuse);
        return alt ? launch_metric<N, A, Ar, VS, GS, 0>(op, x, y, s, xfuse)
                   : launch_metric<N, D, Ar, VS, GS, 0>(op, x, y, s, xfuse);
    }
    return launch_metric<N, D, Ar, VS, GS, 0>(op, x, y, s, xfuse);
}

template <class Ar, class VS, class GS, bool ALL_VARIANTS = true, class GC = typename RCStore<Ar>::type>
cudaError_t launch_degree(const Op &op, const void *x, void *y, cudaStream_t s, int *xfuse = nullptr)
{
    if (xfuse) *xfuse = 0;
    switch (op.n) {
    case 2: return launch_variant<2, Ar, VS, GS, ALL_VARIANTS, GC>(op, x, y, s, xfuse);
    case 3: return launch_variant<3, Ar, VS, GS, ALL_VARIANTS, GC>(op, x, y, s, xfuse);
    case 4: return launch_variant<4, Ar, VS, GS, ALL_VARIANTS, GC>(op, x, y, s, xfuse);
    case 5: return launch_variant<5, Ar, VS, GS, ALL_VARIANTS, GC>(op, x, y, s, xfuse);
    case 6: return launch_variant<6, Ar, VS, GS, ALL_VARIANTS, GC>(op, x, y, s, xfuse);
    case 7: return launch_variant<7, Ar, VS, GS, ALL_VARIANTS, GC>(op, x, y, s, xfuse);
    case 8: return launch_variant<8, Ar, VS, GS, ALL_VARIANTS, GC>(op, x, y, s, xfuse);
    }
    return cudaErrorInvalidValue;
}

// the two cells-per-CTA choices of degree p
inline void cpb_choices(int p, int prec, int out[2])
{
    out[0] = tile_cells(p + 1, prec_f32_arith(prec));
    out[1] = out[0] / 2;
}

}  // namespace cw
