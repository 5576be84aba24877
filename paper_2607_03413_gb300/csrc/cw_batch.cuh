// cw_batch.cuh -- one persistent launch that applies many operators (uneven meshes, mixed degrees,
// several right-hand sides each) to their vectors.
//
// Single mode: work items are (problem, chunk of tiles, right-hand side) with the right-hand side
// fastest, so the R items of one chunk run at nearly the same time and its metric comes from HBM once
// and from L2 for the other R-1. Grouped mode: items are (problem, chunk of tiles), and an item runs all
// R right-hand sides through every tile with the tile's metric staged in shared memory once. A chunk holds about kItemValues cell-wise values, enough work to hide the
// per-item cost (an atomicAdd on the global counter, a search of the problem table). Each CTA
// (128 threads) fetches the number of its next item while it works on the current one; an item
// number past the end ends the CTA (no spinning). The tile size is chosen per degree: the largest
// number of cells whose N*N threads fit in the CTA, or half of it (the remaining cell slots compute
// on zeros). The 1D tables of every degree live in constant memory.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "cw_apply.cuh"
#include "cw_internal.h"

namespace cw {

constexpr int kBatchThreads = 128;
constexpr int kItemValues = 16384;  // target cell-wise values per work item

// cells per tile of degree N (n = N nodes): full or half
__host__ __device__ constexpr int batch_cpt(int N, int half)
{
    return half ? (kBatchThreads / (N * N)) / 2 : kBatchThreads / (N * N);
}
// cell slots the 256 threads cover
__host__ __device__ constexpr int batch_slots(int N) { return (kBatchThreads + N * N - 1) / (N * N); }

struct BatchProb {
    const void *x;      // nrhs vectors of length stride
    void *y;
    const void *geo;    // metric [E][ncomp][n^3]
    int64_t ncells;
    int64_t stride;     // cell-wise length E * n^3
    int64_t item0;      // first work item of this problem (items: chunk * nrhs + rhs)
    int64_t ntiles;     // tiles of cpt cells
    unsigned *status;   // the operator's device status word (an expired bounded wait is recorded there)
    int n, kind, nrhs, cpt, tpi;  // tpi: tiles per chunk
};

template <class C>
struct BatchTables {
    TabMetric<2, C> t2;
    TabMetric<3, C> t3;
    TabMetric<4, C> t4;
    TabMetric<5, C> t5;
    TabMetric<6, C> t6;
    TabMetric<7, C> t7;
    TabMetric<8, C> t8;
};

template <int N, class C>
__device__ __forceinline__ const TabMetric<N, C> &batch_tab(const BatchTables<C> &T)
{
    if constexpr (N == 2) return T.t2;
    else if constexpr (N == 3) return T.t3;
    else if constexpr (N == 4) return T.t4;
    else if constexpr (N == 5) return T.t5;
    else if constexpr (N == 6) return T.t6;
    else if constexpr (N == 7) return T.t7;
    else return T.t8;
}

// one work item of degree N; kept out of line so that each degree gets its own register allocation
// (all seven bodies inlined into one function spill heavily)
template <class Ar, class VS, class GS, int N>
__device__ __noinline__ void batch_item(const BatchProb &P, const BatchTables<typename Ar::C> &T, int64_t local,
                                        unsigned char *smem)
{
    const int64_t chunk = local / P.nrhs, rhs = local - chunk * P.nrhs;
    const VS *x = static_cast<const VS *>(P.x) + rhs * P.stride;
    VS *y = static_cast<VS *>(P.y) + rhs * P.stride;
    const GS *g = static_cast<const GS *>(P.geo);
    const int64_t t0 = chunk * P.tpi, t1 = min(P.ntiles, t0 + P.tpi);
    for (int64_t tile = t0; tile < t1; ++tile) {
        if (tile > t0) __syncthreads();  // the previous tile has finished with shared memory
        // kBatchThreads threads, not N*N*slots: lines stay in thread order (slots past cpt are idle)
        metric_tile<N, batch_slots(N), Ar, VS, GS, 0, false, false, false, false>(
            x, y, g, P.ncells, P.kind, batch_tab<N>(T), tile, P.cpt, smem, nullptr, 0, nullptr, nullptr, P.status);
    }
}

template <class Ar, class VS, class GS>
__device__ __forceinline__ void batch_body(const BatchProb *__restrict__ probs, int nprob, int64_t nitems,
                                           unsigned long long *__restrict__ counter,
                                           const BatchTables<typename Ar::C> &T)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long s_next;
    __shared__ int s_prob;
    if (threadIdx.x == 0) s_next = static_cast<long long>(atomicAdd(counter, 1ull));
    for (;;) {
        __syncthreads();
        const long long it = s_next;
        if (it >= nitems) return;  // block-uniform
        __syncthreads();           // every thread has read s_next
        if (threadIdx.x == 0) {
            s_next = static_cast<long long>(atomicAdd(counter, 1ull));  // next item, used after this one
            int lo = 0, hi = nprob - 1;
            while (lo < hi) {  // last problem whose first item is <= it
                const int mid = (lo + hi + 1) / 2;
                if (__ldg(&probs[mid].item0) <= it) lo = mid;
                else hi = mid - 1;
            }
            s_prob = lo;
        }
        __syncthreads();
        const BatchProb P = probs[s_prob];
        const int64_t local = it - P.item0;
        switch (P.n) {
        case 2: batch_item<Ar, VS, GS, 2>(P, T, local, smem_raw); break;
        case 3: batch_item<Ar, VS, GS, 3>(P, T, local, smem_raw); break;
        case 4: batch_item<Ar, VS, GS, 4>(P, T, local, smem_raw); break;
        case 5: batch_item<Ar, VS, GS, 5>(P, T, local, smem_raw); break;
        case 6: batch_item<Ar, VS, GS, 6>(P, T, local, smem_raw); break;
        case 7: batch_item<Ar, VS, GS, 7>(P, T, local, smem_raw); break;
        default: batch_item<Ar, VS, GS, 8>(P, T, local, smem_raw); break;
        }
    }
}

// the constant-memory tables of one arithmetic's units (specialised where they are defined)
template <class C>
__device__ __forceinline__ const BatchTables<C> &batch_tables();

// One tile of the grouped mode, kept out of line for double-float arithmetic: inlined into the
// persistent item loop, its 1D tables (loop-invariant, two floats per entry) were hoisted into
// registers, which took the kernel from ~80 to 128-166 registers; out of line every table entry
// stays an immediate constant-bank operand, as in the per-operator kernel. (FP32 bodies stay inline:
// the call costs them more than it saves.) gsm: the tile's metric in shared memory (STAGE 3).
template <int N, int CPB, class Ar, class VS, class GS, int STAGE>
__device__ __noinline__ void grouped_tile(const VS *x, VS *y, const GS *g, int64_t ncells, int kind, int64_t tile,
                                          unsigned *status, const GS *gsm)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    metric_tile<N, CPB, Ar, VS, GS, STAGE>(x, y, g, ncells, kind, batch_tab<N>(batch_tables<typename Ar::C>()), tile,
                                           CPB, smem_raw, nullptr, 0, nullptr, nullptr, status, 0, gsm);
}

template <int N, int CPB, class Ar, class VS, class GS, int STAGE>
__device__ __forceinline__ void grouped_one(const VS *x, VS *y, const GS *g, int64_t ncells, int kind, int64_t tile,
                                            unsigned *status, const GS *gsm, unsigned char *smem_raw)
{
    if constexpr (std::is_same<Ar, ArDF>::value)
        grouped_tile<N, CPB, Ar, VS, GS, STAGE>(x, y, g, ncells, kind, tile, status, gsm);
    else
        metric_tile<N, CPB, Ar, VS, GS, STAGE>(x, y, g, ncells, kind, batch_tab<N>(batch_tables<typename Ar::C>()),
                                               tile, CPB, smem_raw, nullptr, 0, nullptr, nullptr, status, 0, gsm);
}

// ---- grouped mode: one persistent kernel per degree, shaped like the per-operator kernel
// (N*N*CPB threads) over the problems of that degree. STAGE 1: work items are (problem, chunk of
// tiles), and an item runs every right-hand side of its problem through each tile with the tile's
// metric moved into shared memory once (a bulk copy on an mbarrier, bounded wait), so a problem with
// R right-hand sides reads its metric from HBM once instead of R times; the right-hand sides' input is
// read directly. STAGE 0 and 2: the per-operator kernel's modes, items (problem, chunk, right-hand
// side) with the right-hand side fastest (the metric of a chunk read again from L2 for each).
template <int N, int CPB, class Ar, class VS, class GS, int STAGE>
__global__ void __launch_bounds__(N *N *CPB) batch_degree_kernel(const BatchProb *__restrict__ probs, int nprob,
                                                                  int64_t nitems, unsigned long long *__restrict__ counter)
{
    using T = typename Ar::T;
    constexpr int N3 = N * N * N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long s_next;
    __shared__ int s_prob;
    // STAGE 1 layout: [line buffers][mbarrier, 16 B][metric tile]
    const size_t offb = 3 * TileLines<N, CPB, sizeof(T), true>::RS * sizeof(T);  // a multiple of 16
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + offb);
    GS *sG = reinterpret_cast<GS *>(smem_raw + offb + 16);
    if (threadIdx.x == 0) s_next = static_cast<long long>(atomicAdd(counter, 1ull));
    for (;;) {
        __syncthreads();
        const long long it = s_next;
        if (it >= nitems) return;  // block-uniform
        __syncthreads();
        if (threadIdx.x == 0) {
            s_next = static_cast<long long>(atomicAdd(counter, 1ull));
            int lo = 0, hi = nprob - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) / 2;
                if (__ldg(&probs[mid].item0) <= it) lo = mid;
                else hi = mid - 1;
            }
            s_prob = lo;
        }
        __syncthreads();
        const BatchProb P = probs[s_prob];
        const int64_t local = it - P.item0;
        // STAGE 1: item = chunk, every right-hand side inside; else item = (chunk, right-hand side),
        // right-hand side fastest, so that one item streams consecutive tiles of one vector
        const int64_t chunk = STAGE == 1 ? local : local / P.nrhs;
        const int r0 = STAGE == 1 ? 0 : static_cast<int>(local - chunk * P.nrhs);
        const int r1 = STAGE == 1 ? P.nrhs : r0 + 1;
        const GS *g = static_cast<const GS *>(P.geo);
        const int64_t t0 = chunk * P.tpi, t1 = min(P.ntiles, t0 + P.tpi);
        const int NC = metric_ncomp(P.kind);
        for (int64_t tile = t0; tile < t1; ++tile) {
            if (tile > t0) __syncthreads();  // the previous tile has finished with shared memory
            bool staged = false;
            if constexpr (STAGE == 1) {
                const int64_t cell0 = tile * CPB;
                const GS *gsrc = g + cell0 * NC * N3;
                const uint32_t gb = CPB * NC * N3 * sizeof(GS);
                staged = cell0 + CPB <= P.ncells && aligned16(gsrc) && gb % 16 == 0;  // block-uniform
                if (staged) {
                    if (threadIdx.x == 0) mbar_init(bar, 1);
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        mbar_expect_tx(bar, gb);
                        bulk_g2s(sG, gsrc, gb, bar);
                    }
                    const bool ok = mbar_wait_bounded(bar, 0, kWaitLimit);
                    if (!ok) {  // reported; the copy is waited for once more, the tile reads from global memory
                        if (P.status) atomicOr(P.status, kDevStatusTimeout);
                        mbar_wait_bounded(bar, 0, kWaitLimit);
                    }
                    staged = !__syncthreads_or(!ok);
                }
            }
            for (int r = r0; r < r1; ++r) {
                if (r > r0) __syncthreads();  // the previous right-hand side has finished with the line buffers
                const VS *x = static_cast<const VS *>(P.x) + r * P.stride;
                VS *y = static_cast<VS *>(P.y) + r * P.stride;
                if constexpr (STAGE == 1) {  // one code path: the metric from shared or from global memory
                    const GS *gm = staged ? sG : g + tile * CPB * NC * N3;
                    grouped_one<N, CPB, Ar, VS, GS, 3>(x, y, g, P.ncells, P.kind, tile, P.status, gm, smem_raw);
                } else {
                    grouped_one<N, CPB, Ar, VS, GS, STAGE>(x, y, g, P.ncells, P.kind, tile, P.status, nullptr, smem_raw);
                }
            }
        }
    }
}

// per-unit launchers of the grouped mode (variant: cells per CTA choice 0/1, staging mode 0/1/2)
cudaError_t batch_degree_launch_df(int n, int cpb_alt, int stage, const Tables1D &tb, const BatchProb *d_probs,
                                   int nprob, int64_t nitems, unsigned long long *counter, int kind_max,
                                   cudaStream_t s);
cudaError_t batch_degree_launch_f32(int n, int cpb_alt, int stage, const Tables1D &tb, const BatchProb *d_probs,
                                    int nprob, int64_t nitems, unsigned long long *counter, int kind_max,
                                    cudaStream_t s);
// cells per CTA of the grouped kernel for degree n (same choices as the per-operator kernel)
inline int degree_cpb(int n, int alt, bool f32)
{
    return alt ? tile_cells(n, f32) / 2 : tile_cells(n, f32);
}

// shared memory one item of degree n needs (all cell slots of the CTA)
template <class T>
inline size_t batch_smem_bytes(int n)
{
    switch (n) {  // the three line buffers of metric_tile in this mode (lines in thread order)
    case 2: return metric_smem_bytes<2, batch_slots(2), T, float, false>(0, 0);
    case 3: return metric_smem_bytes<3, batch_slots(3), T, float, false>(0, 0);
    case 4: return metric_smem_bytes<4, batch_slots(4), T, float, false>(0, 0);
    case 5: return metric_smem_bytes<5, batch_slots(5), T, float, false>(0, 0);
    case 6: return metric_smem_bytes<6, batch_slots(6), T, float, false>(0, 0);
    case 7: return metric_smem_bytes<7, batch_slots(7), T, float, false>(0, 0);
    default: return metric_smem_bytes<8, batch_slots(8), T, float, false>(0, 0);
    }
}

// per-unit entry points (cw_batch_df.cu: double-float on FP64 data; cw_batch_f32.cu: FP32)
cudaError_t batch_upload_tables_df(const Tables1D *const tabs[9]);
cudaError_t batch_upload_tables_f32(const Tables1D *const tabs[9]);
cudaError_t batch_launch_df(const BatchProb *d_probs, int nprob, int64_t nitems, unsigned long long *counter,
                            size_t smem, int grid, cudaStream_t s);
cudaError_t batch_launch_f32(const BatchProb *d_probs, int nprob, int64_t nitems, unsigned long long *counter,
                             size_t smem, int grid, cudaStream_t s);
cudaError_t batch_occupancy_df(size_t smem, int *blocks_per_sm);
cudaError_t batch_occupancy_f32(size_t smem, int *blocks_per_sm);

}  // namespace cw
