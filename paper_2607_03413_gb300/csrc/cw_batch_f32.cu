// Persistent batched apply, FP32 arithmetic on FP32 vectors and metric.
#include "cw_batch.cuh"
#include "cw_launch.cuh"

#include <algorithm>

namespace cw {

__constant__ BatchTables<float> c_batch_tabs_f32;
template <>
__device__ __forceinline__ const BatchTables<float> &batch_tables<float>()
{
    return c_batch_tabs_f32;
}

__global__ void __launch_bounds__(kBatchThreads, 4) batch_kernel_f32(const BatchProb *__restrict__ probs, int nprob,
                                                                   int64_t nitems, unsigned long long *__restrict__ counter)
{
    batch_body<ArF32, float, float>(probs, nprob, nitems, counter, c_batch_tabs_f32);
}

static float mk(double v) { return static_cast<float>(v); }

template <int N, class C>
static void fill(TabMetric<N, C> &t, const Tables1D *tb)
{
    if (tb) fill_metric_tab<N>(t, *tb, mk);
}

cudaError_t batch_upload_tables_f32(const Tables1D *const tabs[9])
{
    BatchTables<float> h{};
    fill<2>(h.t2, tabs[2]);
    fill<3>(h.t3, tabs[3]);
    fill<4>(h.t4, tabs[4]);
    fill<5>(h.t5, tabs[5]);
    fill<6>(h.t6, tabs[6]);
    fill<7>(h.t7, tabs[7]);
    fill<8>(h.t8, tabs[8]);
    return cudaMemcpyToSymbol(c_batch_tabs_f32, &h, sizeof h);
}

cudaError_t batch_occupancy_f32(size_t smem, int *blocks_per_sm)
{
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(batch_kernel_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, batch_kernel_f32, kBatchThreads, smem);
}

cudaError_t batch_launch_f32(const BatchProb *d_probs, int nprob, int64_t nitems, unsigned long long *counter,
                            size_t smem, int grid, cudaStream_t s)
{
    batch_kernel_f32<<<grid, kBatchThreads, smem, s>>>(d_probs, nprob, nitems, counter);
    return cudaGetLastError();
}

template <int N, int CPB, int STAGE>
static cudaError_t grouped(const Tables1D &tb, const BatchProb *d_probs, int nprob, int64_t nitems,
                           unsigned long long *counter, int kind_max, cudaStream_t s)
{
    (void)tb;  // the tables are in constant memory (uploaded at batch creation)
    // shared memory for the largest metric of the group (kind_max components)
    const size_t smem = metric_smem_bytes<N, CPB, typename ArF32::T, float>(metric_ncomp(kind_max), STAGE);
    auto kern = batch_degree_kernel<N, CPB, ArF32, float, float, STAGE>;
    static size_t opted[kMaxDevices] = {};
    static int per_sm_dev[kMaxDevices] = {};
    int per_sm = 0;
    if (cudaError_t e = ensure_smem_occupancy(kern, smem, N * N * CPB, opted, per_sm_dev, &per_sm); e != cudaSuccess)
        return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t grid = std::min<int64_t>(std::max(1, per_sm) * (int64_t)sms, nitems);
    kern<<<(unsigned)std::max<int64_t>(grid, 1), N * N * CPB, smem, s>>>(d_probs, nprob, nitems, counter);
    return cudaGetLastError();
}

template <int N>
static cudaError_t grouped_n(int alt, int stage, const Tables1D &tb, const BatchProb *d_probs, int nprob,
                             int64_t nitems, unsigned long long *counter, int kind_max, cudaStream_t s)
{
    constexpr int D = cpb_default<N, ArF32>(), A = cpb_alt<N, ArF32>();
    if (alt) return stage == 1 ? grouped<N, A, 1>(tb, d_probs, nprob, nitems, counter, kind_max, s)
                   : stage == 2 ? grouped<N, A, 2>(tb, d_probs, nprob, nitems, counter, kind_max, s)
                                : grouped<N, A, 0>(tb, d_probs, nprob, nitems, counter, kind_max, s);
    return stage == 1 ? grouped<N, D, 1>(tb, d_probs, nprob, nitems, counter, kind_max, s)
           : stage == 2 ? grouped<N, D, 2>(tb, d_probs, nprob, nitems, counter, kind_max, s)
                        : grouped<N, D, 0>(tb, d_probs, nprob, nitems, counter, kind_max, s);
}

cudaError_t batch_degree_launch_f32(int n, int cpb_alt, int stage, const Tables1D &tb, const BatchProb *d_probs,
                                   int nprob, int64_t nitems, unsigned long long *counter, int kind_max,
                                   cudaStream_t s)
{
    switch (n) {
    case 2: return grouped_n<2>(cpb_alt, stage, tb, d_probs, nprob, nitems, counter, kind_max, s);
    case 3: return grouped_n<3>(cpb_alt, stage, tb, d_probs, nprob, nitems, counter, kind_max, s);
    case 4: return grouped_n<4>(cpb_alt, stage, tb, d_probs, nprob, nitems, counter, kind_max, s);
    case 5: return grouped_n<5>(cpb_alt, stage, tb, d_probs, nprob, nitems, counter, kind_max, s);
    case 6: return grouped_n<6>(cpb_alt, stage, tb, d_probs, nprob, nitems, counter, kind_max, s);
    case 7: return grouped_n<7>(cpb_alt, stage, tb, d_probs, nprob, nitems, counter, kind_max, s);
    case 8: return grouped_n<8>(cpb_alt, stage, tb, d_probs, nprob, nitems, counter, kind_max, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace cw
