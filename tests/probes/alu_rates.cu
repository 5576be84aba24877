// Throughput probe for the roofline denominators of the double-float operator: FP32 FMA (scalar
// and paired FFMA2), native FP64 FMA, and the double-float multiply-add (TwoProduct + TwoSum, 12 FP32
// instructions). Independent FMA chains per thread, 8 CTAs of 256 threads per SM, CUDA events; every
// loop has a fixed trip count and every store is in bounds.
#include <cstdio>
#include <cuda_runtime.h>

constexpr int kIters = 4096;

__global__ void k_f32(float *out, float a, float b)
{
    float x[8];
    for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 1e-3f + i;
    for (int it = 0; it < kIters; ++it)
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, b);
    float s = 0.0f;
    for (int i = 0; i < 8; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_f32x2(float *out, float a, float b)
{
    float2 x[4];
    for (int i = 0; i < 4; ++i) x[i] = make_float2(threadIdx.x * 1e-3f + 2 * i, threadIdx.x * 1e-3f + 2 * i + 1);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int it = 0; it < kIters; ++it)
#pragma unroll
        for (int i = 0; i < 4; ++i) x[i] = __ffma2_rn(x[i], a2, b2);
    float s = 0.0f;
    for (int i = 0; i < 4; ++i) s += x[i].x + x[i].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_f64(double *out, double a, double b)
{
    double x[8];
    for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 1e-3 + i;
    for (int it = 0; it < kIters / 16; ++it)
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
    double s = 0.0;
    for (int i = 0; i < 8; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

struct DF {
    float h, l;
};

// s += x * b, b = (bh, bl): exact product of the leading parts, TwoSum into s, low parts lazily
__device__ __forceinline__ void df_mad(DF &s, DF x, float bh, float bl)
{
    const float p = x.h * bh;
    float e = fmaf(x.h, bh, -p);
    e = fmaf(x.h, bl, e);
    e = fmaf(x.l, bh, e);
    const float t = s.h + p, v = t - s.h;
    const float w = (s.h - (t - v)) + (p - v);
    s.l = s.l + (w + e);
    s.h = t;
}

__global__ void k_df(float *out, float bh, float bl)
{
    DF s[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    DF x = {threadIdx.x * 1e-3f, 1e-11f};
    for (int it = 0; it < kIters / 8; ++it) {
        df_mad(s[0], x, bh, bl);
        df_mad(s[1], x, bh, -bl);
        df_mad(s[2], x, -bh, bl);
        df_mad(s[3], x, -bh, -bl);
        x.h += 1e-3f;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s[0].h + s[1].h + s[2].h + s[3].h + s[0].l + s[1].l + s[2].l + s[3].l;
}

// FP64 -> (hi, lo) float pair with conversion instructions (F2F, on the FP64 pipe) and a DADD
__global__ void k_split(float *out, const double *in)
{
    double v = in[threadIdx.x];  // in holds blockDim.x values
    float acc = 0.0f;
    for (int it = 0; it < kIters / 16; ++it) {
        const float h = (float)v;
        const float l = (float)(v - (double)h);
        acc += h + l;
        v += 1e-9;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

static float timed(void (*launch)(void), cudaEvent_t a, cudaEvent_t b)
{
    launch();  // warm-up
    cudaEventRecord(a);
    launch();
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
}

static int g_blocks, g_threads;
static float *g_o32;
static double *g_o64, *g_in;

int main()
{
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
    g_blocks = nsm * 8;
    g_threads = 256;
    const double n = (double)g_blocks * g_threads;
    if (cudaMalloc(&g_o32, (size_t)n * sizeof(float)) != cudaSuccess) return 1;
    if (cudaMalloc(&g_o64, (size_t)n * sizeof(double)) != cudaSuccess) return 1;
    if (cudaMalloc(&g_in, g_threads * sizeof(double)) != cudaSuccess) return 1;
    cudaMemset(g_in, 0, g_threads * sizeof(double));
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const float t32 = timed([] { k_f32<<<g_blocks, g_threads>>>(g_o32, 1.0001f, 0.5f); }, a, b);
    const float t32x2 = timed([] { k_f32x2<<<g_blocks, g_threads>>>(g_o32, 1.0001f, 0.5f); }, a, b);
    const float t64 = timed([] { k_f64<<<g_blocks, g_threads>>>(g_o64, 1.0001, 0.5); }, a, b);
    const float tdf = timed([] { k_df<<<g_blocks, g_threads>>>(g_o32, 1.0001f, 1e-9f); }, a, b);
    const float tsp = timed([] { k_split<<<g_blocks, g_threads>>>(g_o32, g_in); }, a, b);
    printf("SMs %d\n", nsm);
    printf("fp32_fma_tflops %.2f\n", 2.0 * 8 * kIters * n / t32 / 1e9);
    printf("fp32_ffma2_tflops %.2f\n", 2.0 * 8 * kIters * n / t32x2 / 1e9);
    printf("fp64_dfma_tflops %.3f\n", 2.0 * 8 * (kIters / 16) * n / t64 / 1e9);
    printf("df64_mad_tper_s %.3f\n", 4.0 * (kIters / 8) * n / tdf / 1e9);
    printf("f2f_split_gper_s %.1f\n", 1.0 * (kIters / 16) * n / tsp / 1e6);
    const cudaError_t e = cudaGetLastError();
    printf("status %s\n", cudaGetErrorString(e));
    return e == cudaSuccess ? 0 : 1;
}
