// cw_batch.cu -- C ABI of the batched apply: many operators (uneven meshes, mixed degrees,
// several right-hand sides each) applied by persistent work-queue kernels, optionally replayed
// from a captured CUDA graph, with the kernel variant of each degree picked by an autotuner.
// Two modes: CW_BATCH_GROUPED (default) runs one persistent kernel per degree present, each shaped
// like the tuned per-operator kernel; CW_BATCH_SINGLE runs every degree in one persistent kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "cw_batch.cuh"

namespace cw {

struct Batch {
    std::vector<Op *> ops;  // sorted by degree (stable)
    std::vector<int> nrhs;
    std::vector<const void *> x;
    std::vector<void *> y;
    int fp64 = 1;  // 1: CW_PREC_F64 (double-float), 0: CW_PREC_F32
    int mode = CW_BATCH_GROUPED;
    int half[9] = {0};     // single mode: half tile per n
    int variant[9] = {0};  // grouped mode: cells-per-CTA choice + 2 * staging, per n
    std::vector<BatchProb> h_probs;
    BatchProb *d_probs = nullptr;
    unsigned long long *d_counter = nullptr;  // [9]: single mode uses [0], grouped mode [n]
    int64_t nitems = 0, values = 0;
    int64_t g_first[9] = {0}, g_count[9] = {0}, g_items[9] = {0};  // grouped: problems and items per n
    int g_kind[9] = {0};                                              // grouped: largest kind per n
    const Tables1D *tabs[9] = {nullptr};
    size_t smem = 0;
    int grid = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    // grouped mode: the degree groups run on their own streams, forked from and joined to the
    // caller's stream, so that one group's CTAs fill the SMs another group's tail leaves idle
    cudaStream_t g_stream[9] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[9] = {};
};

static void batch_free(Batch *b)
{
    // launches still in flight (on the caller's stream or the group streams) read d_probs and
    // d_counter: let them finish before the memory goes back
    cudaDeviceSynchronize();
    if (b->graph) cudaGraphExecDestroy(b->graph);
    cudaFree(b->d_probs);
    cudaFree(b->d_counter);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (int n = 0; n < 9; ++n) {
        if (b->g_stream[n]) cudaStreamDestroy(b->g_stream[n]);
        if (b->ev_join[n]) cudaEventDestroy(b->ev_join[n]);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    delete b;
}

static cw_status batch_rebuild(Batch &b)
{
    b.h_probs.resize(b.ops.size());
    int64_t item = 0;
    b.values = 0;
    size_t smem = 0;
    for (int n = 0; n < 9; ++n) {
        b.g_first[n] = b.g_count[n] = b.g_items[n] = 0;
        b.g_kind[n] = 0;
    }
    for (size_t i = 0; i < b.ops.size(); ++i) {
        const Op &o = *b.ops[i];
        BatchProb &P = b.h_probs[i];
        P.x = b.x[i];
        P.y = b.y[i];
        P.geo = o.d_geo;
        P.status = o.d_status;
        P.ncells = o.E;
        P.stride = o.L;
        P.n = o.n;
        P.kind = o.kind;
        P.nrhs = b.nrhs[i];
        P.cpt = b.mode == CW_BATCH_SINGLE ? batch_cpt(o.n, b.half[o.n]) : degree_cpb(o.n, b.variant[o.n] & 1, !b.fp64);
        P.ntiles = (o.E + P.cpt - 1) / P.cpt;
        // grouped items with the metric staged once (staging mode 1) carry every right-hand side of
        // their tiles: fewer tiles per item
        const bool all_rhs = b.mode == CW_BATCH_GROUPED && (b.variant[o.n] >> 1) == 1;
        const int rh = all_rhs ? P.nrhs : 1;
        P.tpi = std::max(1, kItemValues / (P.cpt * o.n * o.n * o.n * rh));
        if (b.mode == CW_BATCH_GROUPED && b.g_count[o.n] == 0) {  // items restart per degree group
            b.g_first[o.n] = (int64_t)i;
            item = 0;
        }
        P.item0 = item;
        item += (P.ntiles + P.tpi - 1) / P.tpi * (all_rhs ? 1 : P.nrhs);
        b.values += o.L * b.nrhs[i];
        b.g_count[o.n] += 1;
        b.g_items[o.n] = item;
        b.g_kind[o.n] = (b.g_kind[o.n] | o.kind);
        smem = std::max(smem, b.fp64 ? batch_smem_bytes<df64>(o.n) : batch_smem_bytes<float>(o.n));
    }
    b.nitems = item;
    b.smem = smem;
    if (b.mode == CW_BATCH_SINGLE) {
        int per_sm = 0, dev = 0, sms = 0;
        CW_CUDA_TRY(b.fp64 ? batch_occupancy_df(smem, &per_sm) : batch_occupancy_f32(smem, &per_sm));
        CW_CUDA_TRY(cudaGetDevice(&dev));
        CW_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        if (per_sm < 1) return fail(CW_ERR_UNSUPPORTED, "cw_batch: kernel does not fit on an SM");
        b.grid = sms * per_sm;
    }
    // the table is rewritten in place: a launch still running on a non-blocking stream, which a
    // synchronous copy does not wait for, may be reading it
    CW_CUDA_TRY(cudaDeviceSynchronize());
    CW_CUDA_TRY(cudaMemcpy(b.d_probs, b.h_probs.data(), b.h_probs.size() * sizeof(BatchProb), cudaMemcpyHostToDevice));
    if (b.graph) {
        cudaGraphExecDestroy(b.graph);
        b.graph = nullptr;
    }
    return CW_OK;
}

// only >= 2 (grouped mode): enqueue that degree's kernel alone (the tuner times a degree in isolation:
// the degrees run concurrently on their own streams, and timing one degree's variants inside the whole
// batch left its differences below the run-to-run spread of the batch)
static cudaError_t batch_enqueue(const Batch &b, cudaStream_t s, int only = 0)
{
    cudaError_t e = cudaMemsetAsync(b.d_counter, 0, 9 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (b.mode == CW_BATCH_SINGLE)
        return b.fp64 ? batch_launch_df(b.d_probs, (int)b.h_probs.size(), b.nitems, b.d_counter, b.smem, b.grid, s)
                      : batch_launch_f32(b.d_probs, (int)b.h_probs.size(), b.nitems, b.d_counter, b.smem, b.grid, s);
    if ((e = cudaEventRecord(b.ev_fork, s)) != cudaSuccess) return e;
    for (int n = 2; n <= 8; ++n) {
        if (!b.g_count[n] || (only && n != only)) continue;
        const int v = b.variant[n];
        const int kmax = (b.g_kind[n] & 1) ? 3 : 2;  // metric components of the largest kind present
        cudaStream_t gs = b.g_stream[n];
        if ((e = cudaStreamWaitEvent(gs, b.ev_fork, 0)) != cudaSuccess) return e;
        e = b.fp64 ? batch_degree_launch_df(n, v & 1, v >> 1, *b.tabs[n], b.d_probs + b.g_first[n], (int)b.g_count[n],
                                            b.g_items[n], b.d_counter + n, kmax, gs)
                   : batch_degree_launch_f32(n, v & 1, v >> 1, *b.tabs[n], b.d_probs + b.g_first[n], (int)b.g_count[n],
                                             b.g_items[n], b.d_counter + n, kmax, gs);
        if (e != cudaSuccess) return e;
        if ((e = cudaEventRecord(b.ev_join[n], gs)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s, b.ev_join[n], 0)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace cw

using namespace cw;

extern "C" {

cw_status cw_batch_create(const cw_op *ops, const int *nrhs, const void *const *x, void *const *y, int nprob,
                          cw_batch *out)
{
    if (!out) return fail(CW_ERR_ARG, "cw_batch_create: out is NULL");
    *out = nullptr;
    if (!ops || !nrhs || !x || !y || nprob < 1) return fail(CW_ERR_ARG, "cw_batch_create: NULL array or nprob < 1");
    Batch *b = new Batch;
    const Tables1D *tabs[9] = {nullptr};
    std::vector<int> order(nprob);
    for (int i = 0; i < nprob; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        const Op *oa = reinterpret_cast<const Op *>(ops[a]), *oc = reinterpret_cast<const Op *>(ops[c]);
        return (oa ? oa->n : 0) < (oc ? oc->n : 0);
    });
    for (int k = 0; k < nprob; ++k) {
        const int i = order[k];
        Op *o = reinterpret_cast<Op *>(ops[i]);
        if (!o || !x[i] || !y[i] || nrhs[i] < 1) {
            delete b;
            return fail(CW_ERR_ARG, "cw_batch_create: NULL operator or vector, or nrhs < 1");
        }
        if (o->geom != CW_GEOM_METRIC || (o->prec != CW_PREC_F64 && o->prec != CW_PREC_F32)) {
            delete b;
            return fail(CW_ERR_UNSUPPORTED, "cw_batch_create: operators must be CW_GEOM_METRIC, CW_PREC_F64 or CW_PREC_F32");
        }
        const int f = o->prec == CW_PREC_F64;
        if (k == 0) b->fp64 = f;
        if (f != b->fp64) {
            delete b;
            return fail(CW_ERR_ARG, "cw_batch_create: all operators must share one precision");
        }
        if (x[i] == y[i]) {
            delete b;
            return fail(CW_ERR_ARG, "cw_batch_create: x and y must not alias");
        }
        b->ops.push_back(o);
        b->nrhs.push_back(nrhs[i]);
        b->x.push_back(x[i]);
        b->y.push_back(y[i]);
        tabs[o->n] = &o->tab;
        b->tabs[o->n] = &o->tab;
    }
    cudaError_t e = b->fp64 ? batch_upload_tables_df(tabs) : batch_upload_tables_f32(tabs);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_probs, nprob * sizeof(BatchProb));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, 9 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    for (int n = 2; n <= 8 && e == cudaSuccess; ++n) {
        e = cudaStreamCreateWithFlags(&b->g_stream[n], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[n], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_fail(e, "cw_batch_create");
    }
    cw_status st = batch_rebuild(*b);
    if (st != CW_OK) {
        batch_free(b);
        return st;
    }
    *out = reinterpret_cast<cw_batch>(b);
    return CW_OK;
}

cw_status cw_batch_destroy(cw_batch bh)
{
    Batch *b = reinterpret_cast<Batch *>(bh);
    if (!b) return fail(CW_ERR_ARG, "cw_batch_destroy: NULL");
    batch_free(b);
    return CW_OK;
}

int64_t cw_batch_values(cw_batch bh)
{
    Batch *b = reinterpret_cast<Batch *>(bh);
    return b ? b->values : -1;
}

cw_status cw_batch_set_mode(cw_batch bh, int mode)
{
    Batch *b = reinterpret_cast<Batch *>(bh);
    if (!b || (mode != CW_BATCH_GROUPED && mode != CW_BATCH_SINGLE))
        return fail(CW_ERR_ARG, "cw_batch_set_mode: NULL handle or unknown mode");
    b->mode = mode;
    return batch_rebuild(*b);
}

static int variant_count(const Batch &b) { return b.mode == CW_BATCH_SINGLE ? 2 : 6; }

cw_status cw_batch_set_variant(cw_batch bh, int degree, int variant)
{
    Batch *b = reinterpret_cast<Batch *>(bh);
    if (!b || degree < 1 || degree > kMaxDegree || variant < 0 || variant >= variant_count(*b))
        return fail(CW_ERR_ARG, "cw_batch_set_variant: NULL handle, degree outside 1..7 or variant out of range");
    if (b->mode == CW_BATCH_SINGLE) b->half[degree + 1] = variant;
    else b->variant[degree + 1] = variant;
    return batch_rebuild(*b);
}

cw_status cw_batch_get_variant(cw_batch bh, int degree, int *variant, int *cells_per_tile)
{
    Batch *b = reinterpret_cast<Batch *>(bh);
    if (!b || degree < 1 || degree > kMaxDegree) return fail(CW_ERR_ARG, "cw_batch_get_variant: bad arguments");
    const int n = degree + 1;
    if (variant) *variant = b->mode == CW_BATCH_SINGLE ? b->half[n] : b->variant[n];
    if (cells_per_tile)
        *cells_per_tile = b->mode == CW_BATCH_SINGLE ? batch_cpt(n, b->half[n]) : degree_cpb(n, b->variant[n] & 1, !b->fp64);
    return CW_OK;
}

cw_status cw_batch_launch(cw_batch bh, void *stream)
{
    cw::Range nvtx_range("cwfem:cw_batch_launch");
    Batch *b = reinterpret_cast<Batch *>(bh);
    if (!b) return fail(CW_ERR_ARG, "cw_batch_launch: NULL handle");
    CW_CUDA_TRY(batch_enqueue(*b, static_cast<cudaStream_t>(stream)));
    return CW_OK;
}

cw_status cw_batch_graph_launch(cw_batch bh, void *stream)
{
    cw::Range nvtx_range("cwfem:cw_batch_graph_launch");
    Batch *b = reinterpret_cast<Batch *>(bh);
    if (!b) return fail(CW_ERR_ARG, "cw_batch_graph_launch: NULL handle");
    if (!b->graph) {
        cudaGraph_t g;
        CW_CUDA_TRY(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = batch_enqueue(*b, b->cap_stream);
        cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
        if (e != cudaSuccess) return cuda_fail(e, "cw_batch_graph_launch capture");
        if (e2 != cudaSuccess) return cuda_fail(e2, "cw_batch_graph_launch end capture");
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "cw_batch_graph_launch instantiate");
    }
    CW_CUDA_TRY(cudaGraphLaunch(b->graph, static_cast<cudaStream_t>(stream)));
    return CW_OK;
}

cw_status cw_batch_autotune(cw_batch bh, int reps, void *stream, float *best_ms)
{
    cw::Range nvtx_range("cwfem:cw_batch_autotune");
    Batch *b = reinterpret_cast<Batch *>(bh);
    if (!b || reps < 1) return fail(CW_ERR_ARG, "cw_batch_autotune: NULL handle or reps < 1");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    bool present[9] = {false};
    for (Op *o : b->ops) present[o->n] = true;
    struct Events {  // destroyed on every return path
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        ~Events()
        {
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
        }
    } ev;
    CW_CUDA_TRY(cudaEventCreate(&ev.e0));
    CW_CUDA_TRY(cudaEventCreate(&ev.e1));
    cudaEvent_t e0 = ev.e0, e1 = ev.e1;
    // time `reps` launches (after one warm-up) of the batch, or of degree `only` alone
    auto timed = [&](int only, float *ms) -> cudaError_t {
        cudaError_t e = batch_enqueue(*b, s, only);
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = batch_enqueue(*b, s, only);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
        *ms /= reps;
        return e;
    };
    for (int n = 2; n <= 8; ++n) {  // coordinate descent over the degrees present
        if (!present[n]) continue;
        float best = 1e30f;
        int bh_ = 0;
        int *knob = b->mode == CW_BATCH_SINGLE ? &b->half[n] : &b->variant[n];
        for (int h = 0; h < variant_count(*b); ++h) {
            *knob = h;
            cw_status st = batch_rebuild(*b);
            if (st != CW_OK) return st;
            float ms = 0.0f;
            CW_CUDA_TRY(timed(b->mode == CW_BATCH_GROUPED ? n : 0, &ms));
            if (ms < best) {
                best = ms;
                bh_ = h;
            }
        }
        *knob = bh_;
    }
    cw_status st = batch_rebuild(*b);
    if (st != CW_OK) return st;
    float all_ms = 0.0f;
    CW_CUDA_TRY(timed(0, &all_ms));
    if (best_ms) *best_ms = all_ms;
    for (Op *o : b->ops)
        if ((st = op_status_take(o, static_cast<cudaStream_t>(stream), "cw_batch_autotune")) != CW_OK) return st;
    return CW_OK;
}

cw_status cw_apply_batched(const cw_op *ops, const void *const *x, void *const *y, const int *nrhs, int nprob,
                           int flags, void *stream)
{
    cw::Range nvtx_range("cwfem:cw_apply_batched");
    if (flags != CW_APPLY_LOCAL && flags != CW_APPLY_ASSEMBLE)
        return fail(CW_ERR_ARG, "cw_apply_batched: flags must be CW_APPLY_LOCAL or CW_APPLY_ASSEMBLE");
    cw_batch b = nullptr;
    cw_status st = cw_batch_create(ops, nrhs, x, y, nprob, &b);
    if (st != CW_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = cw_batch_launch(b, stream);
    for (int i = 0; st == CW_OK && flags == CW_APPLY_ASSEMBLE && i < nprob; ++i) {
        const Op *o = reinterpret_cast<const Op *>(ops[i]);
        const size_t bytes = (size_t)o->L * (o->prec == CW_PREC_F64 ? sizeof(double) : sizeof(float));
        for (int r = 0; st == CW_OK && r < nrhs[i]; ++r)
            st = cw_dss(ops[i], static_cast<char *>(y[i]) + r * bytes, CW_DSS_SUM, stream);
    }
    const cudaError_t e = cudaStreamSynchronize(s);
    cw_batch_destroy(b);
    if (st != CW_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "cw_apply_batched");
    for (int i = 0; i < nprob; ++i)  // an expired bounded wait left a tile without output
        if ((st = op_status_take(reinterpret_cast<Op *>(ops[i]), s, "cw_apply_batched")) != CW_OK) return st;
    return CW_OK;
}

}  // extern "C"
