// cw_mblock.cu -- multi-block meshes: structured blocks glued face to face in any orientation, and the
// unstructured inter-block DSS of Sec. 4.3 (Algorithm unstruct_dss).
//
// The cell-wise vector of a multi-block mesh is the concatenation of its blocks' cell-wise vectors.
// Within a block the structured DSS (Algorithm struct_dss) sums the copies across interior cell faces;
// after it, every copy of a DoF on the block's boundary holds the block's partial sum. The second phase
// couples the blocks: for every DoF shared by several blocks, the sum of one representative copy per
// sharing block is written to all its copies (Algorithm unstruct_dss). The shared DoFs are partitioned
// by the codimension of the block entity they lie on -- macro-face interiors, macro-line interiors,
// macro-vertices -- into three disjoint sets, one launch each.
//
// Orientation: two blocks may meet in any relative orientation. The set-up identifies every node on a
// block boundary by the global ids of its cell's vertices (block-boundary vertices are matched across
// blocks by exact coordinates) and its position in a canonical frame of the cell entity it lies on: an
// edge runs from its smaller vertex id to the larger, a face starts at its smallest-id corner and runs
// first toward the smaller-id neighbour of that corner. Integer arithmetic alone, at set-up; the
// kernels then read plain index tables (the shared DoFs are a lower-dimensional skeleton, so the
// tables are small).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "cw_internal.h"

namespace cw {

// ------------------------------------------------------------------------------ kernels ----
// One entity per thread: s = sum of its representatives (one copy per sharing block, in block order),
// then s to every copy. Entities touch disjoint copies, so the launch needs no atomics.
template <class VS>
struct MbAcc {
    using A = VS;
    static __device__ __forceinline__ A from(VS v) { return v; }
    static __device__ __forceinline__ VS to(A a) { return a; }
};
template <>
struct MbAcc<__nv_bfloat16> {
    using A = float;
    static __device__ __forceinline__ float from(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 to(float a) { return __float2bfloat16_rn(a); }
};

template <class VS>
__global__ void mb_entity_kernel(VS *__restrict__ v, int64_t nent, const int64_t *__restrict__ rptr,
                                 const int64_t *__restrict__ rep, const int64_t *__restrict__ cptr,
                                 const int64_t *__restrict__ cp)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nent) return;
    typename MbAcc<VS>::A s = MbAcc<VS>::from(v[rep[rptr[e]]]);
    for (int64_t r = rptr[e] + 1; r < rptr[e + 1]; ++r) s = s + MbAcc<VS>::from(v[rep[r]]);
    const VS o = MbAcc<VS>::to(s);
    for (int64_t c = cptr[e]; c < cptr[e + 1]; ++c) v[cp[c]] = o;
}

// v[i] /= kappa[i] (the averaging DSS: every copy gets the mean of its DoF's copies)
template <class VS>
__global__ void mb_divide_kernel(VS *__restrict__ v, const uint8_t *__restrict__ kappa, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t k = kappa[i];
        if (k > 1) v[i] = MbAcc<VS>::to(MbAcc<VS>::from(v[i]) / static_cast<typename MbAcc<VS>::A>(k));
    }
}

// ---------------------------------------------------------------------------- structure ----
struct MbSet {  // one codimension set of shared DoFs, CSR tables on the device
    int64_t nent = 0;
    int64_t *rptr = nullptr, *rep = nullptr, *cptr = nullptr, *cp = nullptr;
};

struct MBlock {
    std::vector<Op *> ops;
    std::vector<int64_t> off;  // first cell-wise entry of every block; off.back() = L
    int p = 0, n = 0, prec = 0;
    int64_t L = 0, NG = 0;
    MbSet sets[3];             // macro-face interiors, macro-line interiors, macro-vertices
    uint8_t *kappa = nullptr;  // number of copies of every entry's DoF
    uint8_t *dirichlet = nullptr;  // 1 on entries of DoFs on the domain boundary (unglued block faces)
    std::vector<int64_t> gidx; // global DoF of every entry (host)
    int64_t bytes = 0;
    // solver scratch (FP64), lazily
    double *r = nullptr, *pv = nullptr, *q = nullptr, *z = nullptr, *dinv = nullptr, *part = nullptr, *scal = nullptr;
};

namespace {

struct VKey {  // a block-boundary vertex, by its exact coordinates
    uint64_t b[3];
    bool operator==(const VKey &o) const { return b[0] == o.b[0] && b[1] == o.b[1] && b[2] == o.b[2]; }
};
struct VKeyHash {
    size_t operator()(const VKey &k) const
    {
        uint64_t h = 1469598103934665603ull;
        for (uint64_t x : k.b) h = (h ^ x) * 1099511628211ull;
        return (size_t)h;
    }
};

// A node on a block boundary: type 0 vertex (a = vertex id), 1 edge interior (a < b the end ids, s
// from a), 2 face interior (a the smallest corner, b the first and c the second neighbour in the
// canonical frame, (s, t) in that frame).
struct NKey {
    int type;
    int64_t a, b, c;
    int s, t;
    bool operator<(const NKey &o) const
    {
        if (type != o.type) return type < o.type;
        if (a != o.a) return a < o.a;
        if (b != o.b) return b < o.b;
        if (c != o.c) return c < o.c;
        if (s != o.s) return s < o.s;
        return t < o.t;
    }
};

struct Copy {
    int block;
    int64_t idx;   // cell-wise entry (global over the concatenated vector)
    int codim;     // 1 block face, 2 block edge, 3 block vertex (in this block's own view)
};

template <class T>
cw_status upload(const std::vector<T> &h, T **d, int64_t &bytes)
{
    if (h.empty()) return CW_OK;
    CW_CUDA_TRY(cudaMalloc(d, h.size() * sizeof(T)));
    CW_CUDA_TRY(cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    bytes += (int64_t)(h.size() * sizeof(T));
    return CW_OK;
}

void free_mblock(MBlock *m)
{
    for (MbSet &s : m->sets) {
        cudaFree(s.rptr);
        cudaFree(s.rep);
        cudaFree(s.cptr);
        cudaFree(s.cp);
    }
    cudaFree(m->kappa);
    cudaFree(m->dirichlet);
    for (double *p : {m->r, m->pv, m->q, m->z, m->dinv, m->part, m->scal}) cudaFree(p);
    delete m;
}

}  // namespace

// Builds the inter-block tables, the valences, the Dirichlet flags and the global numbering.
static cw_status mblock_build(MBlock &mb)
{
    const int p = mb.p, n = mb.n, n3 = n * n * n;
    const int nb = (int)mb.ops.size();
    // 1. global ids of block-boundary vertices, matched across blocks by exact coordinates
    std::unordered_map<VKey, int64_t, VKeyHash> vid;
    std::vector<std::vector<int64_t>> bv(nb);  // per block, per vertex: id (-1 inside the block)
    for (int b = 0; b < nb; ++b) {
        const Mesh &m = *mb.ops[b]->mesh;
        const int64_t nv = (int64_t)(m.nx + 1) * (m.ny + 1) * (m.nz + 1);
        bv[b].assign(nv, -1);
        for (int64_t vz = 0; vz <= m.nz; ++vz)
            for (int64_t vy = 0; vy <= m.ny; ++vy)
                for (int64_t vx = 0; vx <= m.nx; ++vx) {
                    if (!(vx == 0 || vx == m.nx || vy == 0 || vy == m.ny || vz == 0 || vz == m.nz)) continue;
                    const int64_t v = (vz * (m.ny + 1) + vy) * (m.nx + 1) + vx;
                    VKey k;
                    std::memcpy(k.b, &m.h_verts[v * 3], 3 * sizeof(double));
                    auto it = vid.find(k);
                    if (it == vid.end()) it = vid.emplace(k, (int64_t)vid.size()).first;
                    bv[b][v] = it->second;
                }
    }
    // 2. keys of all block-boundary nodes, their copies, and the glued cell faces
    std::map<NKey, std::vector<Copy>> nodes;
    std::map<std::array<int64_t, 4>, int> faces;  // sorted corner ids of block-boundary cell faces -> blocks
    mb.gidx.assign(mb.L, -1);
    std::vector<uint8_t> kap(mb.L, 1), dir(mb.L, 0);
    int64_t ng = 0;
    for (int b = 0; b < nb; ++b) {
        const Mesh &m = *mb.ops[b]->mesh;
        const int64_t dims[3] = {m.nx, m.ny, m.nz};
        auto vtx = [&](int64_t x, int64_t y, int64_t z) { return bv[b][(z * (m.ny + 1) + y) * (m.nx + 1) + x]; };
        // block-interior nodes: a structured number each (p-lattice points not on the block boundary)
        const int64_t gx = dims[0] * p + 1, gy = dims[1] * p + 1;
        for (int64_t e = 0; e < m.ncells(); ++e) {
            const int64_t c[3] = {e % m.nx, (e / m.nx) % m.ny, e / ((int64_t)m.nx * m.ny)};
            for (int loc = 0; loc < n3; ++loc) {
                const int l[3] = {loc % n, (loc / n) % n, loc / (n * n)};
                const int64_t X[3] = {c[0] * p + l[0], c[1] * p + l[1], c[2] * p + l[2]};
                const int64_t t = mb.off[b] + e * n3 + loc;
                int cb = 0, cc = 0;  // block-boundary and cell-boundary coordinates
                for (int a = 0; a < 3; ++a) {
                    cb += (X[a] == 0 || X[a] == dims[a] * p);
                    cc += (l[a] == 0 || l[a] == p);
                }
                // structured valence inside the block: 2 per axis on an interior cell interface
                int kv = 1;
                for (int a = 0; a < 3; ++a)
                    if ((l[a] == 0 && c[a] > 0) || (l[a] == p && c[a] < dims[a] - 1)) kv *= 2;
                kap[t] = (uint8_t)kv;
                if (cb == 0) {  // inside the block: numbered per block below (offset added later)
                    mb.gidx[t] = -2 - (X[0] + gx * (X[1] + gy * X[2]));
                    continue;
                }
                NKey k{};
                const int bits[3] = {l[0] == p, l[1] == p, l[2] == p};
                if (cc == 3) {
                    k.type = 0;
                    k.a = vtx(c[0] + bits[0], c[1] + bits[1], c[2] + bits[2]);
                } else if (cc == 2) {
                    int ax = 0;
                    for (int a = 0; a < 3; ++a)
                        if (l[a] != 0 && l[a] != p) ax = a;
                    int64_t e0[3] = {c[0] + bits[0], c[1] + bits[1], c[2] + bits[2]}, e1[3];
                    e0[ax] = c[ax];
                    std::memcpy(e1, e0, sizeof e0);
                    e1[ax] = c[ax] + 1;
                    const int64_t i0 = vtx(e0[0], e0[1], e0[2]), i1 = vtx(e1[0], e1[1], e1[2]);
                    k.type = 1;
                    if (i0 < i1) k.a = i0, k.b = i1, k.s = l[ax];
                    else k.a = i1, k.b = i0, k.s = p - l[ax];
                } else {  // cc == 1: interior of a cell face on the block boundary
                    int f = 0;
                    for (int a = 0; a < 3; ++a)
                        if (l[a] == 0 || l[a] == p) f = a;
                    const int a1 = f == 0 ? 1 : 0, a2 = f == 2 ? 1 : 2;
                    int64_t ids[2][2];  // [u][v] corner ids along (a1, a2)
                    for (int u = 0; u < 2; ++u)
                        for (int w = 0; w < 2; ++w) {
                            int64_t q[3] = {c[0], c[1], c[2]};
                            q[f] += bits[f];
                            q[a1] += u;
                            q[a2] += w;
                            ids[u][w] = vtx(q[0], q[1], q[2]);
                        }
                    int u0 = 0, w0 = 0;
                    for (int u = 0; u < 2; ++u)
                        for (int w = 0; w < 2; ++w)
                            if (ids[u][w] < ids[u0][w0]) u0 = u, w0 = w;
                    const int64_t n1 = ids[1 - u0][w0], n2 = ids[u0][1 - w0];  // neighbours along a1, a2
                    const int s1 = u0 ? p - l[a1] : l[a1], s2 = w0 ? p - l[a2] : l[a2];
                    k.type = 2;
                    k.a = ids[u0][w0];
                    if (n1 < n2) k.b = n1, k.c = n2, k.s = s1, k.t = s2;
                    else k.b = n2, k.c = n1, k.s = s2, k.t = s1;
                }
                nodes[k].push_back(Copy{b, t, cb});
            }
        }
        // block-boundary cell faces, for the glued / domain-boundary decision
        for (int f = 0; f < 3; ++f)
            for (int side = 0; side < 2; ++side) {
                const int a1 = f == 0 ? 1 : 0, a2 = f == 2 ? 1 : 2;
                for (int64_t i1 = 0; i1 < dims[a1]; ++i1)
                    for (int64_t i2 = 0; i2 < dims[a2]; ++i2) {
                        std::array<int64_t, 4> key;
                        int q = 0;
                        for (int u = 0; u < 2; ++u)
                            for (int w = 0; w < 2; ++w) {
                                int64_t v[3];
                                v[f] = side ? dims[f] : 0;
                                v[a1] = i1 + u;
                                v[a2] = i2 + w;
                                key[q++] = vtx(v[0], v[1], v[2]);
                            }
                        std::sort(key.begin(), key.end());
                        faces[key] += 1;
                    }
            }
    }
    // 3. block-interior numbers: per block, a dense count over its interior lattice points
    for (int b = 0; b < nb; ++b) {
        std::unordered_map<int64_t, int64_t> local;
        for (int64_t t = mb.off[b]; t < mb.off[b + 1]; ++t)
            if (mb.gidx[t] <= -2) {
                auto it = local.find(mb.gidx[t]);
                if (it == local.end()) it = local.emplace(mb.gidx[t], ng++).first;
                mb.gidx[t] = it->second;
            }
    }
    // 4. boundary keys: a global number each; inter-block entities into the three sets
    std::vector<int64_t> rptr[3], rep[3], cptr[3], cp[3];
    for (int s = 0; s < 3; ++s) {
        rptr[s].push_back(0);
        cptr[s].push_back(0);
    }
    for (auto &kv : nodes) {
        std::vector<Copy> &c = kv.second;
        const int64_t g = ng++;
        for (const Copy &x : c) mb.gidx[x.idx] = g;
        if (c.size() > 255) return fail(CW_ERR_UNSUPPORTED, "cw_mblock_create: a DoF with more than 255 copies");
        for (const Copy &x : c) kap[x.idx] = (uint8_t)c.size();
        std::stable_sort(c.begin(), c.end(), [](const Copy &u, const Copy &w) { return u.block < w.block; });
        int nblk = 0;
        for (size_t i = 0; i < c.size(); ++i)
            if (i == 0 || c[i].block != c[i - 1].block) ++nblk;
        if (nblk < 2) {  // one block: its structured DSS already sums it; the valence is the block's
            for (const Copy &x : c) kap[x.idx] = 0;  // restored below from the structure
            continue;
        }
        const int set = std::min(3, c[0].codim) - 1;
        for (size_t i = 0; i < c.size(); ++i) {
            if (i == 0 || c[i].block != c[i - 1].block) rep[set].push_back(c[i].idx);
            cp[set].push_back(c[i].idx);
        }
        rptr[set].push_back((int64_t)rep[set].size());
        cptr[set].push_back((int64_t)cp[set].size());
    }
    // entries whose DoF lives in one block keep the structured valence
    for (int b = 0; b < nb; ++b) {
        const Mesh &m = *mb.ops[b]->mesh;
        const int64_t dims[3] = {m.nx, m.ny, m.nz};
        for (int64_t e = 0; e < m.ncells(); ++e) {
            const int64_t c[3] = {e % m.nx, (e / m.nx) % m.ny, e / ((int64_t)m.nx * m.ny)};
            for (int loc = 0; loc < n3; ++loc) {
                const int64_t t = mb.off[b] + e * n3 + loc;
                if (kap[t] != 0) continue;
                const int l[3] = {loc % n, (loc / n) % n, loc / (n * n)};
                int kv = 1;
                for (int a = 0; a < 3; ++a)
                    if ((l[a] == 0 && c[a] > 0) || (l[a] == p && c[a] < dims[a] - 1)) kv *= 2;
                kap[t] = (uint8_t)kv;
            }
        }
    }
    mb.NG = ng;
    // 5. Dirichlet: every node of a block-boundary cell face that no other block shares
    std::vector<uint8_t> gdir(ng, 0);
    for (int b = 0; b < nb; ++b) {
        const Mesh &m = *mb.ops[b]->mesh;
        const int64_t dims[3] = {m.nx, m.ny, m.nz};
        auto vtx = [&](int64_t x, int64_t y, int64_t z) { return bv[b][(z * (m.ny + 1) + y) * (m.nx + 1) + x]; };
        for (int f = 0; f < 3; ++f)
            for (int side = 0; side < 2; ++side) {
                const int a1 = f == 0 ? 1 : 0, a2 = f == 2 ? 1 : 2;
                for (int64_t i1 = 0; i1 < dims[a1]; ++i1)
                    for (int64_t i2 = 0; i2 < dims[a2]; ++i2) {
                        std::array<int64_t, 4> key;
                        int q = 0;
                        for (int u = 0; u < 2; ++u)
                            for (int w = 0; w < 2; ++w) {
                                int64_t v[3];
                                v[f] = side ? dims[f] : 0;
                                v[a1] = i1 + u;
                                v[a2] = i2 + w;
                                key[q++] = vtx(v[0], v[1], v[2]);
                            }
                        std::sort(key.begin(), key.end());
                        if (faces[key] > 1) continue;  // glued to another block
                        int64_t c[3];
                        c[f] = side ? dims[f] - 1 : 0;
                        c[a1] = i1;
                        c[a2] = i2;
                        const int64_t e = c[0] + m.nx * (c[1] + (int64_t)m.ny * c[2]);
                        for (int loc = 0; loc < n3; ++loc) {
                            const int l[3] = {loc % n, (loc / n) % n, loc / (n * n)};
                            if (l[f] == (side ? p : 0)) gdir[mb.gidx[mb.off[b] + e * n3 + loc]] = 1;
                        }
                    }
            }
    }
    for (int64_t t = 0; t < mb.L; ++t) dir[t] = gdir[mb.gidx[t]];
    // 6. device tables
    for (int s = 0; s < 3; ++s) {
        MbSet &S = mb.sets[s];
        S.nent = (int64_t)rptr[s].size() - 1;
        cw_status st;
        if ((st = upload(rptr[s], &S.rptr, mb.bytes)) != CW_OK) return st;
        if ((st = upload(rep[s], &S.rep, mb.bytes)) != CW_OK) return st;
        if ((st = upload(cptr[s], &S.cptr, mb.bytes)) != CW_OK) return st;
        if ((st = upload(cp[s], &S.cp, mb.bytes)) != CW_OK) return st;
    }
    cw_status st;
    if ((st = upload(kap, &mb.kappa, mb.bytes)) != CW_OK) return st;
    if ((st = upload(dir, &mb.dirichlet, mb.bytes)) != CW_OK) return st;
    return CW_OK;
}

template <class VS>
static cudaError_t mb_dss_typed(const MBlock &mb, VS *v, int flags, cudaStream_t s)
{
    for (size_t b = 0; b < mb.ops.size(); ++b) {  // Algorithm struct_dss inside every block
        cudaError_t e = dss_launch(*mb.ops[b], v + mb.off[b], CW_DSS_SUM, s);
        if (e != cudaSuccess) return e;
    }
    for (const MbSet &S : mb.sets)  // Algorithm unstruct_dss: faces, lines, vertices
        if (S.nent > 0)
            mb_entity_kernel<VS><<<(unsigned)((S.nent + 255) / 256), 256, 0, s>>>(v, S.nent, S.rptr, S.rep, S.cptr,
                                                                                   S.cp);
    if (flags == CW_DSS_AVERAGE)
        mb_divide_kernel<VS><<<1216, 256, 0, s>>>(v, mb.kappa, mb.L);
    return cudaGetLastError();
}

static cudaError_t mb_dss(const MBlock &mb, void *v, int flags, cudaStream_t s)
{
    switch (vec_elem_size(mb.prec)) {
    case 8: return mb_dss_typed(mb, static_cast<double *>(v), flags, s);
    case 4: return mb_dss_typed(mb, static_cast<float *>(v), flags, s);
    default: return mb_dss_typed(mb, static_cast<__nv_bfloat16 *>(v), flags, s);
    }
}

static cudaError_t mb_apply_local(const MBlock &mb, const void *x, void *y, cudaStream_t s)
{
    const size_t es = vec_elem_size(mb.prec);
    for (size_t b = 0; b < mb.ops.size(); ++b) {
        cudaError_t e = apply_local(*mb.ops[b], static_cast<const char *>(x) + mb.off[b] * es,
                                    static_cast<char *>(y) + mb.off[b] * es, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ------------------------------------------------------------------ Jacobi-PCG (FP64) ----
// Primal-dual CG of Sec. 4.4 on the concatenated vector, preconditioner z = D^-1 S r with zeros of the
// inverse diagonal on the domain boundary; FP64 dots, one partial per CTA, the partials summed in a
// fixed order by one CTA (so every run gives the same bits). Per iteration: q = A p block by block,
// <p, q>, one pass for u += alpha p, r -= alpha q and z = r, the DSS of z, one pass for the two dots
// around z <- D^-1 z, and the direction update.
constexpr int kMbBlocks = 1216, kMbThreads = 256;

__device__ __forceinline__ double mb_block_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kMbThreads / 32; ++i) t += sh[i];
    __syncthreads();
    return t;
}

// part[block] = sum a_i b_i (mask: only entries with m[i] == 0, if m)
__global__ void __launch_bounds__(kMbThreads) mb_dot_kernel(const double *__restrict__ a, const double *__restrict__ b,
                                                            const uint8_t *__restrict__ m, int64_t n,
                                                            double *__restrict__ part)
{
    __shared__ double sh[kMbThreads / 32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!m || !m[i]) s = fma(a[i], b[i], s);
    s = mb_block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// out[k] = sum of part[k * nb .. k * nb + nb) for k < nsum (one CTA of kMbThreads: strided sums in a
// fixed order, then the fixed tree of mb_block_sum)
__global__ void __launch_bounds__(kMbThreads) mb_sum_kernel(const double *__restrict__ part, int nb, int nsum,
                                                            double *__restrict__ out)
{
    __shared__ double sh[kMbThreads / 32];
    for (int k = 0; k < nsum; ++k) {
        double s = 0.0;
        for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[(int64_t)k * nb + i];
        s = mb_block_sum(s, sh);
        if (threadIdx.x == 0) out[k] = s;
    }
}

// alpha = num / den: u += alpha p, r -= alpha q, z = r (the DSS input)
__global__ void __launch_bounds__(kMbThreads) mb_update_kernel(double *__restrict__ u, double *__restrict__ r,
                                                               double *__restrict__ z, const double *__restrict__ p,
                                                               const double *__restrict__ q,
                                                               const double *__restrict__ num,
                                                               const double *__restrict__ den, int64_t n)
{
    const double a = (*num) / (*den);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        u[i] = fma(a, p[i], u[i]);
        const double ri = fma(-a, q[i], r[i]);
        r[i] = ri;
        z[i] = ri;
    }
}

// z holds S r: part[block] = <m z, r> (m: entries off the domain boundary, dinv != 0), then
// z <- D^-1 z and part[nb + block] = <r, z>
__global__ void __launch_bounds__(kMbThreads) mb_precond_kernel(double *__restrict__ z, const double *__restrict__ r,
                                                                const double *__restrict__ dinv, int64_t n,
                                                                double *__restrict__ part)
{
    __shared__ double sh[kMbThreads / 32];
    double s1 = 0.0, s2 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double di = dinv[i], ri = r[i], zi = z[i];
        if (di != 0.0) s1 = fma(zi, ri, s1);
        const double zn = di * zi;
        z[i] = zn;
        s2 = fma(ri, zn, s2);
    }
    s1 = mb_block_sum(s1, sh);
    s2 = mb_block_sum(s2, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = s1;
        part[gridDim.x + blockIdx.x] = s2;
    }
}

// p = z + (rho_new / rho_old) p
__global__ void mb_pupdate_kernel(double *__restrict__ p, const double *__restrict__ z, const double *__restrict__ num,
                                  const double *__restrict__ den, int64_t n)
{
    const double beta = (*num) / (*den);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = fma(beta, p[i], z[i]);
}

__global__ void mb_dinv_kernel(const double *__restrict__ d, const uint8_t *__restrict__ dir, double *__restrict__ dinv,
                               int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dinv[i] = dir[i] ? 0.0 : 1.0 / d[i];
}

}  // namespace cw

using namespace cw;

extern "C" {

cw_status cw_mblock_create(const cw_op *ops, int nblocks, cw_mblock *out)
{
    cw::Range nvtx_range("cwfem:cw_mblock_create");
    if (!out) return fail(CW_ERR_ARG, "cw_mblock_create: out is NULL");
    *out = nullptr;
    if (!ops || nblocks < 1) return fail(CW_ERR_ARG, "cw_mblock_create: need at least one block");
    const Op *o0 = reinterpret_cast<const Op *>(ops[0]);
    if (!o0) return fail(CW_ERR_ARG, "cw_mblock_create: NULL operator");
    for (int b = 0; b < nblocks; ++b) {
        const Op *o = reinterpret_cast<const Op *>(ops[b]);
        if (!o) return fail(CW_ERR_ARG, "cw_mblock_create: NULL operator");
        if (o->p != o0->p || o->kind != o0->kind || o->prec != o0->prec)
            return fail(CW_ERR_ARG, "cw_mblock_create: blocks differ in degree, kind or precision");
        for (int c = 0; c < b; ++c)
            if (ops[c] == ops[b] || reinterpret_cast<const Op *>(ops[c])->mesh == o->mesh)
                return fail(CW_ERR_ARG, "cw_mblock_create: a block appears twice");
    }
    MBlock *mb = new (std::nothrow) MBlock;
    if (!mb) return fail(CW_ERR_OOM, "cw_mblock_create: host allocation failed");
    mb->p = o0->p;
    mb->n = o0->n;
    mb->prec = o0->prec;
    mb->off.push_back(0);
    for (int b = 0; b < nblocks; ++b) {
        mb->ops.push_back(reinterpret_cast<Op *>(ops[b]));
        mb->off.push_back(mb->off.back() + mb->ops.back()->L);
    }
    mb->L = mb->off.back();
    cw_status st;
    try {
        st = mblock_build(*mb);
    } catch (const std::bad_alloc &) {
        st = fail(CW_ERR_OOM, "cw_mblock_create: host allocation failed");
    }
    if (st != CW_OK) {
        free_mblock(mb);
        return st;
    }
    *out = reinterpret_cast<cw_mblock>(mb);
    return CW_OK;
}

cw_status cw_mblock_destroy(cw_mblock h)
{
    MBlock *mb = reinterpret_cast<MBlock *>(h);
    if (!mb) return fail(CW_ERR_ARG, "cw_mblock_destroy: NULL");
    cudaDeviceSynchronize();
    free_mblock(mb);
    return CW_OK;
}

int64_t cw_mblock_cellwise_len(cw_mblock h)
{
    MBlock *mb = reinterpret_cast<MBlock *>(h);
    return mb ? mb->L : -1;
}

int64_t cw_mblock_global_len(cw_mblock h)
{
    MBlock *mb = reinterpret_cast<MBlock *>(h);
    return mb ? mb->NG : -1;
}

int64_t cw_mblock_shared_dofs(cw_mblock h, int set)
{
    MBlock *mb = reinterpret_cast<MBlock *>(h);
    if (!mb || set < 0 || set > 2) return -1;
    return mb->sets[set].nent;
}

cw_status cw_mblock_global_index(cw_mblock h, int64_t *out)
{
    MBlock *mb = reinterpret_cast<MBlock *>(h);
    if (!mb || !out) return fail(CW_ERR_ARG, "cw_mblock_global_index: NULL argument");
    std::memcpy(out, mb->gidx.data(), mb->L * sizeof(int64_t));
    return CW_OK;
}

cw_status cw_mblock_dss(cw_mblock h, void *v, int flags, void *stream)
{
    MBlock *mb = reinterpret_cast<MBlock *>(h);
    if (!mb || !v) return fail(CW_ERR_ARG, "cw_mblock_dss: NULL argument");
    if (flags != CW_DSS_SUM && flags != CW_DSS_AVERAGE) return fail(CW_ERR_ARG, "cw_mblock_dss: bad flags");
    CW_CUDA_TRY(mb_dss(*mb, v, flags, static_cast<cudaStream_t>(stream)));
    return CW_OK;
}

cw_status cw_mblock_apply(cw_mblock h, const void *x, void *y, int flags, void *stream)
{
    cw::Range nvtx_range("cwfem:cw_mblock_apply");
    MBlock *mb = reinterpret_cast<MBlock *>(h);
    if (!mb || !x || !y) return fail(CW_ERR_ARG, "cw_mblock_apply: NULL argument");
    if (flags != CW_APPLY_LOCAL && flags != CW_APPLY_ASSEMBLE) return fail(CW_ERR_ARG, "cw_mblock_apply: bad flags");
    if (x == y) return fail(CW_ERR_ARG, "cw_mblock_apply: x and y must not alias");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CW_CUDA_TRY(mb_apply_local(*mb, x, y, s));
    if (flags == CW_APPLY_ASSEMBLE) CW_CUDA_TRY(mb_dss(*mb, y, CW_DSS_SUM, s));
    return CW_OK;
}

cw_status cw_mblock_diagonal(cw_mblock h, double *d, void *stream)
{
    MBlock *mb = reinterpret_cast<MBlock *>(h);
    if (!mb || !d) return fail(CW_ERR_ARG, "cw_mblock_diagonal: NULL argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (size_t b = 0; b < mb->ops.size(); ++b) {  // each block's diagonal, assembled inside the block
        cw_status st = cw_diagonal(reinterpret_cast<cw_op>(mb->ops[b]), d + mb->off[b], stream);
        if (st != CW_OK) return st;
    }
    for (const MbSet &S : mb->sets)  // then across the blocks
        if (S.nent > 0)
            mb_entity_kernel<double><<<(unsigned)((S.nent + 255) / 256), 256, 0, s>>>(d, S.nent, S.rptr, S.rep, S.cptr,
                                                                                       S.cp);
    CW_CUDA_TRY(cudaGetLastError());
    return CW_OK;
}

cw_status cw_mblock_cg_solve(cw_mblock h, const double *b, double *u, double rtol, int maxit, cw_cg_stats *stats,
                             void *stream)
{
    cw::Range nvtx_range("cwfem:cw_mblock_cg_solve");
    MBlock *mb = reinterpret_cast<MBlock *>(h);
    if (!mb || !b || !u) return fail(CW_ERR_ARG, "cw_mblock_cg_solve: NULL argument");
    if (mb->prec != CW_PREC_F64) return fail(CW_ERR_ARG, "cw_mblock_cg_solve: the blocks must be CW_PREC_F64");
    if (!(rtol > 0.0) || maxit < 1) return fail(CW_ERR_ARG, "cw_mblock_cg_solve: rtol must be > 0 and maxit >= 1");
    if (b == u) return fail(CW_ERR_ARG, "cw_mblock_cg_solve: b and u must not alias");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t L = mb->L;
    if (!mb->r) {
        for (double **pp : {&mb->r, &mb->pv, &mb->q, &mb->z, &mb->dinv}) CW_CUDA_TRY(cudaMalloc(pp, L * sizeof(double)));
        CW_CUDA_TRY(cudaMalloc(&mb->part, 2 * kMbBlocks * sizeof(double)));
        CW_CUDA_TRY(cudaMalloc(&mb->scal, 8 * sizeof(double)));
        mb->bytes += 5 * L * (int64_t)sizeof(double) + (2 * kMbBlocks + 8) * (int64_t)sizeof(double);
        cw_status st = cw_mblock_diagonal(h, mb->q, stream);
        if (st != CW_OK) return st;
        mb_dinv_kernel<<<kMbBlocks, kMbThreads, 0, s>>>(mb->q, mb->dirichlet, mb->dinv, L);
        CW_CUDA_TRY(cudaGetLastError());
    }
    cudaEvent_t e0, e1;
    CW_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaError_t e = cudaEventCreate(&e1); e != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(e, "cw_mblock_cg_solve");
    }
    struct Ev {
        cudaEvent_t a, b;
        ~Ev()
        {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } ev{e0, e1};
    CW_CUDA_TRY(cudaEventRecord(e0, s));
    double *r = mb->r, *p = mb->pv, *q = mb->q, *z = mb->z, *sc = mb->scal;
    auto dot = [&](const double *a, const double *bb, double *outp) {
        mb_dot_kernel<<<kMbBlocks, kMbThreads, 0, s>>>(a, bb, nullptr, L, mb->part);
        mb_sum_kernel<<<1, kMbThreads, 0, s>>>(mb->part, kMbBlocks, 1, outp);
    };
    auto host = [&](int i, double *v) -> cw_status {
        CW_CUDA_TRY(cudaMemcpyAsync(v, sc + i, sizeof(double), cudaMemcpyDeviceToHost, s));
        CW_CUDA_TRY(cudaStreamSynchronize(s));
        return CW_OK;
    };
    CW_CUDA_TRY(cudaMemsetAsync(u, 0, L * sizeof(double), s));
    CW_CUDA_TRY(cudaMemcpyAsync(r, b, L * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CW_CUDA_TRY(cudaMemcpyAsync(z, b, L * sizeof(double), cudaMemcpyDeviceToDevice, s));
    // z (= r) <- S z; res = <m z, r> (m: not Dirichlet) = ||m G^T r||^2; z <- D^-1 z; rho = <r, z>
    // (res into sc[res_slot], rho into sc[res_slot + 1])
    auto precond = [&](int res_slot) -> cudaError_t {
        cudaError_t e = mb_dss(*mb, z, CW_DSS_SUM, s);
        if (e != cudaSuccess) return e;
        mb_precond_kernel<<<kMbBlocks, kMbThreads, 0, s>>>(z, r, mb->dinv, L, mb->part);
        mb_sum_kernel<<<1, kMbThreads, 0, s>>>(mb->part, kMbBlocks, 2, sc + res_slot);
        return cudaGetLastError();
    };
    // scalars: 0 rho, 1 <p, q>, 2 res and 3 rho_new of an iteration, 4 res0 (5: rho of the start)
    CW_CUDA_TRY(precond(4));
    CW_CUDA_TRY(cudaMemcpyAsync(sc + 0, sc + 5, sizeof(double), cudaMemcpyDeviceToDevice, s));
    CW_CUDA_TRY(cudaMemcpyAsync(p, z, L * sizeof(double), cudaMemcpyDeviceToDevice, s));
    double res0 = 0.0, res = 0.0;
    cw_status st;
    if ((st = host(4, &res0)) != CW_OK) return st;
    res = res0;
    int it = 0;
    cw_status result = CW_OK;
    while (res0 > 0.0 && res > rtol * rtol * res0) {
        if (it >= maxit) {
            result = fail(CW_ERR_NOT_CONVERGED, "cw_mblock_cg_solve: maxit reached");
            break;
        }
        CW_CUDA_TRY(mb_apply_local(*mb, p, q, s));
        dot(p, q, sc + 1);
        mb_update_kernel<<<kMbBlocks, kMbThreads, 0, s>>>(u, r, z, p, q, sc + 0, sc + 1, L);
        CW_CUDA_TRY(precond(2));
        mb_pupdate_kernel<<<kMbBlocks, kMbThreads, 0, s>>>(p, z, sc + 3, sc + 0, L);
        CW_CUDA_TRY(cudaMemcpyAsync(sc + 0, sc + 3, sizeof(double), cudaMemcpyDeviceToDevice, s));
        CW_CUDA_TRY(cudaGetLastError());
        ++it;
        if ((st = host(2, &res)) != CW_OK) return st;
        if (!std::isfinite(res)) {
            result = fail(CW_ERR_BREAKDOWN, "cw_mblock_cg_solve: non-finite residual");
            break;
        }
    }
    CW_CUDA_TRY(cudaEventRecord(e1, s));
    CW_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    for (Op *o : mb->ops)
        if ((st = op_status_take(o, s, "cw_mblock_cg_solve")) != CW_OK) return st;
    if (stats) {
        stats->iterations = it;
        stats->outer_iterations = 1;
        stats->rel_residual = res0 > 0.0 ? std::sqrt(res / res0) : 0.0;
        stats->energy = 0.0;
        stats->seconds = ms * 1e-3;
    }
    return result;
}

}  // extern "C"
