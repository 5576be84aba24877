// cw_apply.cuh -- sum-factorised cell-local operator kernels (the hot path).
//
// One CTA owns a tile of CPB consecutive cells; a cell is worked by N*N threads. A thread plays
// three roles in turn: owner of an x-line (j,k), of a y-line (i,k) and of a z-pencil (i,j), with
// (r % N, r / N) as its pair of indices, r in [0, N*N). 1D contractions along the owned line run
// in registers; switching axis goes through shared memory (the odd row pitch PI = N|1 spreads a
// cell's line accesses over the banks; where two cells share a warp, as at N = 5, some conflicts
// remain). The 1D tables are kernel parameters (constant bank) so every contraction coefficient is
// an immediate operand.
//
// Curved cells (Sec. 6, "the general cell-wise Laplacian: evaluate gradients, apply the physics,
// integrate gradients"), per cell with u the nodal values:
//   u_q = (B x B x B) u                 interpolation to the n^3 Gauss points
//   g   = (D u_q along x, y, z)         reference gradient by Gauss-point collocation
//   h   = G_q g,  m_q = c_q u_q         metric G_q = w_q detJ J^-1 J^-T, c_q = w_q detJ
//   y   = (B^T x B^T x B^T)(D_x^T h_x + D_y^T h_y + D_z^T h_z + m_q)
// Cartesian cells (Sec. 6, the factored form (D x B x B + B x D x B + B x B x D) det J J^-2 read
// with D, B the 1D stiffness and mass matrices):
//   y = a_x (M x M x K) u + a_y (M x K x M) u + a_z (K x M x M) u + a_m (M x M x M) u
// evaluated as two x-contractions, three y-contractions and two z-contractions.
#pragma once
#include <type_traits>

#include "cw_arith.cuh"
#include "cw_tma.cuh"

namespace cw {

// Even-odd form of an N x N matrix M with reflection symmetry M[N-1-a][N-1-b] = s M[a][b]
// (s = +1 for B and B^T, -1 for D and D^T; the Gauss and Gauss-Lobatto points are symmetric about
// 1/2). With e_b = x_b + x_{N-1-b}, o_b = x_b - x_{N-1-b} (b < N/2) and, for odd N, the middle
// entry x_h:  y_a = sum_b E[a][b] e_b + sum_b O[a][b] o_b + Mid[a] x_h  and
// y_{N-1-a} = s (sum_b E[a][b] e_b - sum_b O[a][b] o_b + Mid[a] x_h), for a < (N+1)/2, where
// E[a][b] = (M[a][b] + M[a][N-1-b])/2, O[a][b] = (M[a][b] - M[a][N-1-b])/2, Mid[a] = M[a][h].
// This halves the multiply-adds of a line contraction (Kronbichler and Kormann's even-odd
// decomposition for sum factorisation).
// For double-float tables the same entries are also stored lane-paired, P[a][b] = (E[a][b], O[a][b])
// and PM[a] = (Mid[a], 0), so that the even and odd sums of an output pair run as one paired
// multiply-add chain with each coefficient pair one 64-bit constant operand.
template <class C>
struct EOPair {
    struct type {};
};
template <>
struct EOPair<df64> {
    using type = df64p;
};
template <>
struct EOPair<float> {
    using type = float2;
};

template <int N, class C>
struct EOMat {
    static constexpr int H = N / 2, NA = (N + 1) / 2;
    C E[NA][H > 0 ? H : 1];
    C O[NA][H > 0 ? H : 1];
    C Mid[NA];
    typename EOPair<C>::type P[NA][H > 0 ? H : 1];
    typename EOPair<C>::type PM[NA];
};

template <int N, class C>
struct TabMetric {
    C B[N][N];  // B[q][m] = l_m(xi_q): Gauss-Lobatto basis at the Gauss points
    C D[N][N];  // D[q][r] = derivative at xi_q of the Lagrange basis on the Gauss points
    EOMat<N, C> Bf, Bt, Df, Dt;  // even-odd forms of B, B^T (s = +1), D, D^T (s = -1)
    C xq[N], wq[N];              // Gauss points and weights on [0,1] (recomputed geometry)
};

// Recomputed geometry: per cell the 21 coefficients a1..a7 (3 components each) of the trilinear
// map x(xi) = a0 + a1 xi + a2 eta + a3 zeta + a4 xi eta + a5 xi zeta + a6 eta zeta + a7 xi eta zeta,
// layout [cell][7][3]; a0 is not needed (only derivatives enter the metric).
constexpr int kTriCoef = 21;

template <int N, class C>
struct TabAffine {
    C M[N][N];  // 1D mass matrix of the Gauss-Lobatto basis on [0,1]
    C K[N][N];  // 1D stiffness matrix
};

// small helpers -------------------------------------------------------------------------------

// sum of two stored values as the structured DSS forms it (BF16: FP32 sum rounded once)
template <class VS>
struct AddOp {
    static __device__ __forceinline__ VS add(VS a, VS b) { return a + b; }
};
template <>
struct AddOp<__nv_bfloat16> {
    static __device__ __forceinline__ __nv_bfloat16 add(__nv_bfloat16 a, __nv_bfloat16 b)
    {
        return __float2bfloat16_rn(__bfloat162float(a) + __bfloat162float(b));
    }
};

template <class S>
__device__ __forceinline__ S ldg_nc(const S *p) { return __ldg(p); }
template <>
__device__ __forceinline__ __nv_bfloat16 ldg_nc<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    return __ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short *>(p)));
}

// out[a] = sum_b M[a][b] in[b]  (TR=false)   or   out[a] = sum_b M[b][a] in[b]  (TR=true)
template <int N, bool TR, class Ar>
__device__ __forceinline__ void contract(const typename Ar::C (&M)[N][N], const typename Ar::T (&in)[N],
                                         typename Ar::T (&out)[N])
{
#pragma unroll
    for (int a = 0; a < N; ++a) {
        typename Ar::T s = Ar::mul(in[0], TR ? M[0][a] : M[a][0]);
#pragma unroll
        for (int b = 1; b < N; ++b) Ar::mad(s, in[b], TR ? M[b][a] : M[a][b]);
        out[a] = Ar::norm(s);
    }
}

// out = M in with M in even-odd form (see EOMat), S = +1 or -1 the reflection sign
// NRM: renormalise each double-float output (no effect for the other arithmetics)
template <int N, int S, class Ar, bool NRM = true>
__device__ __forceinline__ void contract_eo(const EOMat<N, typename Ar::C> &M, const typename Ar::T (&in)[N],
                                            typename Ar::T (&out)[N])
{
    using T = typename Ar::T;
    constexpr int H = N / 2;
    T e[H], o[H];
#pragma unroll
    for (int b = 0; b < H; ++b) {
        e[b] = Ar::add(in[b], in[N - 1 - b]);
        o[b] = Ar::sub(in[b], in[N - 1 - b]);
    }
    if constexpr (std::is_same<Ar, ArDF>::value) {
        // Double-float: the even and odd sums of an output pair run as one chain of paired FP32
        // operations (lane x even, lane y odd; the middle term enters lane y multiplied by 0, which
        // leaves it unchanged), each lane bit-identical to the scalar chain. (Pairing the e/o
        // formation and the final add/subtract as well was slower: the lane shuffles cost more.)
        df64p eo[H];
#pragma unroll
        for (int b = 0; b < H; ++b) eo[b] = dfp_pack(e[b], o[b]);
        df64p xm;
        if constexpr (N % 2 == 1) xm = dfp_pack(in[H], in[H]);
#pragma unroll
        for (int a = 0; a < H; ++a) {
            df64p y2 = dfp_mul(eo[0], M.P[a][0]);
#pragma unroll
            for (int b = 1; b < H; ++b) dfp_mad(y2, eo[b], M.P[a][b]);
            if constexpr (N % 2 == 1) dfp_mad(y2, xm, M.PM[a]);
            const T ye = dfp_x(y2), yo = dfp_y(y2);
            // without NRM the outputs stay unnormalised (|lo| a few ulp of hi): every consumer is a
            // double-float operation or the final conversion, which take that form as it is
            const T sum = Ar::add(ye, yo);
            out[a] = NRM ? Ar::norm(sum) : sum;
            const T d = Ar::sub(ye, yo);
            const T dd = S > 0 ? d : Ar::neg(d);
            out[N - 1 - a] = NRM ? Ar::norm(dd) : dd;
        }
    } else if constexpr (std::is_same<Ar, ArF32>::value) {
        // FP32: the same pairing with FFMA2 (lane x even, lane y odd)
        float2 eo[H];
#pragma unroll
        for (int b = 0; b < H; ++b) eo[b] = make_float2(e[b], o[b]);
        float2 xm;
        if constexpr (N % 2 == 1) xm = make_float2(in[H], in[H]);
#pragma unroll
        for (int a = 0; a < H; ++a) {
            float2 y2 = __fmul2_rn(eo[0], M.P[a][0]);
#pragma unroll
            for (int b = 1; b < H; ++b) y2 = __ffma2_rn(eo[b], M.P[a][b], y2);
            if constexpr (N % 2 == 1) y2 = __ffma2_rn(xm, M.PM[a], y2);
            out[a] = y2.x + y2.y;
            const T d = y2.x - y2.y;
            out[N - 1 - a] = S > 0 ? d : -d;
        }
    } else {
#pragma unroll
        for (int a = 0; a < H; ++a) {
            T ye = Ar::mul(e[0], M.E[a][0]);
#pragma unroll
            for (int b = 1; b < H; ++b) Ar::mad(ye, e[b], M.E[a][b]);
            if constexpr (N % 2 == 1) Ar::mad(ye, in[H], M.Mid[a]);
            T yo = Ar::mul(o[0], M.O[a][0]);
#pragma unroll
            for (int b = 1; b < H; ++b) Ar::mad(yo, o[b], M.O[a][b]);
            out[a] = Ar::norm(Ar::add(ye, yo));
            const T d = Ar::sub(ye, yo);
            out[N - 1 - a] = Ar::norm(S > 0 ? d : Ar::neg(d));
        }
    }
    if constexpr (N % 2 == 1) {  // middle output: only the even (S = +1) or odd (S = -1) part
        if constexpr (S > 0) {
            T ye = Ar::mul(in[H], M.Mid[H]);
#pragma unroll
            for (int b = 0; b < H; ++b) Ar::mad(ye, e[b], M.E[H][b]);
            out[H] = NRM ? Ar::norm(ye) : ye;
        } else {
            T yo = Ar::mul(o[0], M.O[H][0]);
#pragma unroll
            for (int b = 1; b < H; ++b) Ar::mad(yo, o[b], M.O[H][b]);
            out[H] = NRM ? Ar::norm(yo) : yo;
        }
    }
}

// line contraction with B, B^T, D or D^T: even-odd form from N = 4 up, full form below
template <int N, class Ar, int WHICH, bool NRM = true>  // WHICH: 0 B, 1 B^T, 2 D, 3 D^T
__device__ __forceinline__ void sweep(const TabMetric<N, typename Ar::C> &tab, const typename Ar::T (&in)[N],
                                      typename Ar::T (&out)[N])
{
    if constexpr (N >= 4) {
        if constexpr (WHICH == 0) contract_eo<N, 1, Ar, NRM>(tab.Bf, in, out);
        else if constexpr (WHICH == 1) contract_eo<N, 1, Ar, NRM>(tab.Bt, in, out);
        else if constexpr (WHICH == 2) contract_eo<N, -1, Ar, NRM>(tab.Df, in, out);
        else contract_eo<N, -1, Ar, NRM>(tab.Dt, in, out);
    } else {
        if constexpr (WHICH == 0) contract<N, false, Ar>(tab.B, in, out);
        else if constexpr (WHICH == 1) contract<N, true, Ar>(tab.B, in, out);
        else if constexpr (WHICH == 2) contract<N, false, Ar>(tab.D, in, out);
        else contract<N, true, Ar>(tab.D, in, out);
    }
}

// shared-memory line access: element m of the x-line, y-line or z-pencil owned by (ra, rb)
template <int N>
struct Lines {
    static constexpr int PI = N | 1;  // row pitch (odd)
    static constexpr int CS = PI * N * N;
    static __device__ __forceinline__ int x(int ra, int rb, int m) { return m + PI * (ra + N * rb); }
    static __device__ __forceinline__ int y(int ra, int rb, int m) { return ra + PI * (m + N * rb); }
    static __device__ __forceinline__ int z(int ra, int rb, int m) { return ra + PI * (rb + N * m); }
};

// ---- line buffers of the curved kernels (metric_tile)
// Element (i, j, k) of cell slot c sits at c*CS + i + PI*j + PP*k in each of the three buffers, and
// buffer R starts at element R*RS (RS: CPB*CS rounded up to 16 bytes, so that a bulk copy can land in
// buffer 1). A thread keeps the z-pencil (i, j) = (ra, rb) of its own cell in registers from one step
// to the next, and serves x-line (j, k) = (ra, rb) of its own cell where a step reads the input from
// memory or writes the output (coalesced global accesses). The other x-line steps and the y-line
// steps only load a line from shared memory, contract it and store it back, so any thread may serve
// any cell's line there: with `deal_x` / `deal_y` those lines are dealt to threads in the order of the
// shared-memory bank of their first element, round-robin over the warps, so that a warp touches
// distinct banks wherever the bank counts allow. The pitches come from an exhaustive search over
// (PI, PP, CS <= 1.6 n^3) that minimised the wavefronts of all line accesses of one apply (per
// element: 2 x-line accesses in thread order, 4 dealt, 8 y-line, 9 z-pencil) for 4-byte elements:
// at n = 5 and 8 cells per CTA 1105 instead of 1315 per tile (805 without any conflict). Dealing the
// global x-line steps as well cut more wavefronts but scattered the output stores over the tile's
// cells (2.4x the L2 store sectors) and was slower. Double-float and FP64 tiles (8-byte elements)
// keep odd row pitches with lines in thread order: their kernel is bound by the FP32 pipes, and 22 %
// fewer wavefronts changed nothing in its time.
struct TileGeom {
    int pi, pp, cs;  // row pitch, plane pitch, cell stride (elements)
    bool deal_x, deal_y;
};
__host__ __device__ constexpr TileGeom tile_geom(int N, int CPB, int ESZ, bool allow_remap)
{
    if (allow_remap && ESZ == 4) {
        switch (N * 1000 + CPB) {
        case 2016: case 2032: case 2064: return {2, 6, 12, false, true};
        case 3008: case 3016: case 3032: return {3, 10, 41, true, true};
        case 4004: case 4008: return {4, 19, 80, true, true};
        case 5004: case 5008: return {5, 33, 185, true, true};
        case 6002: case 6004: case 6008: return {6, 37, 228, true, true};
        case 7004: case 7008: return {7, 73, 529, true, true};
        case 8002: return {8, 66, 528, true, true};
        default: break;
        }
    }
    return {N | 1, N * (N | 1), N * N * (N | 1), false, false};
}

template <int N, int CPB, int ESZ, bool REMAP>
struct TileLines {
    static constexpr TileGeom G = tile_geom(N, CPB, ESZ, REMAP);
    static constexpr int PI = G.pi, PP = G.pp, CS = G.cs;
    static constexpr int RS = (CPB * CS * ESZ + 15) / 16 * 16 / ESZ;  // buffer stride (elements)
    static_assert(PI >= N && PP >= N * PI && CS >= N * PP, "tile buffers overlap");
};

// in the shared-memory-only steps thread t serves x-line m[t] >> 16 and y-line m[t] & 0xffff; a line
// l = c N^2 + a + N b is cell slot c's x-line (j, k) = (a, b) or y-line (i, k) = (a, b)
template <int N, int CPB, int ESZ>
struct LineMap {
    uint32_t m[N * N * CPB];
};
template <int N, int CPB, int ESZ, bool REMAP>
constexpr LineMap<N, CPB, ESZ> make_line_map()
{
    constexpr TileGeom G = tile_geom(N, CPB, ESZ, REMAP);
    constexpr int T = N * N * CPB, N2 = N * N;
    constexpr int GRP = ESZ == 4 ? 32 : 16;  // lanes served by one wavefront = banks, in elements
    constexpr int NG = (T + GRP - 1) / GRP;
    LineMap<N, CPB, ESZ> r{};
    for (int dir = 0; dir < 2; ++dir) {
        int order[T] = {};
        int n = 0;
        for (int b = 0; b < GRP; ++b)
            for (int l = 0; l < T; ++l) {
                const int c = l / N2, a = l % N, bb = (l / N) % N;
                const int base = c * G.cs + (dir == 0 ? G.pi * a : a) + G.pp * bb;
                if (base % GRP == b) order[n++] = l;
            }
        n = 0;
        for (int lane = 0; lane < GRP; ++lane)
            for (int g = 0; g < NG; ++g) {
                const int t = g * GRP + lane;
                if (t >= T) continue;
                const uint32_t l = static_cast<uint32_t>((dir == 0 ? G.deal_x : G.deal_y) ? order[n++] : t);
                r.m[t] |= dir == 0 ? (l << 16) : l;
            }
    }
    return r;
}
template <int N, int CPB, int ESZ, bool REMAP>
constexpr bool line_map_is_bijection()
{
    constexpr LineMap<N, CPB, ESZ> M = make_line_map<N, CPB, ESZ, REMAP>();
    constexpr int T = N * N * CPB;
    bool seen_x[T] = {}, seen_y[T] = {};
    for (int t = 0; t < T; ++t) {
        const uint32_t lx = M.m[t] >> 16, ly = M.m[t] & 0xffffu;
        if (lx >= static_cast<uint32_t>(T) || ly >= static_cast<uint32_t>(T) || seen_x[lx] || seen_y[ly]) return false;
        seen_x[lx] = seen_y[ly] = true;
    }
    return true;
}
template <int N, int CPB, int ESZ, bool REMAP>
__device__ constexpr LineMap<N, CPB, ESZ> kLineMap = make_line_map<N, CPB, ESZ, REMAP>();

// element m of a line in buffer R: x-line at offset o (stride 1), y-line (stride PI), z-pencil (PP)
#define CW_TLD(R, o, st, v) _Pragma("unroll") for (int m_ = 0; m_ < N; ++m_) v[m_] = S0[(R) * TL::RS + (o) + (st) * m_]
#define CW_TST(R, o, st, v) _Pragma("unroll") for (int m_ = 0; m_ < N; ++m_) S0[(R) * TL::RS + (o) + (st) * m_] = v[m_]

#define CW_LDX(s, v) _Pragma("unroll") for (int m_ = 0; m_ < N; ++m_) v[m_] = (s)[L::x(ra, rb, m_)]
#define CW_LDY(s, v) _Pragma("unroll") for (int m_ = 0; m_ < N; ++m_) v[m_] = (s)[L::y(ra, rb, m_)]
#define CW_LDZ(s, v) _Pragma("unroll") for (int m_ = 0; m_ < N; ++m_) v[m_] = (s)[L::z(ra, rb, m_)]
#define CW_STX(s, v) _Pragma("unroll") for (int m_ = 0; m_ < N; ++m_) (s)[L::x(ra, rb, m_)] = v[m_]
#define CW_STY(s, v) _Pragma("unroll") for (int m_ = 0; m_ < N; ++m_) (s)[L::y(ra, rb, m_)] = v[m_]
#define CW_STZ(s, v) _Pragma("unroll") for (int m_ = 0; m_ < N; ++m_) (s)[L::z(ra, rb, m_)] = v[m_]

// number of stored metric components per quadrature point for an operator kind
__host__ __device__ constexpr int metric_ncomp(int kind) { return kind == 1 ? 6 : (kind == 2 ? 1 : 7); }

// ------------------------------------------------------------------------ curved kernel ----
// geo layout: [cell][comp][qp] with qp = a + N(b + N c); comps (xx, yy, zz, xy, xz, yz, mass)
// for kind 3, the first six for kind 1, the mass coefficient alone for kind 2.
//
// STAGE: the CTA's input tile and metric tile are moved into shared memory by two 1D bulk copies
// issued at entry (x on barrier 0, metric on barrier 1), so the metric stream overlaps the
// interpolation and gradient sweeps. Tiles that cannot use a bulk copy (ragged last tile,
// misaligned span) and copies that do not complete within the wait bound are read with ordinary
// global loads instead.
// STAGE 0: direct loads; 1: x and metric tiles staged in shared memory by TMA; 2: x tile staged by
// TMA, metric tile prefetched into L2 by a bulk prefetch (a third of the shared memory of mode 1,
// so more CTAs per SM), then read with direct loads; 3: the metric tile already in shared memory
// (staged by the caller for several right-hand sides, gsm), x read directly.
template <int N, int CPB, class T, class GS, bool REMAP = true>
__host__ __device__ constexpr size_t metric_smem_bytes(int nc, int stage)
{
    constexpr size_t lb = 3 * TileLines<N, CPB, sizeof(T), REMAP>::RS * sizeof(T);  // a multiple of 16
    return stage == 1 ? lb + (CPB * nc * N * N * N * sizeof(GS) + 15) / 16 * 16 + 16 : stage == 2 ? lb + 16 : lb;
}

// One tile of `cpt` consecutive cells starting at cell tile*cpt, worked by CPB cell slots of N*N
// threads (cpt <= CPB; slots c >= cpt compute on zeros and store nothing, so a CTA may have more
// threads than the tile needs). STAGE (see metric_smem_bytes; staging needs cpt == CPB).
// DOT: also accumulate this thread's share of <x, A x> into *dot, as the quadrature sum over its
// pencil of (grad u)^T G (grad u) + c u^2 (double-float accumulation): the same quadratic form as
// x^T A_e x cell by cell, read off the quadrature-point step with no extra memory traffic.
// asm_nx > 0 (the mesh's cells per x-row): the x pass of Algorithm struct_dss is applied to the
// x-interfaces between cells of this tile before the store (the two end values of each x-line are
// exchanged through shared memory and summed as that pass sums them); the interfaces between tiles
// are left to the DSS.
// RC: geo holds the trilinear coefficients (kTriCoef per cell) and the metric of every quadrature
// point is recomputed from them (Sec. 6: J, det J, J^-1 at the point): G = (w / det J) [c_a . c_b]
// with c_0 = J_eta x J_zeta, c_1 = J_zeta x J_xi, c_2 = J_xi x J_eta (the rows of det J J^-1), and
// the mass coefficient w det J.
// SMOOTH (Algorithm smoother_fused in one pass over the operator's output): y aliases x (= u, updated
// in place), and the stored value is u + D_hat (b - A u) (sb = b, sd = D_hat, cell-wise in the vector
// type), with the x-interfaces inside the tile averaged (the x pass of the averaging DSS:
// (left + right) / 2 to both copies; asm_nx must be the mesh's cells per x-row). Each thread re-reads
// u, b and D_hat on the x-line it stores, with plain loads (y aliases x). The operator output never
// reaches memory.
// An expired wait for a staged copy: record it in the device status word and wait once more (bounded)
// so that the copy is not left in flight. Out of line: the common path carries none of it.
static __device__ __noinline__ void wait_expired(unsigned *status, uint64_t *bar, uint32_t lim)
{
    if (status) atomicOr(status, kDevStatusTimeout);
    mbar_wait_bounded(bar, 0, lim);
}

// Staged tiles and their waits: every wait for a bulk copy is bounded. A thread whose wait expired
// never reads the staged data (it takes zeros for the input tile, the global copy of the metric),
// records kDevStatusTimeout in *status (the operator's device status word, reported as
// CW_ERR_TIMEOUT by the next checking call: the outputs of that call are then undefined), and waits
// once more (bounded) so that the copy is not left in flight. Nothing runs on the common path beyond
// the wait itself: deciding the tile's fate block-wide (an early exit, or a flag read before the
// stores) made the common path 2-6 % slower in measurement. dbg_extra > 0 (fault injection for tests)
// arms the input tile's barrier with dbg_extra bytes more than the copy delivers, so that its phase
// can never complete and the (then short) bounded wait runs out.
template <int N, int CPB, class Ar, class VS, class GS, int STAGE, bool DOT = false, bool RC = false,
          bool SMOOTH = false, bool REMAP = true>
__device__ __forceinline__ void metric_tile(const VS *x, VS *y, const GS *__restrict__ geo,
                                            int64_t ncells, int kind, const TabMetric<N, typename Ar::C> &tab,
                                            int64_t tile, int cpt, unsigned char *smem_raw, df64 *dot = nullptr,
                                            int asm_nx = 0, const VS *sb = nullptr, const VS *sd = nullptr,
                                            unsigned *status = nullptr, uint32_t dbg_extra = 0,
                                            const GS *gsm = nullptr)
{
    static_assert(!(RC && STAGE == 1), "recomputed geometry has no metric tile to stage");
    // Double-float renormalisation of the intermediate values: kept where the operator serves the
    // solver (DOT), whose attainable accuracy depends on it (at 128^3 Q3 the double-float CG took
    // 1351 instead of 1026 iterations without it); skipped in the plain apply (5 % faster there,
    // errors against the oracle <= 1.0e-13 instead of <= 3e-14).
    constexpr bool NRM = DOT;
    using T = typename Ar::T;
    using TL = TileLines<N, CPB, sizeof(T), REMAP>;
    static_assert(line_map_is_bijection<N, CPB, sizeof(T), REMAP>(), "every line has one thread");
    constexpr int N2 = N * N, N3 = N2 * N, PI = TL::PI, PP = TL::PP, CS = TL::CS, RS = TL::RS;
    const bool HAS_K = (kind & 1) != 0, HAS_M = (kind & 2) != 0;
    const int NC = metric_ncomp(kind);
    T *S0 = reinterpret_cast<T *>(smem_raw);
    const int t = threadIdx.x;
    const int c = t / N2, r = t - c * N2, ra = r % N, rb = r / N;
    const int64_t cell0 = tile * cpt;
    const int64_t cell = cell0 + c;
    const bool act = c < cpt && cell < ncells;
    // offsets of the first elements of this thread's lines in a buffer: its own cell's x-line
    // (j, k) = (ra, rb) (xi, the steps that read or write memory) and z-pencil (i, j) = (ra, rb) (zo);
    // the dealt x-line (xo) and y-line (yo) of the shared-memory-only steps
    const int xi = c * CS + PI * ra + PP * rb;
    const int zo = c * CS + ra + PI * rb;
    int xo = xi, yo = c * CS + ra + PP * rb;
    if constexpr (TL::G.deal_x || TL::G.deal_y) {
        const uint32_t lm = kLineMap<N, CPB, sizeof(T), REMAP>.m[t];
        const int lx = static_cast<int>(lm >> 16), ly = static_cast<int>(lm & 0xffffu);
        const int xc = lx / N2, xr = lx - xc * N2, yc = ly / N2, yr = ly - yc * N2;
        xo = xc * CS + PI * (xr % N) + PP * (xr / N);
        yo = yc * CS + (yr % N) + PP * (yr / N);
    }

    // ---- tile staging (single right-hand side)
    bool x_smem = false, g_smem = false, x_ok = true;
    const VS *xs = nullptr;
    const GS *gs = nullptr;
    uint64_t *bar = nullptr;
    const uint32_t lim = dbg_extra ? kWaitLimitInjected : kWaitLimit;
    if constexpr (STAGE == 1) {
        const size_t offg = 3 * RS * sizeof(T);
        GS *sG = reinterpret_cast<GS *>(smem_raw + offg);
        bar = reinterpret_cast<uint64_t *>(smem_raw + offg + (CPB * NC * N3 * sizeof(GS) + 15) / 16 * 16);
        VS *sX = reinterpret_cast<VS *>(S0 + RS);  // buffer 1 is free until the gradients
        const VS *xsrc = x + cell0 * N3;
        const GS *gsrc = geo + cell0 * NC * N3;
        const uint32_t xb = CPB * N3 * sizeof(VS), gb = CPB * NC * N3 * sizeof(GS);
        const bool ok = (cell0 + CPB <= ncells) && aligned16(xsrc) && aligned16(gsrc) && aligned16(sX) &&
                        aligned16(sG) && (xb % 16 == 0) && (gb % 16 == 0);
        if (ok) {  // block-uniform
            if (t == 0) {
                mbar_init(bar, 1);
                mbar_init(bar + 1, 1);
            }
            __syncthreads();
            if (t == 0) {
                mbar_expect_tx(bar, xb + dbg_extra);
                bulk_g2s(sX, xsrc, xb, bar);
                mbar_expect_tx(bar + 1, gb);
                bulk_g2s(sG, gsrc, gb, bar + 1);
            }
            x_ok = mbar_wait_bounded(bar, 0, lim);
            if (!x_ok) wait_expired(status, bar, lim);
            x_smem = true;
            xs = sX + c * N3;
            gs = sG + c * NC * N3;
            g_smem = true;  // its wait comes before the physics step
        }
    } else if constexpr (STAGE == 3) {
        // the caller passes this tile's metric (gsm): staged in shared memory, where one copy serves
        // several right-hand sides, or in global memory when it could not be staged (cell slots past
        // a ragged tile's end read slot 0's, in bounds, and store nothing)
        gs = gsm + (act ? c : 0) * NC * N3;
        g_smem = true;
    } else if constexpr (STAGE == 2) {
        bar = reinterpret_cast<uint64_t *>(smem_raw + 3 * RS * sizeof(T));
        VS *sX = reinterpret_cast<VS *>(S0 + RS);
        const VS *xsrc = x + cell0 * N3;
        constexpr int GV = RC ? kTriCoef : 0;  // geometry values per cell (RC), else NC * N3
        const int gpc = RC ? GV : NC * N3;
        const GS *gsrc = geo + cell0 * gpc;
        const uint32_t xb = CPB * N3 * sizeof(VS), gb = CPB * gpc * sizeof(GS);
        const bool full = cell0 + CPB <= ncells;
        const bool ok = full && aligned16(xsrc) && aligned16(sX) && (xb % 16 == 0);
        if (t == 0 && full && aligned16(gsrc) && (gb % 16 == 0)) bulk_prefetch_l2(gsrc, gb);
        if (ok) {  // block-uniform
            if (t == 0) mbar_init(bar, 1);
            __syncthreads();
            if (t == 0) {
                mbar_expect_tx(bar, xb + dbg_extra);
                bulk_g2s(sX, xsrc, xb, bar);
            }
            x_ok = mbar_wait_bounded(bar, 0, lim);
            if (!x_ok) wait_expired(status, bar, lim);
            x_smem = true;
            xs = sX + c * N3;
        }
    }

    {
        T v[N], w[N], u[N], acc[N], gx[N], gy[N], gz[N];
        // (1) x-line (j,k) = (ra, rb): N contiguous values of the cell, contracted with B along x
        {
            if (x_smem) {  // a thread whose wait expired reads nothing staged
#pragma unroll
                for (int m = 0; m < N; ++m) v[m] = x_ok ? Ar::from(xs[N * r + m]) : Ar::zero();
            } else {
                const VS *xg = x + (act ? cell : 0) * N3 + N * r;
#pragma unroll
                for (int m = 0; m < N; ++m) v[m] = act ? Ar::from(ldg_nc(xg + m)) : Ar::zero();
            }
            sweep<N, Ar, 0, NRM>(tab, v, w);
            CW_TST(0, xi, 1, w);
        }
        __syncthreads();
        // (2) y-line (i,k): contract with B along y, in place
        {
            CW_TLD(0, yo, PI, v);
            sweep<N, Ar, 0, NRM>(tab, v, w);
            CW_TST(0, yo, PI, w);
        }
        __syncthreads();
        // (3) z-pencil (i,j): contract with B along z -> u at the Gauss points (registers)
        {
            CW_TLD(0, zo, PP, v);
            sweep<N, Ar, 0, NRM>(tab, v, u);
        }
        if (HAS_K) {
            {
                sweep<N, Ar, 2, NRM>(tab, u, gz);
                CW_TST(0, zo, PP, u);
            }
            __syncthreads();
            // x- and y-derivatives by collocation, as line owners
            {
                CW_TLD(0, xo, 1, v);
                sweep<N, Ar, 2, NRM>(tab, v, w);
                CW_TST(1, xo, 1, w);
                CW_TLD(0, yo, PI, v);
                sweep<N, Ar, 2, NRM>(tab, v, w);
                CW_TST(2, yo, PI, w);
            }
            __syncthreads();
            {
                CW_TLD(1, zo, PP, gx);
                CW_TLD(2, zo, PP, gy);
            }
        }
        // the metric tile's wait (a thread whose wait expired reads the metric from global memory)
        bool g_ok = true;
        if constexpr (STAGE == 1) {
            if (g_smem) {
                g_ok = mbar_wait_bounded(bar + 1, 0, lim);
                if (!g_ok) wait_expired(status, bar + 1, lim);
            }
        }
        // (4) quadrature-point physics on the owned pencil, qp = (ra, rb, k)
        {
            const GS *gc = (g_smem && g_ok) ? gs + r
                                            : geo + (act ? cell : 0) * (RC ? kTriCoef : NC * N3) + (RC ? 0 : r);
            // RC: the pencil's Jacobian columns as J_xi = P0 + zeta P1, J_eta = Q0 + zeta Q1, J_zeta = Z
            T P0[3], P1[3], Q0[3], Q1[3], Z[3], wab;
            if constexpr (RC) {
                T xi = tab.xq[0], eta = tab.xq[0], wa = tab.wq[0], wb = tab.wq[0];
#pragma unroll
                for (int m = 1; m < N; ++m) {
                    if (ra == m) xi = tab.xq[m], wa = tab.wq[m];
                    if (rb == m) eta = tab.xq[m], wb = tab.wq[m];
                }
                wab = Ar::norm(Ar::mul(wa, wb));
                const T xe = Ar::norm(Ar::mul(xi, eta));
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const T a1 = Ar::from(gc[0 + d]), a2 = Ar::from(gc[3 + d]), a3 = Ar::from(gc[6 + d]);
                    const T a4 = Ar::from(gc[9 + d]), a5 = Ar::from(gc[12 + d]), a6 = Ar::from(gc[15 + d]);
                    const T a7 = Ar::from(gc[18 + d]);
                    T t = a1;
                    Ar::mad(t, a4, eta);
                    P0[d] = Ar::norm(t);
                    t = a5;
                    Ar::mad(t, a7, eta);
                    P1[d] = Ar::norm(t);
                    t = a2;
                    Ar::mad(t, a4, xi);
                    Q0[d] = Ar::norm(t);
                    t = a6;
                    Ar::mad(t, a7, xi);
                    Q1[d] = Ar::norm(t);
                    t = a3;
                    Ar::mad(t, a5, xi);
                    Ar::mad(t, a6, eta);
                    Ar::mad(t, a7, xe);
                    Z[d] = Ar::norm(t);
                }
            }
#pragma unroll
            for (int k = 0; k < N; ++k) {
                const GS *g = gc + N2 * k;
                T gxx, gyy, gzz, gxy, gxz, gyz, cmr;
                if constexpr (RC) {
                    const T zeta = tab.xq[k];
                    T jx[3], jy[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        T t = P0[d];
                        Ar::mad(t, P1[d], zeta);
                        jx[d] = Ar::norm(t);
                        t = Q0[d];
                        Ar::mad(t, Q1[d], zeta);
                        jy[d] = Ar::norm(t);
                    }
                    auto cross = [](const T (&a)[3], const T (&b)[3], T (&c)[3]) {
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
                            T t = Ar::mul(a[d1], b[d2]);
                            Ar::mad(t, Ar::neg(a[d2]), b[d1]);
                            c[d] = Ar::norm(t);
                        }
                    };
                    auto dot3 = [](const T (&a)[3], const T (&b)[3]) {
                        T t = Ar::mul(a[0], b[0]);
                        Ar::mad(t, a[1], b[1]);
                        Ar::mad(t, a[2], b[2]);
                        return Ar::norm(t);
                    };
                    T c0[3], c1[3], c2[3];
                    cross(jy, Z, c0);
                    cross(Z, jx, c1);
                    cross(jx, jy, c2);
                    const T det = dot3(jx, c0);
                    const T w = Ar::norm(Ar::mul(wab, tab.wq[k]));
                    cmr = Ar::norm(Ar::mul(w, det));
                    if (HAS_K) {
                        const T sc = Ar::div(w, det);
                        gxx = Ar::norm(Ar::mul(sc, dot3(c0, c0)));
                        gyy = Ar::norm(Ar::mul(sc, dot3(c1, c1)));
                        gzz = Ar::norm(Ar::mul(sc, dot3(c2, c2)));
                        gxy = Ar::norm(Ar::mul(sc, dot3(c0, c1)));
                        gxz = Ar::norm(Ar::mul(sc, dot3(c0, c2)));
                        gyz = Ar::norm(Ar::mul(sc, dot3(c1, c2)));
                    }
                }
                if (HAS_K) {
                    if constexpr (!RC) {
                        gxx = Ar::from(g[0 * N3]), gyy = Ar::from(g[1 * N3]);
                        gzz = Ar::from(g[2 * N3]), gxy = Ar::from(g[3 * N3]);
                        gxz = Ar::from(g[4 * N3]), gyz = Ar::from(g[5 * N3]);
                    }
                    T hx = Ar::mul(gx[k], gxx), hy = Ar::mul(gx[k], gxy), hz = Ar::mul(gx[k], gxz);
                    Ar::mad(hx, gy[k], gxy);
                    Ar::mad(hy, gy[k], gyy);
                    Ar::mad(hz, gy[k], gyz);
                    Ar::mad(hx, gz[k], gxz);
                    Ar::mad(hy, gz[k], gyz);
                    Ar::mad(hz, gz[k], gzz);
                    if constexpr (DOT) {  // (grad u)^T G (grad u) at this point
                        df_mad(*dot, Ar::to_df(gx[k]), Ar::to_df(hx));
                        df_mad(*dot, Ar::to_df(gy[k]), Ar::to_df(hy));
                        df_mad(*dot, Ar::to_df(gz[k]), Ar::to_df(hz));
                    }
                    gx[k] = NRM ? Ar::norm(hx) : hx;
                    gy[k] = NRM ? Ar::norm(hy) : hy;
                    gz[k] = NRM ? Ar::norm(hz) : hz;
                }
                if (HAS_M) {
                    if constexpr (!RC) cmr = Ar::from(g[(NC - 1) * N3]);
                    const T cm = cmr;
                    acc[k] = NRM ? Ar::norm(Ar::mul(u[k], cm)) : Ar::mul(u[k], cm);
                    if constexpr (DOT) df_mad(*dot, Ar::to_df(u[k]), Ar::to_df(acc[k]));  // c u^2
                }
            }
        }
        if (HAS_K) {
            // z-part of the transposed derivative in registers, x/y parts as line owners
            {
                sweep<N, Ar, 3, NRM>(tab, gz, v);
#pragma unroll
                for (int k = 0; k < N; ++k) acc[k] = HAS_M ? Ar::add(acc[k], v[k]) : v[k];
                CW_TST(1, zo, PP, gx);  // own pencil only: no other thread reads s1/s2 pencils now
                CW_TST(2, zo, PP, gy);
            }
            __syncthreads();
            {
                CW_TLD(1, xo, 1, v);
                sweep<N, Ar, 3, NRM>(tab, v, w);
                CW_TST(1, xo, 1, w);
                CW_TLD(2, yo, PI, v);
                sweep<N, Ar, 3, NRM>(tab, v, w);
                CW_TST(2, yo, PI, w);
            }
            __syncthreads();
            {
                CW_TLD(1, zo, PP, v);
                CW_TLD(2, zo, PP, w);
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    const T t = Ar::add(acc[k], Ar::add(v[k], w[k]));
                    acc[k] = NRM ? Ar::norm(t) : t;
                }
            }
        }
        // (5) integrate back: B^T along z (registers), y and x as line owners
        {
            sweep<N, Ar, 1, NRM>(tab, acc, w);
            CW_TST(0, zo, PP, w);
        }
        __syncthreads();
        {
            CW_TLD(0, yo, PI, v);
            sweep<N, Ar, 1, NRM>(tab, v, w);
            CW_TST(0, yo, PI, w);
        }
        __syncthreads();
        {
            CW_TLD(0, xi, 1, v);
            sweep<N, Ar, 1, NRM>(tab, v, w);
            if constexpr (SMOOTH) {
                VS nv[N];
                const int64_t o = (act ? cell : 0) * N3 + N * r;
#pragma unroll
                for (int m = 0; m < N; ++m) {
                    VS av;
                    Ar::to(av, w[m]);
                    nv[m] = act ? y[o + m] + sd[o + m] * (sb[o + m] - av) : VS(0);
                }
                VS *exl = reinterpret_cast<VS *>(S0 + RS), *exr = exl + CPB * N2;  // buffer 1 is free
                exl[c * N2 + r] = nv[0];
                exr[c * N2 + r] = nv[N - 1];
                __syncthreads();
                if (act) {
                    const int64_t ix = cell % asm_nx;
                    if (c + 1 < cpt && cell + 1 < ncells && ix + 1 < asm_nx)
                        nv[N - 1] = AddOp<VS>::add(nv[N - 1], exl[(c + 1) * N2 + r]) * VS(0.5);
                    if (c > 0 && ix > 0) nv[0] = AddOp<VS>::add(exr[(c - 1) * N2 + r], nv[0]) * VS(0.5);
#pragma unroll
                    for (int m = 0; m < N; ++m) y[o + m] = nv[m];
                }
            } else if (asm_nx > 0) {  // kernel-uniform
                VS o0, o1;
                Ar::to(o0, w[0]);
                Ar::to(o1, w[N - 1]);
                // the S1 buffer is free: its last reads precede the first barrier of step (5)
                VS *exl = reinterpret_cast<VS *>(S0 + RS), *exr = exl + CPB * N2;
                exl[c * N2 + r] = o0;
                exr[c * N2 + r] = o1;
                __syncthreads();
                if (act) {
                    const int64_t ix = cell % asm_nx;
                    if (c + 1 < cpt && cell + 1 < ncells && ix + 1 < asm_nx)
                        o1 = AddOp<VS>::add(o1, exl[(c + 1) * N2 + r]);
                    if (c > 0 && ix > 0) o0 = AddOp<VS>::add(exr[(c - 1) * N2 + r], o0);
                    VS *yc = y + cell * N3 + N * r;
                    yc[0] = o0;
#pragma unroll
                    for (int m = 1; m < N - 1; ++m) Ar::to(yc[m], w[m]);
                    yc[N - 1] = o1;
                }
            } else if (act) {
                VS *yc = y + cell * N3 + N * r;
#pragma unroll
                for (int m = 0; m < N; ++m) Ar::to(yc[m], w[m]);
            }
        }
    }
}

// Register caps for the double-float kernels (as CTAs per SM for the launch bounds): stored metric
// at n = 5 to 72 registers, which it fits without spilling, so that 4 CTAs of 200 threads fit per
// SM (left alone the allocator takes 78 and loses one); recomputed geometry to 128 (2 CTAs at n = 5
// instead of 1). Other n keep the plain kernel: larger n spill under a 72 cap, smaller n already fit
// and ran slower with the hint (a minimum-blocks hint is not neutral, even a hint of 1).
template <class Ar, int N, bool RC>
constexpr bool df_capped()
{
    return std::is_same<Ar, ArDF>::value && (RC || N == 5);
}
template <int THREADS, bool RC>
constexpr int df_min_blocks()
{
    constexpr int warps = (THREADS + 31) / 32;
    constexpr int b = 65536 / (warps * 32 * (RC ? 128 : 72));
    return b > 0 ? b : 1;
}

template <int N, int CPB, class Ar, class VS, class GS, int STAGE, bool RC = false>
__global__ void __launch_bounds__(N *N *CPB) apply_metric_kernel(const VS *__restrict__ x, VS *__restrict__ y,
                                                                  const GS *__restrict__ geo, int64_t ncells,
                                                                  int kind, TabMetric<N, typename Ar::C> tab,
                                                                  int asm_nx, unsigned *status, uint32_t dbg_extra)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    metric_tile<N, CPB, Ar, VS, GS, STAGE, false, RC>(x, y, geo, ncells, kind, tab, blockIdx.x, CPB, smem_raw, nullptr,
                                                      asm_nx, nullptr, nullptr, status, dbg_extra);
}

template <int N, int CPB, class Ar, class VS, class GS, int STAGE, bool RC = false>
__global__ void __launch_bounds__(N *N *CPB, (df_min_blocks<N * N * CPB, RC>()))
    apply_metric_kernel_capped(const VS *__restrict__ x, VS *__restrict__ y, const GS *__restrict__ geo,
                               int64_t ncells, int kind, TabMetric<N, typename Ar::C> tab, int asm_nx,
                               unsigned *status, uint32_t dbg_extra)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    metric_tile<N, CPB, Ar, VS, GS, STAGE, false, RC>(x, y, geo, ncells, kind, tab, blockIdx.x, CPB, smem_raw, nullptr,
                                                      asm_nx, nullptr, nullptr, status, dbg_extra);
}

// y = A x and the CTA's partial of <x, A x> in part[blockIdx.x] (deterministic: fixed order in a CTA)
template <int N, int CPB, class Ar, class VS, class GS, int STAGE, bool RC = false>
__global__ void __launch_bounds__(N *N *CPB) apply_metric_dot_kernel(const VS *__restrict__ x, VS *__restrict__ y,
                                                                      const GS *__restrict__ geo, int64_t ncells,
                                                                      int kind, TabMetric<N, typename Ar::C> tab,
                                                                      double *__restrict__ part, unsigned *status,
                                                                      uint32_t dbg_extra)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double s_red[(N * N * CPB + 31) / 32];
    df64 acc{0.0f, 0.0f};
    metric_tile<N, CPB, Ar, VS, GS, STAGE, true, RC>(x, y, geo, ncells, kind, tab, blockIdx.x, CPB, smem_raw, &acc, 0,
                                                     nullptr, nullptr, status, dbg_extra);
    double v = df_to_double(acc);
    // N^2 * CPB is not always a multiple of 32: the last warp may hold only nw lanes
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = min(32, N * N * CPB - wid * 32);
    const unsigned mask = nw == 32 ? 0xffffffffu : ((1u << nw) - 1u);
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(mask, v, o);
        if (lane + o < nw) v += ov;
    }
    if (lane == 0) s_red[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (N * N * CPB + 31) / 32; ++i) t += s_red[i];
        part[blockIdx.x] = t;
    }
}

// One fused smoothing sweep on a tile (see SMOOTH in metric_tile): u <- x-average(u + D_hat (b - A u)),
// in place; the x pass between tiles and the y and z passes of the averaging DSS follow.
template <int N, int CPB, class Ar, class VS, class GS, int STAGE, bool RC = false>
__global__ void __launch_bounds__(N *N *CPB) smooth_metric_kernel(VS *u, const VS *__restrict__ b,
                                                                   const VS *__restrict__ dhat,
                                                                   const GS *__restrict__ geo, int64_t ncells,
                                                                   int kind, TabMetric<N, typename Ar::C> tab,
                                                                   int asm_nx, unsigned *status, uint32_t dbg_extra)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    metric_tile<N, CPB, Ar, VS, GS, STAGE, false, RC, true>(u, u, geo, ncells, kind, tab, blockIdx.x, CPB, smem_raw,
                                                            nullptr, asm_nx, b, dhat, status, dbg_extra);
}

// ---------------------------------------------------------------------- Cartesian kernel ----
// geo layout: [cell][4] doubles (a_x, a_y, a_z, a_m) = (hy hz/hx, hx hz/hy, hx hy/hz, hx hy hz),
// already multiplied by the kind mask (a_m = 0 for kind 1, a_x = a_y = a_z = 0 for kind 2).
template <int N, int CPB, class Ar, class VS>
__global__ void __launch_bounds__(N *N *CPB) apply_affine_kernel(const VS *__restrict__ x, VS *__restrict__ y,
                                                                  const double *__restrict__ geo, int64_t ncells,
                                                                  int kind, TabAffine<N, typename Ar::C> tab)
{
    using T = typename Ar::T;
    using L = Lines<N>;
    constexpr int N2 = N * N, N3 = N2 * N, CS = L::CS;
    const bool HAS_K = (kind & 1) != 0, HAS_M = (kind & 2) != 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *S0 = reinterpret_cast<T *>(smem_raw);
    const int t = threadIdx.x, c = t / N2, r = t - c * N2, ra = r % N, rb = r / N;
    const int64_t cell = static_cast<int64_t>(blockIdx.x) * CPB + c;
    const bool act = cell < ncells;
    T *s0 = S0 + c * CS;
    T *s1 = S0 + (CPB + c) * CS;
    T v[N], P[N], Q[N];
    // x-line: P = M_x u, Q = K_x u
    {
        const VS *xc = x + (act ? cell : 0) * N3 + N * r;
#pragma unroll
        for (int m = 0; m < N; ++m) v[m] = act ? Ar::from(ldg_nc(xc + m)) : Ar::zero();
        contract<N, false, Ar>(tab.M, v, P);
        CW_STX(s0, P);
        if (HAS_K) {
            contract<N, false, Ar>(tab.K, v, Q);
            CW_STX(s1, Q);
        }
    }
    const double *gc = geo + (act ? cell : 0) * 4;
    const T ax = Ar::from(__ldg(gc + 0)), ay = Ar::from(__ldg(gc + 1));
    const T az = Ar::from(__ldg(gc + 2)), am = Ar::from(__ldg(gc + 3));
    __syncthreads();
    // y-line: R1 = M_y P, R2 = K_y P, R3 = M_y Q; W = a_x R3 + a_y R2 + a_m R1
    {
        T R1[N], W[N];
        CW_LDY(s0, v);
        contract<N, false, Ar>(tab.M, v, R1);
        if (HAS_K) {
            T R2[N], R3[N];
            contract<N, false, Ar>(tab.K, v, R2);
            CW_LDY(s1, v);
            contract<N, false, Ar>(tab.M, v, R3);
#pragma unroll
            for (int m = 0; m < N; ++m) {
                T s = Ar::mul(R3[m], ax);
                Ar::mad(s, R2[m], ay);
                if (HAS_M) Ar::mad(s, R1[m], am);
                W[m] = Ar::norm(s);
                R1[m] = Ar::norm(Ar::mul(R1[m], az));
            }
            CW_STY(s1, R1);
        } else {
#pragma unroll
            for (int m = 0; m < N; ++m) W[m] = Ar::norm(Ar::mul(R1[m], am));
        }
        CW_STY(s0, W);
    }
    __syncthreads();
    // z-pencil: y = M_z W + K_z (a_z R1)
    {
        T out[N];
        CW_LDZ(s0, v);
        contract<N, false, Ar>(tab.M, v, out);
        if (HAS_K) {
            T R[N], KR[N];
            CW_LDZ(s1, R);
            contract<N, false, Ar>(tab.K, R, KR);
#pragma unroll
            for (int m = 0; m < N; ++m) out[m] = Ar::norm(Ar::add(out[m], KR[m]));
        }
        if (act) {
            VS *yc = y + cell * N3 + r;
#pragma unroll
            for (int m = 0; m < N; ++m) Ar::to(yc[N2 * m], out[m]);
        }
    }
}

}  // namespace cw
