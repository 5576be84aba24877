/*
 * cwfem.h -- C ABI of the GB300 (sm_103a) library for matrix-free high-order finite-element
 * operators on cell-wise (redundant, element-local) storage.
 *
 * The method follows "Coalesced Matrix-Free Geometric Multigrid on Persistent Cell-Wise Storage":
 *  - cell-wise storage, primal / dual vectors, gather G and assembly G^T: Sec. 2.1;
 *  - the cell-local operator A: V_cell -> V_cell^*, applied matrix-free: Sec. 2.1,
 *    Eq. (constrained_system) and the paragraph before it;
 *  - the Poisson weak form with Q_p Gauss-Lobatto nodal elements: Sec. 2, Eq. (poisson);
 *  - the Cartesian factored operator with one per-element scalar and the general curved
 *    operator (gradients -> metric -> integrate gradients): Sec. 6, first paragraphs;
 *  - direct stiffness summation S = G G^T: Sec. 4.1, Eq. (dss_operator); its structured
 *    dimension-split realisation: Sec. 4.3, Algorithm struct_dss; averaging DSS: Sec. 5,
 *    Eq. (averaging_dss);
 *  - the Jacobi preconditioner D_cell^-1 S: Sec. 4.1, Eq. (jacobi_recap), with Dirichlet rows
 *    zeroed in the stored inverse diagonal: Sec. 5, "Constraints baked into the diagonal";
 *  - conjugate gradients in primal-dual form on cell-wise data: Sec. 4.4 and Sec. 6 (CG
 *    preconditioned by a consistent operator is iterate-identical to assembled CG).
 *
 * Conventions (all entry points):
 *  - Reference cell [0,1]^3. Degree p in 1..7, n = p+1 Gauss-Lobatto nodes and n Gauss points
 *    per direction.
 *  - A mesh is an nx*ny*nz block of trilinear hexahedra. Cells are numbered cx + nx*(cy + ny*cz).
 *  - Cell-wise vectors have E*n^3 entries, layout [cell][k][j][i] (i along x fastest), a dense
 *    caller-owned DEVICE array. Entry type follows the operator precision: double for CW_PREC_F64
 *    and CW_PREC_F64_NATIVE, float for CW_PREC_F32 and CW_PREC_F32_BF16G, bfloat16 (uint16 bits)
 *    for CW_PREC_BF16.
 *  - Global vectors have (nx*p+1)(ny*p+1)(nz*p+1) doubles, index gx + Gx*(gy + Gy*gz).
 *  - Primal inputs are continuous (all copies of a DoF equal); outputs of CW_APPLY_LOCAL are
 *    unassembled duals (copies hold partial integrals).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream). Every call is
 *    asynchronous on that stream unless stated otherwise; argument errors are detected on the
 *    host before anything is enqueued and returned as a status; device-side errors surface as
 *    CW_ERR_CUDA from the next call that synchronises.
 *  - Ownership: the library owns geometry, tables, diagonals and solver scratch, all allocated
 *    at create time (or at the first call that needs them, as documented). The caller owns every
 *    pointer it passes. Inputs and outputs must not alias unless stated.
 *  - Thread safety: distinct handles may be used from distinct threads; one handle must not be
 *    used by two streams at the same time.
 */
#ifndef CWFEM_H
#define CWFEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cw_mesh_s *cw_mesh;
typedef struct cw_op_s *cw_op;

typedef enum {
    CW_OK = 0,
    CW_ERR_ARG = 1,           /* invalid argument (NULL handle, bad size, unsupported combination) */
    CW_ERR_OOM = 2,           /* device allocation failed */
    CW_ERR_CUDA = 3,          /* a CUDA call failed; cw_last_error() has the message */
    CW_ERR_NOT_CONVERGED = 4, /* solver hit maxit before the tolerance */
    CW_ERR_BREAKDOWN = 5,     /* CG breakdown: <p,Ap> <= 0 or a non-finite scalar */
    CW_ERR_TIMEOUT = 6,       /* a bounded device wait expired */
    CW_ERR_UNSUPPORTED = 7    /* valid request that this library does not implement */
} cw_status;

/* operator kinds */
#define CW_LAPLACE 1      /* K_ij = int grad phi_i . grad phi_j */
#define CW_MASS 2         /* M_ij = int phi_i phi_j */
#define CW_LAPLACE_MASS 3 /* K + M */

/* geometry representations */
#define CW_GEOM_AFFINE 0 /* Cartesian cells: factored 1D stiffness/mass form, per-cell scalars */
#define CW_GEOM_METRIC 1 /* curved trilinear cells: metric w detJ J^-1 J^-T stored per quad. point */
#define CW_GEOM_RECOMPUTE 2 /* curved trilinear cells: metric recomputed at every quadrature point
                               from 21 trilinear-map coefficients per cell (Sec. 6, J and det J) */

/* precisions (vector storage / metric storage / arithmetic) */
#define CW_PREC_F64 0        /* FP64 / FP64 as a rounded float pair (~48 bits) / double-float (FP32 pair,
                                ~47-bit) arithmetic */
#define CW_PREC_F64_NATIVE 1 /* FP64 / IEEE FP64 / native FP64 FMA: the plain IEEE FP64 operator (reference
                                speed baseline; the operator of the solvers' outer residual) */
#define CW_PREC_F32 2        /* FP32 / FP32 / FP32 */
#define CW_PREC_F32_BF16G 3  /* FP32 / BF16 / FP32 */
#define CW_PREC_BF16 4       /* BF16 / BF16 / FP32 accumulate */

/* boundary conditions (used by the diagonal and the solver) */
#define CW_BC_NONE 0
#define CW_BC_DIRICHLET0 1 /* homogeneous Dirichlet on the boundary of the block */

/* apply flags */
#define CW_APPLY_LOCAL 0    /* y = A x, unassembled dual */
#define CW_APPLY_ASSEMBLE 1 /* y = S A x = G A_CG x_g for continuous x */

/* dss flags */
#define CW_DSS_SUM 0     /* v <- S v = G G^T v */
#define CW_DSS_AVERAGE 1 /* v <- S_bar v = G (G^T G)^-1 G^T v */

/* cg modes: every mode keeps u, b and the outer residual b - A u in FP64 (the residual evaluated
   with the IEEE FP64 operator: native FP64 arithmetic, metric stored as IEEE doubles) and refines
   u += d with an inner Jacobi-PCG for A d = S_bar r */
#define CW_CG_F64 0        /* inner CG in FP64 with the double-float operator */
#define CW_CG_IR_F32 1     /* inner CG in FP32 (FP32 vectors and metric, FP64-accumulated dots) */
#define CW_CG_IR_BF16 2    /* inner CG in FP32 with the metric stored in BF16 */
#define CW_CG_F64_NATIVE 3 /* inner CG in FP64 with the IEEE FP64 operator (plain FP64 CG) */
/* flag OR-ed into a cw_cg_solve mode: start from the caller's u (resume a solve, or refine a guess)
   instead of u = 0 */
#define CW_CG_WARM_START 0x100

typedef struct {
    int iterations;        /* total CG iterations (inner iterations summed for IR modes) */
    int outer_iterations;  /* IR refinement steps (1 for CW_CG_F64) */
    double rel_residual;   /* ||m G^T(b - A u)|| / ||m G^T b|| on interior DoFs, in FP64 */
    double energy;         /* eta(u) = <b - A u, u>, Sec. 3.5 Eq. (energy_measure) */
    double seconds;        /* wall time of the solve measured with CUDA events on `stream` */
} cw_cg_stats;

/* Human-readable name of a status code; never NULL. */
const char *cw_status_string(cw_status s);
/* Message of the last error raised on the calling thread ("" if none). */
const char *cw_last_error(void);

/*
 * Create a mesh from host vertex coordinates verts[((vz*(ny+1) + vy)*(nx+1) + vx)*3 + d]
 * (double, (nx+1)(ny+1)(nz+1)*3 entries, copied to the device). Cell (cx,cy,cz) is the trilinear
 * image of [0,1]^3 through its 8 vertices. 1 <= nx, ny, nz <= 65535 and nx*ny*nz <= 2^31, else
 * CW_ERR_ARG; CW_ERR_OOM if the host or device copy cannot be allocated. The mesh must outlive its
 * operators.
 */
cw_status cw_mesh_create(int nx, int ny, int nz, const double *verts_host, cw_mesh *out);

/*
 * Box mesh of the unit cube (the cube meshes of Sec. 7, generated here): nx*ny*nz cells, vertex
 * (ix, iy, iz) at (ix/nx, iy/ny, iz/nz) moved by perturb*h * sin(2 pi f0 X) sin(2 pi f1 Y)
 * sin(2 pi f2 Z) * dir (h = 1/max(nx, ny, nz), dir normalised; the displacement vanishes on the cube's
 * faces, which are kept exact). freq: 3 integers or NULL for (1, 1, 1); direction: 3 doubles or NULL
 * for (1, 1, 1)/sqrt(3). perturb = 0 gives the Cartesian mesh (usable with CW_GEOM_AFFINE).
 * CW_ERR_ARG for sizes outside the limits of cw_mesh_create, a zero or non-finite direction or a
 * non-finite perturb.
 */
cw_status cw_mesh_create_box(int nx, int ny, int nz, double perturb, const int *freq, const double *direction,
                             cw_mesh *out);
/*
 * The library's 1D rules on [0,1] for a degree p in 1..7 (host only): the p+1 Gauss-Lobatto nodes of
 * the nodal basis (local DoF i of a cell along an axis sits at gll_nodes[i] of the reference cell,
 * Sec. 2), and the p+1 Gauss points and weights of the operators' quadrature. Each output (may be
 * NULL) receives p+1 doubles. CW_ERR_ARG for a degree outside 1..7.
 */
cw_status cw_rules_1d(int degree, double *gll_nodes, double *gauss_points, double *gauss_weights);

/*
 * The library's 1D matrices for degree p in 1..7 (host only), each (p+1) x (p+1), row-major, output
 * pointers may be NULL: B[q][m] = l_m(x_q) and Bd[q][m] = l_m'(x_q) (the Gauss-Lobatto basis at the
 * Gauss points), D[q][r] = g_r'(x_q) (the collocation derivative of the Lagrange basis g on the Gauss
 * points), M1[i][j] = int_0^1 l_i l_j and K1[i][j] = int_0^1 l_i' l_j' (the 1D mass and stiffness
 * matrices of the factored Cartesian form, Sec. 6). CW_ERR_ARG for a degree outside 1..7.
 */
cw_status cw_basis_1d(int degree, double *B, double *Bd, double *D, double *M1, double *K1);

/*
 * Vertex array of the uniform refinement of a mesh (the next level of a multigrid hierarchy, Sec. 3:
 * every cell split into 2 x 2 x 2 children by its own trilinear map, so the finite-element spaces of
 * the two meshes are nested). verts: the (nx+1)(ny+1)(nz+1)*3 doubles of cw_mesh_create's layout;
 * out: (2nx+1)(2ny+1)(2nz+1)*3 doubles in the same layout, caller-owned, to pass to cw_mesh_create
 * with 2nx, 2ny, 2nz. Host only (no device work). CW_ERR_ARG for NULL pointers or a refined mesh
 * outside cw_mesh_create's limits; CW_ERR_OOM if host scratch cannot be allocated.
 */
cw_status cw_mesh_refine_vertices(int nx, int ny, int nz, const double *verts, double *out);
cw_status cw_mesh_destroy(cw_mesh m);

/*
 * Create an operator of degree p on a mesh (Sec. 2.1). Allocates and fills the geometry
 * (CW_GEOM_METRIC: ncomp values per quadrature point, ncomp = 6 Laplace, 1 mass, 7 both, stored
 * in the metric precision -- rounded float pairs hi + lo for CW_PREC_F64, IEEE doubles for
 * CW_PREC_F64_NATIVE; CW_GEOM_RECOMPUTE: the 21 coefficients a1..a7 of each cell's trilinear
 * map, as float pairs for CW_PREC_F64, doubles for CW_PREC_F64_NATIVE and floats otherwise -- no
 * per-point storage, the
 * metric is formed in the kernel; CW_GEOM_AFFINE: 4 doubles per cell, and the mesh must be
 * Cartesian -- CW_ERR_ARG otherwise) and the 1D tables. Curved modes check det J > 0 at every
 * quadrature point (CW_ERR_ARG otherwise). CW_ERR_UNSUPPORTED where one DSS axis pass would have
 * 2^32 or more face-node pairs ((p+1)^2 * ny * (nx-1), (p+1)^2 * nx * (ny-1) or (p+1)^2 * nx * (nz-1)).
 * Synchronous.
 */
cw_status cw_op_create(cw_mesh m, int degree, int kind, int geom, int prec, int bc, cw_op *out);
cw_status cw_op_destroy(cw_op op);
int64_t cw_op_cellwise_len(cw_op op); /* E * (p+1)^3, or -1 for a NULL handle */
int64_t cw_op_global_len(cw_op op);   /* (nx p + 1)(ny p + 1)(nz p + 1), or -1 */
/* Bytes of device memory the operator owns (geometry, tables, diagonal, solver scratch). */
int64_t cw_op_device_bytes(cw_op op);

/*
 * Apply-kernel variant (the tuning knobs): cells per CTA -- 0 for the degree's default or one of
 * the two choices cw_op_get_variant reports -- and stage: 0 direct loads; 1 each CTA's input and
 * metric tiles moved into shared memory with bulk asynchronous copies (TMA) at kernel entry; 2 the
 * input tile by TMA and the metric tile prefetched into L2 by a bulk prefetch (less shared memory,
 * more CTAs per SM). Results do not depend on the variant beyond rounding order. CW_PREC_F64_NATIVE has only
 * the default variant (CW_ERR_UNSUPPORTED otherwise). CW_GEOM_RECOMPUTE operators use the default
 * cells per CTA (another choice gives CW_ERR_UNSUPPORTED); stages 1 and 2 both stage the input
 * tile by TMA there (there is no metric tile).
 */
cw_status cw_op_set_variant(cw_op op, int cells_per_cta, int stage);
/* Current variant; choices2 (may be NULL) receives the two cells-per-CTA choices of the degree and
 * arithmetic (the default and half of it; the FP32-arithmetic precisions take larger tiles than the
 * FP64 ones at p = 1, 2, 5, 6). */
cw_status cw_op_get_variant(cw_op op, int *cells_per_cta, int *stage, int *choices2);
/*
 * Autotuner: times every variant of the LOCAL apply on the caller's x, y (device, op vector
 * type, length cw_op_cellwise_len; y is overwritten) with `reps` launches each on `stream`, keeps
 * the fastest on the op and returns its time per launch in *best_ms (may be NULL). Synchronises.
 */
cw_status cw_op_autotune(cw_op op, const void *x, void *y, int reps, void *stream, float *best_ms);

/*
 * Device-side failure report. The operator kernels move tiles into shared memory with bulk copies
 * (TMA) completed on mbarriers, and every wait for such a copy is bounded. If a wait expires, the CTA
 * abandons its tile (no output written for it; no staged data that was not seen to arrive is ever
 * read), waits (bounded) for the copies it issued, and records the event in the operator's device
 * status word. cw_op_check synchronises `stream` and returns CW_ERR_TIMEOUT (clearing the word) if
 * that happened since the last check, else CW_OK; the calls that synchronise anyway (cw_cg_solve,
 * cw_cg_residual, cw_mg_pcg_solve, cw_cg_solve_noalloc, cw_op_autotune, cw_batch_autotune,
 * cw_apply_batched) check their operators' words themselves. The CUDA context stays usable.
 */
cw_status cw_op_check(cw_op op, void *stream);
/*
 * Fault-injection hook for tests of the failure report (on != 0 arms it, 0 disarms it): the
 * operator's kernels then arm the barrier of each staged input tile with 16 bytes more than the copy
 * delivers, so the copy lands but the barrier phase can never complete, the (shortened) bounded wait
 * runs out and the tile is abandoned and reported as above. Tiles read without staging (stage 0, a
 * ragged last tile) are not affected. Not for production use.
 */
cw_status cw_op_inject_stall(cw_op op, int on);

/* x = G u: replicate a device global FP64 vector into cell-wise storage of the op's precision. */
cw_status cw_gather(cw_op op, const double *u_global, void *x, void *stream);

/*
 * y = A x (flags = CW_APPLY_LOCAL) or y = S A x (CW_APPLY_ASSEMBLE). x primal, y dual;
 * both cell-wise device arrays of the op's vector type; x and y must not alias (CW_ERR_ARG).
 * Sec. 2.1 (matrix-free evaluation of the element integrals) and, for ASSEMBLE, Algorithm
 * struct_dss: for curved cells the operator kernel already sums the x-interfaces between the cells
 * of each of its tiles (same sums as the DSS x pass, bit-identical result); the x pass between
 * tiles and the y and z passes follow on `stream`. Asynchronous; errors of the launch are returned,
 * device faults surface at the next synchronisation.
 */
cw_status cw_apply(cw_op op, const void *x, void *y, int flags, void *stream);

/*
 * y = A x or S A x with x and y in HOST memory (layout and type as for cw_apply; page-locked memory
 * gives full copy bandwidth). The cells are processed in slabs of whole z-layers (at most 16): the
 * host-to-device copy of one slab overlaps the work on the previous one, and each slab is copied back
 * as soon as it is final (for CW_APPLY_ASSEMBLE, after the DSS across its interface with the next
 * slab). Asynchronous on `stream`: x and y must stay valid, and y must not be read, until `stream`
 * reaches the end of the call. The first call allocates two device vectors, three streams and events
 * owned by the op.
 */
cw_status cw_apply_host(cw_op op, const void *x_host, void *y_host, int flags, void *stream);

/*
 * In-place DSS on a cell-wise device array of the op's vector type: v <- S v (CW_DSS_SUM,
 * Algorithm struct_dss: three sequential axis passes over all interior faces) or
 * v <- S_bar v (CW_DSS_AVERAGE: the sum divided by the DoF valence).
 */
cw_status cw_dss(cw_op op, void *v, int flags, void *stream);

/*
 * Cell-wise assembled diagonal: d = G diag(A_CG) (FP64, E*n^3 doubles), Sec. 4.1. With
 * bc = CW_BC_DIRICHLET0 the entries of boundary DoFs are those of A_CG all the same.
 */
cw_status cw_diagonal(cw_op op, double *d, void *stream);

/*
 * Unassembled load vector b_K,i = sum_q w_q detJ f(x_q) phi_i(x_q) (FP64 cell-wise) for the
 * manufactured problems: which = 0: f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z); which = 1:
 * f = 2[y(1-y)z(1-z) + x(1-x)z(1-z) + x(1-x)y(1-y)]. Formed from the mesh vertices (any geometry mode).
 */
cw_status cw_load_vector(cw_op op, int which, double *b, void *stream);

/*
 * Solve A_CG u_g = G^T b for the Poisson / K+M operator with homogeneous Dirichlet conditions
 * (op bc must be CW_BC_DIRICHLET0, precision CW_PREC_F64), by Jacobi-preconditioned CG on
 * cell-wise data from u = 0 (Sec. 4.1 Eq. (jacobi_recap); Sec. 4.4). b: FP64 cell-wise dual;
 * u: FP64 cell-wise primal output; with CW_CG_WARM_START in mode, also the input iterate (a continuous
 * cell-wise vector, e.g. the u of an earlier call: checkpoint = copy u out, resume = call again with
 * the flag): the first residual b - A u is then evaluated with the IEEE FP64 operator, the stopping
 * measure stays relative to b, the corrections vanish on boundary DoFs (their values in u are kept:
 * zero for the homogeneous problem), and a non-finite initial residual returns CW_ERR_BREAKDOWN with
 * u untouched; with b = 0 the solve returns u = 0. Stops when rel_residual <= rtol or after maxit iterations
 * (CW_ERR_NOT_CONVERGED; u then holds the last iterate). mode selects the inner solver (see the
 * CW_CG_* modes); the relative residual is always measured with the IEEE FP64 operator (a twin of
 * op with precision CW_PREC_F64_NATIVE, its metric stored as doubles). The inner right-hand side
 * is the averaged residual S_bar r (same assembly G^T r, every copy small), so that rounding it to
 * FP32 keeps the assembled residual. The first call on an op allocates the solver vectors and the
 * IEEE twin (and, for the CW_CG_IR_* modes, the FP32 inner operator); cw_op_device_bytes counts
 * them. Synchronises `stream`. stats may be NULL. Errors of the inner solve (breakdown, CUDA
 * failures) end the solve with their status.
 */
cw_status cw_cg_solve(cw_op op, const double *b, double *u, double rtol, int maxit, int mode,
                      cw_cg_stats *stats, void *stream);

/*
 * Relative residual ||m G^T (b - A u)|| / ||m G^T b|| on interior DoFs (the measure of
 * cw_cg_solve) of a cell-wise FP64 iterate u for the FP64 dual b, with A evaluated in precision
 * `prec`: CW_PREC_F64_NATIVE, the IEEE FP64 operator (the twin cw_cg_solve uses), or CW_PREC_F64,
 * the op's own double-float arithmetic on its float-pair metric. op: CW_PREC_F64 with
 * CW_BC_DIRICHLET0 (else CW_ERR_ARG). The first call allocates the solver scratch and the IEEE
 * twin, as cw_cg_solve does. Synchronises `stream`.
 */
cw_status cw_cg_residual(cw_op op, const double *b, const double *u, int prec, double *rel_residual, void *stream);

/*
 * Batched apply (not in the paper): y_i = A_i x_i (LOCAL, unassembled) for nprob operators at
 * once -- uneven meshes and mixed degrees -- each with nrhs[i] right-hand sides, in ONE persistent
 * kernel launch. x[i] / y[i] are caller-owned device pointers to nrhs[i] consecutive cell-wise
 * vectors of ops[i] (stride cw_op_cellwise_len(ops[i]); x[i] and y[i] must not overlap); they are
 * bound at create and used by every launch. All operators must be CW_GEOM_METRIC and share one
 * precision, CW_PREC_F64 (double-float arithmetic) or CW_PREC_F32; they must outlive the batch.
 * Work items are taken from a device counter by persistent CTAs (no waiting: an item number past the
 * end ends a CTA). Mode CW_BATCH_GROUPED (default): one persistent kernel per degree present, shaped
 * like the per-operator kernel (variant = cells-per-CTA choice + 2 * staging mode, 0..5); an item is a
 * (problem, chunk of tiles) pair and runs every right-hand side of the problem through each tile. With
 * staging mode 1 a tile's metric is moved into shared memory once and serves all right-hand sides (a
 * problem with R right-hand sides reads its metric from HBM once, not R times); modes 0 and 2 are the
 * per-operator kernel's, per right-hand side. Mode
 * CW_BATCH_SINGLE: all degrees in ONE persistent kernel of 128-thread CTAs (variant = 0 full tile,
 * 1 half tile; items are (problem, chunk of tiles, right-hand side), right-hand side fastest); its 1D
 * tables live in the library's constant memory, uploaded at create, so only one single-mode batch per
 * precision may be launched at a time.
 */
#define CW_BATCH_GROUPED 0
#define CW_BATCH_SINGLE 1
typedef struct cw_batch_s *cw_batch;
cw_status cw_batch_create(const cw_op *ops, const int *nrhs, const void *const *x, void *const *y, int nprob,
                          cw_batch *out);
cw_status cw_batch_destroy(cw_batch b); /* waits for the device to finish first */
/* total cell-wise values one launch processes: sum_i nrhs[i] * cw_op_cellwise_len(ops[i]) */
int64_t cw_batch_values(cw_batch b);
/* one launch: clears the work counter and starts the persistent kernel on `stream` */
cw_status cw_batch_launch(cw_batch b, void *stream);
/* the same two operations captured once into a CUDA graph (on an internal stream) and replayed on
   `stream`; changing a variant re-captures at the next call */
cw_status cw_batch_graph_launch(cw_batch b, void *stream);
/* launch mode (CW_BATCH_GROUPED or CW_BATCH_SINGLE); variants are kept per mode. This call and
   cw_batch_set_variant rewrite the device-side problem table and so wait for the device first */
cw_status cw_batch_set_mode(cw_batch b, int mode);
/* kernel variant of one degree in the current mode (see above); cells_per_tile (may be NULL)
   receives the resulting cells per tile */
cw_status cw_batch_set_variant(cw_batch b, int degree, int variant);
cw_status cw_batch_get_variant(cw_batch b, int degree, int *variant, int *cells_per_tile);
/* autotuner: for each degree present, times every variant of the current mode over `reps`
   launches of the whole batch on `stream` (overwriting every y) and keeps the fastest;
   synchronises */
cw_status cw_batch_autotune(cw_batch b, int reps, void *stream, float *best_ms);

/*
 * One-shot batched apply: cw_batch_create over the same arguments (same requirements and argument
 * errors; default mode and variants), one cw_batch_launch on `stream`, then for flags ==
 * CW_APPLY_ASSEMBLE a DSS sum (cw_dss, CW_DSS_SUM) of every right-hand side of every problem, so
 * that y_i = S A_i x_i as in cw_apply. flags: CW_APPLY_LOCAL or CW_APPLY_ASSEMBLE, else CW_ERR_ARG.
 * Synchronises `stream` and frees the batch before it returns; device errors come back here.
 * Callers that apply the same batch repeatedly should keep a cw_batch instead (no set-up per call).
 */
cw_status cw_apply_batched(const cw_op *ops, const void *const *x, void *const *y, const int *nrhs, int nprob,
                           int flags, void *stream);

/*
 * Geometric multigrid on a uniform mesh hierarchy (Sec. 3, Algorithm mg_vcycle; Sec. 5 for the
 * realisation). levels[0] is the coarsest level, levels[l+1] an operator on the uniform refinement of
 * levels[l]'s mesh (twice the cells per direction, vertices from cw_mesh_refine_vertices, so that
 * the spaces are nested: checked on the vertices, CW_ERR_ARG otherwise). All levels share degree,
 * kind and precision -- CW_PREC_F64 (double-float cycle), CW_PREC_F64_NATIVE (IEEE FP64 cycle) or
 * CW_PREC_F32 (FP32 cycle, the mixed-precision preconditioner of cw_mg_pcg_solve) -- and use
 * CW_BC_DIRICHLET0; geometry modes may differ. nu1 / nu2 pre- / post-smoothing sweeps (0..64),
 * omega in (0, 2) the damping of the Jacobi smoother.
 *  - Smoother: one sweep is Algorithm smoother_fused: v = A u, u += D_hat (b - v) per copy,
 *    u = S_bar u, with D_hat = omega K_cell D_cell^-1 (valence baked in, Eq. (valence_baking), zeros
 *    on Dirichlet DoFs: "Constraints baked into the diagonal").
 *  - Transfers: Algorithms prolongation and restriction, the restriction fed b - A u as two operands
 *    (fused residual restriction, Sec. 5). Cells are lexicographic on every level.
 *  - Coarse solve A_0^-1: the interior block of level 0's assembled matrix (element matrices in FP64)
 *    inverted once at create on the host; at most 4096 interior DoFs on level 0 (CW_ERR_UNSUPPORTED
 *    beyond).
 * The create call allocates the level vectors (right-hand side, iterate, operator output) and the
 * inverse diagonals, and synchronises the device. The operators must outlive the hierarchy, and a
 * hierarchy must not be used by two streams at once (its level vectors are shared by all calls).
 */
typedef struct cw_mg_s *cw_mg;
cw_status cw_mg_create(const cw_op *levels, int nlevels, int nu1, int nu2, double omega, cw_mg *out);
cw_status cw_mg_destroy(cw_mg mg); /* waits for the device first */
int64_t cw_mg_device_bytes(cw_mg mg);
/*
 * One V-cycle on the finest level: u <- MG(b, u) (Algorithm mg_vcycle). b: raw (unassembled) dual,
 * u: continuous primal, both cell-wise vectors of the levels' type and of the finest level's length.
 * zero_guess != 0: u enters as zero (its content is ignored; the first smoothing sweep skips the
 * operator). Asynchronous on `stream`, no host synchronisation (can be captured into a CUDA graph).
 */
cw_status cw_mg_vcycle(cw_mg mg, const void *b, void *u, int zero_guess, void *stream);
/* uf = P uc: Algorithm prolongation from level-1 to level (1 <= level < nlevels), overwriting uf */
cw_status cw_mg_prolong(cw_mg mg, int level, const void *uc, void *uf, void *stream);
/* rc = R rf: Algorithm restriction from level to level-1 (additive over the children) */
cw_status cw_mg_restrict(cw_mg mg, int level, const void *rf, void *rc, void *stream);
/* `sweeps` smoothing sweeps (Algorithm smoother_fused) on a level: u <- S(b, u); b raw dual, u continuous */
cw_status cw_mg_smooth(cw_mg mg, int level, const void *b, void *u, int sweeps, void *stream);
/* u = A_0^-1 b on the coarsest level (interior DoFs; zero on the boundary), b a raw dual */
cw_status cw_mg_coarse_solve(cw_mg mg, const void *b, void *u, void *stream);
/*
 * Solve A_CG u_g = G^T b with CG preconditioned by one V-cycle of `mg` from a zero initial guess
 * (Sec. 5), in the cell-wise primal-dual form, inside the FP64 outer refinement of cw_cg_solve (same
 * stopping measure, residual with the IEEE FP64 operator; the inner CG restarts at every outer step).
 * op: CW_PREC_F64, CW_BC_DIRICHLET0, on the finest level's mesh with its degree and kind; its
 * double-float operator runs the CG. The cycle is fed the averaged residual S_bar r (same assembly
 * G^T r, every copy small; rounded to FP32 for an FP32 hierarchy, whose output is widened back to
 * FP64). One CG iteration is captured into a CUDA graph and replayed; the host reads the device flags
 * after each. Allocates as cw_cg_solve on first use (plus two FP32 vectors for an FP32 hierarchy).
 * Synchronises `stream`; stats as cw_cg_solve (iterations = CG iterations = V-cycles).
 */
cw_status cw_mg_pcg_solve(cw_mg mg, cw_op op, const double *b, double *u, double rtol, int maxit, cw_cg_stats *stats,
                          void *stream);

/*
 * Multi-block meshes (Sec. 4.3, unstructured inter-block interfaces; Algorithm unstruct_dss): nblocks
 * operators, one per structured block, of one degree, kind and precision. The blocks are glued where
 * their boundaries meet: face to face and conforming (a shared block face has the same cells on both
 * sides), in any relative orientation, with the shared block-boundary vertices bit-identical in the
 * meshes' vertex arrays (they are matched by exact coordinates). The multi-block cell-wise vector is
 * the concatenation of the blocks' cell-wise vectors (block 0 first, each in its own [cell][k][j][i]
 * layout; cw_mblock_cellwise_len entries). Set-up (host, synchronous) identifies every node on a block
 * boundary by the global ids of its cell's vertices and its position in a canonical frame of the edge
 * or face it lies on (orientation reconciled by integer arithmetic) and builds index tables of the DoFs
 * shared by several blocks, split by the codimension of the block entity they lie on (set 0 macro-face
 * interiors, 1 macro-line interiors, 2 macro-vertices), the number of copies of every entry, and the
 * Dirichlet flags of the domain boundary (the block faces no other block shares). The operators must
 * outlive the multi-block handle.
 */
typedef struct cw_mblock_s *cw_mblock;
cw_status cw_mblock_create(const cw_op *ops, int nblocks, cw_mblock *out);
cw_status cw_mblock_destroy(cw_mblock mb); /* waits for the device first */
int64_t cw_mblock_cellwise_len(cw_mblock mb);
int64_t cw_mblock_global_len(cw_mblock mb); /* distinct DoFs of the whole mesh */
/* number of DoFs shared by several blocks in codimension set 0, 1 or 2 (-1 for a bad argument) */
int64_t cw_mblock_shared_dofs(cw_mblock mb, int set);
/* the library's global DoF of every cell-wise entry (host array of cw_mblock_cellwise_len int64) */
cw_status cw_mblock_global_index(cw_mblock mb, int64_t *out);
/*
 * v <- S v (CW_DSS_SUM) or S_bar v (CW_DSS_AVERAGE) on the multi-block cell-wise device vector of the
 * blocks' vector type: Algorithm struct_dss inside every block, then Algorithm unstruct_dss across
 * the blocks (three launches: faces, lines, vertices; each shared DoF gets the sum of one copy per
 * sharing block), then, for AVERAGE, division by the number of copies.
 */
cw_status cw_mblock_dss(cw_mblock mb, void *v, int flags, void *stream);
/* y = A x (CW_APPLY_LOCAL: every block's operator on its part) or S A x (CW_APPLY_ASSEMBLE) */
cw_status cw_mblock_apply(cw_mblock mb, const void *x, void *y, int flags, void *stream);
/* d = G diag(A_CG) of the whole multi-block mesh (FP64 cell-wise device vector) */
cw_status cw_mblock_diagonal(cw_mblock mb, double *d, void *stream);
/*
 * Solve A_CG u = G^T b on the multi-block mesh with homogeneous Dirichlet conditions on the domain
 * boundary by Jacobi-preconditioned CG in primal-dual form (Sec. 4.4), FP64 (blocks of CW_PREC_F64),
 * from u = 0, until ||m G^T r|| <= rtol ||m G^T b|| (recursive residual) or maxit (CW_ERR_NOT_CONVERGED).
 * b: FP64 cell-wise dual, u: FP64 cell-wise primal output. The first call allocates five vectors.
 * Synchronises `stream` (the host reads the residual every iteration). stats may be NULL.
 */
cw_status cw_mblock_cg_solve(cw_mblock mb, const double *b, double *u, double rtol, int maxit, cw_cg_stats *stats,
                             void *stream);

/*
 * Allocation-free variant of cw_cg_solve. The paper has no counterpart; this entry point exists
 * for callers that must not allocate device memory while solving -- e.g. code that runs inside a
 * caller-managed memory pool or an allocator callback, a real-time loop whose memory is fixed at
 * start-up, or a host whose policy forbids cudaMalloc/cudaFree after initialisation. It solves the
 * same system with the same operator, preconditioner and stopping measure as cw_cg_solve for mode
 * CW_CG_F64 or CW_CG_F64_NATIVE (arguments, outputs and statuses as there; always from u = 0:
 * CW_CG_WARM_START is rejected with CW_ERR_ARG), with three differences: the inner CG restarts at every outer refinement step (no search direction carried
 * over), the outer loop stops after 50 steps, and both the native-arithmetic inner operator and the
 * outer residual read the op's own float-pair metric (cw_cg_solve builds an IEEE-metric twin for
 * them, which would need an allocation). Iteration counts and round-off may therefore differ
 * slightly from cw_cg_solve. Every scratch vector comes from one fixed file-scope device array of
 * about 17 MB, which every GPU that loads this library holds until the process exits. It calls no
 * cudaMalloc, cudaFree or other allocating routine, creates no stream, event or graph, and runs on
 * `stream` directly, synchronising it. Limit: cw_op_cellwise_len(op) <= 262144 (2^18);
 * larger operators are rejected with CW_ERR_ARG and a message naming the limit, before any GPU
 * work. The op itself must have been created beforehand (cw_op_create allocates its geometry).
 * Every call resolves the array's device address (cudaGetSymbolAddress) with the caller's device
 * current; the first call on a device may load the library's device code there, so make it before
 * any stream capture. All calls share the one array and leave their data in it; each call
 * re-initialises what it reads. Calls that overlap on the GPU (from two streams or two threads)
 * race on the array and must be serialised by the caller. stats->seconds is host wall time.
 */
cw_status cw_cg_solve_noalloc(cw_op op, const double *b, double *u, double rtol, int maxit, int mode,
                              cw_cg_stats *stats, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* CWFEM_H */
