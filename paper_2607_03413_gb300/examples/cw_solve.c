/*
 * cw_solve.c -- the C ABI from plain C (no Python, no PyTorch): the manufactured Poisson problem
 * -lap u = 3 pi^2 sin(pi x) sin(pi y) sin(pi z) with homogeneous Dirichlet conditions on a curved
 * n^3 mesh of the unit cube, Q_p elements.
 *
 *   1. cell-wise load vector (cw_load_vector) and a loose solve (rtol 1e-4) by Jacobi-PCG, FP32 inner
 *      CG inside the FP64 refinement (Sec. 4.1 Eq. (jacobi_recap), Sec. 4.4);
 *   2. checkpoint: the iterate copied to host memory, the device copy overwritten;
 *   3. resume from the checkpoint (CW_CG_WARM_START) to rtol 1e-10, and the relative residual
 *      evaluated again with the IEEE FP64 operator (cw_cg_residual);
 *   4. the nodal error of the discrete solution against u* at every cell-wise node, the node
 *      positions formed here from the box mesh's vertex formula, the library's Gauss-Lobatto
 *      nodes (cw_rules_1d) and the trilinear cell map;
 *   5. the assembled apply y = S A u (cw_apply, CW_APPLY_ASSEMBLE) and the device status check.
 *
 * Build (CUDA_HOME the toolkit, LIB the directory of libcwfem.so):
 *   gcc -std=c11 -O2 -I include -I $CUDA_HOME/include cw_solve.c -L $LIB -lcwfem \
 *       -L $CUDA_HOME/lib64 -lcudart -lm -Wl,-rpath,$LIB -o cw_solve
 * Run: ./cw_solve [cells per direction, default 16] [degree, default 3]. Prints "ok" and exits 0
 * when the resumed solve reaches 1e-10 and the nodal error is below 1e-3 (p >= 2).
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime_api.h>

#include "cwfem.h"

#define CW_CHECK(call)                                                                                  \
    do {                                                                                                \
        cw_status s_ = (call);                                                                          \
        if (s_ != CW_OK) {                                                                              \
            fprintf(stderr, "%s: %s (%s)\n", #call, cw_status_string(s_), cw_last_error());             \
            return 1;                                                                                   \
        }                                                                                               \
    } while (0)

#define CUDA_CHECK(call)                                                                                \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) {                                                                        \
            fprintf(stderr, "%s: %s\n", #call, cudaGetErrorString(e_));                                 \
            return 1;                                                                                   \
        }                                                                                               \
    } while (0)

static const double kPi = 3.14159265358979323846;

/* vertex (ix, iy, iz) of the n^3 box mesh moved by perturb * h * sin(2 pi X) sin(2 pi Y) sin(2 pi Z)
   along (1, 1, 1)/sqrt(3): the cw_mesh_create_box formula with its default frequencies and direction */
static void box_vertex(int n, double perturb, int ix, int iy, int iz, double *x)
{
    const double X = (double)ix / n, Y = (double)iy / n, Z = (double)iz / n;
    const double d = perturb / n * sin(2 * kPi * X) * sin(2 * kPi * Y) * sin(2 * kPi * Z) / sqrt(3.0);
    x[0] = X + d;
    x[1] = Y + d;
    x[2] = Z + d;
}

int main(int argc, char **argv)
{
    const int n = argc > 1 ? atoi(argv[1]) : 16;
    const int p = argc > 2 ? atoi(argv[2]) : 3;
    const double perturb = 0.1;
    if (n < 1 || p < 1 || p > 7) {
        fprintf(stderr, "usage: cw_solve [cells per direction >= 1] [degree 1..7]\n");
        return 2;
    }
    cw_mesh mesh = NULL;
    cw_op op = NULL;
    CW_CHECK(cw_mesh_create_box(n, n, n, perturb, NULL, NULL, &mesh));
    CW_CHECK(cw_op_create(mesh, p, CW_LAPLACE, CW_GEOM_METRIC, CW_PREC_F64, CW_BC_DIRICHLET0, &op));
    const int64_t L = cw_op_cellwise_len(op);
    const size_t bytes = (size_t)L * sizeof(double);
    double *b = NULL, *u = NULL, *y = NULL;
    CUDA_CHECK(cudaMalloc((void **)&b, bytes));
    CUDA_CHECK(cudaMalloc((void **)&u, bytes));
    CUDA_CHECK(cudaMalloc((void **)&y, bytes));
    double *host = (double *)malloc(bytes);
    if (!host) return 1;

    /* 1. loose solve */
    CW_CHECK(cw_load_vector(op, 0, b, NULL));
    cw_cg_stats st1, st2;
    CW_CHECK(cw_cg_solve(op, b, u, 1e-4, 100000, CW_CG_IR_F32, &st1, NULL));
    /* 2. checkpoint on the host; the device iterate is lost */
    CUDA_CHECK(cudaMemcpy(host, u, bytes, cudaMemcpyDeviceToHost));
    CUDA_CHECK(cudaMemset(u, 0xff, bytes)); /* NaN bit patterns */
    /* 3. resume */
    CUDA_CHECK(cudaMemcpy(u, host, bytes, cudaMemcpyHostToDevice));
    CW_CHECK(cw_cg_solve(op, b, u, 1e-10, 100000, CW_CG_IR_F32 | CW_CG_WARM_START, &st2, NULL));
    double rel = 0.0;
    CW_CHECK(cw_cg_residual(op, b, u, CW_PREC_F64_NATIVE, &rel, NULL));

    /* 4. nodal error against u* = sin(pi x) sin(pi y) sin(pi z) */
    CUDA_CHECK(cudaMemcpy(host, u, bytes, cudaMemcpyDeviceToHost));
    double gll[8], gq[8], wq[8];
    CW_CHECK(cw_rules_1d(p, gll, gq, wq));
    const int nn = p + 1;
    double err = 0.0, umax = 0.0;
    for (int cz = 0; cz < n; ++cz)
        for (int cy = 0; cy < n; ++cy)
            for (int cx = 0; cx < n; ++cx) {
                double V[8][3];
                for (int v = 0; v < 8; ++v) box_vertex(n, perturb, cx + (v & 1), cy + ((v >> 1) & 1), cz + (v >> 2), V[v]);
                const int64_t cell = cx + (int64_t)n * (cy + (int64_t)n * cz);
                for (int k = 0; k < nn; ++k)
                    for (int j = 0; j < nn; ++j)
                        for (int i = 0; i < nn; ++i) {
                            const double s[3] = {gll[i], gll[j], gll[k]};
                            double x[3] = {0.0, 0.0, 0.0};
                            for (int v = 0; v < 8; ++v) {
                                const double N = ((v & 1) ? s[0] : 1 - s[0]) * (((v >> 1) & 1) ? s[1] : 1 - s[1]) *
                                                 ((v >> 2) ? s[2] : 1 - s[2]);
                                for (int a = 0; a < 3; ++a) x[a] += N * V[v][a];
                            }
                            const double ue = sin(kPi * x[0]) * sin(kPi * x[1]) * sin(kPi * x[2]);
                            const double uh = host[cell * nn * nn * nn + i + nn * (j + nn * k)];
                            err = fmax(err, fabs(uh - ue));
                            umax = fmax(umax, fabs(ue));
                        }
            }

    /* 5. assembled apply of the solution, then the operator's device status */
    CW_CHECK(cw_apply(op, u, y, CW_APPLY_ASSEMBLE, NULL));
    CW_CHECK(cw_op_check(op, NULL));
    CUDA_CHECK(cudaDeviceSynchronize());

    printf("mesh %d^3 Q%d, %lld cell-wise values\n", n, p, (long long)L);
    printf("loose solve: %d iterations, rel residual %.3e\n", st1.iterations, st1.rel_residual);
    printf("resumed solve: %d iterations in %d outer steps, rel residual %.3e (IEEE FP64 operator %.3e)\n",
           st2.iterations, st2.outer_iterations, st2.rel_residual, rel);
    printf("max nodal error %.3e (max |u*| %.3f)\n", err, umax);
    const int ok = rel <= 1e-10 && st2.rel_residual <= 1e-10 && (p < 2 || err / umax < 1e-3);
    printf("%s\n", ok ? "ok" : "FAILED");

    free(host);
    cudaFree(b);
    cudaFree(u);
    cudaFree(y);
    CW_CHECK(cw_op_destroy(op));
    CW_CHECK(cw_mesh_destroy(mesh));
    return ok ? 0 : 1;
}
