/*
 * oracle.c -- plain FP64 CPU reference for the cell-wise high-order FEM hot path.
 *
 * TEST INFRASTRUCTURE ONLY. This file is compiled into liboracle.so, which only the tests,
 * the smoke check and the benchmark's CPU-baseline leg load. The CUDA library never links,
 * includes or calls it, and it shares no code, tables or constants with the CUDA path.
 *
 * What it computes (the plain definitions, no sum factorisation, no tensor-product tricks):
 *  - 1D Gauss-Legendre rule with q points and the Gauss-Lobatto nodes of degree p on [0,1]
 *    (the Q_p Gauss-Lobatto nodal basis of the Poisson discretisation, Sec. 2, Eq. (poisson));
 *  - per cell, with the trilinear map x(xi) of its 8 vertices, the element stiffness matrix
 *    K_ij = sum_q w_q detJ (J^-T grad phi_i).(J^-T grad phi_j) and the element mass matrix
 *    M_ij = sum_q w_q detJ phi_i phi_j, by explicit loops over i, j and the 3D quadrature points;
 *  - the cell-local operator A: V_cell -> V_cell^* as y_K = A_K x_K (Sec. 2.1, the local operator
 *    that maps a primal vector to an unassembled dual vector);
 *  - the global numbering, the gather G and the additive assembly G^T (Sec. 2.1), and the direct
 *    stiffness summation S = G G^T (Sec. 4.1, Eq. (dss_operator)) by global index;
 *  - the assembled diagonal d = G^T diag(A_K) (Sec. 4.1, Eq. (jacobi_recap));
 *  - the load vector b_K,i = sum_q w_q detJ f(x_q) phi_i(x_q) and L2 / H1 errors against the
 *    manufactured solution u = sin(pi x) sin(pi y) sin(pi z), f = 3 pi^2 u;
 *  - the cell-wise inter-grid transfers of a uniform mesh hierarchy (Sec. 3, Algorithms
 *    prolongation and restriction): per parent cell and child, the Kronecker product of the 1D
 *    child prolongation matrices, written out entry by entry.
 *
 * Conventions: reference cell [0,1]^3; local DoF index i + n*(j + n*k) with i along x;
 * cells numbered cx + nx*(cy + ny*cz); vertices V[((vz*(ny+1) + vy)*(nx+1) + vx)*3 + d];
 * global DoF gx + (nx*p+1)*(gy + (ny*p+1)*gz) with gx = cx*p + i.
 * Quadrature for the operators and the load vector: q = p+1 Gauss points per direction.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXN 16

/* ---------------------------------------------------------------- 1D rules ---- */

/* Legendre polynomial P_n(t) and its derivative by the three-term recurrence. */
static void legendre(int n, double t, double *P, double *dP)
{
    double p0 = 1.0, p1 = t;
    if (n == 0) { *P = 1.0; *dP = 0.0; return; }
    for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    *P = p1;
    /* derivative from (t^2-1) P_n' = n (t P_n - P_{n-1}); only used away from t = +-1 */
    *dP = n * (t * p1 - p0) / (t * t - 1.0);
}

/* q-point Gauss-Legendre rule on [0,1], nodes ascending. Returns 0 on success. */
int orc_gauss(int q, double *x, double *w)
{
    if (q < 1 || q > ORC_MAXN) return -1;
    for (int i = 0; i < q; ++i) {
        double t = cos(M_PI * (i + 0.75) / (q + 0.5)), P, dP;
        for (int it = 0; it < 100; ++it) {
            legendre(q, t, &P, &dP);
            double dt = P / dP;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        legendre(q, t, &P, &dP);
        /* t_i descending in i; store ascending on [0,1] */
        x[q - 1 - i] = 0.5 * (1.0 + t);
        w[q - 1 - i] = 0.5 * 2.0 / ((1.0 - t * t) * dP * dP);
    }
    return 0;
}

/* Gauss-Lobatto nodes of degree p (p+1 nodes) on [0,1]: the end points and the roots of P_p'. */
int orc_gll(int p, double *x)
{
    if (p < 1 || p + 1 > ORC_MAXN) return -1;
    x[0] = 0.0;
    x[p] = 1.0;
    for (int i = 1; i < p; ++i) {
        double t = -cos(M_PI * i / p); /* ascending initial guesses */
        for (int it = 0; it < 100; ++it) {
            double P, dP;
            legendre(p, t, &P, &dP);
            /* Legendre ODE: (1-t^2) P'' = 2 t P' - p(p+1) P */
            double d2P = (2.0 * t * dP - p * (p + 1.0) * P) / (1.0 - t * t);
            double dt = dP / d2P;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        x[i] = 0.5 * (1.0 + t);
    }
    return 0;
}

/* Lagrange basis of the n nodes and its derivative at xi, by the product formula. */
void orc_lagrange(int n, const double *nodes, double xi, double *l, double *dl)
{
    for (int i = 0; i < n; ++i) {
        double prod = 1.0;
        for (int m = 0; m < n; ++m)
            if (m != i) prod *= (xi - nodes[m]) / (nodes[i] - nodes[m]);
        l[i] = prod;
        double s = 0.0;
        for (int k = 0; k < n; ++k) {
            if (k == i) continue;
            double t = 1.0 / (nodes[i] - nodes[k]);
            for (int m = 0; m < n; ++m)
                if (m != i && m != k) t *= (xi - nodes[m]) / (nodes[i] - nodes[m]);
            s += t;
        }
        dl[i] = s;
    }
}

/* ------------------------------------------------------------ geometry ---- */

static void cell_vertices(int nx, int ny, const double *V, int64_t e, int nxc, int nyc, double X[8][3])
{
    (void)nyc;
    int64_t cx = e % nxc, cy = (e / nxc) % ny, cz = e / ((int64_t)nxc * ny);
    for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                int v = a + 2 * b + 4 * c;
                int64_t vid = ((cz + c) * (ny + 1) + (cy + b)) * (int64_t)(nx + 1) + (cx + a);
                for (int d = 0; d < 3; ++d) X[v][d] = V[vid * 3 + d];
            }
}

/* Trilinear map at xi: physical point x, Jacobian J[r][s] = dx_r / dxi_s. */
static void trilinear(const double X[8][3], const double xi[3], double x[3], double J[3][3])
{
    for (int r = 0; r < 3; ++r) {
        x[r] = 0.0;
        for (int s = 0; s < 3; ++s) J[r][s] = 0.0;
    }
    for (int v = 0; v < 8; ++v) {
        int bit[3] = {v & 1, (v >> 1) & 1, (v >> 2) & 1};
        double f[3], df[3];
        for (int d = 0; d < 3; ++d) {
            f[d] = bit[d] ? xi[d] : 1.0 - xi[d];
            df[d] = bit[d] ? 1.0 : -1.0;
        }
        double N = f[0] * f[1] * f[2];
        double dN[3] = {df[0] * f[1] * f[2], f[0] * df[1] * f[2], f[0] * f[1] * df[2]};
        for (int r = 0; r < 3; ++r) {
            x[r] += X[v][r] * N;
            for (int s = 0; s < 3; ++s) J[r][s] += X[v][r] * dN[s];
        }
    }
}

/* detJ and inverse by the adjugate. */
static double inverse3(const double J[3][3], double Ji[3][3])
{
    double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
               - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
               + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    return det;
}

/* 1D tables of the nodal basis at nq points: L[a*n+i] = l_i(xi_a), dL likewise. */
static void basis_tables(int p, int nq, const double *xq, double *L, double *dL)
{
    int n = p + 1;
    double nodes[ORC_MAXN];
    orc_gll(p, nodes);
    for (int a = 0; a < nq; ++a) orc_lagrange(n, nodes, xq[a], L + a * n, dL + a * n);
}

/*
 * Element matrices of one cell (n^3 x n^3, row-major). K or M may be NULL.
 * Returns 0, or -1 when detJ <= 0 at some quadrature point.
 */
int orc_element_matrices(int p, const double *X24, double *K, double *M)
{
    const int n = p + 1, q = p + 1, n3 = n * n * n;
    double X[8][3];
    memcpy(X, X24, sizeof X);
    double xq[ORC_MAXN], wq[ORC_MAXN], L[ORC_MAXN * ORC_MAXN], dL[ORC_MAXN * ORC_MAXN];
    orc_gauss(q, xq, wq);
    basis_tables(p, q, xq, L, dL);
    double *phi = malloc(sizeof(double) * n3), *gphi = malloc(sizeof(double) * 3 * n3);
    if (K) memset(K, 0, sizeof(double) * n3 * n3);
    if (M) memset(M, 0, sizeof(double) * n3 * n3);
    int bad = 0;
    for (int c = 0; c < q; ++c)
        for (int b = 0; b < q; ++b)
            for (int a = 0; a < q; ++a) {
                double xi[3] = {xq[a], xq[b], xq[c]}, x[3], J[3][3], Ji[3][3];
                trilinear(X, xi, x, J);
                double det = inverse3(J, Ji);
                if (!(det > 0.0)) bad = 1;
                double W = wq[a] * wq[b] * wq[c] * det;
                for (int k = 0; k < n; ++k)
                    for (int j = 0; j < n; ++j)
                        for (int i = 0; i < n; ++i) {
                            int id = i + n * (j + n * k);
                            double la = L[a * n + i], lb = L[b * n + j], lc = L[c * n + k];
                            double g[3] = {dL[a * n + i] * lb * lc, la * dL[b * n + j] * lc,
                                           la * lb * dL[c * n + k]};
                            phi[id] = la * lb * lc;
                            /* physical gradient: J^-T g, (J^-T)_{rs} = Ji[s][r] */
                            for (int r = 0; r < 3; ++r)
                                gphi[3 * id + r] = Ji[0][r] * g[0] + Ji[1][r] * g[1] + Ji[2][r] * g[2];
                        }
                for (int i = 0; i < n3; ++i)
                    for (int j = i; j < n3; ++j) {
                        if (K) {
                            double s = gphi[3 * i] * gphi[3 * j] + gphi[3 * i + 1] * gphi[3 * j + 1]
                                     + gphi[3 * i + 2] * gphi[3 * j + 2];
                            K[(int64_t)i * n3 + j] += W * s;
                        }
                        if (M) M[(int64_t)i * n3 + j] += W * phi[i] * phi[j];
                    }
            }
    /* the loops above filled the upper triangle; both matrices are symmetric by definition */
    for (int i = 0; i < n3; ++i)
        for (int j = 0; j < i; ++j) {
            if (K) K[(int64_t)i * n3 + j] = K[(int64_t)j * n3 + i];
            if (M) M[(int64_t)i * n3 + j] = M[(int64_t)j * n3 + i];
        }
    free(phi);
    free(gphi);
    return bad ? -1 : 0;
}

/* Vertices of cell e of an nx*ny*nz box mesh as a flat [8][3] array. */
void orc_cell_vertices(int nx, int ny, int nz, const double *V, int64_t e, double *X24)
{
    (void)nz;
    double X[8][3];
    cell_vertices(nx, ny, V, e, nx, ny, X);
    memcpy(X24, X, sizeof X);
}

/*
 * Cell-local operator y_K = (kind&1 ? K_K : 0) x_K + (kind&2 ? M_K : 0) x_K for the listed cells
 * (all cells when cells == NULL); x and y are full cell-wise arrays, only listed cells of y are
 * written. Element matrices are built explicitly per cell. Returns the number of cells with a
 * non-positive Jacobian determinant.
 */
int64_t orc_apply_local(int nx, int ny, int nz, const double *V, int p, int kind, const double *x,
                        double *y, int64_t ncl, const int64_t *cells)
{
    const int n = p + 1, n3 = n * n * n;
    const int64_t E = (int64_t)nx * ny * nz, cnt = cells ? ncl : E;
    int64_t nbad = 0;
#pragma omp parallel reduction(+ : nbad)
    {
        double *K = malloc(sizeof(double) * n3 * n3), *M = malloc(sizeof(double) * n3 * n3);
#pragma omp for schedule(dynamic, 4)
        for (int64_t t = 0; t < cnt; ++t) {
            int64_t e = cells ? cells[t] : t;
            double X[8][3];
            cell_vertices(nx, ny, V, e, nx, ny, X);
            if (orc_element_matrices(p, &X[0][0], (kind & 1) ? K : NULL, (kind & 2) ? M : NULL))
                ++nbad;
            const double *xe = x + e * n3;
            double *ye = y + e * n3;
            for (int i = 0; i < n3; ++i) {
                double s = 0.0;
                for (int j = 0; j < n3; ++j) {
                    double a = 0.0;
                    if (kind & 1) a += K[(int64_t)i * n3 + j];
                    if (kind & 2) a += M[(int64_t)i * n3 + j];
                    s += a * xe[j];
                }
                ye[i] = s;
            }
        }
        free(K);
        free(M);
    }
    (void)nz;
    return nbad;
}

/* ------------------------------------------------- numbering, G, G^T, S ---- */

/* Global index of every cell-wise entry: map[e*n^3 + local]. */
void orc_global_index(int nx, int ny, int nz, int p, int64_t *map)
{
    const int n = p + 1, n3 = n * n * n;
    const int64_t gnx = (int64_t)nx * p + 1, gny = (int64_t)ny * p + 1;
    const int64_t E = (int64_t)nx * ny * nz;
#pragma omp parallel for
    for (int64_t e = 0; e < E; ++e) {
        int64_t cx = e % nx, cy = (e / nx) % ny, cz = e / ((int64_t)nx * ny);
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i)
                    map[e * n3 + i + n * (j + n * k)] =
                        (cx * p + i) + gnx * ((cy * p + j) + gny * (cz * p + k));
    }
}

/* Gather G: replicate each global coefficient into all its cell-local copies. */
void orc_gather(int nx, int ny, int nz, int p, const double *ug, double *xc)
{
    const int n = p + 1, n3 = n * n * n;
    const int64_t L = (int64_t)nx * ny * nz * n3;
    int64_t *map = malloc(sizeof(int64_t) * L);
    orc_global_index(nx, ny, nz, p, map);
#pragma omp parallel for
    for (int64_t t = 0; t < L; ++t) xc[t] = ug[map[t]];
    free(map);
}

/* Additive assembly G^T: sum all cell-local copies into the global entry (sequential, exact order). */
void orc_scatter_add(int nx, int ny, int nz, int p, const double *yc, double *fg)
{
    const int n = p + 1, n3 = n * n * n;
    const int64_t L = (int64_t)nx * ny * nz * n3;
    const int64_t NG = ((int64_t)nx * p + 1) * ((int64_t)ny * p + 1) * ((int64_t)nz * p + 1);
    int64_t *map = malloc(sizeof(int64_t) * L);
    orc_global_index(nx, ny, nz, p, map);
    memset(fg, 0, sizeof(double) * NG);
    for (int64_t t = 0; t < L; ++t) fg[map[t]] += yc[t];
    free(map);
}

/* Direct stiffness summation S = G G^T, out of place. */
void orc_dss(int nx, int ny, int nz, int p, const double *yc, double *zc)
{
    const int64_t NG = ((int64_t)nx * p + 1) * ((int64_t)ny * p + 1) * ((int64_t)nz * p + 1);
    double *fg = malloc(sizeof(double) * NG);
    orc_scatter_add(nx, ny, nz, p, yc, fg);
    orc_gather(nx, ny, nz, p, fg, zc);
    free(fg);
}

/* Assembled diagonal d = G^T diag(A_K) as a global vector. */
void orc_diagonal(int nx, int ny, int nz, const double *V, int p, int kind, double *dg)
{
    const int n = p + 1, n3 = n * n * n;
    const int64_t E = (int64_t)nx * ny * nz;
    double *dc = malloc(sizeof(double) * E * n3);
#pragma omp parallel
    {
        double *K = malloc(sizeof(double) * n3 * n3), *M = malloc(sizeof(double) * n3 * n3);
#pragma omp for schedule(dynamic, 4)
        for (int64_t e = 0; e < E; ++e) {
            double X[8][3];
            cell_vertices(nx, ny, V, e, nx, ny, X);
            orc_element_matrices(p, &X[0][0], (kind & 1) ? K : NULL, (kind & 2) ? M : NULL);
            for (int i = 0; i < n3; ++i) {
                double a = 0.0;
                if (kind & 1) a += K[(int64_t)i * n3 + i];
                if (kind & 2) a += M[(int64_t)i * n3 + i];
                dc[e * n3 + i] = a;
            }
        }
        free(K);
        free(M);
    }
    orc_scatter_add(nx, ny, nz, p, dc, dg);
    free(dc);
    (void)nz;
}

/* All element matrices of the mesh, [E][n^3][n^3] (for assembling small global matrices). */
int64_t orc_all_element_matrices(int nx, int ny, int nz, const double *V, int p, int kind, double *A)
{
    const int n = p + 1, n3 = n * n * n;
    const int64_t E = (int64_t)nx * ny * nz, sz = (int64_t)n3 * n3;
    int64_t nbad = 0;
#pragma omp parallel reduction(+ : nbad)
    {
        double *K = malloc(sizeof(double) * sz), *M = malloc(sizeof(double) * sz);
#pragma omp for schedule(dynamic, 4)
        for (int64_t e = 0; e < E; ++e) {
            double X[8][3];
            cell_vertices(nx, ny, V, e, nx, ny, X);
            if (orc_element_matrices(p, &X[0][0], (kind & 1) ? K : NULL, (kind & 2) ? M : NULL)) ++nbad;
            for (int64_t t = 0; t < sz; ++t)
                A[e * sz + t] = ((kind & 1) ? K[t] : 0.0) + ((kind & 2) ? M[t] : 0.0);
        }
        free(K);
        free(M);
    }
    (void)nz;
    return nbad;
}

/* ------------------------------------------- load vector and error norms ---- */

/*
 * Manufactured problems for -Laplace(u) = f on the unit cube, u = 0 on the boundary:
 *  which = 0: u = sin(pi x) sin(pi y) sin(pi z),      f = 3 pi^2 u;
 *  which = 1: u = x(1-x) y(1-y) z(1-z) (in Q_2),      f = 2 [y(1-y)z(1-z) + x(1-x)z(1-z) + x(1-x)y(1-y)].
 */
static void exact_solution(int which, const double x[3], double *u, double g[3], double *f)
{
    if (which == 0) {
        double s[3] = {sin(M_PI * x[0]), sin(M_PI * x[1]), sin(M_PI * x[2])};
        double c[3] = {cos(M_PI * x[0]), cos(M_PI * x[1]), cos(M_PI * x[2])};
        *u = s[0] * s[1] * s[2];
        g[0] = M_PI * c[0] * s[1] * s[2];
        g[1] = M_PI * s[0] * c[1] * s[2];
        g[2] = M_PI * s[0] * s[1] * c[2];
        *f = 3.0 * M_PI * M_PI * *u;
    } else {
        double b[3], db[3];
        for (int d = 0; d < 3; ++d) {
            b[d] = x[d] * (1.0 - x[d]);
            db[d] = 1.0 - 2.0 * x[d];
        }
        *u = b[0] * b[1] * b[2];
        g[0] = db[0] * b[1] * b[2];
        g[1] = b[0] * db[1] * b[2];
        g[2] = b[0] * b[1] * db[2];
        *f = 2.0 * (b[1] * b[2] + b[0] * b[2] + b[0] * b[1]);
    }
}

/* Unassembled load vector b_K,i = sum_q w_q detJ f(x_q) phi_i(x_q) of problem `which`, q = p+1. */
void orc_load_vector(int nx, int ny, int nz, const double *V, int p, int which, double *b)
{
    const int n = p + 1, q = p + 1, n3 = n * n * n;
    const int64_t E = (int64_t)nx * ny * nz;
    double xq[ORC_MAXN], wq[ORC_MAXN], L[ORC_MAXN * ORC_MAXN], dL[ORC_MAXN * ORC_MAXN];
    orc_gauss(q, xq, wq);
    basis_tables(p, q, xq, L, dL);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t e = 0; e < E; ++e) {
        double X[8][3];
        cell_vertices(nx, ny, V, e, nx, ny, X);
        double *be = b + e * n3;
        for (int i = 0; i < n3; ++i) be[i] = 0.0;
        for (int c = 0; c < q; ++c)
            for (int bb = 0; bb < q; ++bb)
                for (int a = 0; a < q; ++a) {
                    double xi[3] = {xq[a], xq[bb], xq[c]}, x[3], J[3][3], Ji[3][3];
                    trilinear(X, xi, x, J);
                    double det = inverse3(J, Ji);
                    double uu, gg[3], f;
                    exact_solution(which, x, &uu, gg, &f);
                    double W = wq[a] * wq[bb] * wq[c] * det * f;
                    for (int k = 0; k < n; ++k)
                        for (int j = 0; j < n; ++j)
                            for (int i = 0; i < n; ++i)
                                be[i + n * (j + n * k)] += W * L[a * n + i] * L[bb * n + j] * L[c * n + k];
                }
    }
    (void)nz;
}

/*
 * L2 error and H1 seminorm error of the cell-wise primal u against the exact solution of problem
 * `which`, with nq Gauss points per direction (nq = p+3 recommended). out = {||e||_L2, |e|_H1}.
 */
void orc_error_norms(int nx, int ny, int nz, const double *V, int p, int which, int nq, const double *u,
                     double *out)
{
    const int n = p + 1, n3 = n * n * n;
    const int64_t E = (int64_t)nx * ny * nz;
    double xq[ORC_MAXN], wq[ORC_MAXN], L[ORC_MAXN * ORC_MAXN], dL[ORC_MAXN * ORC_MAXN];
    orc_gauss(nq, xq, wq);
    basis_tables(p, nq, xq, L, dL);
    double l2 = 0.0, h1 = 0.0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : l2, h1)
    for (int64_t e = 0; e < E; ++e) {
        double X[8][3];
        cell_vertices(nx, ny, V, e, nx, ny, X);
        const double *ue = u + e * n3;
        for (int c = 0; c < nq; ++c)
            for (int bb = 0; bb < nq; ++bb)
                for (int a = 0; a < nq; ++a) {
                    double xi[3] = {xq[a], xq[bb], xq[c]}, x[3], J[3][3], Ji[3][3];
                    trilinear(X, xi, x, J);
                    double det = inverse3(J, Ji);
                    double W = wq[a] * wq[bb] * wq[c] * det;
                    double uh = 0.0, g[3] = {0.0, 0.0, 0.0};
                    for (int k = 0; k < n; ++k)
                        for (int j = 0; j < n; ++j)
                            for (int i = 0; i < n; ++i) {
                                double v = ue[i + n * (j + n * k)];
                                double la = L[a * n + i], lb = L[bb * n + j], lc = L[c * n + k];
                                uh += v * la * lb * lc;
                                g[0] += v * dL[a * n + i] * lb * lc;
                                g[1] += v * la * dL[bb * n + j] * lc;
                                g[2] += v * la * lb * dL[c * n + k];
                            }
                    double gx[3];
                    for (int r = 0; r < 3; ++r) gx[r] = Ji[0][r] * g[0] + Ji[1][r] * g[1] + Ji[2][r] * g[2];
                    double ue_, ge[3], fe;
                    exact_solution(which, x, &ue_, ge, &fe);
                    l2 += W * (uh - ue_) * (uh - ue_);
                    for (int r = 0; r < 3; ++r) h1 += W * (gx[r] - ge[r]) * (gx[r] - ge[r]);
                }
    }
    out[0] = sqrt(l2);
    out[1] = sqrt(h1);
    (void)nz;
}

/* Physical coordinates of every cell-wise node (for interpolating exact functions). */
void orc_node_coords(int nx, int ny, int nz, const double *V, int p, double *xyz)
{
    const int n = p + 1, n3 = n * n * n;
    const int64_t E = (int64_t)nx * ny * nz;
    double nodes[ORC_MAXN];
    orc_gll(p, nodes);
#pragma omp parallel for
    for (int64_t e = 0; e < E; ++e) {
        double X[8][3];
        cell_vertices(nx, ny, V, e, nx, ny, X);
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    double xi[3] = {nodes[i], nodes[j], nodes[k]}, x[3], J[3][3];
                    trilinear(X, xi, x, J);
                    for (int r = 0; r < 3; ++r) xyz[(e * n3 + i + n * (j + n * k)) * 3 + r] = x[r];
                }
    }
    (void)nz;
}

/* ------------------------------------------------ inter-grid transfers ---- */

/* The 1D prolongation matrices of the two children of an interval (Sec. 3, inter-grid transfers):
   child b in {0, 1} covers [b/2, (b+1)/2] of the parent's reference interval, so its node xi_i
   sits at (xi_i + b)/2 there, and P_b[i][a] = l_a((xi_i + b)/2) with l_a the parent's Lagrange
   basis on the Gauss-Lobatto nodes. */
void orc_prolong_1d(int p, double *P0, double *P1)
{
    const int n = p + 1;
    double xi[ORC_MAXN], l[ORC_MAXN], dl[ORC_MAXN];
    orc_gll(p, xi);
    for (int b = 0; b < 2; ++b)
        for (int i = 0; i < n; ++i) {
            orc_lagrange(n, xi, 0.5 * (xi[i] + b), l, dl);
            for (int a = 0; a < n; ++a) (b ? P1 : P0)[i * n + a] = l[a];
        }
}

/* Child c = bx + 2 by + 4 bz of coarse cell (cx, cy, cz) is fine cell (2cx+bx, 2cy+by, 2cz+bz) of
   the 2ncx x 2ncy x 2ncz mesh; bit d of c selects P_0 or P_1 along axis d. */
static int64_t child_cell(int ncx, int ncy, int64_t cx, int64_t cy, int64_t cz, int c)
{
    const int64_t nfx = 2 * (int64_t)ncx, nfy = 2 * (int64_t)ncy;
    return (2 * cx + (c & 1)) + nfx * ((2 * cy + ((c >> 1) & 1)) + nfy * (2 * cz + ((c >> 2) & 1)));
}

/* Algorithm prolongation: for every coarse cell K and child K_c,
   u_f|K_c = (P_bz (x) P_by (x) P_bx) u_c|K, the Kronecker product written out entry by entry:
   u_f[i,j,k] = sum_{a,b,c} P_bx[i][a] P_by[j][b] P_bz[k][c] u_c[a,b,c]. Every fine cell is the
   child of exactly one coarse cell, so the zero-initialised accumulation of the algorithm is an
   assignment here. */
void orc_prolong(int ncx, int ncy, int ncz, int p, const double *uc, double *uf)
{
    const int n = p + 1, n3 = n * n * n;
    double P[2][ORC_MAXN * ORC_MAXN];
    orc_prolong_1d(p, P[0], P[1]);
    const int64_t E = (int64_t)ncx * ncy * ncz;
#pragma omp parallel for
    for (int64_t e = 0; e < E; ++e) {
        const int64_t cx = e % ncx, cy = (e / ncx) % ncy, cz = e / ((int64_t)ncx * ncy);
        const double *u = uc + e * n3;
        for (int ch = 0; ch < 8; ++ch) {
            const double *Px = P[ch & 1], *Py = P[(ch >> 1) & 1], *Pz = P[(ch >> 2) & 1];
            double *y = uf + child_cell(ncx, ncy, cx, cy, cz, ch) * n3;
            for (int k = 0; k < n; ++k)
                for (int j = 0; j < n; ++j)
                    for (int i = 0; i < n; ++i) {
                        double s = 0.0;
                        for (int c = 0; c < n; ++c)
                            for (int b = 0; b < n; ++b)
                                for (int a = 0; a < n; ++a)
                                    s += Px[i * n + a] * Py[j * n + b] * Pz[k * n + c] * u[a + n * (b + n * c)];
                        y[i + n * (j + n * k)] = s;
                    }
        }
    }
    (void)ncz;
}

/* Algorithm restriction: for every coarse cell K, r_c|K = sum over its children K_c of
   (P_bz^T (x) P_by^T (x) P_bx^T) r_f|K_c, i.e.
   r_c[a,b,c] = sum_c sum_{i,j,k} P_bx[i][a] P_by[j][b] P_bz[k][c] r_f|K_c[i,j,k]. Acts on raw
   (unassembled) dual vectors: no assembly and no weights. */
void orc_restrict(int ncx, int ncy, int ncz, int p, const double *rf, double *rc)
{
    const int n = p + 1, n3 = n * n * n;
    double P[2][ORC_MAXN * ORC_MAXN];
    orc_prolong_1d(p, P[0], P[1]);
    const int64_t E = (int64_t)ncx * ncy * ncz;
#pragma omp parallel for
    for (int64_t e = 0; e < E; ++e) {
        const int64_t cx = e % ncx, cy = (e / ncx) % ncy, cz = e / ((int64_t)ncx * ncy);
        double *r = rc + e * n3;
        for (int q = 0; q < n3; ++q) r[q] = 0.0;
        for (int ch = 0; ch < 8; ++ch) {
            const double *Px = P[ch & 1], *Py = P[(ch >> 1) & 1], *Pz = P[(ch >> 2) & 1];
            const double *y = rf + child_cell(ncx, ncy, cx, cy, cz, ch) * n3;
            for (int c = 0; c < n; ++c)
                for (int b = 0; b < n; ++b)
                    for (int a = 0; a < n; ++a) {
                        double s = 0.0;
                        for (int k = 0; k < n; ++k)
                            for (int j = 0; j < n; ++j)
                                for (int i = 0; i < n; ++i)
                                    s += Px[i * n + a] * Py[j * n + b] * Pz[k * n + c] * y[i + n * (j + n * k)];
                        r[a + n * (b + n * c)] += s;
                    }
        }
    }
    (void)ncz;
}
