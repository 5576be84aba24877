// cw_tables.cpp -- the library's 1D Gauss / Gauss-Lobatto rules and basis tables.
//
// Computed once per operator on the host in long double: Gauss-Legendre points as roots of P_n
// (Newton from Tricomi-type initial guesses), Gauss-Lobatto nodes as the end points plus the roots
// of P_p' (Newton on the Legendre ODE), Lagrange bases in barycentric form (Berrut & Trefethen,
// "Barycentric Lagrange interpolation", SIAM Review 2004), and the 1D mass / stiffness matrices of
// the Gauss-Lobatto basis by (p+1)-point Gauss quadrature, which is exact for both.
#include <cmath>

#include "cw_internal.h"

namespace cw {

namespace {
typedef long double ld;
const ld kPi = 3.141592653589793238462643383279502884L;

// P_n(t), P_n'(t) with the Bonnet recurrence
void legendre_pair(int n, ld t, ld &P, ld &dP)
{
    ld a = 1.0L, b = t;
    if (n == 0) {
        P = 1.0L;
        dP = 0.0L;
        return;
    }
    for (int k = 2; k <= n; ++k) {
        ld c = ((2 * k - 1) * t * b - (k - 1) * a) / k;
        a = b;
        b = c;
    }
    P = b;
    dP = n * (a - t * b) / (1.0L - t * t);
}

void gauss_rule(int n, ld *x, ld *w)
{
    for (int i = 0; i < n; ++i) {
        // i-th root in ascending order; initial guess -cos(pi (i + 3/4) / (n + 1/2))
        ld t = -std::cos(kPi * (i + 0.75L) / (n + 0.5L)), P, dP;
        for (int it = 0; it < 60; ++it) {
            legendre_pair(n, t, P, dP);
            ld dt = P / dP;
            t -= dt;
            if (std::fabs(dt) < 1e-19L) break;
        }
        legendre_pair(n, t, P, dP);
        x[i] = (t + 1.0L) / 2.0L;
        w[i] = 1.0L / ((1.0L - t * t) * dP * dP);  // 2/((1-t^2)P'^2) halved for [0,1]
    }
}

void lobatto_nodes(int p, ld *x)
{
    x[0] = 0.0L;
    x[p] = 1.0L;
    for (int i = 1; i < p; ++i) {
        ld t = -std::cos(kPi * i / p);
        for (int it = 0; it < 60; ++it) {
            ld P, dP;
            legendre_pair(p, t, P, dP);
            ld d2P = (2.0L * t * dP - p * (p + 1.0L) * P) / (1.0L - t * t);
            ld dt = dP / d2P;
            t -= dt;
            if (std::fabs(dt) < 1e-19L) break;
        }
        x[i] = (t + 1.0L) / 2.0L;
    }
}

// barycentric weights lambda_j = 1 / prod_{k != j} (x_j - x_k)
void bary_weights(int n, const ld *x, ld *lam)
{
    for (int j = 0; j < n; ++j) {
        ld prod = 1.0L;
        for (int k = 0; k < n; ++k)
            if (k != j) prod *= (x[j] - x[k]);
        lam[j] = 1.0L / prod;
    }
}

// values and derivatives of the Lagrange basis of nodes x at point s
void basis_at(int n, const ld *x, const ld *lam, ld s, ld *l, ld *dl)
{
    for (int j = 0; j < n; ++j) {
        if (s == x[j]) {  // at a node: l = delta, derivative from the differentiation matrix
            for (int m = 0; m < n; ++m) l[m] = (m == j) ? 1.0L : 0.0L;
            ld diag = 0.0L;
            for (int m = 0; m < n; ++m) {
                if (m == j) continue;
                dl[m] = (lam[m] / lam[j]) / (x[j] - x[m]);
                diag -= dl[m];
            }
            dl[j] = diag;
            return;
        }
    }
    // l_m(s) = lam_m / (s - x_m) * prod_k (s - x_k); derivative by the product rule
    ld ell = 1.0L;
    for (int k = 0; k < n; ++k) ell *= (s - x[k]);
    ld sum_inv = 0.0L;
    for (int k = 0; k < n; ++k) sum_inv += 1.0L / (s - x[k]);
    for (int m = 0; m < n; ++m) {
        l[m] = ell * lam[m] / (s - x[m]);
        dl[m] = l[m] * (sum_inv - 1.0L / (s - x[m]));
    }
}
}  // namespace

void build_tables(int p, Tables1D &t)
{
    const int n = p + 1;
    t.p = p;
    t.n = n;
    ld g[kMaxN], xq[kMaxN], wq[kMaxN], lamg[kMaxN], lamq[kMaxN];
    lobatto_nodes(p, g);
    gauss_rule(n, xq, wq);
    bary_weights(n, g, lamg);
    bary_weights(n, xq, lamq);
    ld B[kMaxN][kMaxN], Bd[kMaxN][kMaxN];
    for (int q = 0; q < n; ++q) {
        ld l[kMaxN], dl[kMaxN];
        basis_at(n, g, lamg, xq[q], l, dl);
        for (int m = 0; m < n; ++m) {
            B[q][m] = l[m];
            Bd[q][m] = dl[m];
        }
        ld lq[kMaxN], dlq[kMaxN];
        basis_at(n, xq, lamq, xq[q], lq, dlq);
        for (int r = 0; r < n; ++r) t.D[q][r] = (double)dlq[r];
    }
    for (int i = 0; i < n; ++i) {
        t.gll[i] = (double)g[i];
        t.xq[i] = (double)xq[i];
        t.wq[i] = (double)wq[i];
        for (int j = 0; j < n; ++j) {
            ld m = 0.0L, k = 0.0L;
            for (int q = 0; q < n; ++q) {
                m += wq[q] * B[q][i] * B[q][j];
                k += wq[q] * Bd[q][i] * Bd[q][j];
            }
            t.M1[i][j] = (double)m;
            t.K1[i][j] = (double)k;
        }
        for (int q = 0; q < n; ++q) {
            t.B[q][i] = (double)B[q][i];
            t.Bd[q][i] = (double)Bd[q][i];
        }
    }
    // 1D prolongation matrices of the two children of [0,1] (Sec. 3, Algorithm prolongation): node
    // i of child b sits at (g_i + b)/2 of the parent, where the parent's basis is evaluated
    for (int b = 0; b < 2; ++b)
        for (int i = 0; i < n; ++i) {
            ld l[kMaxN], dl[kMaxN];
            basis_at(n, g, lamg, (g[i] + b) / 2.0L, l, dl);
            for (int a = 0; a < n; ++a) (b ? t.P1 : t.P0)[i][a] = (double)l[a];
        }
}

}  // namespace cw
