/*
 * Oracle operator tables (TEST INFRASTRUCTURE ONLY; shares no code with the CUDA library).
 *
 * Flux reconstruction on tensor-product elements (Sec. 2.1, the FR method the paper
 * builds on): Gauss-Legendre solution points, Lagrange interpolation to the element
 * faces, the nodal derivative matrix and the DG-recovering correction functions
 * g_L = (-1)^p/2 (P_p - P_{p+1}), g_R = (P_p + P_{p+1})/2.
 * The L2 restriction and prolongation operators follow Eqs. (17)-(18) (Sec. 3.1):
 * Gamma = (M^{p1})^{-1} M^{p1 p0},  Pi = (M^{p0})^{-1} M^{p0 p1}, mass matrices of the
 * Lagrange bases on the standard element.
 *
 * Everything is evaluated in binary128 from the plain definitions (product formulas,
 * quadrature-built mass matrices solved by Gaussian elimination) and rounded to double
 * once.  Values whose exact value is zero are stored as exact zeros (|v| < 1e-25).
 */
#include <math.h>
#include <string.h>
#include "oracle.h"

typedef _Float128 qf;

static double rnd(qf v) {
    double d = (double)v;
    if (fabs(d) < 1e-25) d = 0.0;
    return d;
}

/* Legendre P_k(x) and P_k'(x) for k = 0..kmax by the three-term recurrences. */
static void legendre(int kmax, qf x, qf *P, qf *dP) {
    P[0] = 1; dP[0] = 0;
    if (kmax == 0) return;
    P[1] = x; dP[1] = 1;
    for (int k = 1; k < kmax; ++k) {
        P[k + 1] = ((2 * k + 1) * x * P[k] - k * P[k - 1]) / (k + 1);
        dP[k + 1] = dP[k - 1] + (2 * k + 1) * P[k];
    }
}

/* roots of P_n in ascending order, Newton in binary128 */
static void gauss_legendre(int n, qf *x, qf *w) {
    qf P[OR_MAXN + 2], dP[OR_MAXN + 2];
    for (int i = 0; i < n; ++i) {
        qf xi = -cos(M_PI * (4.0 * i + 3.0) / (4.0 * n + 2.0));
        for (int it = 0; it < 40; ++it) {
            legendre(n, xi, P, dP);
            xi = xi - P[n] / dP[n];
        }
        if (n % 2 == 1 && i == n / 2) xi = 0;
        legendre(n, xi, P, dP);
        x[i] = xi;
        w[i] = 2 / ((1 - xi * xi) * dP[n] * dP[n]);
    }
}

/* Lagrange basis l_m of nodes xs (count n) at y, and its derivative (product formulas) */
static qf lag(int n, const qf *xs, int m, qf y) {
    qf v = 1;
    for (int k = 0; k < n; ++k)
        if (k != m) v *= (y - xs[k]) / (xs[m] - xs[k]);
    return v;
}
static qf dlag(int n, const qf *xs, int m, qf y) {
    qf s = 0;
    for (int j = 0; j < n; ++j) {
        if (j == m) continue;
        qf t = 1 / (xs[m] - xs[j]);
        for (int k = 0; k < n; ++k)
            if (k != m && k != j) t *= (y - xs[k]) / (xs[m] - xs[k]);
        s += t;
    }
    return s;
}

void or_make_tab(or_tab *T, int p, int g) {
    memset(T, 0, sizeof(*T));
    int n = p + 1;
    T->p = p; T->n = n; T->g = g;
    qf x[OR_MAXN], w[OR_MAXN];
    gauss_legendre(n, x, w);
    for (int i = 0; i < n; ++i) { T->x[i] = rnd(x[i]); T->w[i] = rnd(w[i]); }
    for (int i = 0; i < n; ++i)
        for (int m = 0; m < n; ++m) T->D[i][m] = rnd(dlag(n, x, m, x[i]));
    for (int m = 0; m < n; ++m) {
        T->lm[m] = rnd(lag(n, x, m, -1));
        T->lp[m] = rnd(lag(n, x, m, 1));
        T->dlm[m] = rnd(dlag(n, x, m, -1));
        T->dlp[m] = rnd(dlag(n, x, m, 1));
    }
    /* correction function derivatives */
    qf P[OR_MAXN + 2], dP[OR_MAXN + 2];
    qf sgn = (p % 2 == 0) ? 1 : -1;
    for (int i = 0; i < n; ++i) {
        legendre(p + 1, x[i], P, dP);
        T->gLd[i] = rnd(sgn / 2 * (dP[p] - dP[p + 1]));
        T->gRd[i] = rnd((dP[p] + dP[p + 1]) / 2);
    }
    legendre(p + 1, -1, P, dP);
    T->gLf = rnd(sgn / 2 * (dP[p] - dP[p + 1]));
    legendre(p + 1, 1, P, dP);
    T->gRf = rnd((dP[p] + dP[p + 1]) / 2);
    /* geometry basis: Lobatto nodes of degree g (g = 1: {-1,1}; g = 2: {-1,0,1}) */
    qf gx[3];
    if (g == 1) { gx[0] = -1; gx[1] = 1; }
    else { gx[0] = -1; gx[1] = 0; gx[2] = 1; }
    for (int t = 0; t < n + 2; ++t) {
        qf y = (t < n) ? x[t] : (t == n ? -1 : 1);
        for (int a = 0; a <= g; ++a) {
            T->gb[t][a] = rnd(lag(g + 1, gx, a, y));
            T->gdb[t][a] = rnd(dlag(g + 1, gx, a, y));
        }
    }
}

/* Gaussian elimination with partial pivoting in binary128: A X = B, A is n x n, B n x m */
static void qsolve(int n, int m, qf A[OR_MAXN][OR_MAXN], qf B[OR_MAXN][OR_MAXN]) {
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int i = k + 1; i < n; ++i)
            if (fabs((double)A[i][k]) > fabs((double)A[piv][k])) piv = i;
        if (piv != k) {
            for (int j = 0; j < n; ++j) { qf t = A[k][j]; A[k][j] = A[piv][j]; A[piv][j] = t; }
            for (int j = 0; j < m; ++j) { qf t = B[k][j]; B[k][j] = B[piv][j]; B[piv][j] = t; }
        }
        for (int i = k + 1; i < n; ++i) {
            qf f = A[i][k] / A[k][k];
            for (int j = k; j < n; ++j) A[i][j] -= f * A[k][j];
            for (int j = 0; j < m; ++j) B[i][j] -= f * B[k][j];
        }
    }
    for (int k = n - 1; k >= 0; --k)
        for (int j = 0; j < m; ++j) {
            qf s = B[k][j];
            for (int i = k + 1; i < n; ++i) s -= A[k][i] * B[i][j];
            B[k][j] = s / A[k][k];
        }
}

/* Eqs. (17)-(18): mass matrices on [-1,1] built by Gauss-Legendre quadrature with
 * p0+1 points (exact for all the products of degree <= p0+p1 <= 2 p0 + 1 involved). */
void or_make_transfer(int p0, int p1, double Gam[OR_MAXN][OR_MAXN], double Pi[OR_MAXN][OR_MAXN]) {
    int n0 = p0 + 1, n1 = p1 + 1;
    qf x0[OR_MAXN], w0[OR_MAXN], x1[OR_MAXN], w1[OR_MAXN];
    gauss_legendre(n0, x0, w0);
    gauss_legendre(n1, x1, w1);
    qf M1[OR_MAXN][OR_MAXN], M10[OR_MAXN][OR_MAXN], M0[OR_MAXN][OR_MAXN], M01[OR_MAXN][OR_MAXN];
    memset(M1, 0, sizeof M1); memset(M10, 0, sizeof M10);
    memset(M0, 0, sizeof M0); memset(M01, 0, sizeof M01);
    for (int q = 0; q < n0; ++q) {
        qf l1[OR_MAXN], l0[OR_MAXN];
        for (int i = 0; i < n1; ++i) l1[i] = lag(n1, x1, i, x0[q]);
        for (int i = 0; i < n0; ++i) l0[i] = lag(n0, x0, i, x0[q]);
        for (int i = 0; i < n1; ++i) {
            for (int j = 0; j < n1; ++j) M1[i][j] += w0[q] * l1[i] * l1[j];
            for (int j = 0; j < n0; ++j) M10[i][j] += w0[q] * l1[i] * l0[j];
        }
        for (int i = 0; i < n0; ++i) {
            for (int j = 0; j < n0; ++j) M0[i][j] += w0[q] * l0[i] * l0[j];
            for (int j = 0; j < n1; ++j) M01[i][j] += w0[q] * l0[i] * l1[j];
        }
    }
    qsolve(n1, n0, M1, M10);   /* M10 <- Gamma */
    qsolve(n0, n1, M0, M01);   /* M01 <- Pi    */
    for (int i = 0; i < OR_MAXN; ++i)
        for (int j = 0; j < OR_MAXN; ++j) { Gam[i][j] = 0; Pi[i][j] = 0; }
    for (int i = 0; i < n1; ++i)
        for (int j = 0; j < n0; ++j) Gam[i][j] = rnd(M10[i][j]);
    for (int i = 0; i < n0; ++i)
        for (int j = 0; j < n1; ++j) Pi[i][j] = rnd(M01[i][j]);
}
