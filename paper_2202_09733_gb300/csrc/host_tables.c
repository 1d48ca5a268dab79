/*
 * Operator tables of the flux-reconstruction discretisation (host, binary128).
 *
 * Per degree p (n = p + 1 Gauss-Legendre solution points per direction):
 *   x, w          Gauss-Legendre nodes (Newton on the Legendre recurrence) and weights
 *                 w = 2 (1 - x^2) / (n P_{n-1}(x))^2
 *   D[i][m]       l_m'(x_i) from barycentric weights (diagonal by the negative row sum)
 *   lm, lp        l_m(-1), l_m(+1)        dlm, dlp   l_m'(-1), l_m'(+1)
 *   gLd, gRd      derivatives at the nodes of the DG (right/left Radau) correction functions
 *                 g_L = (-1)^p (P_p - P_{p+1}) / 2,  g_R = (P_p + P_{p+1}) / 2
 *   gLf, gRf      g_L'(-1) = -(p+1)^2 / 2,  g_R'(+1) = (p+1)^2 / 2
 *   gb, gdb       Lobatto Lagrange basis of the geometry (degree 1 or 2) and its
 *                 derivative at the nodes and at -1, +1
 * Transfers between degrees p0 > p1 (Sec. 3.1, Eqs. 17-18), in closed form for
 * Gauss-Legendre nodal bases (both mass matrices are exact and diagonal under the
 * (p0+1)-point rule):  Gamma[i][j] = w0_j l^{p1}_i(x0_j) / w1_i,   Pi[i][j] = l^{p1}_j(x0_i).
 * Every value is the double nearest to its binary128 evaluation; magnitudes below 1e-25
 * (exact zeros) are stored as 0.
 */
#include <math.h>
#include <string.h>
#include "host_tables.h"

typedef _Float128 Q;

static Q sqrtq_(Q v) {
    Q r = (Q)sqrt((double)v);
    for (int it = 0; it < 3; ++it) r = (r + v / r) / 2;
    return r;
}

static double to_d(Q v) {
    double d = (double)v;
    return fabs(d) < 1e-25 ? 0.0 : d;
}

static void legendre_pair(int n, Q x, Q *Pn, Q *Pn1, Q *dPn) {
    /* P_n, P_{n-1} and P_n' */
    Q p0 = 1, p1 = x;
    if (n == 0) { *Pn = 1; *Pn1 = 0; *dPn = 0; return; }
    for (int k = 2; k <= n; ++k) {
        Q p2 = ((Q)(2 * k - 1) * x * p1 - (Q)(k - 1) * p0) / (Q)k;
        p0 = p1; p1 = p2;
    }
    *Pn = p1; *Pn1 = p0;
    *dPn = (Q)n * (p0 - x * p1) / (1 - x * x);
}

static void gauss_nodes(int n, Q *x, Q *w) {
    for (int i = 0; i < n; ++i) {
        /* guess for the i-th root counted from -1 */
        Q xi = -cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 50; ++it) {
            Q Pn, Pn1, dPn;
            legendre_pair(n, xi, &Pn, &Pn1, &dPn);
            xi -= Pn / dPn;
        }
        if ((n & 1) && i == n / 2) xi = 0;
        Q Pn, Pn1, dPn;
        legendre_pair(n, xi, &Pn, &Pn1, &dPn);
        x[i] = xi;
        w[i] = 2 * (1 - xi * xi) / ((Q)n * Pn1 * (Q)n * Pn1);
    }
}

static void bary_weights(int n, const Q *x, Q *lam) {
    for (int m = 0; m < n; ++m) {
        Q p = 1;
        for (int k = 0; k < n; ++k)
            if (k != m) p *= x[m] - x[k];
        lam[m] = 1 / p;
    }
}

/* value and derivative of every basis function l_m at y (y may coincide with a node) */
static void bary_eval(int n, const Q *x, const Q *lam, Q y, Q *val, Q *der) {
    int hit = -1;
    for (int k = 0; k < n; ++k)
        if (y == x[k]) hit = k;
    if (hit >= 0) {
        for (int m = 0; m < n; ++m) val[m] = (m == hit) ? 1 : 0;
        if (der) {
            Q s = 0;
            for (int m = 0; m < n; ++m) {
                if (m == hit) continue;
                der[m] = (lam[m] / lam[hit]) / (x[hit] - x[m]);
                s += der[m];
            }
            der[hit] = -s;
        }
        return;
    }
    Q ell = 1, sinv = 0;
    for (int k = 0; k < n; ++k) { ell *= y - x[k]; sinv += 1 / (y - x[k]); }
    for (int m = 0; m < n; ++m) {
        val[m] = ell * lam[m] / (y - x[m]);
        if (der) der[m] = val[m] * (sinv - 1 / (y - x[m]));
    }
}

static void radau_derivs(int p, Q y, Q *dgL, Q *dgR) {
    /* P_p'(y), P_{p+1}'(y) by differentiating the recurrence */
    Q P[8], dP[8];
    P[0] = 1; dP[0] = 0; P[1] = y; dP[1] = 1;
    for (int k = 1; k <= p; ++k) {
        P[k + 1] = ((Q)(2 * k + 1) * y * P[k] - (Q)k * P[k - 1]) / (Q)(k + 1);
        dP[k + 1] = ((Q)(2 * k + 1) * (P[k] + y * dP[k]) - (Q)k * dP[k - 1]) / (Q)(k + 1);
    }
    Q sg = (p & 1) ? -1 : 1;
    *dgL = sg * (dP[p] - dP[p + 1]) / 2;
    *dgR = (dP[p] + dP[p + 1]) / 2;
}

static void geometry_basis(int g, Q y, Q *b, Q *db) {
    if (g == 1) {
        b[0] = (1 - y) / 2; b[1] = (1 + y) / 2;
        db[0] = -(Q)0.5; db[1] = (Q)0.5;
    } else {
        b[0] = y * (y - 1) / 2; b[1] = 1 - y * y; b[2] = y * (y + 1) / 2;
        db[0] = y - (Q)0.5; db[1] = -2 * y; db[2] = y + (Q)0.5;
    }
}

void frh_make_tables(int p, int g, frh_tab *T) {
    memset(T, 0, sizeof(*T));
    int n = p + 1;
    T->p = p; T->n = n; T->g = g;
    Q x[FRH_MAXN], w[FRH_MAXN], lam[FRH_MAXN];
    gauss_nodes(n, x, w);
    bary_weights(n, x, lam);
    for (int i = 0; i < n; ++i) { T->x[i] = to_d(x[i]); T->w[i] = to_d(w[i]); }
    for (int i = 0; i < n; ++i) {
        Q val[FRH_MAXN], der[FRH_MAXN];
        bary_eval(n, x, lam, x[i], val, der);
        for (int m = 0; m < n; ++m) T->D[i][m] = to_d(der[m]);
    }
    Q val[FRH_MAXN], der[FRH_MAXN];
    bary_eval(n, x, lam, -1, val, der);
    for (int m = 0; m < n; ++m) { T->lm[m] = to_d(val[m]); T->dlm[m] = to_d(der[m]); }
    bary_eval(n, x, lam, 1, val, der);
    for (int m = 0; m < n; ++m) { T->lp[m] = to_d(val[m]); T->dlp[m] = to_d(der[m]); }
    for (int i = 0; i < n; ++i) {
        Q a, b;
        radau_derivs(p, x[i], &a, &b);
        T->gLd[i] = to_d(a);
        T->gRd[i] = to_d(b);
    }
    T->gLf = -(double)((p + 1) * (p + 1)) / 2.0;
    T->gRf = (double)((p + 1) * (p + 1)) / 2.0;
    for (int t = 0; t < n + 2; ++t) {
        Q y = (t < n) ? x[t] : (t == n ? (Q)-1 : (Q)1);
        Q b[3], db[3];
        geometry_basis(g, y, b, db);
        for (int a = 0; a <= g; ++a) { T->gb[t][a] = to_d(b[a]); T->gdb[t][a] = to_d(db[a]); }
    }
}

void frh_make_transfer(int p0, int p1, double Gam[FRH_MAXN][FRH_MAXN], double Pi[FRH_MAXN][FRH_MAXN]) {
    int n0 = p0 + 1, n1 = p1 + 1;
    Q x0[FRH_MAXN], w0[FRH_MAXN], x1[FRH_MAXN], w1[FRH_MAXN], lam1[FRH_MAXN];
    gauss_nodes(n0, x0, w0);
    gauss_nodes(n1, x1, w1);
    bary_weights(n1, x1, lam1);
    memset(Gam, 0, sizeof(double) * FRH_MAXN * FRH_MAXN);
    memset(Pi, 0, sizeof(double) * FRH_MAXN * FRH_MAXN);
    for (int j = 0; j < n0; ++j) {
        Q val[FRH_MAXN];
        bary_eval(n1, x1, lam1, x0[j], val, 0);
        for (int i = 0; i < n1; ++i) {
            Gam[i][j] = to_d(w0[j] * val[i] / w1[i]);
            Pi[j][i] = to_d(val[i]);
        }
    }
}

/* Sec. 3.3 spectral-decay indicator: M[a][i] = w_i phi_a(x_i), phi_a = sqrt((2a + 1)/2) P_a
 * the orthonormal Legendre polynomials, so that sum_i M[a][i] s_i is the coefficient of
 * phi_a in the degree-p polynomial through the nodal values s (the (p+1)-point rule is
 * exact for the products). */
void frh_modal(int p, double M[FRH_MAXN][FRH_MAXN]) {
    int n = p + 1;
    Q x[FRH_MAXN], w[FRH_MAXN];
    gauss_nodes(n, x, w);
    memset(M, 0, sizeof(double) * FRH_MAXN * FRH_MAXN);
    for (int i = 0; i < n; ++i) {
        Q P0 = 1, P1 = x[i];
        for (int a = 0; a < n; ++a) {
            Q Pa;
            if (a == 0) Pa = 1;
            else if (a == 1) Pa = x[i];
            else {
                Q P2 = ((Q)(2 * a - 1) * x[i] * P1 - (Q)(a - 1) * P0) / (Q)a;
                P0 = P1; P1 = P2; Pa = P2;
            }
            M[a][i] = to_d(w[i] * sqrtq_((Q)(2 * a + 1) / 2) * Pa);
        }
    }
}
