/*
 * Oracle mesh levels: geometric factors and face-point connectivity
 * (TEST INFRASTRUCTURE ONLY; shares no code with the CUDA library).
 *
 * Elements are curved tensor-product maps of geometry degree qg (1 or 2, Lobatto
 * nodes).  Level p uses geometry degree g = min(qg, p): the degree-g Lobatto
 * interpolant of the element map (for g = 1 < qg = 2: the corner nodes), which keeps
 * the polynomial metric terms inside the FR solution space on every p-level.
 *   Jm[c][dd] = dx_c/dxi_dd      (nested fma chains over the geometry nodes, xi0 inner)
 *   S[dd][c]  = J dxi_dd/dx_c    (cofactors; 2-D: (-1)^(dd+c) Jm[1-c][1-dd];
 *                                 3-D: Jm[c1][d1] Jm[c2][d2] - Jm[c1][d2] Jm[c2][d1], cyclic)
 *   J         = sum_dd Jm[0][dd] S[dd][0]   (fma chain)
 *   G[dd][c]  = S[dd][c] / J ;   invJ = 1 / J
 * Face numbering f = 2*dir + side (side 0: xi_dir = -1, 1: +1); face points are ordered
 * by the tangential directions in increasing order, first tangential index fastest.
 * Face list rows: eL fL eR fR orient bc (eR < 0: boundary with bc 1 far field, 2 wall).
 * orient: 2-D bit0 reverses the tangential index; 3-D: bit2 swaps (a,b), then bit0 flips
 * the first and bit1 the second index of the R side.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static double gnode(const or_ctx *C, int g, int e, const int *b, int c) {
    int qg = C->qg, d = C->d, a[3];
    for (int k = 0; k < d; ++k) a[k] = (g == qg) ? b[k] : 2 * b[k];
    int m = qg + 1;
    int idx = (d == 2) ? a[0] + m * a[1] : a[0] + m * (a[1] + m * a[2]);
    return C->gnodes[((size_t)e * (d == 2 ? m * m : m * m * m) + idx) * d + c];
}

/* rows t[k] of the geometry tables per direction (0..n-1 GL node, n: -1, n+1: +1) */
static void metric_at(const or_ctx *C, const or_tab *T, int e, const int *t,
                      double S[3][3], double G[3][3], double *Jdet, double *invJ) {
    int d = C->d, g = T->g;
    double Jm[3][3];
    for (int c = 0; c < d; ++c)
        for (int dd = 0; dd < d; ++dd) {
            const double *B[3];
            for (int k = 0; k < d; ++k) B[k] = (k == dd) ? T->gdb[t[k]] : T->gb[t[k]];
            int b[3] = {0, 0, 0};
            double s2 = 0.0;
            int n2 = (d == 3) ? g + 1 : 1;
            for (b[2] = 0; b[2] < n2; ++b[2]) {
                double s1 = 0.0;
                for (b[1] = 0; b[1] <= g; ++b[1]) {
                    double s0 = 0.0;
                    for (b[0] = 0; b[0] <= g; ++b[0]) s0 = fma(B[0][b[0]], gnode(C, g, e, b, c), s0);
                    s1 = fma(B[1][b[1]], s0, s1);
                }
                if (d == 3) s2 = fma(B[2][b[2]], s1, s2);
                else s2 = s1;
            }
            Jm[c][dd] = s2;
        }
    if (d == 2) {
        for (int dd = 0; dd < 2; ++dd)
            for (int c = 0; c < 2; ++c) {
                double v = Jm[1 - c][1 - dd];
                S[dd][c] = ((dd + c) % 2 == 0) ? v : -v;
            }
    } else {
        for (int dd = 0; dd < 3; ++dd)
            for (int c = 0; c < 3; ++c) {
                int c1 = (c + 1) % 3, c2 = (c + 2) % 3, d1 = (dd + 1) % 3, d2 = (dd + 2) % 3;
                S[dd][c] = Jm[c1][d1] * Jm[c2][d2] - Jm[c1][d2] * Jm[c2][d1];
            }
    }
    double J = 0.0;
    for (int dd = 0; dd < d; ++dd) J = fma(Jm[0][dd], S[dd][0], J);
    for (int dd = 0; dd < d; ++dd)
        for (int c = 0; c < d; ++c) G[dd][c] = S[dd][c] / J;
    *Jdet = J;
    *invJ = 1.0 / J;
}

static int tau_map(int d, int n, int orient, int t) {
    if (d == 2) return (orient & 1) ? n - 1 - t : t;
    int a = t % n, b = t / n, u = a, v = b;
    if (orient & 4) { u = b; v = a; }
    if (orient & 1) u = n - 1 - u;
    if (orient & 2) v = n - 1 - v;
    return u + n * v;
}

void or_level_init(or_ctx *C, int l, int p) {
    or_level *L = &C->L[l];
    int d = C->d, E = C->E, nv = C->nv;
    memset(L, 0, sizeof(*L));
    L->p = p; L->n = p + 1;
    L->np = (d == 2) ? L->n * L->n : L->n * L->n * L->n;
    L->nf1 = (d == 2) ? L->n : L->n * L->n;
    L->nfp = 2 * d * L->nf1;
    int g = (p < C->qg) ? p : C->qg;
    or_make_tab(&L->T, p, g);
    int n = L->n, np = L->np, nfp = L->nfp;
    L->S = malloc(sizeof(double) * d * d * np * E);
    L->G = malloc(sizeof(double) * d * d * np * E);
    L->invJ = malloc(sizeof(double) * np * E);
    L->Jdet = malloc(sizeof(double) * np * E);
    L->Sf = malloc(sizeof(double) * d * d * nfp * E);
    L->Gf = malloc(sizeof(double) * d * d * nfp * E);
    for (int e = 0; e < E; ++e) {
        for (int i = 0; i < np; ++i) {
            int t[3] = {i % n, (i / n) % n, (d == 3) ? i / (n * n) : 0};
            double S[3][3], G[3][3], J, iJ;
            metric_at(C, &L->T, e, t, S, G, &J, &iJ);
            for (int dd = 0; dd < d; ++dd)
                for (int c = 0; c < d; ++c) {
                    L->S[((size_t)(dd * d + c) * np + i) * E + e] = S[dd][c];
                    L->G[((size_t)(dd * d + c) * np + i) * E + e] = G[dd][c];
                }
            L->Jdet[(size_t)i * E + e] = J;
            L->invJ[(size_t)i * E + e] = iJ;
        }
        for (int k = 0; k < nfp; ++k) {
            int f = k / L->nf1, tt = k % L->nf1, df = f / 2, s = f % 2, t[3], td[2] = {0, 0}, j = 0;
            for (int c = 0; c < d; ++c) if (c != df) td[j++] = c;
            t[df] = n + s;
            t[td[0]] = tt % n;
            if (d == 3) t[td[1]] = tt / n;
            double S[3][3], G[3][3], J, iJ;
            metric_at(C, &L->T, e, t, S, G, &J, &iJ);
            for (int dd = 0; dd < d; ++dd)
                for (int c = 0; c < d; ++c) {
                    L->Sf[((size_t)(dd * d + c) * nfp + k) * E + e] = S[dd][c];
                    L->Gf[((size_t)(dd * d + c) * nfp + k) * E + e] = G[dd][c];
                }
        }
    }
    /* face-point pairs */
    int nf1 = L->nf1;
    L->npairs = C->nfaces * nf1;
    L->pe = malloc(sizeof(int) * 2 * L->npairs);
    L->pk = malloc(sizeof(int) * 2 * L->npairs);
    L->bc = malloc(sizeof(int) * L->npairs);
    L->epair = malloc(sizeof(int) * nfp * E);
    for (int i = 0; i < nfp * E; ++i) L->epair[i] = -1;
    for (int F = 0; F < C->nfaces; ++F) {
        const int *fr = &C->faces[6 * F];
        for (int t = 0; t < nf1; ++t) {
            int P = F * nf1 + t;
            L->pe[2 * P] = fr[0];
            L->pk[2 * P] = fr[1] * nf1 + t;
            L->bc[P] = (fr[2] < 0) ? fr[5] : 0;
            L->epair[(size_t)L->pk[2 * P] * E + fr[0]] = P;
            if (fr[2] >= 0) {
                L->pe[2 * P + 1] = fr[2];
                L->pk[2 * P + 1] = fr[3] * nf1 + tau_map(d, n, fr[4], t);
                L->epair[(size_t)L->pk[2 * P + 1] * E + fr[2]] = P;
            } else {
                L->pe[2 * P + 1] = -1;
                L->pk[2 * P + 1] = -1;
            }
        }
    }
    L->qf = malloc(sizeof(double) * nv * nfp * E);
    L->dq = malloc(sizeof(double) * nv * nfp * E);
    L->fn = malloc(sizeof(double) * nv * nfp * E);
    L->Q = malloc(sizeof(double) * d * nv * np * E);
    L->gface = malloc(sizeof(double) * d * nv * nfp * E);
    L->Qf = malloc(sizeof(double) * d * nv * nfp * E);
}

void or_level_free(or_level *L) {
    free(L->S); free(L->G); free(L->invJ); free(L->Jdet); free(L->Sf); free(L->Gf);
    free(L->pe); free(L->pk); free(L->bc); free(L->epair);
    free(L->qf); free(L->dq); free(L->fn); free(L->Q); free(L->gface); free(L->Qf);
}
