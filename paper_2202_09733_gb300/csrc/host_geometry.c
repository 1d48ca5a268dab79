/*
 * Geometric factors and connectivity (host, double).
 *
 * The element map of level p has degree g = min(qg, p) (for g = 1 < qg = 2 the corner
 * nodes).  At a point with table rows t_k per direction:
 *   Jm[c][dd] = dx_c / dxi_dd        nested fma chains over the geometry nodes:
 *               s0 over b0 (innermost), then s1 over b1, then s2 over b2
 *   S[dd][c]  = J dxi_dd / dx_c      cofactors (2-D: +-Jm[1-c][1-dd]; 3-D: cyclic
 *               Jm[c1][d1] Jm[c2][d2] - Jm[c1][d2] Jm[c2][d1])
 *   J         = fma chain over dd of Jm[0][dd] S[dd][0];  G = S / J;  invJ = 1 / J.
 * Compiled with -ffp-contract=off.
 */
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include "host_tables.h"

static void metric(int d, int g, int qg, const double *gn /* this element */, const frh_tab *T,
                   const int *t, double *S, double *G, double *Jdet, double *invJ) {
    int m = qg + 1, stride = (g == qg) ? 1 : 2;
    double Jm[3][3];
    for (int c = 0; c < d; ++c)
        for (int dd = 0; dd < d; ++dd) {
            const double *B0 = (dd == 0) ? T->gdb[t[0]] : T->gb[t[0]];
            const double *B1 = (dd == 1) ? T->gdb[t[1]] : T->gb[t[1]];
            const double *B2 = (d == 3) ? ((dd == 2) ? T->gdb[t[2]] : T->gb[t[2]]) : 0;
            double s2 = 0.0;
            for (int b2 = 0; b2 < (d == 3 ? g + 1 : 1); ++b2) {
                double s1 = 0.0;
                for (int b1 = 0; b1 <= g; ++b1) {
                    double s0 = 0.0;
                    for (int b0 = 0; b0 <= g; ++b0) {
                        int a = b0 * stride + m * (b1 * stride + m * (b2 * stride));
                        s0 = fma(B0[b0], gn[a * d + c], s0);
                    }
                    s1 = fma(B1[b1], s0, s1);
                }
                s2 = (d == 3) ? fma(B2[b2], s1, s2) : s1;
            }
            Jm[c][dd] = s2;
        }
    double Sl[3][3];
    if (d == 2) {
        Sl[0][0] = Jm[1][1]; Sl[0][1] = -Jm[0][1];
        Sl[1][0] = -Jm[1][0]; Sl[1][1] = Jm[0][0];
    } else {
        for (int dd = 0; dd < 3; ++dd)
            for (int c = 0; c < 3; ++c) {
                int c1 = (c + 1) % 3, c2 = (c + 2) % 3, d1 = (dd + 1) % 3, d2 = (dd + 2) % 3;
                Sl[dd][c] = Jm[c1][d1] * Jm[c2][d2] - Jm[c1][d2] * Jm[c2][d1];
            }
    }
    double J = 0.0;
    for (int dd = 0; dd < d; ++dd) J = fma(Jm[0][dd], Sl[dd][0], J);
    for (int dd = 0; dd < d; ++dd)
        for (int c = 0; c < d; ++c) {
            S[dd * d + c] = Sl[dd][c];
            G[dd * d + c] = Sl[dd][c] / J;
        }
    *Jdet = J;
    *invJ = 1.0 / J;
}

void frh_geometry(int d, int E, int qg, const double *gnodes, const frh_tab *T,
                  double *S, double *G, double *invJ, double *Jdet, double *Sf, double *Gf) {
    int n = T->n, g = T->g, m = qg + 1;
    int ng = (d == 2) ? m * m : m * m * m;
    int np = (d == 2) ? n * n : n * n * n, nf1 = (d == 2) ? n : n * n, nfp = 2 * d * nf1;
    for (int e = 0; e < E; ++e) {
        const double *gn = gnodes + (size_t)e * ng * d;
        double s[9], gg[9], J, iJ;
        for (int i = 0; i < np; ++i) {
            int t[3] = {i % n, (i / n) % n, (d == 3) ? i / (n * n) : 0};
            metric(d, g, qg, gn, T, t, s, gg, &J, &iJ);
            for (int r = 0; r < d * d; ++r) {
                S[((size_t)r * np + i) * E + e] = s[r];
                G[((size_t)r * np + i) * E + e] = gg[r];
            }
            invJ[(size_t)i * E + e] = iJ;
            Jdet[(size_t)i * E + e] = J;
        }
        for (int k = 0; k < nfp; ++k) {
            int f = k / nf1, tt = k % nf1, df = f / 2, side = f % 2, t[3] = {0, 0, 0};
            int ta = (df == 0) ? 1 : 0, tb = (df == 2) ? 1 : 2;   /* tangential directions */
            t[df] = n + side;
            t[ta] = tt % n;
            if (d == 3) t[tb] = tt / n;
            metric(d, g, qg, gn, T, t, s, gg, &J, &iJ);
            for (int r = 0; r < d * d; ++r) {
                Sf[((size_t)r * nfp + k) * E + e] = s[r];
                Gf[((size_t)r * nfp + k) * E + e] = gg[r];
            }
        }
    }
}

static int tangential_map(int d, int n, int orient, int t) {
    if (d == 2) return (orient & 1) ? n - 1 - t : t;
    int a = t % n, b = t / n;
    if (orient & 4) { int s = a; a = b; b = s; }
    if (orient & 1) a = n - 1 - a;
    if (orient & 2) b = n - 1 - b;
    return a + n * b;
}

typedef struct { int eL, kL, eR, kR, bc; } pair_t;
static int cmp_pair(const void *a, const void *b) {
    const pair_t *x = a, *y = b;
    if (x->kL != y->kL) return x->kL - y->kL;
    return x->eL - y->eL;
}

int frh_pairs(int d, int n, int E, int nfaces, const int *faces, int *pairs, int *bc) {
    int nf1 = (d == 2) ? n : n * n;
    int nfp = 2 * d * nf1;
    int P = nfaces * nf1;
    pair_t *tmp = malloc(sizeof(pair_t) * (size_t)P);
    char *seen = calloc((size_t)nfp * E, 1);
    int ok = 1;
    for (int F = 0; F < nfaces && ok; ++F) {
        const int *fr = faces + 6 * F;
        if (fr[0] < 0 || fr[0] >= E || fr[1] < 0 || fr[1] >= 2 * d) ok = 0;
        if (fr[2] >= 0 && (fr[2] >= E || fr[3] < 0 || fr[3] >= 2 * d)) ok = 0;
        if (fr[2] < 0 && fr[5] != 1 && fr[5] != 2) ok = 0;
        if (!ok) break;
        for (int t = 0; t < nf1; ++t) {
            pair_t *q = &tmp[F * nf1 + t];
            q->eL = fr[0]; q->kL = fr[1] * nf1 + t;
            if (fr[2] >= 0) { q->eR = fr[2]; q->kR = fr[3] * nf1 + tangential_map(d, n, fr[4], t); q->bc = 0; }
            else { q->eR = -1; q->kR = -1; q->bc = fr[5]; }
            if (seen[(size_t)q->kL * E + q->eL]++) ok = 0;
            if (q->eR >= 0 && seen[(size_t)q->kR * E + q->eR]++) ok = 0;
        }
    }
    /* every face point of every element must belong to exactly one pair */
    for (size_t i = 0; ok && i < (size_t)nfp * E; ++i) if (seen[i] != 1) ok = 0;
    if (ok) {
        qsort(tmp, (size_t)P, sizeof(pair_t), cmp_pair);
        for (int i = 0; i < P; ++i) {
            pairs[4 * i] = tmp[i].eL; pairs[4 * i + 1] = tmp[i].kL;
            pairs[4 * i + 2] = tmp[i].eR; pairs[4 * i + 3] = tmp[i].kR;
            bc[i] = tmp[i].bc;
        }
    }
    free(tmp); free(seen);
    return ok ? P : -1;
}

int frh_color(int E, int nfaces, const int *faces, int *color) {
    /* adjacency lists */
    int *deg = calloc((size_t)E + 1, sizeof(int));
    for (int F = 0; F < nfaces; ++F)
        if (faces[6 * F + 2] >= 0 && faces[6 * F + 2] != faces[6 * F]) { deg[faces[6 * F]]++; deg[faces[6 * F + 2]]++; }
    int *off = malloc(sizeof(int) * ((size_t)E + 1));
    off[0] = 0;
    for (int e = 0; e < E; ++e) off[e + 1] = off[e] + deg[e];
    int *adj = malloc(sizeof(int) * (size_t)(off[E] > 0 ? off[E] : 1));
    memset(deg, 0, sizeof(int) * (size_t)E);
    for (int F = 0; F < nfaces; ++F) {
        int a = faces[6 * F], b = faces[6 * F + 2];
        if (b < 0 || a == b) continue;
        adj[off[a] + deg[a]++] = b;
        adj[off[b] + deg[b]++] = a;
    }
    int ncol = 0;
    for (int e = 0; e < E; ++e) color[e] = -1;
    for (int e = 0; e < E; ++e) {
        unsigned long long used = 0;
        for (int k = off[e]; k < off[e + 1]; ++k)
            if (color[adj[k]] >= 0 && color[adj[k]] < 64) used |= 1ull << color[adj[k]];
        int c = 0;
        while (c < 64 && (used >> c) & 1ull) ++c;
        color[e] = c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    free(deg); free(off); free(adj);
    return ncol;
}

int frh_neighbours(int E, int nf, int nfaces, const int *faces, int *nbr) {
    for (long long i = 0; i < (long long)E * nf; ++i) nbr[i] = -1;
    for (int F = 0; F < nfaces; ++F) {
        int a = faces[6 * F], fa = faces[6 * F + 1], b = faces[6 * F + 2], fb = faces[6 * F + 3];
        if (b < 0 || a == b) continue;
        if (fa < 0 || fa >= nf || fb < 0 || fb >= nf) return -1;
        nbr[(long long)fa * E + a] = b;
        nbr[(long long)fb * E + b] = a;
    }
    for (int e = 0; e < E; ++e)
        for (int f = 1; f < nf; ++f) {
            int n = nbr[(long long)f * E + e];
            if (n < 0) continue;
            for (int g = 0; g < f; ++g)
                if (nbr[(long long)g * E + e] == n) { nbr[(long long)f * E + e] = -1; break; }
        }
    return 0;
}

int frh_color2(int E, int nf, const int *nbr, int *color) {
    enum { MAXC = 1024 };
    int *stamp = malloc(sizeof(int) * MAXC);
    for (int c = 0; c < MAXC; ++c) stamp[c] = -1;
    for (int e = 0; e < E; ++e) color[e] = -1;
    int ncol = 0;
    for (int e = 0; e < E; ++e) {
        /* mark the colours of every element within two face steps */
        for (int f = 0; f < nf; ++f) {
            int n = nbr[(long long)f * E + e];
            if (n < 0) continue;
            if (color[n] >= 0) stamp[color[n]] = e;
            for (int g = 0; g < nf; ++g) {
                int m = nbr[(long long)g * E + n];
                if (m >= 0 && m != e && color[m] >= 0) stamp[color[m]] = e;
            }
        }
        int c = 0;
        while (c < MAXC && stamp[c] == e) ++c;
        if (c == MAXC) { free(stamp); return -1; }
        color[e] = c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    free(stamp);
    return ncol;
}
