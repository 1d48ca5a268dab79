/*
 * Oracle entry points for the Python test harness (TEST INFRASTRUCTURE ONLY).
 */
#include <stdlib.h>
#include <string.h>
#include "oracle.h"
#ifdef _OPENMP
#include <omp.h>
#endif

/* threads of the element loops (OpenMP builds; results do not depend on the count) */
void or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_level_init(or_ctx *C, int l, int p);
void or_level_free(or_level *L);

or_ctx *or_create(int d, int E, int qg, const double *gnodes, int nfaces, const int *faces,
                  int nlev, const int *plev, const double *phys) {
    or_ctx *C = calloc(1, sizeof(or_ctx));
    C->d = d; C->nv = d + 2; C->E = E; C->qg = qg; C->nlev = nlev;
    C->ph.gamma = phys[0]; C->ph.Pr = phys[1]; C->ph.mu = phys[2]; C->ph.eta = phys[3];
    for (int v = 0; v < C->nv; ++v) C->ph.qinf[v] = phys[4 + v];
    C->ph.flux = (int)phys[9];        /* phys = gamma, Pr, mu, eta, qinf[5], flux code, Ur floor */
    C->ph.ws_umin = phys[10];
    int m = qg + 1, ng = (d == 2) ? m * m : m * m * m;
    C->gnodes = malloc(sizeof(double) * (size_t)E * ng * d);
    memcpy(C->gnodes, gnodes, sizeof(double) * (size_t)E * ng * d);
    C->nfaces = nfaces;
    C->faces = malloc(sizeof(int) * 6 * nfaces);
    memcpy(C->faces, faces, sizeof(int) * 6 * nfaces);
    for (int l = 0; l < nlev; ++l) or_level_init(C, l, plev[l]);
    for (int l = 0; l + 1 < nlev; ++l) or_make_transfer(plev[l], plev[l + 1], C->Gam[l], C->Pi[l]);
    return C;
}

void or_destroy(or_ctx *C) {
    if (!C) return;
    for (int l = 0; l < C->nlev; ++l) or_level_free(&C->L[l]);
    free(C->gnodes); free(C->faces); free(C);
}

int or_level_np(const or_ctx *C, int l) { return C->L[l].np; }
int or_level_nfp(const or_ctx *C, int l) { return C->L[l].nfp; }

/* tables for pins: out = [x(n), w(n), D(n*n), lm, lp, dlm, dlp, gLd, gRd, gLf, gRf] */
void or_table(int p, int g, double *out) {
    or_tab T;
    or_make_tab(&T, p, g);
    int n = p + 1, o = 0;
    for (int i = 0; i < n; ++i) out[o++] = T.x[i];
    for (int i = 0; i < n; ++i) out[o++] = T.w[i];
    for (int i = 0; i < n; ++i) for (int m = 0; m < n; ++m) out[o++] = T.D[i][m];
    for (int i = 0; i < n; ++i) out[o++] = T.lm[i];
    for (int i = 0; i < n; ++i) out[o++] = T.lp[i];
    for (int i = 0; i < n; ++i) out[o++] = T.dlm[i];
    for (int i = 0; i < n; ++i) out[o++] = T.dlp[i];
    for (int i = 0; i < n; ++i) out[o++] = T.gLd[i];
    for (int i = 0; i < n; ++i) out[o++] = T.gRd[i];
    out[o++] = T.gLf; out[o++] = T.gRf;
}

void or_transfer(int p0, int p1, double *Gam, double *Pi) {
    double G[OR_MAXN][OR_MAXN], P[OR_MAXN][OR_MAXN];
    or_make_transfer(p0, p1, G, P);
    for (int i = 0; i <= p1; ++i) for (int j = 0; j <= p0; ++j) Gam[i * (p0 + 1) + j] = G[i][j];
    for (int i = 0; i <= p0; ++i) for (int j = 0; j <= p1; ++j) Pi[i * (p1 + 1) + j] = P[i][j];
}

/* geometry export: Jdet[i][e] at solution points (for quadrature-based pins) */
void or_jacobian(const or_ctx *C, int l, double *Jdet) {
    memcpy(Jdet, C->L[l].Jdet, sizeof(double) * C->L[l].np * C->E);
}
/* scaled outward normals of the L side of every face-point pair: [P][d], and bc */
int or_pairs(const or_ctx *C, int l, int *pe, int *pk, int *bc) {
    const or_level *L = &C->L[l];
    memcpy(pe, L->pe, sizeof(int) * 2 * L->npairs);
    memcpy(pk, L->pk, sizeof(int) * 2 * L->npairs);
    memcpy(bc, L->bc, sizeof(int) * L->npairs);
    return L->npairs;
}
