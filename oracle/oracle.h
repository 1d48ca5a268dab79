/*
 * FP64 CPU oracle for the JFNK-pMG hot path — TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference leg may
 * load this code.  It shares no code with the CUDA library: every table, geometric
 * factor and arithmetic step below is written independently.
 *
 * Arithmetic convention (so a reader can re-derive every rounding):
 *   - every sum of products  sum_k a_k b_k  is an fma chain in ascending k that
 *     starts from +0.0:   s = 0; s = fma(a_k, b_k, s);
 *   - divisions by the density are multiplications by one reciprocal rinv = 1/rho;
 *   - every other expression is evaluated exactly as parenthesised in the source,
 *     compiled with -ffp-contract=off (no implicit contraction, no reassociation);
 *   - operator tables are the correctly rounded doubles of their exact values
 *     (computed in binary128 and rounded once).
 *
 * Layouts: a state on level l is q[v][i][e]  (v < nv, i < Np, e < E; element fastest).
 */
#ifndef FR_ORACLE_H
#define FR_ORACLE_H
#include <stddef.h>

#define OR_MAXN 6          /* points per direction: p <= 5 */
#define OR_MAXLEV 4

typedef struct {
    int p, n;                          /* degree, points per direction (n = p+1)   */
    double x[OR_MAXN], w[OR_MAXN];     /* Gauss-Legendre nodes / weights          */
    double D[OR_MAXN][OR_MAXN];        /* D[i][m] = l_m'(x_i)                     */
    double lm[OR_MAXN], lp[OR_MAXN];   /* l_m(-1), l_m(+1)                        */
    double dlm[OR_MAXN], dlp[OR_MAXN]; /* l_m'(-1), l_m'(+1)                      */
    double gLd[OR_MAXN], gRd[OR_MAXN]; /* g_L'(x_i), g_R'(x_i)  (DG / Radau)      */
    double gLf, gRf;                   /* g_L'(-1), g_R'(+1)                      */
    /* geometry basis (degree g Lobatto Lagrange) at x_0..x_{n-1}, -1, +1 */
    int g;
    double gb[OR_MAXN + 2][3], gdb[OR_MAXN + 2][3];
} or_tab;

typedef struct {
    double gamma, Pr, mu, eta;         /* ratio of heats, Prandtl, viscosity, BR2 penalty */
    double qinf[5];                    /* free-stream conservative state (far field ghost) */
    int flux;                          /* inviscid common flux: 0 Rusanov, 1 Roe,
                                          2 Roe with Weiss-Smith low-Mach preconditioning */
    double ws_umin;                    /* Weiss-Smith: floor of the reference velocity     */
} or_phys;

typedef struct {
    int p, n, np, nf1, nfp;            /* degree, n = p+1, Np = n^d, n^(d-1), Nfp = 2d n^(d-1) */
    or_tab T;
    double *S, *G, *invJ, *Jdet;       /* S,G: [d][c][i][e]; invJ, Jdet: [i][e]   */
    double *Sf, *Gf;                   /* [d][c][k][e]                             */
    /* scratch for one residual evaluation */
    double *qf, *dq, *Q, *gface, *Qf, *fn;
    int *pe, *pk, *bc;                 /* per face-point pair: L/R element, L/R point, bc */
    int npairs;
    int *epair;                        /* per element and face point: pair index (k order) */
} or_level;

typedef struct {
    int d, nv, E, qg, nlev;
    or_phys ph;
    double *gnodes;                    /* [E][(qg+1)^d][d] */
    int nfaces;
    int *faces;                        /* [F][6] eL fL eR fR orient bc */
    or_level L[OR_MAXLEV];
    double Gam[OR_MAXLEV][OR_MAXN][OR_MAXN];  /* restriction l -> l+1 : [i1][i0] */
    double Pi[OR_MAXLEV][OR_MAXN][OR_MAXN];   /* prolongation l+1 -> l : [i0][i1] */
} or_ctx;

/* tables.c */
void or_make_tab(or_tab *T, int p, int g);
void or_make_transfer(int p0, int p1, double Gam[OR_MAXN][OR_MAXN], double Pi[OR_MAXN][OR_MAXN]);

/* residual.c */
void or_residual(or_ctx *C, int l, const double *q, double *R);
void or_elem_residual(or_ctx *C, int l, const double *q, int e, const double *qe, double *Re);
void or_flux_inviscid(const or_ctx *C, const double *q, double f[3][5]);
void or_flux_viscous(const or_ctx *C, const double *q, double Q[3][5], int adiabatic, double f[3][5]);
void or_rusanov(const or_ctx *C, const double *qL, const double *qR, const double *n, double *F);
void or_roe(const or_ctx *C, const double *qL, const double *qR, const double *n, double *F);
void or_weiss_smith(const or_ctx *C, const double *qL, const double *qR, const double *n, double *F);

#endif
