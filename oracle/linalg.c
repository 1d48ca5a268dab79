/*
 * Oracle element-Jacobi blocks, dense LU and p-transfer operators
 * (TEST INFRASTRUCTURE ONLY; shares no code with the CUDA library).
 *
 * Element blocks (Sec. 2.2, Eq. 9; Sec. 3.2): the diagonal block of the shifted
 * Jacobian, M_e = shift I - dR_e/dq_e, where R_e depends on q_e with every other element
 * held fixed.  Column j is the forward difference with step eps_j = 1e-7 max(1,|q_j|):
 *     M[r][j] = (r == j ? shift : 0) - (R_e(q + eps_j e_j)[r] - R_e(q)[r]) / eps_j.
 * The element degree of freedom index is r = v*Np + i; blocks are stored row-major per
 * element, M[e][r][j].
 *
 * Dense LU: Gaussian elimination with partial pivoting (first maximal |pivot|, rows
 * swapped), multipliers l = a/u, trailing updates a = fma(-l, u, a) in ascending
 * elimination order; the factor keeps the reciprocal 1/u_kk in place of each pivot
 * (the paper leaves the LU arithmetic open; one division per pivot instead of one per
 * solve).  Triangular solves as fma chains in the order the unknowns become known
 * (ascending column index forward, descending column index backward), x_k = s_k (1/u_kk).
 * or_lu_factor_div / or_lu_solve_div are the textbook division form of the same
 * elimination (x_k = s_k / u_kk), kept for the pin that the two forms agree.
 *
 * Transfers (Eqs. 17-18): the 1-D Gamma / Pi applied along direction 0, then 1, then 2.
 *
 * Element loops may run on several OpenMP threads: every element's result is computed by
 * the same operations in the same order whatever the thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

void or_elem_blocks(or_ctx *C, int l, const double *q, double shift, const int *elems, int ne, double *M) {
    or_level *L = &C->L[l];
    int E = C->E, nv = C->nv, np = L->np, nd = nv * np;
    double *R = malloc(sizeof(double) * nd * E);
    or_residual(C, l, q, R);
#pragma omp parallel
    {
    double *qe = malloc(sizeof(double) * nd), *qp = malloc(sizeof(double) * nd);
    double *R0 = malloc(sizeof(double) * nd), *Rp = malloc(sizeof(double) * nd);
#pragma omp for schedule(dynamic)
    for (int t = 0; t < ne; ++t) {
        int e = elems[t];
        for (int r = 0; r < nd; ++r) qe[r] = q[(size_t)r * E + e];
        or_elem_residual(C, l, q, e, qe, R0);
        double *Me = &M[(size_t)t * nd * nd];
        for (int j = 0; j < nd; ++j) {
            double eps = 1e-7 * fmax(1.0, fabs(qe[j]));
            memcpy(qp, qe, sizeof(double) * nd);
            qp[j] = qe[j] + eps;
            or_elem_residual(C, l, q, e, qp, Rp);
            for (int r = 0; r < nd; ++r) {
                double m = (Rp[r] - R0[r]) / eps;
                Me[(size_t)r * nd + j] = (r == j) ? shift - m : -m;
            }
        }
    }
    free(qe); free(qp); free(R0); free(Rp);
    }
    free(R);
}

/* the elimination; u_kk stays on the diagonal */
static void lu_eliminate(int n, double *A, int *piv) {
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(A[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i) {
            double a = fabs(A[(size_t)i * n + k]);
            if (a > best) { best = a; p = i; }
        }
        piv[k] = p;
        if (p != k)
            for (int j = 0; j < n; ++j) {
                double t = A[(size_t)k * n + j];
                A[(size_t)k * n + j] = A[(size_t)p * n + j];
                A[(size_t)p * n + j] = t;
            }
        for (int i = k + 1; i < n; ++i) {
            double li = A[(size_t)i * n + k] / A[(size_t)k * n + k];
            A[(size_t)i * n + k] = li;
            for (int j = k + 1; j < n; ++j)
                A[(size_t)i * n + j] = fma(-li, A[(size_t)k * n + j], A[(size_t)i * n + j]);
        }
    }
}

void or_lu_factor(int n, double *A, int *piv) {
    lu_eliminate(n, A, piv);
    for (int k = 0; k < n; ++k) A[(size_t)k * n + k] = 1.0 / A[(size_t)k * n + k];
}

/* Textbook form of the same factor and solve, for the pin that the reciprocal form above
 * changes nothing beyond round-off: the diagonal keeps u_kk and the backward substitution
 * divides, x_k = s_k / u_kk. */
void or_lu_factor_div(int n, double *A, int *piv) { lu_eliminate(n, A, piv); }
void or_lu_solve_div(int n, const double *A, const int *piv, double *b) {
    for (int k = 0; k < n; ++k)
        if (piv[k] != k) { double t = b[k]; b[k] = b[piv[k]]; b[piv[k]] = t; }
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s = fma(-A[(size_t)i * n + k], b[k], s);
        b[i] = s;
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int k = n - 1; k > i; --k) s = fma(-A[(size_t)i * n + k], b[k], s);
        b[i] = s / A[(size_t)i * n + i];
    }
}

void or_lu_solve(int n, const double *A, const int *piv, double *b) {
    for (int k = 0; k < n; ++k)
        if (piv[k] != k) { double t = b[k]; b[k] = b[piv[k]]; b[piv[k]] = t; }
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s = fma(-A[(size_t)i * n + k], b[k], s);
        b[i] = s;
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int k = n - 1; k > i; --k) s = fma(-A[(size_t)i * n + k], b[k], s);
        b[i] = s * A[(size_t)i * n + i];
    }
}

/* apply a 1-D operator Op[m_out][m_in] along every direction of a [nv][n_in^d][E] field */
static void tensor_apply(int d, int nv, int E, int nin, int nout, double Op[OR_MAXN][OR_MAXN],
                         const double *x, double *y) {
    int nmax = nin > nout ? nin : nout;
    size_t blk = (size_t)nmax * nmax * nmax;
    int npin = d == 2 ? nin * nin : nin * nin * nin;
    int npout = d == 2 ? nout * nout : nout * nout * nout;
#pragma omp parallel
    {
    double *a = malloc(sizeof(double) * blk), *b = malloc(sizeof(double) * blk);
#pragma omp for schedule(static)
    for (int e = 0; e < E; ++e)
        for (int v = 0; v < nv; ++v) {
            int dims[3] = {nin, nin, d == 3 ? nin : 1};
            for (int i = 0; i < npin; ++i) a[i] = x[((size_t)v * npin + i) * E + e];
            for (int dir = 0; dir < d; ++dir) {
                int nd[3] = {dims[0], dims[1], dims[2]};
                nd[dir] = nout;
                for (int i2 = 0; i2 < nd[2]; ++i2)
                    for (int i1 = 0; i1 < nd[1]; ++i1)
                        for (int i0 = 0; i0 < nd[0]; ++i0) {
                            int o[3] = {i0, i1, i2}, src[3] = {i0, i1, i2};
                            double s = 0.0;
                            for (int m = 0; m < nin; ++m) {
                                src[dir] = m;
                                s = fma(Op[o[dir]][m], a[src[0] + dims[0] * (src[1] + dims[1] * src[2])], s);
                            }
                            b[i0 + nd[0] * (i1 + nd[1] * i2)] = s;
                        }
                memcpy(dims, nd, sizeof dims);
                double *t = a; a = b; b = t;
            }
            for (int i = 0; i < npout; ++i) y[((size_t)v * npout + i) * E + e] = a[i];
        }
    free(a); free(b);
    }
}

void or_restrict(or_ctx *C, int l, const double *x0, double *x1) {
    tensor_apply(C->d, C->nv, C->E, C->L[l].n, C->L[l + 1].n, C->Gam[l], x0, x1);
}
void or_prolong(or_ctx *C, int l, const double *x1, double *x0) {
    tensor_apply(C->d, C->nv, C->E, C->L[l + 1].n, C->L[l].n, C->Pi[l], x1, x0);
}
