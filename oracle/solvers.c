/*
 * Oracle solvers (TEST INFRASTRUCTURE ONLY; shares no code with the CUDA library):
 * FD Jacobian-vector product, nonlinear pMG preconditioner, flexible GMRES, ESDIRK with
 * pseudo-transient continuation, Rosenbrock-Wanner steps and steady PTC with SER.
 *
 *  - Jv (Eq. 8):  A v = shift v - (R(q + eps v) - R(q)) / eps,  eps fixed (1e-6).
 *  - pMG preconditioner (Sec. 3.2, Eqs. 22-26, with the V-cycle of Sec. 3.1,
 *    Eqs. 11-16): Y approximates A^{-1} X by pseudo-time marching the nonlinear system
 *    0 = X + R(qh) - c qh - R(q) + c q.  On level l the system is F_l(qh) = S_l with
 *    F_l(y) = c y - R_l(y); each smoothing step is the linearised backward-Euler pseudo
 *    step with element-diagonal blocks M_l = (1/dtau* + c) I - J_l,ee:
 *        qh <- qh + M_l^{-1} (S_l - F_l(qh)).
 *    S_l - F_l(qh) is evaluated as  d_l - (c (qh - b_l) - (R_l(qh) - R_l(b_l))),  where
 *    b_0 = q, d_0 = X and, on coarser levels, b_{l+1} = Gamma qh_l^a and
 *    d_{l+1} = Gamma (S_l - F_l(qh_l^a)) (Eqs. 13-15); grouping the differences keeps
 *    the small preconditioned vector out of the cancellation.  When qh = b the
 *    difference terms are exact zeros, so the first smoothing step on a level uses d_l
 *    directly.  One V-cycle per application; Y = qh_0 - q.
 *  - FGMRES (right preconditioned, restarted, modified Gram-Schmidt), stopping when the
 *    Arnoldi least-squares residual estimate falls to tol ||b|| (the FD product is not
 *    exactly linear, so the true residual floors near eps |R''|/|J|; it is recomputed
 *    only to start a new cycle after a restart).  The FD product of Eq. (8) is
 *    only ever applied to unit 2-norm directions, as it is for unpreconditioned Krylov
 *    vectors: each preconditioned direction Z_j = P^{-1} V_j is normalised (FGMRES is
 *    invariant to the scale of Z_j) and A x is evaluated as ||x|| A (x/||x||).
 *  - ESDIRK stage equation (Eq. 5) solved by PTC/Newton (Eqs. 6-7):
 *        F(q) = (q - s_i) / (a_ii dt) - R(q),  s_i = q^n + dt sum_{j<i} a_ij R(q_j);
 *    converged when RMS(a_ii dt F) <= tol.  q^{n+1} = q^n + dt sum_i b_i R(q_i) (Eq. 2).
 *  - ROW (Eq. 3): (I/(gamma dt) - dR/dq(q^n)) Y_i = R(q^n + sum a_ij Y_j) + (1/dt) sum c_ij Y_j;
 *    q^{n+1} = q^n + sum m_j Y_j.
 *  - Steady PTC with SER (Eq. 10, read with the ratio ||F^k|| / ||F^{k+1}|| so that the
 *    pseudo step grows as the residual falls).
 *  - Matrix-based Newton-Krylov smoother of the coarsest level (Sec. 3.2): the level's
 *    shifted Jacobian assembled as element blocks plus face-neighbour blocks (forward
 *    differences of the whole level residual, one dof at a time), and each smoothing
 *    step's block solve replaced by GMRES (modified Gram-Schmidt, Givens) from zero,
 *    right-preconditioned by the element blocks (block-Jacobi where the paper used ILU0),
 *    stopping at the first iteration whose estimate meets the relative tolerance.
 *  - pMG nonlinear solver: steady (one cycle with X = R(q) per SER pseudo step) and for
 *    the ESDIRK stages (one cycle with X = -F per pseudo-time update, Sec. 3.1).
 * Every function here is pinned by tests/test_oracle_*.py (the pins are listed in each
 * file's docstring).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

void or_residual(or_ctx *C, int l, const double *q, double *R);
void or_elem_blocks(or_ctx *C, int l, const double *q, double shift, const int *elems, int ne, double *M);
void or_lu_factor(int n, double *A, int *piv);
void or_lu_solve(int n, const double *A, const int *piv, double *b);
void or_restrict(or_ctx *C, int l, const double *x0, double *x1);
void or_prolong(or_ctx *C, int l, const double *x1, double *x0);

/* ------------------------------------------------------------------ vectors */
static size_t vlen(const or_ctx *C, int l) { return (size_t)C->nv * C->L[l].np * C->E; }
static double dot(size_t N, const double *a, const double *b) {
    double s = 0.0;
    for (size_t i = 0; i < N; ++i) s = fma(a[i], b[i], s);
    return s;
}

/* ------------------------------------------------------------------ Jv, Eq. (8) */
void or_jvp(or_ctx *C, const double *q, const double *Rq, const double *v, double eps, double shift, double *Av) {
    size_t N = vlen(C, 0);
    double *qp = malloc(sizeof(double) * N), *Rp = malloc(sizeof(double) * N);
    for (size_t i = 0; i < N; ++i) qp[i] = q[i] + eps * v[i];
    or_residual(C, 0, qp, Rp);
    for (size_t i = 0; i < N; ++i) Av[i] = shift * v[i] - (Rp[i] - Rq[i]) / eps;
    free(qp); free(Rp);
}

/* ------------------------------------------------------------------ face neighbours */
/* nbr[e * 2d + f] = the element across local face f of element e, or -1 where that face
 * is a boundary, where it wraps onto e itself (a periodic mesh one element wide: that
 * coupling belongs to the diagonal block) or where an earlier face of e already reaches
 * the same element (a periodic mesh two elements wide: the first such face's block then
 * holds the whole coupling).  Faces rows are (eL, fL, eR, fR, orient, bc). */
void or_neighbours(const or_ctx *C, int *nbr) {
    int nf = 2 * C->d, E = C->E;
    for (int i = 0; i < E * nf; ++i) nbr[i] = -1;
    for (int F = 0; F < C->nfaces; ++F) {
        const int *fc = &C->faces[6 * F];
        if (fc[2] < 0 || fc[2] == fc[0]) continue;
        nbr[fc[0] * nf + fc[1]] = fc[2];
        nbr[fc[2] * nf + fc[3]] = fc[0];
    }
    for (int e = 0; e < E; ++e)
        for (int f = 0; f < nf; ++f)
            for (int g = 0; g < f; ++g)
                if (nbr[e * nf + f] >= 0 && nbr[e * nf + g] == nbr[e * nf + f]) nbr[e * nf + f] = -1;
}

/* Off-diagonal blocks of the shifted Jacobian A = shift I - dR/dq on level l at q: for
 * element e and face slot f with neighbour n = nbr[e][f], block (e, f) is -dR_e/dq_n,
 * column j the forward difference of the whole residual with the step
 * eps_j = 1e-7 max(1, |q_n,j|) on dof j of element n alone (the element blocks' step).
 * Stored row-major per block: O[((e * 2d + f) * nd + r) * nd + j]. */
void or_nbr_blocks(or_ctx *C, int l, const double *q, const int *nbr, double *O) {
    or_level *L = &C->L[l];
    int E = C->E, nd = C->nv * L->np, nf = 2 * C->d;
    size_t N = (size_t)nd * E;
    double *R0 = malloc(sizeof(double) * N), *Rp = malloc(sizeof(double) * N), *qp = malloc(sizeof(double) * N);
    memset(O, 0, sizeof(double) * (size_t)E * nf * nd * nd);
    or_residual(C, l, q, R0);
    memcpy(qp, q, sizeof(double) * N);
    for (int n = 0; n < E; ++n)
        for (int j = 0; j < nd; ++j) {
            double x = q[(size_t)j * E + n];
            double eps = 1e-7 * fmax(1.0, fabs(x));
            qp[(size_t)j * E + n] = x + eps;
            or_residual(C, l, qp, Rp);
            qp[(size_t)j * E + n] = x;
            for (int e = 0; e < E; ++e)
                for (int f = 0; f < nf; ++f) {
                    if (nbr[e * nf + f] != n) continue;
                    double *B = &O[(size_t)(e * nf + f) * nd * nd];
                    for (int r = 0; r < nd; ++r) {
                        double m = (Rp[(size_t)r * E + e] - R0[(size_t)r * E + e]) / eps;
                        B[(size_t)r * nd + j] = -m;
                    }
                }
        }
    free(R0); free(Rp); free(qp);
}

/* ------------------------------------------------------------------ pMG */
typedef struct {
    int nlev, nsmooth[OR_MAXLEV];
    double c, inv_dtau_star;
    double *M[OR_MAXLEV];
    int *piv[OR_MAXLEV];
    /* matrix-based Newton-Krylov smoother on the coarsest level (Sec. 3.2) */
    int mbnk, mbnk_maxit;
    double mbnk_tol;
    double *Md, *O;                    /* unfactored diagonal blocks, neighbour blocks */
    int *nbr;
    int mbnk_last_iters;
    double mbnk_last_relres;
    int ready;
} or_pmg;

static or_pmg g_pmg;

static void pmg_free(void) {
    for (int l = 0; l < OR_MAXLEV; ++l) { free(g_pmg.M[l]); free(g_pmg.piv[l]); g_pmg.M[l] = 0; g_pmg.piv[l] = 0; }
    free(g_pmg.Md); free(g_pmg.O); free(g_pmg.nbr);
    g_pmg.Md = 0; g_pmg.O = 0; g_pmg.nbr = 0;
    g_pmg.ready = 0;
}

/* blocks at the reference state q_ref (restricted level by level) and their LU factors;
 * mbnk != 0: the coarsest level also keeps its assembled operator (diagonal and neighbour
 * blocks) for the matrix-based smoother, GMRES of at most mbnk_maxit iterations to the
 * relative tolerance mbnk_tol */
void or_pmg_setup(or_ctx *C, const double *q_ref, int nlev, const int *nsmooth, double c, double inv_dtau_star,
                  int mbnk, int mbnk_maxit, double mbnk_tol) {
    pmg_free();
    g_pmg.nlev = nlev; g_pmg.c = c; g_pmg.inv_dtau_star = inv_dtau_star;
    g_pmg.mbnk = mbnk; g_pmg.mbnk_maxit = mbnk_maxit; g_pmg.mbnk_tol = mbnk_tol;
    for (int l = 0; l < nlev; ++l) g_pmg.nsmooth[l] = nsmooth[l];
    int E = C->E;
    int *all = malloc(sizeof(int) * E);
    for (int e = 0; e < E; ++e) all[e] = e;
    double *qr = malloc(sizeof(double) * vlen(C, 0));
    memcpy(qr, q_ref, sizeof(double) * vlen(C, 0));
    for (int l = 0; l < nlev; ++l) {
        int nd = C->nv * C->L[l].np;
        g_pmg.M[l] = malloc(sizeof(double) * (size_t)nd * nd * E);
        g_pmg.piv[l] = malloc(sizeof(int) * (size_t)nd * E);
        or_elem_blocks(C, l, qr, inv_dtau_star + c, all, E, g_pmg.M[l]);
        if (mbnk && l == nlev - 1) {
            int nf = 2 * C->d;
            g_pmg.Md = malloc(sizeof(double) * (size_t)nd * nd * E);
            memcpy(g_pmg.Md, g_pmg.M[l], sizeof(double) * (size_t)nd * nd * E);
            g_pmg.nbr = malloc(sizeof(int) * (size_t)E * nf);
            or_neighbours(C, g_pmg.nbr);
            g_pmg.O = malloc(sizeof(double) * (size_t)E * nf * nd * nd);
            or_nbr_blocks(C, l, qr, g_pmg.nbr, g_pmg.O);
        }
#pragma omp parallel for schedule(static)
        for (int e = 0; e < E; ++e)
            or_lu_factor(nd, &g_pmg.M[l][(size_t)e * nd * nd], &g_pmg.piv[l][(size_t)e * nd]);
        if (l + 1 < nlev) {
            double *qn = malloc(sizeof(double) * vlen(C, l + 1));
            or_restrict(C, l, qr, qn);
            free(qr);
            qr = qn;
        }
    }
    free(qr); free(all);
    g_pmg.ready = 1;
}

/* apply M_l^{-1} element by element, in place on x[v][i][e] */
static void block_solve(or_ctx *C, int l, double *x) {
    int E = C->E, nd = C->nv * C->L[l].np;
#pragma omp parallel
    {
    double *b = malloc(sizeof(double) * nd);
#pragma omp for schedule(static)
    for (int e = 0; e < E; ++e) {
        for (int r = 0; r < nd; ++r) b[r] = x[(size_t)r * E + e];
        or_lu_solve(nd, &g_pmg.M[l][(size_t)e * nd * nd], &g_pmg.piv[l][(size_t)e * nd], b);
        for (int r = 0; r < nd; ++r) x[(size_t)r * E + e] = b[r];
    }
    free(b);
    }
}
void or_block_solve(or_ctx *C, int l, double *x) { block_solve(C, l, x); }

/* rhs = d - (c (qh - b) - (Rqh - Rb)) */
static void pmg_rhs(size_t N, double c, const double *d, const double *qh, const double *b,
                    const double *Rqh, const double *Rb, double *rhs) {
    for (size_t i = 0; i < N; ++i) {
        double t1 = qh[i] - b[i], t2 = Rqh[i] - Rb[i];
        rhs[i] = d[i] - (c * t1 - t2);
    }
}

/* y = A x with the assembled operator of the coarsest level:
 * y_e = Md_e x_e + sum_f O_(e,f) x_nbr(e,f) */
void or_mbnk_matvec(or_ctx *C, int l, const double *x, double *y) {
    int E = C->E, nd = C->nv * C->L[l].np, nf = 2 * C->d;
    for (int e = 0; e < E; ++e)
        for (int r = 0; r < nd; ++r) {
            double acc = 0.0;
            const double *Me = &g_pmg.Md[(size_t)e * nd * nd + (size_t)r * nd];
            for (int j = 0; j < nd; ++j) acc = fma(Me[j], x[(size_t)j * E + e], acc);
            for (int f = 0; f < nf; ++f) {
                int n = g_pmg.nbr[e * nf + f];
                if (n < 0) continue;
                const double *B = &g_pmg.O[(size_t)(e * nf + f) * nd * nd + (size_t)r * nd];
                for (int j = 0; j < nd; ++j) acc = fma(B[j], x[(size_t)j * E + n], acc);
            }
            y[(size_t)r * E + e] = acc;
        }
}

/* one matrix-based Newton-Krylov smoothing solve (Sec. 3.2): GMRES on A delta = r from
 * delta = 0, right-preconditioned by the element blocks (delta = Md^{-1} V y), modified
 * Gram-Schmidt, Givens rotations; it stops after the first iteration k whose residual
 * estimate |g_k+1| is <= mbnk_tol ||r||, or after mbnk_maxit iterations.  In place:
 * x holds r on entry and delta on return. */
void or_mbnk_solve(or_ctx *C, int l, double *x) {
    size_t N = vlen(C, l);
    int m = g_pmg.mbnk_maxit;
    double *V = calloc((size_t)(m + 1) * N, sizeof(double)), *w = malloc(sizeof(double) * N);
    double *z = malloc(sizeof(double) * N);
    double *H = calloc((size_t)(m + 1) * m, sizeof(double));      /* H[i * m + k] */
    double *cs = calloc(m, sizeof(double)), *sn = calloc(m, sizeof(double)), *g = calloc(m + 1, sizeof(double));
    double *y = calloc(m, sizeof(double));
    double beta = sqrt(dot(N, x, x));
    int k_used = 0;
    g_pmg.mbnk_last_relres = 0.0;
    if (beta > 0.0) {
        for (size_t i = 0; i < N; ++i) V[i] = x[i] / beta;
        g[0] = beta;
        for (int k = 0; k < m; ++k) {
            double *vk = &V[(size_t)k * N], *vn = &V[(size_t)(k + 1) * N];
            memcpy(z, vk, sizeof(double) * N);
            block_solve(C, l, z);
            or_mbnk_matvec(C, l, z, w);
            for (int i = 0; i <= k; ++i) {
                double h = dot(N, w, &V[(size_t)i * N]);
                H[i * m + k] = h;
                for (size_t t = 0; t < N; ++t) w[t] = w[t] - h * V[(size_t)i * N + t];
            }
            double hn = sqrt(dot(N, w, w));
            H[(k + 1) * m + k] = hn;
            if (hn > 0.0)
                for (size_t t = 0; t < N; ++t) vn[t] = w[t] / hn;
            /* earlier rotations on the new column, then the rotation that zeroes H[k+1][k] */
            for (int i = 0; i < k; ++i) {
                double a = H[i * m + k], b = H[(i + 1) * m + k];
                H[i * m + k] = cs[i] * a + sn[i] * b;
                H[(i + 1) * m + k] = -sn[i] * a + cs[i] * b;
            }
            double a = H[k * m + k], b = H[(k + 1) * m + k], rr = hypot(a, b);
            cs[k] = rr > 0.0 ? a / rr : 1.0;
            sn[k] = rr > 0.0 ? b / rr : 0.0;
            H[k * m + k] = rr;
            H[(k + 1) * m + k] = 0.0;
            g[k + 1] = -sn[k] * g[k];
            g[k] = cs[k] * g[k];
            k_used = k + 1;
            if (fabs(g[k + 1]) <= g_pmg.mbnk_tol * beta) break;
        }
        g_pmg.mbnk_last_relres = fabs(g[k_used]) / beta;
        for (int i = k_used - 1; i >= 0; --i) {
            double t = g[i];
            for (int j = i + 1; j < k_used; ++j) t = t - H[i * m + j] * y[j];
            y[i] = H[i * m + i] != 0.0 ? t / H[i * m + i] : 0.0;
        }
    }
    for (size_t t = 0; t < N; ++t) {
        double acc = 0.0;
        for (int j = 0; j < k_used; ++j) acc = acc + y[j] * V[(size_t)j * N + t];
        x[t] = acc;
    }
    block_solve(C, l, x);
    g_pmg.mbnk_last_iters = k_used;
    free(V); free(w); free(z); free(H); free(cs); free(sn); free(g); free(y);
}

int or_mbnk_last_iters(void) { return g_pmg.mbnk_last_iters; }
double or_mbnk_last_relres(void) { return g_pmg.mbnk_last_relres; }

static void smooth(or_ctx *C, int l, int nsteps, const double *b, const double *Rb, const double *d,
                   double *qh, int first_is_base) {
    size_t N = vlen(C, l);
    double *Rqh = malloc(sizeof(double) * N), *rhs = malloc(sizeof(double) * N);
    for (int s = 0; s < nsteps; ++s) {
        if (s == 0 && first_is_base) memcpy(rhs, d, sizeof(double) * N);
        else {
            or_residual(C, l, qh, Rqh);
            pmg_rhs(N, g_pmg.c, d, qh, b, Rqh, Rb, rhs);
        }
        if (g_pmg.mbnk && l == g_pmg.nlev - 1) or_mbnk_solve(C, l, rhs);
        else block_solve(C, l, rhs);
        for (size_t i = 0; i < N; ++i) qh[i] = qh[i] + rhs[i];
    }
    free(Rqh); free(rhs);
}

static void vcycle(or_ctx *C, int l, const double *b, const double *Rb, const double *d, double *qh) {
    size_t N = vlen(C, l);
    int n = g_pmg.nsmooth[l];
    smooth(C, l, n, b, Rb, d, qh, 1);
    if (l + 1 >= g_pmg.nlev) return;
    size_t N1 = vlen(C, l + 1);
    double *Rqh = malloc(sizeof(double) * N), *r = malloc(sizeof(double) * N);
    double *b1 = malloc(sizeof(double) * N1), *Rb1 = malloc(sizeof(double) * N1);
    double *d1 = malloc(sizeof(double) * N1), *qh1 = malloc(sizeof(double) * N1);
    double *C0 = malloc(sizeof(double) * N);
    /* defect d_l = S_l - F_l(qh^a), Eq. (13) */
    if (n == 0) memcpy(r, d, sizeof(double) * N);
    else {
        or_residual(C, l, qh, Rqh);
        pmg_rhs(N, g_pmg.c, d, qh, b, Rqh, Rb, r);
    }
    /* restriction and coarse forcing, Eqs. (14)-(15) */
    or_restrict(C, l, qh, b1);
    or_restrict(C, l, r, d1);
    or_residual(C, l + 1, b1, Rb1);
    memcpy(qh1, b1, sizeof(double) * N1);
    vcycle(C, l + 1, b1, Rb1, d1, qh1);
    /* prolongation of the coarse correction, Eq. (16) */
    for (size_t i = 0; i < N1; ++i) qh1[i] = qh1[i] - b1[i];
    or_prolong(C, l, qh1, C0);
    for (size_t i = 0; i < N; ++i) qh[i] = qh[i] + C0[i];
    /* post-smoothing */
    smooth(C, l, n, b, Rb, d, qh, 0);
    free(Rqh); free(r); free(b1); free(Rb1); free(d1); free(qh1); free(C0);
}

void or_pmg_apply(or_ctx *C, const double *q, const double *Rq, const double *X, double *Y) {
    size_t N = vlen(C, 0);
    double *qh = malloc(sizeof(double) * N);
    memcpy(qh, q, sizeof(double) * N);
    vcycle(C, 0, q, Rq, X, qh);
    for (size_t i = 0; i < N; ++i) Y[i] = qh[i] - q[i];
    free(qh);
}

/* ------------------------------------------------------------------ FGMRES */
typedef struct { int iters, restarts; double relres; } or_gmres_stats;

int or_gmres(or_ctx *C, const double *q, const double *Rq, const double *b, double *x,
             int kdim, double tol, int maxit, double shift, double eps, int use_pmg,
             or_gmres_stats *st) {
    size_t N = vlen(C, 0);
    double **V = malloc(sizeof(double *) * (kdim + 1)), **Z = malloc(sizeof(double *) * kdim);
    for (int j = 0; j <= kdim; ++j) V[j] = malloc(sizeof(double) * N);
    for (int j = 0; j < kdim; ++j) Z[j] = malloc(sizeof(double) * N);
    double *H = calloc((size_t)(kdim + 1) * kdim, sizeof(double));
    double *cs = malloc(sizeof(double) * kdim), *sn = malloc(sizeof(double) * kdim);
    double *g = malloc(sizeof(double) * (kdim + 1)), *y = malloc(sizeof(double) * kdim);
    double *w = malloc(sizeof(double) * N), *r = malloc(sizeof(double) * N);
    memset(x, 0, sizeof(double) * N);
    memcpy(r, b, sizeof(double) * N);
    double bnorm = sqrt(dot(N, b, b)), beta = bnorm, est = bnorm;
    int total = 0, restarts = 0;
    st->iters = 0; st->restarts = 0; st->relres = 0.0;
    if (bnorm == 0.0) goto done;
    for (;;) {
        for (size_t i = 0; i < N; ++i) V[0][i] = r[i] / beta;
        for (int j = 0; j <= kdim; ++j) g[j] = 0.0;
        g[0] = beta;
        int jj = 0;
        for (int j = 0; j < kdim; ++j) {
            if (use_pmg) {
                or_pmg_apply(C, q, Rq, V[j], Z[j]);
                double zn = sqrt(dot(N, Z[j], Z[j]));
                for (size_t t = 0; t < N; ++t) Z[j][t] = Z[j][t] / zn;
            } else memcpy(Z[j], V[j], sizeof(double) * N);
            or_jvp(C, q, Rq, Z[j], eps, shift, w);
            for (int i = 0; i <= j; ++i) {
                double h = dot(N, w, V[i]);
                H[i * kdim + j] = h;
                for (size_t t = 0; t < N; ++t) w[t] = w[t] - h * V[i][t];
            }
            double hn = sqrt(dot(N, w, w));
            H[(j + 1) * kdim + j] = hn;
            for (size_t t = 0; t < N; ++t) V[j + 1][t] = w[t] / hn;
            for (int i = 0; i < j; ++i) {
                double a = H[i * kdim + j], bb = H[(i + 1) * kdim + j];
                H[i * kdim + j] = cs[i] * a + sn[i] * bb;
                H[(i + 1) * kdim + j] = -sn[i] * a + cs[i] * bb;
            }
            double a = H[j * kdim + j], bb = H[(j + 1) * kdim + j];
            double rr = hypot(a, bb);
            cs[j] = a / rr; sn[j] = bb / rr;
            H[j * kdim + j] = rr; H[(j + 1) * kdim + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++total; jj = j + 1;
            est = fabs(g[j + 1]);
            if (est <= tol * bnorm || total >= maxit || hn == 0.0) break;
        }
        for (int i = jj - 1; i >= 0; --i) {
            double s = g[i];
            for (int k = i + 1; k < jj; ++k) s -= H[i * kdim + k] * y[k];
            y[i] = s / H[i * kdim + i];
        }
        for (int i = 0; i < jj; ++i)
            for (size_t t = 0; t < N; ++t) x[t] = x[t] + y[i] * Z[i][t];
        if (est <= tol * bnorm || total >= maxit) break;
        /* restart: true residual, A x through the unit direction x/||x|| */
        double xn = sqrt(dot(N, x, x));
        for (size_t t = 0; t < N; ++t) r[t] = x[t] / xn;
        or_jvp(C, q, Rq, r, eps, shift, w);
        for (size_t t = 0; t < N; ++t) r[t] = b[t] - xn * w[t];
        beta = sqrt(dot(N, r, r));
        ++restarts;
    }
    st->iters = total; st->restarts = restarts; st->relres = est / bnorm;
done:
    for (int j = 0; j <= kdim; ++j) free(V[j]);
    for (int j = 0; j < kdim; ++j) free(Z[j]);
    free(V); free(Z); free(H); free(cs); free(sn); free(g); free(y); free(w); free(r);
    return 0;
}

/* ------------------------------------------------------------------ drivers */
typedef struct {
    int kdim, maxit_gmres, max_ptc, nlev, nsmooth[OR_MAXLEV], use_pmg;
    double tol_gmres, tol_newton, eps, dtau, inv_dtau_star;
    int mbnk, mbnk_maxit;              /* matrix-based smoother on the coarsest level */
    double mbnk_tol;
    int nonlinear;                     /* ESDIRK stage solver: 0 JFNK, 1 pMG V-cycles */
} or_solve_opts;

typedef struct { int n_ptc, n_gmres, converged; double final_res; } or_step_stats;

static double rms_scaled(size_t N, double a, const double *F) {
    double s = 0.0;
    for (size_t i = 0; i < N; ++i) { double t = a * F[i]; s = fma(t, t, s); }
    return sqrt(s / (double)N);
}

/* ESDIRK step, Eqs. (2), (5)-(8); A is s x s row-major, b length s.
 * o->nonlinear 0: each stage's pseudo-time Newton iteration solves (Eq. 8) A dq = -F by
 * FGMRES (JFNK).  1: the pMG nonlinear solver (Sec. 3.1): dq is one V-cycle of the
 * stage's pseudo-time equation, the preconditioner's cycle with X = -F, i.e. the FAS
 * cycle for (1/dtau + 1/(a_ii dt)) dq - (R(q + dq) - R(q)) = -F(q). */
int or_esdirk_step(or_ctx *C, int s, const double *A, const double *bw, double dt, double *q,
                   const or_solve_opts *o, or_step_stats *st) {
    size_t N = vlen(C, 0);
    double *qn = malloc(sizeof(double) * N), *Rs = malloc(sizeof(double) * N * s);
    double *sv = malloc(sizeof(double) * N), *F = malloc(sizeof(double) * N);
    double *Rk = malloc(sizeof(double) * N), *dq = malloc(sizeof(double) * N);
    memcpy(qn, q, sizeof(double) * N);
    or_residual(C, 0, qn, Rs);
    memset(st, 0, sizeof(*st));
    st->converged = 1;
    double aii = A[1 * s + 1];
    double c = 1.0 / o->dtau + 1.0 / (aii * dt);
    if (o->use_pmg) or_pmg_setup(C, qn, o->nlev, o->nsmooth, c, o->inv_dtau_star, o->mbnk, o->mbnk_maxit, o->mbnk_tol);
    for (int i = 1; i < s; ++i) {
        double adt = A[i * s + i] * dt;
        for (size_t t = 0; t < N; ++t) {
            double acc = 0.0;
            for (int j = 0; j < i; ++j) acc = fma(A[i * s + j], Rs[(size_t)j * N + t], acc);
            sv[t] = qn[t] + dt * acc;
        }
        /* guess q^n */
        memcpy(q, qn, sizeof(double) * N);
        int k, conv = 0;
        double res = 0.0;
        for (k = 0; k <= o->max_ptc; ++k) {
            or_residual(C, 0, q, Rk);
            for (size_t t = 0; t < N; ++t) F[t] = (q[t] - sv[t]) / adt - Rk[t];
            res = rms_scaled(N, adt, F);
            if (res <= o->tol_newton) { conv = 1; break; }
            if (k == o->max_ptc) break;
            for (size_t t = 0; t < N; ++t) F[t] = -F[t];
            if (o->nonlinear == 1) {
                or_pmg_apply(C, q, Rk, F, dq);
            } else {
                or_gmres_stats gs;
                or_gmres(C, q, Rk, F, dq, o->kdim, o->tol_gmres, o->maxit_gmres, c, o->eps, o->use_pmg, &gs);
                st->n_gmres += gs.iters;
            }
            for (size_t t = 0; t < N; ++t) q[t] = q[t] + dq[t];
            st->n_ptc++;
        }
        if (!conv) st->converged = 0;
        st->final_res = res;
        memcpy(&Rs[(size_t)i * N], Rk, sizeof(double) * N);
    }
    for (size_t t = 0; t < N; ++t) {
        double acc = 0.0;
        for (int j = 0; j < s; ++j) acc = fma(bw[j], Rs[(size_t)j * N + t], acc);
        q[t] = qn[t] + dt * acc;
    }
    free(qn); free(Rs); free(sv); free(F); free(Rk); free(dq);
    return st->converged ? 0 : 1;
}

/* ROW step, Eq. (3): a, cc are the s x s strictly lower transformed coefficients, m the weights */
int or_row_step(or_ctx *C, int s, double gam, const double *a, const double *cc, const double *m,
                double dt, double *q, const or_solve_opts *o, or_step_stats *st) {
    size_t N = vlen(C, 0);
    double *qn = malloc(sizeof(double) * N), *Rn = malloc(sizeof(double) * N);
    double *Y = malloc(sizeof(double) * N * s), *qi = malloc(sizeof(double) * N);
    double *rhs = malloc(sizeof(double) * N), *Ri = malloc(sizeof(double) * N);
    memcpy(qn, q, sizeof(double) * N);
    or_residual(C, 0, qn, Rn);
    memset(st, 0, sizeof(*st));
    st->converged = 1;
    double c = 1.0 / (gam * dt);
    if (o->use_pmg) or_pmg_setup(C, qn, o->nlev, o->nsmooth, c, o->inv_dtau_star, o->mbnk, o->mbnk_maxit, o->mbnk_tol);
    for (int i = 0; i < s; ++i) {
        for (size_t t = 0; t < N; ++t) {
            double acc = 0.0;
            for (int j = 0; j < i; ++j) acc = fma(a[i * s + j], Y[(size_t)j * N + t], acc);
            qi[t] = qn[t] + acc;
        }
        if (i == 0) memcpy(Ri, Rn, sizeof(double) * N);
        else or_residual(C, 0, qi, Ri);
        for (size_t t = 0; t < N; ++t) {
            double acc = 0.0;
            for (int j = 0; j < i; ++j) acc = fma(cc[i * s + j], Y[(size_t)j * N + t], acc);
            rhs[t] = Ri[t] + acc / dt;
        }
        or_gmres_stats gs;
        or_gmres(C, qn, Rn, rhs, &Y[(size_t)i * N], o->kdim, o->tol_gmres, o->maxit_gmres, c, o->eps,
                 o->use_pmg, &gs);
        st->n_gmres += gs.iters;
        if (gs.relres > o->tol_gmres) st->converged = 0;
        st->final_res = gs.relres;
    }
    for (size_t t = 0; t < N; ++t) {
        double acc = 0.0;
        for (int j = 0; j < s; ++j) acc = fma(m[j], Y[(size_t)j * N + t], acc);
        q[t] = qn[t] + acc;
    }
    free(qn); free(Rn); free(Y); free(qi); free(rhs); free(Ri);
    return st->converged ? 0 : 1;
}

/* steady PTC with SER; Eq. (7) without the dt terms, Eq. (10) with the growth reading */
int or_ptc_steady(or_ctx *C, double *q, double dtau_init, double dtau_max, double tol_rel, int max_it,
                  const or_solve_opts *o, or_step_stats *st, double *hist) {
    size_t N = vlen(C, 0);
    double *R = malloc(sizeof(double) * N), *dq = malloc(sizeof(double) * N);
    memset(st, 0, sizeof(*st));
    or_residual(C, 0, q, R);
    double r0 = sqrt(dot(N, R, R)), rk = r0, dtau = dtau_init;
    if (hist) hist[0] = r0;
    int k;
    for (k = 0; k < max_it; ++k) {
        if (rk <= tol_rel * r0) break;
        double c = 1.0 / dtau;
        if (o->use_pmg)
            or_pmg_setup(C, q, o->nlev, o->nsmooth, c, o->inv_dtau_star < 0 ? c : o->inv_dtau_star, o->mbnk,
                         o->mbnk_maxit, o->mbnk_tol);
        or_gmres_stats gs;
        or_gmres(C, q, R, R, dq, o->kdim, o->tol_gmres, o->maxit_gmres, c, o->eps, o->use_pmg, &gs);
        st->n_gmres += gs.iters;
        for (size_t t = 0; t < N; ++t) q[t] = q[t] + dq[t];
        or_residual(C, 0, q, R);
        double rn = sqrt(dot(N, R, R));
        dtau = fmin(dtau * (rk / rn), dtau_max);
        rk = rn;
        st->n_ptc++;
        if (hist) hist[k + 1] = rn;
    }
    st->final_res = rk / r0;
    st->converged = rk <= tol_rel * r0;
    free(R); free(dq);
    return st->converged ? 0 : 1;
}

/* The pMG nonlinear solver for steady problems (Sec. 3.1, Eqs. 11-16): every iteration is
 * one nonlinear V-cycle of pseudo-time marching on R(q) = 0 started from the current
 * state.  The preconditioner's cycle solves 0 = X + R(qh) - c (qh - q) - R(q); with
 * X = R(q) that is the backward-Euler pseudo step R(qh) - c (qh - q) = 0, c = 1/dtau, so the
 * iteration is q <- q + P(q, R(q), R(q)); dtau follows the same SER rule as the PTC
 * driver.  Element blocks are formed at every iteration's q. */
int or_pmg_steady(or_ctx *C, double *q, double dtau_init, double dtau_max, double tol_rel, int max_it,
                  const or_solve_opts *o, or_step_stats *st, double *hist) {
    size_t N = vlen(C, 0);
    double *R = malloc(sizeof(double) * N), *Y = malloc(sizeof(double) * N);
    memset(st, 0, sizeof(*st));
    or_residual(C, 0, q, R);
    double r0 = sqrt(dot(N, R, R)), rk = r0, dtau = dtau_init;
    if (hist) hist[0] = r0;
    for (int k = 0; k < max_it; ++k) {
        if (rk <= tol_rel * r0) break;
        double c = 1.0 / dtau;
        or_pmg_setup(C, q, o->nlev, o->nsmooth, c, o->inv_dtau_star < 0 ? c : o->inv_dtau_star, o->mbnk,
                     o->mbnk_maxit, o->mbnk_tol);
        or_pmg_apply(C, q, R, R, Y);
        for (size_t t = 0; t < N; ++t) q[t] = q[t] + Y[t];
        or_residual(C, 0, q, R);
        double rn = sqrt(dot(N, R, R));
        dtau = fmin(dtau * (rk / rn), dtau_max);
        rk = rn;
        st->n_ptc++;
        if (hist) hist[k + 1] = rn;
    }
    st->final_res = rk / r0;
    st->converged = rk <= tol_rel * r0;
    free(R); free(Y);
    return st->converged ? 0 : 1;
}
