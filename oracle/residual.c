/*
 * Oracle FR residual R(q) for the compressible Navier-Stokes equations
 * (TEST INFRASTRUCTURE ONLY; shares no code with the CUDA library).
 *
 * Eq. (1): dq/dt + div f = 0, f = f_inv(q) - f_visc(q, grad q).  The semi-discrete
 * operator is used with the sign R = -div f so that dq/dt = R, which is the sign the
 * ESDIRK (Eq. 2), Rosenbrock (Eq. 3) and Jacobian-vector (Eq. 8) formulas need.
 * Spatial discretisation: flux reconstruction (Sec. 2.1) on tensor-product elements with
 * Gauss-Legendre solution points and DG (Radau) correction functions; Rusanov common
 * inviscid flux; BR2 common viscous flux.  Stages:
 *   1 interpolate q to the flux points of every element
 *   2 per face-point pair: common solution qs = (qL+qR)/2, jumps dq = qs - q_side
 *   3 per element: corrected gradient at solution points; face gradient traces
 *     (uncorrected) plus the BR2 face lifting eta g'(face) dq in the face-normal
 *     reference direction
 *   4 per face-point pair: common normal flux  Rusanov(qL,qR,n) - f_v(qs, avg grad).n
 *   5 per element: transformed flux, divergence with FR corrections, R = -div / J.
 * Arithmetic convention: see oracle.h.
 */
#include <math.h>
#include <string.h>
#include <stdlib.h>
#include "oracle.h"

#define NVMAX 5
#define NPMAX (OR_MAXN * OR_MAXN * OR_MAXN)

/* ---------------------------------------------------------------- indexing */
static int sp_idx(int n, int d, const int *ii) {
    return d == 2 ? ii[0] + n * ii[1] : ii[0] + n * (ii[1] + n * ii[2]);
}
static void sp_coords(int n, int d, int i, int *ii) {
    ii[0] = i % n; ii[1] = (i / n) % n; ii[2] = (d == 3) ? i / (n * n) : 0;
}
static void tang_dirs(int d, int df, int *td) {
    int j = 0;
    for (int c = 0; c < d; ++c) if (c != df) td[j++] = c;
}
/* face point k -> normal dir df, side s, coordinates ii (ii[df] left unset) */
static void fp_decode(int n, int d, int nf1, int k, int *df, int *s, int *ii) {
    int f = k / nf1, t = k % nf1, td[2] = {0, 0};
    *df = f / 2; *s = f % 2;
    tang_dirs(d, *df, td);
    ii[0] = ii[1] = ii[2] = 0;
    ii[td[0]] = t % n;
    if (d == 3) ii[td[1]] = t / n;
}
static int fp_encode(int n, int d, int nf1, int df, int s, const int *ii) {
    int td[2] = {0, 0};
    tang_dirs(d, df, td);
    int t = ii[td[0]] + (d == 3 ? n * ii[td[1]] : 0);
    return (2 * df + s) * nf1 + t;
}

/* ---------------------------------------------------------------- physics */
void or_flux_inviscid(const or_ctx *C, const double *q, double f[3][5]) {
    int d = C->d;
    double gm1 = C->ph.gamma - 1.0;
    double rho = q[0], E = q[d + 1], u[3], ke = 0.0, rinv = 1.0 / rho;
    for (int j = 0; j < d; ++j) u[j] = q[1 + j] * rinv;
    for (int j = 0; j < d; ++j) ke = fma(q[1 + j], u[j], ke);
    double p = gm1 * (E - 0.5 * ke);
    for (int c = 0; c < d; ++c) {
        f[c][0] = q[1 + c];
        for (int j = 0; j < d; ++j) {
            double t = q[1 + c] * u[j];
            if (j == c) t = t + p;
            f[c][1 + j] = t;
        }
        f[c][d + 1] = (E + p) * u[c];
    }
}

void or_flux_viscous(const or_ctx *C, const double *q, double Q[3][5], int adiabatic, double f[3][5]) {
    int d = C->d;
    double gamma = C->ph.gamma, mu = C->ph.mu;
    double kappa = (gamma * mu) / C->ph.Pr, c23 = 2.0 / 3.0;
    double rho = q[0], E = q[d + 1], u[3], rinv = 1.0 / rho, Er = E * rinv;
    double du[3][3], de[3], tau[3][3];
    for (int j = 0; j < d; ++j) u[j] = q[1 + j] * rinv;
    for (int j = 0; j < d; ++j)
        for (int c = 0; c < d; ++c) du[j][c] = (Q[c][1 + j] - u[j] * Q[c][0]) * rinv;
    for (int c = 0; c < d; ++c) {
        double s = 0.0;
        for (int j = 0; j < d; ++j) s = fma(u[j], du[j][c], s);
        de[c] = (Q[c][d + 1] - Er * Q[c][0]) * rinv;
        de[c] = de[c] - s;
    }
    double divu = 0.0;
    for (int j = 0; j < d; ++j) divu = divu + du[j][j];
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double t = du[i][j] + du[j][i];
            if (i == j) t = t - c23 * divu;
            tau[i][j] = mu * t;
        }
    for (int c = 0; c < d; ++c) {
        f[c][0] = 0.0;
        for (int j = 0; j < d; ++j) f[c][1 + j] = tau[j][c];
        double s = 0.0;
        for (int j = 0; j < d; ++j) s = fma(u[j], tau[j][c], s);
        if (!adiabatic) s = s + kappa * de[c];
        f[c][d + 1] = s;
    }
}

/* Rusanov (local Lax-Friedrichs) flux along the scaled normal n */
void or_rusanov(const or_ctx *C, const double *qL, const double *qR, const double *n, double *F) {
    int d = C->d, nv = C->nv;
    double gamma = C->ph.gamma, gm1 = gamma - 1.0;
    double fL[3][5], fR[3][5];
    or_flux_inviscid(C, qL, fL);
    or_flux_inviscid(C, qR, fR);
    double nn = 0.0;
    for (int c = 0; c < d; ++c) nn = fma(n[c], n[c], nn);
    double nmag = sqrt(nn);
    double lam[2];
    for (int side = 0; side < 2; ++side) {
        const double *q = side ? qR : qL;
        double rho = q[0], E = q[d + 1], u[3], ke = 0.0, vn = 0.0, rinv = 1.0 / rho;
        for (int j = 0; j < d; ++j) u[j] = q[1 + j] * rinv;
        for (int j = 0; j < d; ++j) ke = fma(q[1 + j], u[j], ke);
        double p = gm1 * (E - 0.5 * ke);
        double a = sqrt((gamma * p) * rinv);
        for (int c = 0; c < d; ++c) vn = fma(u[c], n[c], vn);
        lam[side] = fabs(vn) + a * nmag;
    }
    double lmax = fmax(lam[0], lam[1]);
    for (int v = 0; v < nv; ++v) {
        double FnL = 0.0, FnR = 0.0;
        for (int c = 0; c < d; ++c) FnL = fma(fL[c][v], n[c], FnL);
        for (int c = 0; c < d; ++c) FnR = fma(fR[c][v], n[c], FnR);
        F[v] = 0.5 * (FnL + FnR) - 0.5 * lmax * (qR[v] - qL[v]);
    }
}

/* Roe's approximate Riemann solver along the scaled normal n (Sec. 4.2 names the original
 * Roe solver as the inviscid common flux of the unsteady cases; no entropy fix).  Written from
 * the textbook construction: Roe-averaged density sqrt(rhoL rhoR) and sqrt(rho)-weighted
 * velocity and total enthalpy; the jump qR - qL split into the acoustic waves vn -/+ c
 * (strengths (dp -/+ rho c dvn) / (2 c^2)), the entropy wave (drho - dp / c^2) and the shear
 * waves (rho (du - dvn nh)), the last two at speed vn.  F = (FnL + FnR)/2 - |n| D / 2, with D
 * the sum over waves of |speed| x strength x right eigenvector along the unit normal nh. */
void or_roe(const or_ctx *C, const double *qL, const double *qR, const double *n, double *F) {
    int d = C->d, nv = C->nv;
    double gm1 = C->ph.gamma - 1.0;
    double fL[3][5], fR[3][5];
    or_flux_inviscid(C, qL, fL);
    or_flux_inviscid(C, qR, fR);
    double nn = 0.0;
    for (int c = 0; c < d; ++c) nn = fma(n[c], n[c], nn);
    double nmag = sqrt(nn);
    double nh[3];
    for (int c = 0; c < d; ++c) nh[c] = n[c] / nmag;
    double rho[2], u[2][3], p[2], H[2];
    for (int side = 0; side < 2; ++side) {
        const double *q = side ? qR : qL;
        double rinv = 1.0 / q[0], ke = 0.0;
        rho[side] = q[0];
        for (int j = 0; j < d; ++j) u[side][j] = q[1 + j] * rinv;
        for (int j = 0; j < d; ++j) ke = fma(q[1 + j], u[side][j], ke);
        p[side] = gm1 * (q[d + 1] - 0.5 * ke);
        H[side] = (q[d + 1] + p[side]) * rinv;
    }
    /* Roe average */
    double sL = sqrt(rho[0]), sR = sqrt(rho[1]), wt = 1.0 / (sL + sR);
    double ut[3], q2 = 0.0, vn = 0.0, du[3], dvn = 0.0, udu = 0.0;
    for (int j = 0; j < d; ++j) ut[j] = (sL * u[0][j] + sR * u[1][j]) * wt;
    double Ht = (sL * H[0] + sR * H[1]) * wt;
    for (int j = 0; j < d; ++j) q2 = fma(ut[j], ut[j], q2);
    for (int j = 0; j < d; ++j) vn = fma(ut[j], nh[j], vn);
    double c2 = gm1 * (Ht - 0.5 * q2);
    double ct = sqrt(c2);
    double rt = sL * sR;
    /* jumps and wave strengths */
    double drho = rho[1] - rho[0], dp = p[1] - p[0];
    for (int j = 0; j < d; ++j) du[j] = u[1][j] - u[0][j];
    for (int j = 0; j < d; ++j) dvn = fma(du[j], nh[j], dvn);
    for (int j = 0; j < d; ++j) udu = fma(ut[j], du[j], udu);
    double a1 = (dp - rt * ct * dvn) / (2.0 * c2);
    double a3 = (dp + rt * ct * dvn) / (2.0 * c2);
    double a2 = drho - dp / c2;
    double l1 = fabs(vn - ct), l2 = fabs(vn), l3 = fabs(vn + ct);
    double w1 = l1 * a1, w2 = l2 * a2, w3 = l3 * a3, ws = l2 * rt;
    /* |A_nh| (qR - qL) */
    double Dv[5];
    Dv[0] = w1 + w2 + w3;
    for (int j = 0; j < d; ++j)
        Dv[1 + j] = w1 * (ut[j] - ct * nh[j]) + w2 * ut[j] + ws * (du[j] - dvn * nh[j]) + w3 * (ut[j] + ct * nh[j]);
    Dv[d + 1] = w1 * (Ht - ct * vn) + w2 * (0.5 * q2) + ws * (udu - vn * dvn) + w3 * (Ht + ct * vn);
    for (int v = 0; v < nv; ++v) {
        double FnL = 0.0, FnR = 0.0;
        for (int c = 0; c < d; ++c) FnL = fma(fL[c][v], n[c], FnL);
        for (int c = 0; c < d; ++c) FnR = fma(fR[c][v], n[c], FnR);
        F[v] = 0.5 * (FnL + FnR) - 0.5 * nmag * Dv[v];
    }
}

/* Weiss-Smith low-Mach preconditioning of Roe's dissipation (Sec. 4.1 uses it with Roe's
 * solver for the steady low-Mach sphere).  In the primitive variables Q = (p, u, T), with the
 * gas constant 1 (T = p / rho, C_p = gamma / (gamma - 1), c^2 = gamma T), the dissipation is
 *     D = Gamma |Gamma^{-1} A_n| (Q_R - Q_L)
 * at the Roe-averaged state (rho, u, H of Roe's solver), where A_n = dF_n/dQ along the unit
 * normal and Gamma = dW/dQ with drho/dp replaced by theta = 1/Ur^2 - rho_T / (rho C_p); the
 * reference velocity Ur = min(c, max(|u|, umin)).  Gamma^{-1} A_n has the eigenvalues vn
 * (d times) and u' +- c', u' = vn (1 - alpha), c' = sqrt(alpha^2 vn^2 + Ur^2), alpha =
 * (1 - Ur^2 / c^2) / 2: three distinct values (Ur > 0).  So |Gamma^{-1} A_n| is the
 * quadratic p(B) = a0 + a1 B + a2 B^2 that takes |lambda| at them, and
 *     D = a0 Gamma dQ + a1 A_n dQ + a2 A_n Gamma^{-1} A_n dQ.
 * With Ur = c, Gamma = dW/dQ and D is Roe's |A| dW to first order in the jump. */
typedef struct { double rho, u[3], H, T, rp, rT, cp, theta, vn, nh[3]; int d; } ws_state;

static void ws_apply_A(const ws_state *S, const double *x, double *y) {
    int d = S->d;
    double nx = 0.0, ux = 0.0;
    for (int j = 0; j < d; ++j) nx = fma(S->nh[j], x[1 + j], nx);
    for (int j = 0; j < d; ++j) ux = fma(S->u[j], x[1 + j], ux);
    double r = S->rp * S->vn * x[0] + S->rho * nx + S->rT * S->vn * x[d + 1];
    y[0] = r;
    for (int i = 0; i < d; ++i) y[1 + i] = S->u[i] * r + S->nh[i] * x[0] + S->rho * S->vn * x[1 + i];
    y[d + 1] = S->H * r + S->rho * S->vn * ux + S->rho * S->cp * S->vn * x[d + 1];
}
static void ws_apply_G(const ws_state *S, const double *x, double *y) {
    int d = S->d;
    double ux = 0.0;
    for (int j = 0; j < d; ++j) ux = fma(S->u[j], x[1 + j], ux);
    double r = S->theta * x[0] + S->rT * x[d + 1];
    y[0] = r;
    for (int i = 0; i < d; ++i) y[1 + i] = S->u[i] * r + S->rho * x[1 + i];
    y[d + 1] = S->H * r - x[0] + S->rho * ux + S->rho * S->cp * x[d + 1];
}
/* z = Gamma^{-1} y: the velocity rows give z_u, the energy row minus H times the first
 * leaves -z_p + rho C_p z_T = s, which with theta z_p + rho_T z_T = y_0 fixes z_p, z_T */
static void ws_solve_G(const ws_state *S, const double *y, double *z) {
    int d = S->d;
    double r0 = y[0], sum = 0.0;
    for (int i = 0; i < d; ++i) {
        double t = y[1 + i] - S->u[i] * r0;
        z[1 + i] = t / S->rho;
        sum = fma(S->u[i], t, sum);
    }
    double s = y[d + 1] - S->H * r0 - sum;
    double det = S->theta * S->rho * S->cp + S->rT;
    z[0] = (r0 * S->rho * S->cp - S->rT * s) / det;
    z[d + 1] = (S->theta * s + r0) / det;
}

void or_weiss_smith(const or_ctx *C, const double *qL, const double *qR, const double *n, double *F) {
    int d = C->d, nv = C->nv;
    double gamma = C->ph.gamma, gm1 = gamma - 1.0;
    double fL[3][5], fR[3][5];
    or_flux_inviscid(C, qL, fL);
    or_flux_inviscid(C, qR, fR);
    double nn = 0.0;
    for (int c = 0; c < d; ++c) nn = fma(n[c], n[c], nn);
    double nmag = sqrt(nn);
    ws_state S;
    S.d = d;
    for (int c = 0; c < d; ++c) S.nh[c] = n[c] / nmag;
    double rho[2], u[2][3], p[2], H[2], T[2];
    for (int side = 0; side < 2; ++side) {
        const double *q = side ? qR : qL;
        double rinv = 1.0 / q[0], ke = 0.0;
        rho[side] = q[0];
        for (int j = 0; j < d; ++j) u[side][j] = q[1 + j] * rinv;
        for (int j = 0; j < d; ++j) ke = fma(q[1 + j], u[side][j], ke);
        p[side] = gm1 * (q[d + 1] - 0.5 * ke);
        H[side] = (q[d + 1] + p[side]) * rinv;
        T[side] = p[side] * rinv;
    }
    double sL = sqrt(rho[0]), sR = sqrt(rho[1]), wt = 1.0 / (sL + sR), q2 = 0.0;
    for (int j = 0; j < d; ++j) S.u[j] = (sL * u[0][j] + sR * u[1][j]) * wt;
    S.H = (sL * H[0] + sR * H[1]) * wt;
    for (int j = 0; j < d; ++j) q2 = fma(S.u[j], S.u[j], q2);
    S.vn = 0.0;
    for (int j = 0; j < d; ++j) S.vn = fma(S.u[j], S.nh[j], S.vn);
    double c2 = gm1 * (S.H - 0.5 * q2);
    S.rho = sL * sR;
    S.cp = gamma / gm1;
    S.T = c2 / gamma;
    S.rp = 1.0 / S.T;
    S.rT = -S.rho / S.T;
    double ur = fmin(sqrt(c2), fmax(sqrt(q2), C->ph.ws_umin));
    S.theta = 1.0 / (ur * ur) - S.rT / (S.rho * S.cp);
    double alpha = 0.5 * (1.0 - (ur * ur) / c2);
    double up = S.vn * (1.0 - alpha), cq = sqrt(alpha * alpha * S.vn * S.vn + ur * ur);
    double l1 = S.vn, l2 = up + cq, l3 = up - cq;
    double f1 = fabs(l1), f2 = fabs(l2), f3 = fabs(l3);
    double s21 = (f2 - f1) / (l2 - l1), s31 = (f3 - f1) / (l3 - l1);
    double a2 = (s31 - s21) / (l3 - l2);
    double a1 = s21 - a2 * (l1 + l2);
    double a0 = f1 - a1 * l1 - a2 * (l1 * l1);
    double dQ[5], g[5], y1[5], z[5], y2[5], Dv[5];
    dQ[0] = p[1] - p[0];
    for (int j = 0; j < d; ++j) dQ[1 + j] = u[1][j] - u[0][j];
    dQ[d + 1] = T[1] - T[0];
    ws_apply_G(&S, dQ, g);
    ws_apply_A(&S, dQ, y1);
    ws_solve_G(&S, y1, z);
    ws_apply_A(&S, z, y2);
    for (int v = 0; v < nv; ++v) Dv[v] = a0 * g[v] + a1 * y1[v] + a2 * y2[v];
    for (int v = 0; v < nv; ++v) {
        double FnL = 0.0, FnR = 0.0;
        for (int c = 0; c < d; ++c) FnL = fma(fL[c][v], n[c], FnL);
        for (int c = 0; c < d; ++c) FnR = fma(fR[c][v], n[c], FnR);
        F[v] = 0.5 * (FnL + FnR) - 0.5 * nmag * Dv[v];
    }
}

/* boundary ghost state: 1 = far field (free stream), 2 = no-slip adiabatic wall */
static void ghost(const or_ctx *C, int bc, const double *qL, double *qR) {
    int d = C->d;
    if (bc == 1) {
        for (int v = 0; v < C->nv; ++v) qR[v] = C->ph.qinf[v];
    } else {
        qR[0] = qL[0];
        for (int j = 0; j < d; ++j) qR[1 + j] = -qL[1 + j];
        qR[d + 1] = qL[d + 1];
    }
}

/* outward scaled normal of the L side of pair P */
static void pair_normal(const or_ctx *C, const or_level *L, int P, double *nrm) {
    int d = C->d, E = C->E, df, s, ii[3];
    int eL = L->pe[2 * P], kL = L->pk[2 * P];
    fp_decode(L->n, d, L->nf1, kL, &df, &s, ii);
    for (int c = 0; c < d; ++c) {
        double v = L->Sf[((size_t)(df * d + c) * L->nfp + kL) * E + eL];
        nrm[c] = s ? v : -v;
    }
}

/* --------------------------------------------------- per-element building blocks */
/* stage 1: qfe[v][k] from qe[v][i] */
static void interp_faces(const or_ctx *C, const or_level *L, const double *qe, double *qfe) {
    int d = C->d, n = L->n, np = L->np, nfp = L->nfp;
    for (int k = 0; k < nfp; ++k) {
        int df, s, ii[3];
        fp_decode(n, d, L->nf1, k, &df, &s, ii);
        const double *l = s ? L->T.lp : L->T.lm;
        for (int v = 0; v < C->nv; ++v) {
            double acc = 0.0;
            for (int m = 0; m < n; ++m) {
                ii[df] = m;
                acc = fma(l[m], qe[v * np + sp_idx(n, d, ii)], acc);
            }
            qfe[v * nfp + k] = acc;
        }
    }
}

/* face gradient with BR2 lifting from uncorrected reference gradient gf[dd] at face point k */
static void face_grad(const or_ctx *C, const or_level *L, int e, int k, double gf[3][5],
                      const double *dqk, double Qk[3][5]) {
    int d = C->d, E = C->E, df, s, ii[3];
    fp_decode(L->n, d, L->nf1, k, &df, &s, ii);
    double etag = C->ph.eta * (s ? L->T.gRf : L->T.gLf);
    for (int v = 0; v < C->nv; ++v) {
        double comp[3];
        for (int dd = 0; dd < d; ++dd) comp[dd] = gf[dd][v];
        comp[df] = fma(etag, dqk[v], gf[df][v]);
        for (int c = 0; c < d; ++c) {
            double acc = 0.0;
            for (int dd = 0; dd < d; ++dd)
                acc = fma(L->Gf[((size_t)(dd * d + c) * L->nfp + k) * E + e], comp[dd], acc);
            Qk[c][v] = acc;
        }
    }
}

/* stage 3 for element e.  Outputs: Qe[c][v][i] corrected physical gradient,
 * gfe[dd][v][k] uncorrected reference gradient at face points, Qfe[c][v][k] face gradient
 * with lifting. */
static void grad_elem(const or_ctx *C, const or_level *L, int e, const double *qe,
                      const double *qfe, const double *dqe, double *Qe, double *gfe, double *Qfe) {
    int d = C->d, E = C->E, n = L->n, np = L->np, nfp = L->nfp, nv = C->nv;
    const or_tab *T = &L->T;
    for (int i = 0; i < np; ++i) {
        int ii[3], jj[3];
        sp_coords(n, d, i, ii);
        for (int v = 0; v < nv; ++v) {
            double gr[3];
            for (int dd = 0; dd < d; ++dd) {
                double t = 0.0;
                memcpy(jj, ii, sizeof jj);
                for (int m = 0; m < n; ++m) {
                    jj[dd] = m;
                    t = fma(T->D[ii[dd]][m], qe[v * np + sp_idx(n, d, jj)], t);
                }
                int kL = fp_encode(n, d, L->nf1, dd, 0, ii), kR = fp_encode(n, d, L->nf1, dd, 1, ii);
                t = fma(T->gLd[ii[dd]], dqe[v * nfp + kL], t);
                t = fma(T->gRd[ii[dd]], dqe[v * nfp + kR], t);
                gr[dd] = t;
            }
            for (int c = 0; c < d; ++c) {
                double acc = 0.0;
                for (int dd = 0; dd < d; ++dd)
                    acc = fma(L->G[((size_t)(dd * d + c) * np + i) * E + e], gr[dd], acc);
                Qe[(c * nv + v) * np + i] = acc;
            }
        }
    }
    for (int k = 0; k < nfp; ++k) {
        int df, s, ii[3], td[2], jj[3];
        fp_decode(n, d, L->nf1, k, &df, &s, ii);
        tang_dirs(d, df, td);
        const double *dl = s ? T->dlp : T->dlm;
        double gf[3][5], dqk[5], Qk[3][5];
        for (int v = 0; v < nv; ++v) {
            double t = 0.0;
            memcpy(jj, ii, sizeof jj);
            for (int m = 0; m < n; ++m) {
                jj[df] = m;
                t = fma(dl[m], qe[v * np + sp_idx(n, d, jj)], t);
            }
            gf[df][v] = t;
            for (int j = 0; j < d - 1; ++j) {
                int tdir = td[j];
                double u = 0.0;
                memcpy(jj, ii, sizeof jj);
                for (int m = 0; m < n; ++m) {
                    jj[tdir] = m;
                    u = fma(T->D[ii[tdir]][m], qfe[v * nfp + fp_encode(n, d, L->nf1, df, s, jj)], u);
                }
                gf[tdir][v] = u;
            }
            dqk[v] = dqe[v * nfp + k];
        }
        for (int dd = 0; dd < d; ++dd)
            for (int v = 0; v < nv; ++v) gfe[(dd * nv + v) * nfp + k] = gf[dd][v];
        face_grad(C, L, e, k, gf, dqk, Qk);
        for (int c = 0; c < d; ++c)
            for (int v = 0; v < nv; ++v) Qfe[(c * nv + v) * nfp + k] = Qk[c][v];
    }
}

/* stage 4 for pair P given both traces (qR, QR ignored on boundary pairs) */
static void pair_flux(const or_ctx *C, const or_level *L, int P, const double *qL, const double *qRin,
                      double QL[3][5], double QR[3][5], double *F) {
    int d = C->d, nv = C->nv, bc = L->bc[P];
    double nrm[3], qR[5], qs[5], Qs[3][5], Fr[5], fv[3][5];
    pair_normal(C, L, P, nrm);
    if (bc == 0) memcpy(qR, qRin, sizeof(double) * nv);
    else ghost(C, bc, qL, qR);
    for (int v = 0; v < nv; ++v) qs[v] = 0.5 * (qL[v] + qR[v]);
    for (int c = 0; c < d; ++c)
        for (int v = 0; v < nv; ++v) Qs[c][v] = (bc == 0) ? 0.5 * (QL[c][v] + QR[c][v]) : QL[c][v];
    if (C->ph.flux == 2) or_weiss_smith(C, qL, qR, nrm, Fr);
    else if (C->ph.flux == 1) or_roe(C, qL, qR, nrm, Fr);
    else or_rusanov(C, qL, qR, nrm, Fr);
    or_flux_viscous(C, qs, Qs, bc == 2, fv);
    for (int v = 0; v < nv; ++v) {
        double Fv = 0.0;
        for (int c = 0; c < d; ++c) Fv = fma(fv[c][v], nrm[c], Fv);
        F[v] = Fr[v] - Fv;
    }
}

/* stage 5 for element e: R_e from q_e, Q_e and the common normal fluxes fne[v][k] */
static void div_elem(const or_ctx *C, const or_level *L, int e, const double *qe, const double *Qe,
                     const double *fne, double *Re) {
    int d = C->d, E = C->E, n = L->n, np = L->np, nfp = L->nfp, nv = C->nv;
    const or_tab *T = &L->T;
    static _Thread_local double Ft[3 * NVMAX * NPMAX];
    for (int i = 0; i < np; ++i) {
        double qi[5], Qi[3][5], fi[3][5], fvi[3][5];
        for (int v = 0; v < nv; ++v) qi[v] = qe[v * np + i];
        for (int c = 0; c < d; ++c)
            for (int v = 0; v < nv; ++v) Qi[c][v] = Qe[(c * nv + v) * np + i];
        or_flux_inviscid(C, qi, fi);
        or_flux_viscous(C, qi, Qi, 0, fvi);
        for (int dd = 0; dd < d; ++dd)
            for (int v = 0; v < nv; ++v) {
                double acc = 0.0;
                for (int c = 0; c < d; ++c)
                    acc = fma(L->S[((size_t)(dd * d + c) * np + i) * E + e], fi[c][v] - fvi[c][v], acc);
                Ft[(dd * nv + v) * np + i] = acc;
            }
    }
    for (int i = 0; i < np; ++i) {
        int ii[3], jj[3];
        sp_coords(n, d, i, ii);
        for (int v = 0; v < nv; ++v) {
            double div = 0.0;
            for (int dd = 0; dd < d; ++dd) {
                const double *F = &Ft[(dd * nv + v) * np];
                double t = 0.0, FL = 0.0, FR = 0.0;
                memcpy(jj, ii, sizeof jj);
                for (int m = 0; m < n; ++m) {
                    jj[dd] = m;
                    t = fma(T->D[ii[dd]][m], F[sp_idx(n, d, jj)], t);
                }
                for (int m = 0; m < n; ++m) {
                    jj[dd] = m;
                    FL = fma(T->lm[m], F[sp_idx(n, d, jj)], FL);
                }
                for (int m = 0; m < n; ++m) {
                    jj[dd] = m;
                    FR = fma(T->lp[m], F[sp_idx(n, d, jj)], FR);
                }
                int kL = fp_encode(n, d, L->nf1, dd, 0, ii), kR = fp_encode(n, d, L->nf1, dd, 1, ii);
                double FsL = -fne[v * nfp + kL], FsR = fne[v * nfp + kR];
                t = fma(T->gLd[ii[dd]], FsL - FL, t);
                t = fma(T->gRd[ii[dd]], FsR - FR, t);
                div = div + t;
            }
            Re[v * np + i] = -(div * L->invJ[(size_t)i * E + e]);
        }
    }
}

/* ------------------------------------------------------------ gather/scatter */
static void gather(const double *g, int nrow, int E, int e, double *loc) {
    for (int r = 0; r < nrow; ++r) loc[r] = g[(size_t)r * E + e];
}
static void scatter(double *g, int nrow, int E, int e, const double *loc) {
    for (int r = 0; r < nrow; ++r) g[(size_t)r * E + e] = loc[r];
}

/* ------------------------------------------------------------ full residual */
void or_residual(or_ctx *C, int l, const double *q, double *R) {
    or_level *L = &C->L[l];
    int d = C->d, E = C->E, nv = C->nv, np = L->np, nfp = L->nfp;
    static _Thread_local double qe[NVMAX * NPMAX], qfe[NVMAX * NPMAX], dqe[NVMAX * NPMAX];
    static _Thread_local double Qe[3 * NVMAX * NPMAX], gfe[3 * NVMAX * NPMAX], Qfe[3 * NVMAX * NPMAX];
    static _Thread_local double fne[NVMAX * NPMAX], Re[NVMAX * NPMAX];
    /* stage 1 */
#pragma omp parallel for schedule(static)
    for (int e = 0; e < E; ++e) {
        gather(q, nv * np, E, e, qe);
        interp_faces(C, L, qe, qfe);
        scatter(L->qf, nv * nfp, E, e, qfe);
    }
    /* stage 2 */
#pragma omp parallel for schedule(static)
    for (int P = 0; P < L->npairs; ++P) {
        int eL = L->pe[2 * P], kL = L->pk[2 * P], eR = L->pe[2 * P + 1], kR = L->pk[2 * P + 1];
        double qL[5], qR[5];
        for (int v = 0; v < nv; ++v) qL[v] = L->qf[((size_t)v * nfp + kL) * E + eL];
        if (L->bc[P] == 0)
            for (int v = 0; v < nv; ++v) qR[v] = L->qf[((size_t)v * nfp + kR) * E + eR];
        else ghost(C, L->bc[P], qL, qR);
        for (int v = 0; v < nv; ++v) {
            double qs = 0.5 * (qL[v] + qR[v]);
            L->dq[((size_t)v * nfp + kL) * E + eL] = qs - qL[v];
            if (L->bc[P] == 0) L->dq[((size_t)v * nfp + kR) * E + eR] = qs - qR[v];
        }
    }
    /* stage 3 */
#pragma omp parallel for schedule(static)
    for (int e = 0; e < E; ++e) {
        gather(q, nv * np, E, e, qe);
        gather(L->qf, nv * nfp, E, e, qfe);
        gather(L->dq, nv * nfp, E, e, dqe);
        grad_elem(C, L, e, qe, qfe, dqe, Qe, gfe, Qfe);
        scatter(L->Q, d * nv * np, E, e, Qe);
        scatter(L->gface, d * nv * nfp, E, e, gfe);
        scatter(L->Qf, d * nv * nfp, E, e, Qfe);
    }
    /* stage 4 */
#pragma omp parallel for schedule(static)
    for (int P = 0; P < L->npairs; ++P) {
        int eL = L->pe[2 * P], kL = L->pk[2 * P], eR = L->pe[2 * P + 1], kR = L->pk[2 * P + 1];
        int bc = L->bc[P];
        double qL[5], qR[5], QL[3][5], QR[3][5], F[5];
        for (int v = 0; v < nv; ++v) {
            qL[v] = L->qf[((size_t)v * nfp + kL) * E + eL];
            qR[v] = bc == 0 ? L->qf[((size_t)v * nfp + kR) * E + eR] : 0.0;
            for (int c = 0; c < d; ++c) {
                QL[c][v] = L->Qf[((size_t)(c * nv + v) * nfp + kL) * E + eL];
                QR[c][v] = bc == 0 ? L->Qf[((size_t)(c * nv + v) * nfp + kR) * E + eR] : 0.0;
            }
        }
        pair_flux(C, L, P, qL, qR, QL, QR, F);
        for (int v = 0; v < nv; ++v) {
            L->fn[((size_t)v * nfp + kL) * E + eL] = F[v];
            if (bc == 0) L->fn[((size_t)v * nfp + kR) * E + eR] = -F[v];
        }
    }
    /* stage 5 */
#pragma omp parallel for schedule(static)
    for (int e = 0; e < E; ++e) {
        gather(q, nv * np, E, e, qe);
        gather(L->Q, d * nv * np, E, e, Qe);
        gather(L->fn, nv * nfp, E, e, fne);
        div_elem(C, L, e, qe, Qe, fne, Re);
        scatter(R, nv * np, E, e, Re);
    }
}

/* --------------------------------------------------------- element-local residual
 * R restricted to element e when only q_e is replaced by qe_new and every other
 * element keeps its value in q: exactly the stages above evaluated on e and on the
 * neighbour traces that touch e (the neighbour's BR2 lifting depends on q_e through the
 * common solution, so it is recomputed).  Requires or_residual(C, l, q, .) to have been
 * called on the same q (it leaves the neighbours' traces in the level scratch). */
void or_elem_residual(or_ctx *C, int l, const double *q, int e, const double *qe_new, double *Re) {
    or_level *L = &C->L[l];
    int d = C->d, E = C->E, nv = C->nv, nfp = L->nfp;
    (void)q;
    static _Thread_local double qfe[NVMAX * NPMAX], dqe[NVMAX * NPMAX];
    static _Thread_local double Qe[3 * NVMAX * NPMAX], gfe[3 * NVMAX * NPMAX], Qfe[3 * NVMAX * NPMAX];
    static _Thread_local double fne[NVMAX * NPMAX];
    static _Thread_local double dqn[NVMAX * NPMAX];   /* neighbour-side jump at e's face point k */
    interp_faces(C, L, qe_new, qfe);
    for (int k = 0; k < nfp; ++k) {
        int P = L->epair[(size_t)k * E + e];
        int bc = L->bc[P];
        int isL = (L->pe[2 * P] == e && L->pk[2 * P] == k);
        double qme[5], qo[5];
        for (int v = 0; v < nv; ++v) qme[v] = qfe[v * nfp + k];
        if (bc == 0) {
            int eo = isL ? L->pe[2 * P + 1] : L->pe[2 * P];
            int ko = isL ? L->pk[2 * P + 1] : L->pk[2 * P];
            for (int v = 0; v < nv; ++v) qo[v] = L->qf[((size_t)v * nfp + ko) * E + eo];
        } else {
            ghost(C, bc, qme, qo);
        }
        for (int v = 0; v < nv; ++v) {
            double qs = 0.5 * (qme[v] + qo[v]);
            dqe[v * nfp + k] = qs - qme[v];
            dqn[v * nfp + k] = qs - qo[v];
        }
    }
    grad_elem(C, L, e, qe_new, qfe, dqe, Qe, gfe, Qfe);
    for (int k = 0; k < nfp; ++k) {
        int P = L->epair[(size_t)k * E + e];
        int bc = L->bc[P];
        int isL = (L->pe[2 * P] == e && L->pk[2 * P] == k);
        double qme[5], qo[5], Qme[3][5], Qo[3][5], F[5];
        for (int v = 0; v < nv; ++v) {
            qme[v] = qfe[v * nfp + k];
            for (int c = 0; c < d; ++c) Qme[c][v] = Qfe[(c * nv + v) * nfp + k];
        }
        if (bc == 0) {
            int eo = isL ? L->pe[2 * P + 1] : L->pe[2 * P];
            int ko = isL ? L->pk[2 * P + 1] : L->pk[2 * P];
            double gf[3][5], dqk[5];
            for (int v = 0; v < nv; ++v) {
                qo[v] = L->qf[((size_t)v * nfp + ko) * E + eo];
                for (int dd = 0; dd < d; ++dd) gf[dd][v] = L->gface[((size_t)(dd * nv + v) * nfp + ko) * E + eo];
                dqk[v] = dqn[v * nfp + k];
            }
            face_grad(C, L, eo, ko, gf, dqk, Qo);
        } else {
            for (int v = 0; v < nv; ++v) qo[v] = 0.0;
        }
        if (isL) pair_flux(C, L, P, qme, qo, Qme, Qo, F);
        else pair_flux(C, L, P, qo, qme, Qo, Qme, F);
        for (int v = 0; v < nv; ++v) fne[v * nfp + k] = isL ? F[v] : -F[v];
    }
    div_elem(C, L, e, qe_new, Qe, fne, Re);
}
