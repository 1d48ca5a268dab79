// Internal interface between the orchestration layer (lib.cu) and the kernel
// translation units (kernels64.cu).  Not part of the public C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#define FRL_MAXLEV 4

// device-resident data of one p-level
struct FrLevel {
    int d, p, n, np, nf1, nfp, nv, E;
    long long ndof;               // nv * np * E
    int nd;                       // nv * np (element block size)
    int npairs;
    int4 *pairs;                  // (eL, kL, eR, kR), sorted by (kL, eL)
    int *bc;
    double *S, *G, *invJ, *Sf, *Gf;
    // residual workspace
    double *qf, *dq, *Q, *Qf, *fn, *Ft, *Ftf;
    double etagL, etagR;
};

struct FrPhysH {
    double gamma, gm1, mu, kappa, c23, qinf[5];
};

// tables: per degree p (0..5) and transfers per (p0, p1)
struct FrTabH {
    double D[6][6], lm[6], lp[6], dlm[6], dlp[6], gLd[6], gRd[6];
};

int frk64_upload_tables(const FrTabH *tabs /* [6] */, const double *gam /* [6][6][6][6] */,
                        const double *pi /* [6][6][6][6] */);
int frk64_residual(const FrLevel &L, const FrPhysH &ph, const double *q, double *R, cudaStream_t s);

// elementwise helpers
void frk64_axpy_perturb(long long n, const double *q, double eps, const double *v, double *qp, cudaStream_t s);
void frk64_jv_finish(long long n, double shift, const double *v, const double *Rp, const double *Rq, double eps,
                     double *Av, cudaStream_t s);
void frk64_scale(long long n, double a, const double *x, double *y, cudaStream_t s);      // y = x * a
void frk64_div_scalar(long long n, const double *x, double a, double *y, cudaStream_t s);  // y = x / a
void frk64_copy(long long n, const double *x, double *y, cudaStream_t s);
void frk64_add(long long n, const double *a, const double *b, double *y, cudaStream_t s);  // y = a + b
void frk64_sub(long long n, const double *a, const double *b, double *y, cudaStream_t s);  // y = a - b
void frk64_neg(long long n, const double *x, double *y, cudaStream_t s);
// rhs = d - (c (qh - b) - (Rqh - Rb))
void frk64_pmg_rhs(long long n, double c, const double *d, const double *qh, const double *b, const double *Rqh,
                   const double *Rb, double *rhs, cudaStream_t s);
// y[i] = sum_j coef[j] * X[j][i]  (fma chain over j, X rows of stride n), y = base + acc * scale
void frk64_lincomb(long long n, int m, const double *coef_host, const double *const *X, const double *base,
                   double scale, double *y, cudaStream_t s);
// F = (q - sv) / adt - R
void frk64_stage_F(long long n, const double *q, const double *sv, double adt, const double *R, double *F,
                   cudaStream_t s);
// rhs = Ri + acc / dt with acc = sum_j c_j Y_j
// (done by lincomb with base = NULL then frk64_add_scaled)
void frk64_add_div(long long n, const double *a, const double *acc, double dt, double *y, cudaStream_t s);

// reductions (fixed two-level tree), results written to device array out (m values)
int frk64_multidot(long long n, int m, const double *w, const double *const *V, double *out_dev, cudaStream_t s);
// w -= sum_j h[j] V[j] with h on the device
void frk64_multi_axpy(long long n, int m, const double *h_dev, const double *const *V, double *w, cudaStream_t s);
// x += sum_j y[j] Z[j] (host coefficients)
void frk64_update_x(long long n, int m, const double *y_host, const double *const *Z, double *x, cudaStream_t s);

// element blocks by colours
void frk64_perturb_color(const FrLevel &L, const int *color, int col, int j, const double *q, double *qp,
                         cudaStream_t s);
void frk64_restore_color(const FrLevel &L, const int *color, int col, int j, const double *q, double *qp,
                         cudaStream_t s);
void frk64_block_column(const FrLevel &L, const int *color, int col, int j, const double *q, const double *R0,
                        const double *Rp, double shift, double *M, cudaStream_t s);
int frk64_lu_factor(const FrLevel &L, double *M, int *perm, int *info_dev, cudaStream_t s);
int frk64_lu_solve(const FrLevel &L, const double *M, const int *perm, double *x, cudaStream_t s);
int frk64_transfer(const FrLevel &Lf, const FrLevel &Lc, bool restrict_, const double *x, double *y, cudaStream_t s);

unsigned long long frk64_launch_count();
