// Internal interface between the orchestration layer (lib.cu) and the kernel
// translation units (kernels64.cu: FP64, kernels32.cu: FP32).  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include "fr_dual.cuh"

#define FRL_MAXLEV 4

// device-resident data of one p-level in scalar type T
template <typename T>
struct FrLevelT {
    int d, p, n, np, nf1, nfp, nv, E;
    long long ndof;               // nv * np * E
    int nd;                       // nv * np (element block size)
    int npairs;
    int4 *pairs;                  // (eL, kL, eR, kR), sorted by (kL, eL)
    int *bc;
    typename FrBase<T>::type *S, *G, *invJ, *Sf, *Gf;
    // residual workspace: traces, jumps, face gradients, common fluxes, transformed fluxes
    // (volume and at the faces); the corrected volume gradient lives in registers only
    T *qf, *dq, *Qf, *fn, *Ft, *Ftf;
    double etagL, etagR;
    // launch shapes (0 = default): CTA size of the residual kernels (0 interpolation,
    // 1 common solution, 2 gradient + volume flux, 3 face gradients, 4 face flux, 5 unused,
    // 6 face values of the transformed flux, 7 divergence); block solve: columns
    // in flight of the register kernel (2, 4, 8) or 1 = the bulk-copy (TMA) kernel
    short tile[8];
    short lu_g;
};
typedef FrLevelT<double> FrLevel;
typedef FrLevelT<float> FrLevel32;
typedef FrLevelT<DualT> FrLevelAD;

struct FrPhysH {
    double gamma, gm1, mu, kappa, c23, qinf[5];
    int flux;   // 0 Rusanov, 1 Roe, 2 Roe with Weiss-Smith preconditioning
    double ws_umin;   // Weiss-Smith: floor of the reference velocity
};

// tables: per degree p (0..5) and transfers per (p0, p1)
struct FrTabH {
    double D[6][6], lm[6], lp[6], dlm[6], dlp[6], gLd[6], gRd[6];
};

#define FRK_DECLARE(P, T)                                                                                   \
    unsigned long long P##_launch_count();                                                                  \
    int P##_upload_tables(const FrTabH *tabs, const double *gam, const double *pi);                         \
    int P##_residual(const FrLevelT<T> &L, const FrPhysH &ph, const T *q, T *R, cudaStream_t s);            \
    void P##_copy(long long n, const T *x, T *y, cudaStream_t s);                                           \
    void P##_add(long long n, const T *a, const T *b, T *y, cudaStream_t s);                                \
    void P##_sub(long long n, const T *a, const T *b, T *y, cudaStream_t s);                                \
    void P##_pmg_rhs(long long n, double c, const T *d, const T *qh, const T *b, const T *Rqh, const T *Rb,  \
                     T *rhs, cudaStream_t s);                                                               \
    void P##_perturb_color(const FrLevelT<T> &L, const int *color, int col, int j, const T *q, T *qp,       \
                           double epsrel, cudaStream_t s);                                                  \
    void P##_restore_color(const FrLevelT<T> &L, const int *color, int col, int j, const T *q, T *qp,       \
                           cudaStream_t s);                                                                 \
    void P##_block_column(const FrLevelT<T> &L, const int *color, int col, int j, const T *q, const T *R0,  \
                          const T *Rp, double shift, double epsrel, T *M, cudaStream_t s);                  \
    int P##_lu_factor(const FrLevelT<T> &L, T *M, int *perm, int *info_dev, cudaStream_t s);               \
    int P##_lu_solve(const FrLevelT<T> &L, const T *M, const int *perm, T *x, cudaStream_t s);             \
    void P##_lu_solve_prepare();                                                                            \
    int P##_lu_solve_error(int clear);                                                                      \
    void P##_wait_selftest(int limit, cudaStream_t s);                                                      \
    int P##_transfer(const FrLevelT<T> &Lf, const FrLevelT<T> &Lc, bool restrict_, const T *x, T *y,       \
                     cudaStream_t s);                                                                       \
    void P##_halo_pack(int rows, long long E, int nsend, const int *idx, const T *x, T *buf, cudaStream_t s);  \
    void P##_halo_unpack(int rows, long long E, int n_owned, int nrecv, const T *buf, T *x, cudaStream_t s);

FRK_DECLARE(frk64, double)
FRK_DECLARE(frk32, float)

// FP64-only: Jacobian-vector product, Krylov and time-stepping vector kernels
void frk64_axpy_perturb(long long n, const double *q, double eps, const double *v, double *qp, cudaStream_t s);
void frk64_jv_finish(long long n, double shift, const double *v, const double *Rp, const double *Rq, double eps,
                     double *Av, cudaStream_t s);
void frk64_scale(long long n, double a, const double *x, double *y, cudaStream_t s);      // y = x * a
void frk64_div_scalar(long long n, const double *x, double a, double *y, cudaStream_t s);  // y = x / a
void frk64_neg(long long n, const double *x, double *y, cudaStream_t s);
// y = base + scale * sum_j coef[j] X[j]  (fma chain over j; base may be NULL)
void frk64_lincomb(long long n, int m, const double *coef_host, const double *const *X, const double *base,
                   double scale, double *y, cudaStream_t s);
void frk64_stage_F(long long n, const double *q, const double *sv, double adt, const double *R, double *F,
                   cudaStream_t s);                                                    // F = (q - sv)/adt - R
void frk64_add_div(long long n, const double *a, const double *acc, double dt, double *y, cudaStream_t s);
// out_dev[j] = w . V_j over rows x n_owned entries of [rows][E] vectors (n_owned = E: all);
// partial: frk64_multidot_scratch(rows * n_owned) doubles of the caller's
long long frk64_multidot_scratch(long long n);
int frk64_multidot(long long rows, long long E, long long n_owned, int m, const double *w, const double *const *V,
                   double *out_dev, double *partial, cudaStream_t s);
void frk64_multi_axpy(long long n, int m, const double *h_dev, const double *const *V, double *w, cudaStream_t s);
void frk64_update_x(long long n, int m, const double *y_host, const double *const *Z, double *x, cudaStream_t s);

// precision boundary of the mixed preconditioner
void frk32_d2f(long long n, const double *x, float *y, cudaStream_t s);
void frk32_d2f_scaled(long long n, const double *x, const double *xmax_dev, double target, float *y, cudaStream_t s);
// per-variable max |x| of a [nv][per] vector into out_dev[0..nv)
int frk32_absmax_var(int nv, long long per, const double *x, double *out_dev, cudaStream_t s);
int frk32_absmax_var_f(int nv, long long per, const float *x, double *out_dev, cudaStream_t s);
int frk32_absmax(long long n, const double *x, double *out_dev, cudaStream_t s);
// the same over the owned elements (first n_owned of E) of [rows][E] vectors
int frk32_absmax_owned(long long rows, long long E, long long n_owned, const double *x, double *out_dev, cudaStream_t s);
int frk32_absmax_var_owned(int nv, long long np, long long E, long long n_owned, const double *x, double *out_dev,
                           cudaStream_t s);
int frk32_absmax_var_owned_f(int nv, long long np, long long E, long long n_owned, const float *x, double *out_dev,
                             cudaStream_t s);
void frk32_f2d_unscale(long long n, const float *x, const double *xmax_dev, double target, double *y, cudaStream_t s);

void frk32_d2f_scaled_dev(long long n, const double *x, const double *xmax_dev, const double *target_dev, float *y,
                          cudaStream_t s);
void frk32_f2d_unscale_dev(long long n, const float *x, const double *xmax_dev, const double *target_dev, double *y,
                           cudaStream_t s);
void frk32_next_target(int nv, const double *ymax_dev, const double *qref_dev, double want, double *target_dev,
                       cudaStream_t s);

// tensor-core LU of FP32 element blocks (lu_tc.cu): supported block sizes, the factor
// (same layout and permutation as P##_lu_factor), its time-out flag (4 if set)
unsigned long long frktc_launch_count();
int frktc_lu_supported(int nd);
// l21: scratch of frktc_lu_scratch_floats(E, nd) floats (each phase's split L21 operand)
size_t frktc_lu_scratch_floats(int E, int nd);
int frktc_lu_factor(int E, int nd, float *M, int *perm, int *info, float *l21, cudaStream_t s);
int frktc_lu_error(int clear);
// half-width factors for the solves: binary16 L and column-scaled U (columns frktc_half_ld(nd)
// halves apart), per column (1/u_kk, g_k)
int frktc_half_ld(int nd);
int frktc_lu_to_half(int E, int nd, const float *M, void *H, float *dg, cudaStream_t s);
int frktc_lu_solve_half(int E, int nd, int g, const void *H, const float *dg, const int *perm, float *x,
                        cudaStream_t s);

// p-adaptation indicator and marking (padapt.cu)
unsigned long long frpa_launch_count();
int frpa_upload(const double *modal /* [6][6][6]: [p][a][i] */);
int frpa_spectral_decay(int d, int p, int E, const double *q, int var, double *eta, double *emax_dev, cudaStream_t s);
void frpa_mark(int E, const double *eta, const double *emax_dev, const int *p_in, int p_min, int p_max,
               double nu_min, double nu_max, int *p_out, cudaStream_t s);

// segmented vector kernels of the batched solver (batch_kernels.cu)
unsigned long long frkb_launch_count();
int frkb_segdots(int rows, int E, int nitems, const int4 *items, int nprob, const int *item_off, const double *w,
                 int m, const double *const *V, double *partial, double *out, int ld, cudaStream_t s);
void frkb_seg_invnorm(int nprob, const double *sq, int ld, const double *mask, double *nrm, double *inv,
                      cudaStream_t s);
void frkb_seg_scale(long long n, int E, const int *ep, const double *f, const double *x, double *y, cudaStream_t s);
void frkb_seg_multi_axpy(long long n, int E, const int *ep, int m, const double *h, int ld, const double *const *V,
                         double *w, cudaStream_t s);
void frkb_seg_update_x(long long n, int E, const int *ep, int m, const double *y, int ld, const double *const *Z,
                       double *x, cudaStream_t s);
void frkb_gather(int rows, int Ei, const double *qi, double *Q, int E, int off, cudaStream_t s);
void frkb_scatter(int rows, int Ei, const double *Q, int E, int off, double *qi, cudaStream_t s);

// FP32 element blocks by forward-mode differentiation of the residual (kernelsad.cu),
// FR_AD_K columns per residual evaluation
unsigned long long frkad_launch_count();
int frkad_upload_tables(const FrTabH *tabs);
int frkad_residual(const FrLevelAD &L, const FrPhysH &ph, const DualT *q, DualT *R, cudaStream_t s);
void frkad_init(long long n, const float *q, DualT *qd, cudaStream_t s);          // qd = (q, 0)
void frkad_seed(const FrLevelAD &L, const int *color, int col, int j0, DualT *qd, float seed, cudaStream_t s);
void frkad_block_column(const FrLevelAD &L, const int *color, int col, int j0, const DualT *Rd, double shift,
                        float *M, cudaStream_t s);

void frkad_nbr_column(const FrLevelAD &L, int nf, const int *nbr, const int *color2, int col, int j0,
                      const DualT *Rd, float *O, cudaStream_t s);
// element-local FP32 blocks (fr_ad_elem.cuh): qf, Qf are the FP32 residual workspace's
// traces and face gradients at q (a residual at q must precede the call); NT (floats,
// frkad_elem_nt_floats) and BCk (nfp E bytes) are scratch
long long frkad_elem_nt_floats(const FrLevel32 &L);
int frkad_elem_blocks(const FrLevel32 &L, const FrPhysH &h, const float *q, const float *qf, const float *Qf,
                      float *NT, signed char *BCk, double shift, float *M, cudaStream_t s);

// matrix-based Newton-Krylov smoother of the coarsest level (mbnk.cu).  Device scratch
// gm (FRMB_GM doubles): Hessenberg H[i m + k] at 0, Gram-Schmidt coefficients at
// FRMB_H, ||r|| at FRMB_BETA, y at FRMB_Y, iterations used at FRMB_KUSED, relative
// residual estimate at FRMB_REL; partial sums: FRMB_MAXBLK x (FRMB_MAXIT + 1) doubles.
#define FRMB_MAXIT 16
#define FRMB_MAXBLK 608
#define FRMB_H ((FRMB_MAXIT + 1) * FRMB_MAXIT)
#define FRMB_BETA (FRMB_H + FRMB_MAXIT + 1)
#define FRMB_Y (FRMB_BETA + 1)
#define FRMB_KUSED (FRMB_Y + FRMB_MAXIT)
#define FRMB_REL (FRMB_KUSED + 1)
#define FRMB_GM (FRMB_REL + 1)
unsigned long long frmb_launch_count();
void frmb_nbr_column(int E, int nd, int nf, const int *nbr, const int *color2, int col, int j, const double *q,
                     const double *R0, const double *Rp, double epsrel, double *O, cudaStream_t s);
void frmb_bsr_mv(int E, int nd, int nf, const int *nbr, const double *Md, const double *O, const double *x, double *y,
                 cudaStream_t s);
void frmb_bsr_mv(int E, int nd, int nf, const int *nbr, const float *Md, const float *O, const float *x, float *y,
                 cudaStream_t s);
void frmb_start(long long N, const double *r, double *V, double *partial, double *gm, cudaStream_t s);
void frmb_start(long long N, const float *r, float *V, double *partial, double *gm, cudaStream_t s);
void frmb_arnoldi(long long N, int m, int k, double *V, double *w, double *partial, double *gm, cudaStream_t s);
void frmb_arnoldi(long long N, int m, int k, float *V, float *w, double *partial, double *gm, cudaStream_t s);
void frmb_small_solve(int m, double tol, double *gm, cudaStream_t s);
void frmb_combine(long long N, int m, const double *V, const double *gm, double *u, cudaStream_t s);
void frmb_combine(long long N, int m, const float *V, const double *gm, float *u, cudaStream_t s);

// learned initial guess (mlp.cu)
struct fr_mlp;
unsigned long long frkmlp_launch_count();
void frkmlp_features(int E, int nv, int Np, int K0, const double *qn, const double *q1, const double *q2,
                     const double *Rn, double dt, const double *invJ, double c, const double *s_dev,
                     const double *sig_dev, const double *qinf_dev, unsigned short *X, cudaStream_t st);
void frkmlp_extrap(long long n, const double *qn, const double *q1, const double *q2, double c, double *qex,
                   cudaStream_t st);
void frkmlp_targets(int E, int nv, int Np, const double *qs, const double *qex, const double *s_dev, float *T,
                    cudaStream_t st);
void frkmlp_guess(int E, int nv, int Np, const double *qex, const double *s_dev, const float *Y, double *g,
                  cudaStream_t st);
int frkmlp_forward(fr_mlp *M, int B, const unsigned short *X, float *Y, cudaStream_t s);
int frkmlp_dims(const fr_mlp *M, int *in, int *hid, int *out);
int frkmlp_var_stats(int nv, long long per, const double *a, const double *b, const double *qinf_dev, double *part,
                     double *out_dev, cudaStream_t s);
long long frkmlp_state_floats(const fr_mlp *M);
int frkmlp_state_save(const fr_mlp *M, int *dims4, float *buf);
int frkmlp_state_load(fr_mlp *M, const int *dims4, const float *buf);
