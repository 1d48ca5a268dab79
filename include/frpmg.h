/*
 * frpmg — GB300 (sm_103a) JFNK-pMG hot path for flux-reconstruction Navier-Stokes.
 *
 * C ABI.  Every array argument is a plain pointer; the comment of each call says whether
 * it is a host or a device pointer.  Device pointers are owned by the caller (the
 * library never frees them); the library owns the workspaces it allocates in fr_create
 * and pmg_setup and frees them in fr_destroy.  Work is enqueued on the caller's CUDA
 * stream (`stream` is a cudaStream_t passed as void*, NULL = legacy default stream);
 * calls that return scalars to the host (gmres_solve, esdirk_step, row_step,
 * ptc_steady) synchronise that stream.  A context is not thread safe: one host thread
 * at a time per context.
 *
 * Errors: every call returns an int status (FR_OK = 0, negative = error) and leaves a
 * message retrievable with fr_last_error() (thread local).  Invalid arguments are
 * rejected before any work is enqueued.  A CUDA error is reported as FR_ERR_CUDA and
 * leaves the context usable only for fr_destroy.
 *
 * Layouts.  d = dimension (2 or 3), nv = d + 2 conservative variables
 * (rho, rho u_1..rho u_d, E), level l has degree p_l, n = p_l + 1 Gauss-Legendre
 * points per direction, Np = n^d solution points; a state on level l is a
 * double array q[v][i][e] of nv * Np * E values, element index fastest, solution
 * point i = i0 + n (i1 + n i2).  An element block is nd x nd with nd = nv * Np and
 * degree-of-freedom index r = v * Np + i; blocks are stored column-major per element:
 * M[(e * nd + j) * nd + r] holds entry (row r, column j).
 *
 * Arithmetic.  The FP64 residual, Jacobian-vector product, element blocks, block LU,
 * block solves, transfers and preconditioner cycle evaluate every sum of products as an
 * fma chain in a fixed order with no other contraction, so they are reproducible bit
 * for bit run to run.  GMRES inner products (the outer FGMRES and the matrix-based
 * coarse smoother's) use fixed-order two-level reductions, so they too repeat bit for bit.
 */
#ifndef FRPMG_H
#define FRPMG_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
    FR_OK = 0,
    FR_ERR_INVALID_ARG = -1,
    FR_ERR_CUDA = -2,
    FR_ERR_OOM = -3,
    FR_ERR_NOT_CONVERGED = -4,
    FR_ERR_NONFINITE = -5,
    FR_ERR_BREAKDOWN = -6,
    FR_ERR_UNIMPLEMENTED = -7,
    FR_ERR_NOT_READY = -8
};

typedef struct fr_ctx fr_ctx;

/* Mesh (all host pointers, copied during fr_create).
 *   gnodes  [nelem][(qg+1)^dim][dim] geometry nodes on the Lobatto points {-1,(0),1} of
 *           degree qg (1 or 2), node a = a0 + (qg+1)(a1 + (qg+1) a2)
 *   faces   [nfaces][6] rows (eL, fL, eR, fR, orient, bc); face f = 2*dir + side, side 0
 *           at xi_dir = -1; eR = -1 marks a boundary face with bc 1 = far field (ghost =
 *           free stream) or 2 = no-slip adiabatic wall; orient (interior faces): 2-D bit 0
 *           reverses the tangential index of the R side; 3-D bit 2 swaps the two
 *           tangential indices, then bit 0 / bit 1 reverse the first / second.
 *   plevels [nlevels] polynomial degree per p-level, finest first (p in 1..4 for 2-D,
 *           1..3 for 3-D).  Geometry of level p has degree min(qg, p).
 *   nelem   1 .. 2,097,120 (= 32 x 65535) elements per context. */
typedef struct {
    int dim, nelem, qg;
    const double *gnodes;
    int nfaces;
    const int *faces;
    int nlevels;
    const int *plevels;
} fr_mesh_desc;

/* gamma, Prandtl number, dynamic viscosity (1/Re in the dimensionless set-up of Sec. 2.2),
 * BR2 penalty, free-stream conservative state (nv values) used by far-field faces, and the
 * inviscid common flux: 0 Rusanov (local Lax-Friedrichs), 1 Roe (the original Roe solver
 * the paper uses in Sec. 4.2: |A| of the Roe-averaged state, no entropy fix), 2 Roe with
 * the Weiss-Smith low-Mach preconditioning of its dissipation (Sec. 4.1, the steady
 * low-Mach case): Gamma |Gamma^{-1} A_n| dQ in the primitive variables (p, u, T), Gamma =
 * dW/dQ with drho/dp replaced by 1/Ur^2 - rho_T/(rho C_p), reference velocity
 * Ur = min(c, max(|u|, ws_umin)) at the Roe-averaged state (ws_umin > 0, used with flux 2
 * only).  Any other flux value is FR_ERR_INVALID_ARG. */
typedef struct {
    double gamma, prandtl, mu, eta;
    double qinf[5];
    int flux;
    double ws_umin;
} fr_physics;

/* Create a context: operator tables, geometric factors of every level, connectivity and
 * workspaces on the current CUDA device.  *out receives the context (NULL on error). */
int fr_create(fr_ctx **out, const fr_mesh_desc *mesh, const fr_physics *phys);
int fr_destroy(fr_ctx *ctx);
const char *fr_last_error(void);
/* number of CUDA kernels this library has launched in the process so far (host counter) */
unsigned long long fr_kernel_launches(void);
/* sizes of level l (host out-pointers, any may be NULL): degree, Np, nv*Np*E */
int fr_level_info(const fr_ctx *ctx, int level, int *p, int *np, long long *ndof);
/* number of element colours used to assemble the element blocks (host int*) */
int fr_num_colors(const fr_ctx *ctx, int *ncolors);

/* Sec. 2.1, Eq. (1): R(q) = -div f(q, grad q) on level `level` (flux reconstruction with
 * Gauss-Legendre points and DG correction functions, Rusanov inviscid + BR2 viscous
 * common fluxes), so that dq/dt = R.  q, R: device, [nv][Np][E]; q and R must not alias. */
int fr_residual(fr_ctx *ctx, int level, const double *q, double *R, void *stream);

/* The same residual as fr_residual (same kernels, same result bit for bit), for callers
 * that cannot allocate device memory when they call it: code under CUDA stream capture
 * in the global capture mode, where cudaMalloc is refused; hosts whose device memory is
 * owned by another allocator with a fixed budget; real-time loops that must not pay for,
 * or risk the failure of, an allocation.  The paper has no counterpart: this is a
 * property of the library, not of the method.  The stage scratch (flux-point traces,
 * gradients, common fluxes) comes from one file-scope device array of 16 MiB
 * (2 Mi doubles) that every GPU loading the library holds until the process exits; no
 * cudaMalloc, cudaFree or allocating routine is called.  A level whose scratch needs
 * more than the array (4 nv Nfp E + 2 d nv Np E + d nv Nfp E doubles, each part rounded
 * up to 32) is rejected with FR_ERR_INVALID_ARG.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress), so make it before any stream
 * capture.  Every scratch value is written before it is read within a call; all calls
 * share the array, so calls whose GPU work overlaps (other streams, contexts or host
 * threads) race on it.  q, R: device [nv][Np][E], not aliased. */
int fr_residual_noalloc(fr_ctx *ctx, int level, const double *q, double *R, void *stream);

/* Eq. (8): Av = shift v - (R(q + eps v) - Rq) / eps on the finest level; Rq must be R(q).
 * q, Rq, v, Av: device [nv][Np][E]; Av must not alias the inputs. */
int fr_jvp(fr_ctx *ctx, const double *q, const double *Rq, const double *v, double eps,
           double shift, double *Av, void *stream);

/* Sec. 2.2, Eq. (9) and Sec. 3.2 smoother: element-diagonal blocks of the shifted
 * Jacobian M_e = shift I - dR_e/dq_e at q (every other element fixed), column j by the
 * forward difference with step 1e-7 max(1, |q_j|).  q: device level state; M: device,
 * E * nd * nd doubles, column-major per element (see Layouts). */
int fr_elem_blocks(fr_ctx *ctx, int level, const double *q, double shift, double *M, void *stream);
/* The same blocks in FP32 (the mixed preconditioner's), exact derivatives of the FP32
 * residual instead of differences: q device FP32 [nv][Np][E] level state, M device FP32,
 * E nd^2 values column-major per element.  method 0: element by element, each element's
 * residual differentiated with its neighbours' face traces and face gradients frozen
 * (the neighbour's face gradient still follows the common solution through its BR2
 * lifting); method 1: whole-level forward-mode residuals over an element colouring, a few
 * columns per evaluation.  The two agree to FP32 rounding; method 0 is refused
 * (FR_ERR_INVALID_ARG) on meshes where a face joins an element to itself. */
int fr_elem_blocks_f32(fr_ctx *ctx, int level, const float *q, double shift, float *M, int method, void *stream);
/* the method (as above) that pmg_setup uses for its FP32 blocks; 0 by default (meshes with
 * a face joining an element to itself always use 1) */
int fr_set_block_method(fr_ctx *ctx, int method);

/* Sec. 3.2 matrix-based smoother: the element blocks M (as fr_elem_blocks) and the face
 * neighbour blocks O of the shifted Jacobian on a level in one pass over a distance-2
 * colouring: O[((e nf + f) nd + j) nd + r] (column-major per block, nf = 2d slots per
 * element) = -dR_e[r]/dq_n[j] for the neighbour n = nbr[f E + e], by the forward difference
 * with step 1e-7 max(1, |q_n,j|); zero where nbr is -1.  q: device level state; M, O:
 * device, E nd^2 and E nf nd^2 doubles. */
int fr_nbr_blocks(fr_ctx *ctx, int level, const double *q, double shift, double *M, double *O, void *stream);
/* face-neighbour table nbr[f E + e] (host, 2d E ints): the element across local face f of
 * element e; -1 for a boundary face, a face wrapping onto e itself (that coupling is in
 * the element block) and any face after the first reaching the same element (the first
 * slot's block holds the whole coupling). */
int fr_neighbour_table(const fr_ctx *ctx, int *nbr);
/* copy of the coarsest level's assembled operator of the last pmg_setup with
 * coarse_smoother 1: unfactored element blocks Md (E nd^2) and neighbour blocks O
 * (E 2d nd^2), layouts as fr_nbr_blocks, in the cycle's precision (FP32 values when the
 * setup was mixed, else FP64).  Md, O: device; FR_ERR_NOT_READY without such a setup. */
int fr_mbnk_operator(const fr_ctx *ctx, void *Md, void *O, void *stream);
/* iterations and relative residual estimate of the last matrix-based smoothing solve
 * (synchronises); FR_ERR_NOT_READY before the first one. */
int fr_mbnk_last(const fr_ctx *ctx, int *iters, double *relres);

/* In-place LU with partial pivoting of every block (first maximal |pivot|).  M as above,
 * receives L (unit, below the diagonal), U (above) and 1/u_kk on the diagonal; perm:
 * device int [E][nd], receives the row permutation (row i of LU is row perm[i] of the
 * input block).  Returns FR_ERR_BREAKDOWN (after the whole batch) if a zero pivot was met. */
int fr_block_factor(fr_ctx *ctx, int level, double *M, int *perm, void *stream);
/* x <- M_e^{-1} x for every element using the factors of fr_block_factor.
 * x: device [nv][Np][E], overwritten. */
int fr_block_solve(fr_ctx *ctx, int level, const double *M, const int *perm, double *x, void *stream);
/* The same factorisation of FP32 blocks (those of fr_elem_blocks_f32, which the mixed
 * preconditioner factors in pmg_setup): M device FP32, E nd^2 values column-major per
 * element, factored in place (L, U, 1/u_kk as above); perm as above.  method 0: the
 * tensor-core factorisation where the block size allows it (65 <= nd <= 384), else the
 * CUDA-core kernels; 1: the CUDA-core kernels (FP32 fma, one block per CTA); 2: the
 * tensor-core factorisation (FR_ERR_UNIMPLEMENTED outside 65..384).  The tensor-core path
 * eliminates in 32-column panels with the same pivot rule; its trailing updates
 * A22 - L21 U12 run as tcgen05 TF32 products of split operands (x = hi + lo, three
 * products), which keeps them at FP32 accuracy, so its factors differ from method 1's
 * by rounding only.  Synchronises the stream; FR_ERR_BREAKDOWN on a zero pivot;
 * FR_ERR_CUDA if a bounded wait for the tensor cores ran out. */
int fr_block_factor_f32(fr_ctx *ctx, int level, float *M, int *perm, int method, void *stream);
/* x <- M_e^{-1} x with FP32 factors of fr_block_factor_f32; x device FP32 [nv][Np][E]. */
int fr_block_solve_f32(fr_ctx *ctx, int level, const float *M, const int *perm, float *x, void *stream);
/* the FP32 factorisation pmg_setup uses for the mixed preconditioner's blocks: 0 (the
 * default) as method 0 above, 1 the CUDA-core kernels */
int fr_set_lu_method(fr_ctx *ctx, int method);
/* Factors stored at half width for the FP32 block solves (not in the paper: a storage
 * format of the mixed preconditioner, which the block solves read once per smoothing step
 * and which bound them by memory bandwidth).  From FP32 factors M (fr_block_factor_f32):
 * H device binary16 [E][nd][ldh] column-major with ldh = nd rounded up to even (column k
 * at H + (e nd + k) ldh; the pad row is 0), L below the diagonal (|l| <= 1), column k of U
 * (rows < k) divided by its largest magnitude g_k (g_k = 1 for an all-zero column), 0 on
 * the diagonal; dg device FP32 [E][nd][2] = (1/u_kk, g_k).  binary16 keeps 10
 * mantissa bits (TF32's): entries carry a relative error up to 2^-11 (below 2^-14 of the
 * column's scale, an absolute one up to 2^-25 of it). */
int fr_block_to_half(fr_ctx *ctx, int level, const float *M, void *H, float *dg, void *stream);
/* x <- M_e^{-1} x with the half-width factors (x device FP32 [nv][Np][E]); perm as from
 * fr_block_factor_f32.  FR_ERR_UNIMPLEMENTED for blocks of more than 384 rows. */
int fr_block_solve_half(fr_ctx *ctx, int level, const void *H, const float *dg, const int *perm, float *x,
                        void *stream);
/* ------------------------------------------------------------------ p-adaptation
 * Sec. 3.3: the spectral-decay smoothness indicator eta_e = ||s_p - s_{p-1}|| / ||s_p||
 * (L2 norms on the reference element) of variable var (the paper's default: 1, the
 * x-momentum) of the level state q (device FP64 [nv][Np][E]), per element into eta
 * (device, E doubles): s_p's expansion in tensor products of orthonormal Legendre
 * polynomials, s_{p-1} the modes whose largest index is below p, so eta_e^2 is the
 * energy of the others over all; 0 for s = 0.  FR_ERR_UNIMPLEMENTED beyond p = 5 (2-D)
 * or p = 4 (3-D). */
int fr_spectral_decay(fr_ctx *ctx, int level, const double *q, int var, double *eta, void *stream);
/* Sec. 3.3 marking rule: p_out[e] = p_in[e] + 1 where eta_e > nu_max max(eta) (if below
 * p_max), p_in[e] - 1 where eta_e < nu_min max(eta) (if above p_min), else p_in[e]; the
 * paper takes nu_max = 0.2, nu_min = 1e-3, p_min = 1.  eta, p_in, p_out: device, E each. */
int fr_padapt_mark(fr_ctx *ctx, const double *eta, const int *p_in, int p_min, int p_max, double nu_min,
                   double nu_max, int *p_out, void *stream);
/* Sec. 3.3 nested p-hierarchy of an element of degree p over nlevels sublevels with order
 * gap: degrees[0] = p, degrees[l] = min(max(p - gap l, nlevels - 1 - l), max(degrees[l-1]
 * - 1, 0)) (host; this rule reproduces the paper's eight examples, e.g. gap 2: p{4-2-0},
 * p{3-1-0}, p{2-1-0}, p{1-0-0}). */
int fr_nested_hierarchy(int p_elem, int gap, int nlevels, int *degrees);

/* 1: the FP64 preconditioner cycle (pmg_setup precision 0, as used by FGMRES) is driven
 * like the FP32 one: X scaled so that the correction is about 1e-2 of the state per
 * variable, the result scaled back (a nonlinear preconditioner; FGMRES allows it).  For
 * states whose magnitude dwarfs a unit-norm Krylov vector (the pressure ~ 1/(gamma Ma^2)
 * at low Mach) an unscaled correction is lost in the rounding of R(q + Y) - R(q).  0 (the
 * default): unscaled, the oracle's cycle.  The nonlinear pMG solvers are never scaled.
 * Takes effect at the next pmg_setup. */
int fr_set_cycle_scaling(fr_ctx *ctx, int on);
/* ptc_steady with the FP32 preconditioner: 1 (the default) switches to the FP64 cycle
 * when FGMRES stalls (all its iterations used and the residual fell by less than half, or
 * five pseudo steps in a row each gained less than 10%); 0 keeps the FP32 cycle. */
int fr_set_precision_fallback(fr_ctx *ctx, int on);
/* 1: pmg_setup also stores the mixed preconditioner's FP32 factors at half width and the
 * smoother's block solves read those (half the bytes per solve; levels whose blocks have
 * more than 384 rows keep FP32 factors); 0 (the default): FP32 factors.  Takes effect at
 * the next pmg_setup. */
int fr_set_lu_storage(fr_ctx *ctx, int half);

/* Eqs. (17)-(18): L2 restriction level -> level+1 and prolongation level+1 -> level,
 * tensor-product 1-D operators applied along direction 0, 1, 2 in turn.  Device arrays. */
int fr_restrict(fr_ctx *ctx, int level, const double *x_fine, double *x_coarse, void *stream);
int fr_prolong(fr_ctx *ctx, int level, const double *x_coarse, double *x_fine, void *stream);

/* Nonlinear pMG preconditioner, Sec. 3.2, Eqs. (22)-(26) with the V-cycle of Sec. 3.1,
 * Eqs. (11)-(16).  c = 1/dtau + 1/(a_ii dt) (ESDIRK) or 1/(gamma dt) (ROW);
 * inv_dtau_star = 1/dtau* of the preconditioner's own pseudo step (0 = infinite).
 * nsmooth[l] = smoothing steps on level l (pre and post on levels with a coarser one).
 * pmg_setup evaluates and factors the element blocks (1/dtau* + c) I - J_ee on every level
 * at q_ref restricted level by level (device state), and keeps them until the next
 * pmg_setup or fr_destroy.
 * precision 0: everything in FP64 (reproducible, see Arithmetic).  precision 1 (mixed):
 * the cycle, its residuals on every level, the element blocks and their LU factors and
 * solves run in FP32, the blocks' columns by forward-mode differentiation of the FP32
 * residual (exact derivatives, no finite-difference noise); X is scaled on the
 * device so that max_v ||Y_v||_inf / max|q_ref,v| ~ 1e-2 inside the cycle (keeping
 * R(qh) - R(q) clear of FP32 rounding; the scale starts from the gain 1/((c + 1/dtau*)
 * min_v max|q_ref,v|) and follows the gain measured by the previous call, and a call
 * that lands more than 30x off repeats its cycle once at the measured gain), and Y is
 * scaled back and returned in FP64.  Each mixed call reads nv maxima back to the host
 * (one stream synchronisation).
 * coarse_smoother 0: element-Jacobi smoothing on every level.  1: the matrix-based
 * Newton-Krylov (MBNK) smoother of Sec. 3.2 on the coarsest level: its linearised operator
 * (1/dtau* + c) I - dR/dq is assembled at q_ref as the element blocks plus one block per
 * face neighbour (finite differences in FP64, forward-mode derivatives in FP32, over a
 * distance-2 colouring), and each smoothing step there solves it by GMRES (classical
 * Gram-Schmidt with one re-orthogonalisation) from zero, right-preconditioned by the
 * factored element blocks, stopping at the first iteration whose residual estimate is
 * <= mbnk_tol ||rhs|| or after mbnk_maxit (1..16) iterations; the paper uses 5 and 1e-1,
 * with per-block ILU0 where this uses the element blocks.  The whole GMRES runs on the
 * device with no host synchronisation (iterations after the stopping one are computed
 * and discarded), so the cycle stays capturable.  Extra device memory on the coarsest
 * level: E (2d + 1) nd^2 + (mbnk_maxit + 3) N values of the cycle's precision. */
typedef struct {
    int nlevels;
    int nsmooth[4];
    double c;
    double inv_dtau_star;
    int precision;
    int coarse_smoother, mbnk_maxit;
    double mbnk_tol;
} fr_pmg_opts;
int pmg_setup(fr_ctx *ctx, const double *q_ref, const fr_pmg_opts *opts, void *stream);
/* Y ~ A^{-1} X: one V-cycle of pseudo-time marching of
 * 0 = X + R(qh) - c qh - R(q) + c q from qh = q; Y = qh - q.  q, Rq (= R(q)), X, Y: device
 * finest-level vectors; Y must not alias the inputs. */
int pmg_precondition(fr_ctx *ctx, const double *q, const double *Rq, const double *X, double *Y,
                     void *stream);

/* Restarted right-preconditioned flexible GMRES (CGS2 orthogonalisation) for
 * A x = b with A v = shift v - (R(q + eps v) - R(q))/eps (Eq. 8) and, if use_pmg, the
 * preconditioner of the last pmg_setup.  The FD product is applied to unit-norm
 * directions only.  Stops when the Arnoldi least-squares residual estimate is
 * <= tol ||b|| or after maxit iterations (stats->relres is that estimate / ||b||); the
 * true residual is recomputed at each restart to start the next cycle.
 * q, Rq, b, x: device; stats: host (may be NULL). */
typedef struct {
    int kdim, maxit, use_pmg;
    double tol, eps, shift;
} fr_gmres_opts;
typedef struct {
    int iters, restarts;
    double relres;
} fr_gmres_stats;
int gmres_solve(fr_ctx *ctx, const double *q, const double *Rq, const double *b, double *x,
                const fr_gmres_opts *opts, fr_gmres_stats *stats, void *stream);

/* Solver options for the time steppers (host struct). */
typedef struct {
    int kdim, maxit_gmres, max_ptc, nlevels, nsmooth[4], use_pmg;
    double tol_gmres, tol_newton, eps, dtau, inv_dtau_star;
    int precision;   /* preconditioner precision, as fr_pmg_opts.precision */
    /* Newton initial guess of the ESDIRK stages (esdirk_step only; the paper uses q^n):
     * 0: q^n; 1: the better (smaller FP64 stage residual RMS(a_ii dt F)) of q^n and the
     * quadratic extrapolation in time of the last three converged steps to t_n + c_i dt;
     * 2: as 1 plus the extrapolation corrected by the attached network (fr_set_mlp): the
     * network's correction d enters scaled by the beta in [-1, 2] that minimises the
     * linearised ||F(qex + beta d)|| (one extra residual), or unscaled if that is better.
     * Only converged steps join the history, so a step that returns FR_ERR_NOT_CONVERGED
     * leaves it as it was; a step whose dt differs from the history's spacing restarts
     * the history from the current state (no extrapolation until three states of that
     * spacing exist).
     * train_iters > 0: after the step, the converged stages join a training ring (the
     * last six steps) and the network takes train_iters Adam steps of train_batch
     * samples at learning rate lr. */
    int guess, train_iters, train_batch;
    double lr;
    int coarse_smoother, mbnk_maxit;   /* as fr_pmg_opts (when use_pmg) */
    double mbnk_tol;
    /* ESDIRK stage solver (esdirk_step only): 0 JFNK (each pseudo-time Newton update by
     * FGMRES, Eq. 8); 1 the pMG nonlinear solver of Sec. 3.1: each update is one V-cycle
     * of the stage's pseudo-time equation, (1/dtau + 1/(a_ii dt)) dq - (R(q + dq) - R(q))
     * = -F(q), i.e. pmg_precondition with X = -F; max_ptc bounds the cycles per stage.
     * Needs use_pmg and precision 0; row_step and the batched step refuse it. */
    int nonlinear;
} fr_solve_opts;
typedef struct {
    int n_ptc, n_gmres, converged;
    double final_res;
    double guess_rms[3];   /* mean over stages of RMS(a_ii dt F) of q^n, extrapolation, network guess */
    int guess_pick[3];     /* how many stages started from each candidate */
    double guess_beta;     /* mean step along the network's correction (guess 2) */
    double train_loss;     /* loss of the last training step (train_iters > 0) */
    int prec_switch_it;    /* ptc_steady: pseudo step after which the FP32 preconditioner
                              stalled and the FP64 one took over (-1: never) */
} fr_step_stats;

/* ESDIRK step, Eq. (2): stages solved by PTC/Newton (Eqs. 5-7) with FGMRES, the
 * preconditioner set up once per step at q^n; stage converged when
 * RMS(a_ii dt F(q_i)) <= tol_newton.  A: host [stages][stages] row-major (A[0][*] = 0),
 * b: host [stages]; q: device, q^n in, q^{n+1} out.  Returns FR_ERR_NOT_CONVERGED (with
 * q^{n+1} written) when a stage missed the tolerance within max_ptc iterations. */
typedef struct {
    int stages;
    double A[36];
    double b[6];
} fr_esdirk_tableau;
int esdirk_step(fr_ctx *ctx, const fr_esdirk_tableau *tab, double dt, double *q,
                const fr_solve_opts *opts, fr_step_stats *stats, void *stream);

/* Per-element network for the Newton initial guess (not in the paper; see fr_solve_opts.guess):
 *   h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = W3 h2 + b3,
 * bfloat16 operands and FP32 accumulation on the tensor cores, FP32 master weights and
 * Adam moments.  params (host float): W1[hidden][in], b1[hidden], W2[hidden][hidden],
 * b2[hidden], W3[out][hidden], b3[out]; the caller draws the initial values.  Features of
 * element e: (q^n - q^{n-1})/s_v, (q^{n-1} - q^{n-2})/s_v, (q^n - qinf_v)/sig_v,
 * dt R(q^n)/s_v, log J / 10, the stage abscissa c_i, zero padding (s_v, sig_v: per-variable
 * RMS of q^n - q^{n-1} and q^n - qinf over the mesh);
 * output: the stage state's correction of the extrapolation, in units of s_v. */
typedef struct fr_mlp fr_mlp;
int mlp_create(fr_mlp **out, int in_dim, int hidden, int out_dim, const float *params);
int mlp_destroy(fr_mlp *mlp);
int mlp_get_params(const fr_mlp *mlp, float *params /* host */);
/* X: device bfloat16 [B][in] (as unsigned short), Y: device float [B][out] */
int mlp_forward(fr_mlp *mlp, int B, const unsigned short *X, float *Y, void *stream);
/* one step: forward, mean-squared loss against T (device float [B][out]), backward, Adam.
 * loss (host, may be NULL) synchronises the stream; grads (device float, parameter
 * layout, may be NULL) receives the gradients before the update. */
int mlp_train_step(fr_mlp *mlp, int B, const unsigned short *X, const float *T, float lr, float *loss, float *grads,
                   void *stream);
/* network sizes the context expects (in = 4 nd + Np + 1 rounded up to 16, out = nd) */
int fr_mlp_dims(const fr_ctx *ctx, int *in_dim, int *out_dim);
int fr_set_mlp(fr_ctx *ctx, fr_mlp *mlp);
/* the network's inputs for states q^n, q^{n-1}, q^{n-2} (device, level-0 layout), R(q^n),
 * dt and stage abscissa c: X device bfloat16 [E][in]; scales (host double[10], may be
 * NULL) receives s_0..s_4 and sig_0..sig_4 (entries past nv unused). */
int fr_guess_features(fr_ctx *ctx, const double *qn, const double *q1, const double *q2, const double *Rn, double dt,
                      double c, unsigned short *X, double *scales, void *stream);
/* forget the converged-state history and the training ring (start of a new trajectory) */
int fr_reset_history(fr_ctx *ctx);

/* Rosenbrock-Wanner step in the variables of Eq. (3):
 * (I/(gamma dt) - dR/dq(q^n)) Y_i = R(q^n + sum_j a_ij Y_j) + (1/dt) sum_j c_ij Y_j,
 * q^{n+1} = q^n + sum_j m_j Y_j.  a, c: host [stages][stages] row-major strictly lower. */
typedef struct {
    int stages;
    double gamma;
    double a[36];
    double c[36];
    double m[6];
} fr_row_tableau;
int row_step(fr_ctx *ctx, const fr_row_tableau *tab, double dt, double *q, const fr_solve_opts *opts,
             fr_step_stats *stats, void *stream);

/* Steady PTC (Eq. 7 without the dt terms) with the SER pseudo-step of Eq. (10), read as
 * dtau <- min(dtau ||R^k|| / ||R^{k+1}||, dtau_max); preconditioner re-set at every
 * iteration with c = 1/dtau (inv_dtau_star < 0 selects 1/dtau* = c).  Stops at
 * ||R|| <= tol_rel ||R_0||.  hist: host [max_it+1] residual norms (may be NULL).
 * precision = 1: the FP32 cycle until a pseudo step where FGMRES used all maxit_gmres
 * iterations and ||R|| fell by less than half, or the fifth pseudo step in a row that cut
 * ||R|| by less than 10%; from then on the FP64 cycle (stats->prec_switch_it records the
 * step). */
int ptc_steady(fr_ctx *ctx, double *q, double dtau_init, double dtau_max, double tol_rel, int max_it,
               const fr_solve_opts *opts, fr_step_stats *stats, double *hist, void *stream);

/* Checkpoint of a time-stepping run's library-side state (the paper resumes runs from
 * saved solutions, Sec. 4): the learned guess's three converged states and training ring,
 * and (mlp != NULL) the network's weights and Adam state.  The caller keeps q, t and the
 * step count beside it; launch shapes have their own file (fr_autotune_save).  Loading
 * into a context of the same mesh and levels, with a network of the same sizes, and
 * stepping on reproduces the uninterrupted run bit for bit.  buf: host memory of at least
 * fr_checkpoint_size bytes; save and load synchronise the device. */
int fr_checkpoint_size(const fr_ctx *ctx, const fr_mlp *mlp, long long *bytes);
int fr_checkpoint_save(const fr_ctx *ctx, const fr_mlp *mlp, void *buf, long long bytes);
int fr_checkpoint_load(fr_ctx *ctx, fr_mlp *mlp, const void *buf, long long bytes);

/* The pMG nonlinear solver for steady problems (Sec. 3.1, Eqs. 11-16), the paper's
 * comparison method: each iteration is one nonlinear V-cycle of pseudo-time marching on
 * R(q) = 0 from the current state — the preconditioner's cycle with X = R(q), which turns
 * its equation into the backward-Euler pseudo step R(qh) - c (qh - q) = 0, c = 1/dtau —
 * then q <- qh; element blocks at every iteration's q; dtau by the SER rule of ptc_steady.
 * Uses opts->nlevels, nsmooth, inv_dtau_star (< 0: = c); FP64 only (precision 0).
 * q: device, updated in place; hist: host [max_it+1] residual norms (may be NULL). */
int pmg_solve_steady(fr_ctx *ctx, double *q, double dtau_init, double dtau_max, double tol_rel, int max_it,
                     const fr_solve_opts *opts, fr_step_stats *stats, double *hist, void *stream);

/* ---------------------------------------------------------------- autotuner
 * Launch shapes (not in the paper; no result bit depends on them): the CTA size (elements
 * per CTA tile, 64/128/256) of each of the 7 kernels of the residual, per level and
 * precision, and the columns in flight G (2/4/8) of the block solve.  fr_autotune times
 * the candidates with CUDA events on the context's own levels (reps launches each after
 * a warm-up; a coordinate-descent pass over the residual kernels, then the solve variant
 * on the level's factored blocks if pmg_setup has run in that precision) and keeps the
 * fastest.  Solve variants: the register kernel with G = 2, 4 or 8 columns in flight, or
 * (G = 1) the kernel that streams the factor through shared memory with bulk async
 * copies (rows of a column that the pass needs only; nd * sizeof(scalar) % 16 == 0).  flags:
 * bit 0 FP64 levels, bit 1 FP32 levels, bit 2 re-tune even if cached.  Results are kept
 * in a process-wide cache keyed by (device name, d, p, precision, floor(log2 E)), safe
 * to use from several host threads; new contexts pick cached shapes up.  report (host, may be NULL): one line per level.
 * Uses the legacy default stream and synchronises the device. */
int fr_autotune(fr_ctx *ctx, int flags, int reps, char *report, int report_len);
/* tiles[9]: 8 CTA-size slots (the residual's 7 kernels, slot 5 unused; 0 = default 128;
 * else a multiple of 32 in 32..256) and G
 * (0 = default, 1 = bulk-copy kernel, 2, 4 or 8) of level `level` in precision 0 (FP64)
 * or 1 (FP32) */
int fr_get_tiles(const fr_ctx *ctx, int level, int precision, int *tiles);
int fr_set_tiles(fr_ctx *ctx, int level, int precision, const int *tiles);
/* the cache as a text file: one line "device d p precision log2E tile0..tile7 G" per key
 * (load skips malformed lines and out-of-range values) */
int fr_autotune_save(const char *path);
int fr_autotune_load(const char *path);
/* bounded device-side waits that ran out since the last clear (bit 0: block-solve stage
 * barriers); such a kernel records the failure and returns instead of hanging.  Bit 1:
 * the bulk-copy block solve also gave up waiting for its own copies in flight, which may
 * then land in shared memory after its CTA exited: treat the device as unusable.  Bit 2:
 * a trailing update of the tensor-core LU gave up waiting for its operand copy or its
 * products (its block's factors are then wrong); if it also gave up waiting for the copy
 * to drain, bit 1 is set as well. */
int fr_kernel_timeouts(int clear);
/* runs the time-out path of those waits on purpose (a barrier that nothing completes,
 * 4096 polls) so that callers can check that it reports through fr_kernel_timeouts and
 * leaves the context usable; synchronises the device */
int fr_selftest_wait_timeout(void);

/* ------------------------------------------------------------------ element partition
 * One process per GPU, each solving its part of one mesh (the paper's runs split the mesh
 * over four MPI processes, Sec. 4; the interface is this library's).  A process's context
 * is created on its local mesh: its owned elements first (0 .. n_owned-1), then ghost
 * copies of the other processes' elements that share a face with an owned element, in
 * the order the communicator delivers them.  A ghost's faces towards elements that are
 * neither owned nor ghost enter as far-field faces: they change only the ghost's own
 * residual, which nothing reads.  With a communicator set on the context:
 *  - before every residual evaluation of a state whose ghosts may be stale (fr_residual,
 *    the Jacobian-vector product, every pMG level, the steppers), the library packs the
 *    owned elements send_idx[0 .. nsend) of that level vector into send_buf (element by
 *    element: nv Np_level values of the level's precision each, concatenated in send_idx
 *    order) and calls halo(user, level, precision, elem_bytes, stream) with the stream
 *    synchronised; on return recv_buf must hold the E - n_owned ghost elements' values
 *    (ghost order, elem_bytes each), which the library copies into the ghosts.  A finite
 *    difference column of the element blocks exchanges nothing (each process perturbs
 *    its own elements only);
 *  - every inner product and norm runs over the owned elements and is summed over the
 *    processes by allreduce(user, buf, n, 0) on a host buffer; the FP32 cycle's maxima
 *    by allreduce(.., 1) (max); RMS norms divide by the global unknown count
 *    (n_owned_total elements); fr_set_comm itself communicates nothing;
 *  - so each process's owned values follow the single-process computation step for step;
 *    results differ from it only in the summation order of inner products.
 * fr_residual and fr_jvp overwrite the ghost entries of their state inputs with the
 * owners' values.  A non-zero return from a callback fails the call with FR_ERR_CUDA.
 * Refused while a communicator is set: the network guess and its training (guess 2,
 * train_iters > 0), the matrix-based coarse smoother, fr_residual_noalloc.
 * send_buf and recv_buf: device memory of the caller, at least nsend (and E - n_owned)
 * elements of nv Np_0 doubles. */
typedef struct {
    int n_owned;
    long long n_owned_total;  /* owned elements over all processes (RMS norms divide by it) */
    int nsend;
    const int *send_idx;      /* host, nsend owned element indices (copied by the call) */
    void *send_buf, *recv_buf;
    int (*halo)(void *user, int level, int precision, long long elem_bytes, void *stream);
    int (*allreduce)(void *user, double *buf, int n, int op);
    void *user;
} fr_comm;
/* comm NULL: single process again */
int fr_set_comm(fr_ctx *ctx, const fr_comm *comm);

/* ------------------------------------------------------------------ batches
 * Many independent problems advanced together (not in the paper: a throughput mode).
 * Problems sharing the dimension, geometry degree and p-levels are solved on one merged
 * mesh per group, so each kernel of the step runs once per group; Newton and FGMRES stay
 * per problem (segmented norms and inner products, own Hessenberg matrix, stopping test
 * and restarts; a converged problem is masked out).  Every problem of a batch takes the
 * same dt, solver options and physics (an ensemble advancing in lockstep); a group with
 * fewer p-levels than opts->nlevels uses all it has.  The Arnoldi
 * step of a group runs as a CUDA graph captured once per Krylov index and operator
 * parameters (fr_batch_set_graphs(b, 0) launches the kernels one by one instead).  With
 * precision 1 the FP32 cycle keeps its scale on the device: each call's measured gain
 * sets the next call's input scale (no repeat of a call).  The work runs on the batch's
 * own stream, ordered after and before the caller's stream. */
typedef struct fr_batch fr_batch;
/* meshes: host array of nprob descriptions (copied); physics shared by all problems */
int fr_batch_create(fr_batch **out, int nprob, const fr_mesh_desc *meshes, const fr_physics *phys);
int fr_batch_destroy(fr_batch *batch);
/* host outs (any may be NULL): number of groups, group of each problem [nprob], first
 * element of each problem in its group's merged mesh [nprob] */
int fr_batch_info(const fr_batch *batch, int *ngroups, int *group_of, int *elem_offset);
int fr_batch_set_graphs(fr_batch *batch, int on);
/* R(q_k) for every problem: q, R host arrays of nprob device pointers ([nv][Np][E_k] each) */
int fr_batch_residual(fr_batch *batch, double *const *q, double *const *R, void *stream);
/* one ESDIRK step (as esdirk_step, guess 0, kdim <= 62, element-Jacobi smoothing on every
 * level: coarse_smoother 1 is FR_ERR_UNIMPLEMENTED) of every problem: q host array of
 * nprob device pointers, updated in place; stats host [nprob] (may be NULL).  Returns
 * FR_ERR_NOT_CONVERGED if any problem missed the Newton tolerance (all states are still
 * advanced). */
int fr_batch_esdirk_step(fr_batch *batch, const fr_esdirk_tableau *tab, double dt, double *const *q,
                         const fr_solve_opts *opts, fr_step_stats *stats, void *stream);
/* fr_autotune on every group of the batch (drops the captured graphs) */
int fr_batch_autotune(fr_batch *batch, int flags, int reps, char *report, int report_len);

#ifdef __cplusplus
}
#endif
#endif
