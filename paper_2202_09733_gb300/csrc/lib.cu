// frpmg C ABI: context set-up and the host-side orchestration of the JFNK-pMG hot path
// (pMG V-cycle in FP64 or FP32, FGMRES with CGS2, ESDIRK/PTC, ROW, steady PTC/SER).
// Every arithmetic step on solution vectors runs in the kernels of kernels64.cu and
// kernels32.cu; the host only keeps the Krylov scalars (Hessenberg matrix, Givens
// rotations) and the iteration logic.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <nvtx3/nvToolsExt.h>
#include <vector>
#include "../../include/frpmg.h"
#include "fr_lib.h"
#include "host_tables.h"

static thread_local char g_err[1024] = "";

static int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t _e = (call);                                                              \
        if (_e != cudaSuccess)                                                                \
            return fail(FR_ERR_CUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(_e)); \
    } while (0)

#define CKLAUNCH()                                                                            \
    do {                                                                                      \
        cudaError_t _e = cudaGetLastError();                                                  \
        if (_e != cudaSuccess)                                                                \
            return fail(FR_ERR_CUDA, "%s:%d kernel launch: %s", __FILE__, __LINE__, cudaGetErrorString(_e)); \
    } while (0)

// NVTX range for a profiler's timeline (a no-op unless a tool is attached): time steps,
// stages, pseudo-time updates, FGMRES solves, pMG set-ups and V-cycle levels
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
static const char *const kVcycleRange[FRL_MAXLEV] = {"vcycle level 0", "vcycle level 1", "vcycle level 2",
                                                     "vcycle level 3"};

#define TRY(x)                       \
    do {                             \
        int _r = (x);                \
        if (_r != FR_OK) return _r;  \
    } while (0)

// options of the coarsest level's smoother (fr_pmg_opts / fr_solve_opts)
static int check_coarse_opts(int coarse, int maxit, double tol) {
    if (coarse != 0 && coarse != 1)
        return fail(FR_ERR_INVALID_ARG, "coarse_smoother must be 0 (element-Jacobi) or 1 (matrix-based)");
    if (coarse == 1 && (maxit < 1 || maxit > FRMB_MAXIT))
        return fail(FR_ERR_INVALID_ARG, "mbnk_maxit outside 1..%d", FRMB_MAXIT);
    if (coarse == 1 && !(tol >= 0.0)) return fail(FR_ERR_INVALID_ARG, "mbnk_tol must be >= 0");
    return FR_OK;
}
static void coarse_opts_copy(const fr_solve_opts *o, fr_pmg_opts *po) {
    po->coarse_smoother = o->coarse_smoother;
    po->mbnk_maxit = o->mbnk_maxit;
    po->mbnk_tol = o->mbnk_tol;
}

template <typename T>
struct PmgBuf {
    T *M[FRL_MAXLEV];
    int *perm[FRL_MAXLEV];
    size_t M_cap[FRL_MAXLEV];
    T *b[FRL_MAXLEV], *Rb[FRL_MAXLEV], *d[FRL_MAXLEV], *qh[FRL_MAXLEV], *Rqh[FRL_MAXLEV], *rhs[FRL_MAXLEV],
        *C[FRL_MAXLEV];
    T *blk_R0, *blk_Rp, *blk_qp;  // element-block assembly temporaries (finest-level size)
    // matrix-based smoother of the coarsest level: unfactored diagonal blocks, neighbour
    // blocks, Krylov basis (FRMB_MAXIT + 1 vectors), two work vectors; capacities in T
    T *Md, *O, *V, *mz, *mw;
    size_t Md_cap, O_cap, V_cap, w_cap;
    // FP32 factors also stored at half width for the solves (binary16 entries, per-column
    // (1/u_kk, g_k) in FP32) when the context asks for it; half_ok[l]: current for M[l]
    void *H[FRL_MAXLEV];
    float *dg[FRL_MAXLEV];
    size_t H_cap[FRL_MAXLEV];
    int half_ok[FRL_MAXLEV];
};

struct fr_ctx {
    int d, nv, E, qg, nlev;
    FrPhysH ph;
    double eta;
    FrLevel L[FRL_MAXLEV];
    FrLevel32 L32[FRL_MAXLEV];    // FP32 copies of the levels (mixed preconditioner)
    FrLevelAD LA[FRL_MAXLEV];     // forward-mode (FP32 dual) residual workspace for the FP32 blocks
    int have32, haveAD;
    DualT *qd, *Rd;
    int ncolor;
    int *color;
    int self_face;                // a face joins an element to itself (periodic, one element wide)
    int ad_method;                // FP32 blocks: 0 element by element, 1 whole-level colours
    int lu_method;                // FP32 LU: 0 tensor cores where the block size allows, 1 CUDA cores
    int lu_half;                  // FP32 block solves from half-width factors (pmg_setup converts)
    int scale64;                  // the FP64 cycle driven with a scaled X, as the FP32 cycle is
    int no_fallback;              // ptc_steady: keep the FP32 cycle when it stalls
    double *x64s;                 // the scaled FP64 cycle's right-hand side
    double *pa_max;               // max of the spectral-decay indicators (device)
    float *lu_scr;                // tensor-core LU: each phase's split L21 operand
    size_t lu_scr_cap;
    float *ad_nt;                 // element-local FP32 blocks: the other sides' frozen face data
    signed char *ad_bck;          //   and the boundary code of every element face point
    int ncolor2;
    int *color2;                  // distance-2 colouring (assembly of the neighbour blocks)
    int *nbr;                     // face neighbours nbr[f E + e], -1 none
    int mbnk, mbnk_maxit;         // matrix-based smoother on the coarsest level (last pmg_setup)
    double mbnk_tol;
    double *mb_partial, *mb_gm;
    int *info;
    std::vector<void *> allocs;
    double *jv_qp, *jv_Rp;
    double *dots;                 // device scratch for inner products (64)
    // pMG
    int pmg_ready, pmg_nlev, pmg_prec, nsmooth[FRL_MAXLEV];
    double pmg_c, pmg_ids, pmg_qref[5];
    double pmg_gain;   // mixed cycle: last measured max_v ||Y_v||_inf / qref_v per ||X||_inf
    const double *q32_of;   // q whose FP32 copy and residual q32/Rq32 hold (NULL: none); set
                            // only while an FGMRES solve keeps q fixed
    double *ymax;
    PmgBuf<double> p64;
    PmgBuf<float> p32;
    float *x32, *q32, *Rq32, *y32;
    double *xmax;
    // GMRES
    std::vector<double *> V, Z;
    double *gw, *gr, *gtmp;
    // steppers
    std::vector<double *> stv;
    // initial guess: last three converged states, extrapolation, learned correction
    double *hist[3];              // q^{n-2}, q^{n-1}, q^n
    int nhist;
    double hist_dt;               // step between the history states (0: not yet spaced)
    fr_mlp *mlp;
    int K0, O, mlp_steps;
    double *qex, *qcand, *Rtmp, *Ftmp, *Fex, *sdev, *qinf_dev, *vpart;
    unsigned short *Xf, *ringX;
    float *Yf, *Tf, *ringT;
    int ring_cap, ring_n, ring_head, train_cursor;
    // element partition (fr_set_comm): ghosts are elements n_owned .. E-1
    int has_comm;
    fr_comm comm;
    int *send_idx_dev;
    double ndof_rms;              // unknowns the RMS norms divide by (over all processes)
    double *partial;              // this context's reduction partials
};

static int dalloc(fr_ctx *C, void **p, size_t bytes) {
    if (bytes == 0) bytes = 8;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(FR_ERR_OOM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    }
    C->allocs.push_back(*p);
    return FR_OK;
}
template <typename T>
static int dalloc_t(fr_ctx *C, T **p, size_t count) {
    return dalloc(C, (void **)p, sizeof(T) * count);
}
static void dfree(fr_ctx *C, void *p) {
    if (!p) return;
    for (size_t i = 0; i < C->allocs.size(); ++i)
        if (C->allocs[i] == p) { C->allocs.erase(C->allocs.begin() + i); break; }
    cudaFree(p);
}

static cudaStream_t S_(void *s) { return (cudaStream_t)s; }
static void apply_cached_tiles(fr_ctx *C, int prec);

extern "C" const char *fr_last_error(void) { return g_err; }

static std::atomic<unsigned long long> g_graph_kernels{0};    // kernels run by CUDA graph replays
static std::atomic<unsigned long long> g_capture_kernels{0};  // launch-counter increments made while capturing graphs

extern "C" unsigned long long fr_kernel_launches(void) {
    return frk64_launch_count() + frk32_launch_count() + frkad_launch_count() + frkmlp_launch_count() +
           frkb_launch_count() + frmb_launch_count() + frktc_launch_count() + frpa_launch_count() - g_capture_kernels + g_graph_kernels;
}

// ---------------------------------------------------------------- context set-up
static int upload_tables() {
    static FrTabH tabs[6];
    static double gam[6][6][6][6], pi[6][6][6][6];
    memset(tabs, 0, sizeof tabs);
    memset(gam, 0, sizeof gam);
    memset(pi, 0, sizeof pi);
    for (int p = 1; p <= 5; ++p) {
        frh_tab T;
        frh_make_tables(p, p < 2 ? p : 2, &T);
        memcpy(tabs[p].D, T.D, sizeof T.D);
        memcpy(tabs[p].lm, T.lm, sizeof T.lm);
        memcpy(tabs[p].lp, T.lp, sizeof T.lp);
        memcpy(tabs[p].dlm, T.dlm, sizeof T.dlm);
        memcpy(tabs[p].dlp, T.dlp, sizeof T.dlp);
        memcpy(tabs[p].gLd, T.gLd, sizeof T.gLd);
        memcpy(tabs[p].gRd, T.gRd, sizeof T.gRd);
        for (int p1 = 1; p1 <= p; ++p1) {
            double G[FRH_MAXN][FRH_MAXN], P[FRH_MAXN][FRH_MAXN];
            frh_make_transfer(p, p1, G, P);
            memcpy(gam[p][p1], G, sizeof G);
            memcpy(pi[p][p1], P, sizeof P);
        }
    }
    static double modal[6][6][6];
    memset(modal, 0, sizeof modal);
    for (int p = 0; p <= 5; ++p) {
        double Mp[FRH_MAXN][FRH_MAXN];
        frh_modal(p, Mp);
        for (int a = 0; a <= p; ++a)
            for (int i = 0; i <= p; ++i) modal[p][a][i] = Mp[a][i];
    }
    if (frk64_upload_tables(tabs, &gam[0][0][0][0], &pi[0][0][0][0]) != 0 ||
        frk32_upload_tables(tabs, &gam[0][0][0][0], &pi[0][0][0][0]) != 0 || frkad_upload_tables(tabs) != 0 ||
        frpa_upload(&modal[0][0][0]) != 0)
        return fail(FR_ERR_CUDA, "uploading operator tables: %s", cudaGetErrorString(cudaGetLastError()));
    return FR_OK;
}

static int setup_level(fr_ctx *C, int l, int p, const fr_mesh_desc *m) {
    FrLevel &L = C->L[l];
    int d = C->d, E = C->E;
    L.d = d; L.p = p; L.n = p + 1; L.E = E; L.nv = C->nv;
    L.np = d == 2 ? L.n * L.n : L.n * L.n * L.n;
    L.nf1 = d == 2 ? L.n : L.n * L.n;
    L.nfp = 2 * d * L.nf1;
    L.nd = L.nv * L.np;
    L.ndof = (long long)L.nd * E;
    frh_tab T;
    int g = p < C->qg ? p : C->qg;
    frh_make_tables(p, g, &T);
    L.etagL = C->eta * T.gLf;
    L.etagR = C->eta * T.gRf;
    size_t nsp = (size_t)d * d * L.np * E, nfpt = (size_t)d * d * L.nfp * E;
    std::vector<double> S(nsp), G(nsp), iJ((size_t)L.np * E), J((size_t)L.np * E), Sf(nfpt), Gf(nfpt);
    frh_geometry(d, E, C->qg, m->gnodes, &T, S.data(), G.data(), iJ.data(), J.data(), Sf.data(), Gf.data());
    for (size_t i = 0; i < J.size(); ++i)
        if (!(J[i] > 0.0)) return fail(FR_ERR_INVALID_ARG, "level %d: non-positive Jacobian in element %zu", l, i % E);
    std::vector<int> pairs((size_t)4 * m->nfaces * L.nf1), bc((size_t)m->nfaces * L.nf1);
    int np_ = frh_pairs(d, L.n, E, m->nfaces, m->faces, pairs.data(), bc.data());
    if (np_ < 0) return fail(FR_ERR_INVALID_ARG, "face list does not pair every face point exactly once");
    L.npairs = np_;
    TRY(dalloc_t(C, &L.S, nsp)); TRY(dalloc_t(C, &L.G, nsp)); TRY(dalloc_t(C, &L.invJ, (size_t)L.np * E));
    TRY(dalloc_t(C, &L.Sf, nfpt)); TRY(dalloc_t(C, &L.Gf, nfpt));
    TRY(dalloc_t(C, &L.pairs, (size_t)np_)); TRY(dalloc_t(C, &L.bc, (size_t)np_));
    CK(cudaMemcpy(L.S, S.data(), sizeof(double) * nsp, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(L.G, G.data(), sizeof(double) * nsp, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(L.invJ, iJ.data(), sizeof(double) * iJ.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(L.Sf, Sf.data(), sizeof(double) * nfpt, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(L.Gf, Gf.data(), sizeof(double) * nfpt, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(L.pairs, pairs.data(), sizeof(int) * pairs.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(L.bc, bc.data(), sizeof(int) * bc.size(), cudaMemcpyHostToDevice));
    size_t nfv = (size_t)C->nv * L.nfp * E, npv = (size_t)C->nv * L.np * E;
    TRY(dalloc_t(C, &L.qf, nfv)); TRY(dalloc_t(C, &L.dq, nfv)); TRY(dalloc_t(C, &L.fn, nfv));
    TRY(dalloc_t(C, &L.Ftf, nfv)); TRY(dalloc_t(C, &L.Ft, d * npv));
    TRY(dalloc_t(C, &L.Qf, d * nfv));
    return FR_OK;
}

extern "C" int fr_destroy(fr_ctx *C) {
    if (!C) return FR_OK;
    for (void *p : C->allocs) cudaFree(p);
    delete C;
    return FR_OK;
}

extern "C" int fr_create(fr_ctx **out, const fr_mesh_desc *m, const fr_physics *ph) {
    if (!out) return fail(FR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!m || !ph) return fail(FR_ERR_INVALID_ARG, "mesh or physics is NULL");
    if (m->dim != 2 && m->dim != 3) return fail(FR_ERR_INVALID_ARG, "dim must be 2 or 3");
    if (m->qg != 1 && m->qg != 2) return fail(FR_ERR_INVALID_ARG, "geometry degree must be 1 or 2");
    if (m->nelem <= 0 || !m->gnodes || !m->faces || m->nfaces <= 0)
        return fail(FR_ERR_INVALID_ARG, "empty mesh");
    // the residual's grids put element chunks (CTA size >= 32) on the y axis, at most 65535
    if (m->nelem > 32LL * 65535)
        return fail(FR_ERR_INVALID_ARG, "at most %lld elements per context", 32LL * 65535);
    if (m->nlevels < 1 || m->nlevels > FRL_MAXLEV || !m->plevels)
        return fail(FR_ERR_INVALID_ARG, "nlevels must be 1..%d", FRL_MAXLEV);
    int pmax = m->dim == 2 ? 4 : 3;
    for (int l = 0; l < m->nlevels; ++l) {
        if (m->plevels[l] < 1 || m->plevels[l] > pmax)
            return fail(FR_ERR_INVALID_ARG, "level %d degree %d outside 1..%d", l, m->plevels[l], pmax);
        if (l > 0 && m->plevels[l] > m->plevels[l - 1])
            return fail(FR_ERR_INVALID_ARG, "levels must be ordered finest first");
    }
    if (!(ph->gamma > 1.0) || !(ph->prandtl > 0.0) || !(ph->mu >= 0.0) || !(ph->eta >= 0.0))
        return fail(FR_ERR_INVALID_ARG, "invalid physical parameters");
    if (ph->flux < 0 || ph->flux > 2) return fail(FR_ERR_INVALID_ARG, "flux must be 0 (Rusanov), 1 (Roe) or 2 (Weiss-Smith)");
    if (ph->flux == 2 && !(ph->ws_umin > 0.0)) return fail(FR_ERR_INVALID_ARG, "Weiss-Smith needs a positive ws_umin");
    fr_ctx *C = new fr_ctx();
    C->d = m->dim; C->nv = m->dim + 2; C->E = m->nelem; C->qg = m->qg; C->nlev = m->nlevels;
    C->eta = ph->eta;
    C->ph.gamma = ph->gamma;
    C->ph.gm1 = ph->gamma - 1.0;
    C->ph.mu = ph->mu;
    C->ph.kappa = (ph->gamma * ph->mu) / ph->prandtl;
    C->ph.c23 = 2.0 / 3.0;
    for (int v = 0; v < 5; ++v) C->ph.qinf[v] = v < C->nv ? ph->qinf[v] : 0.0;
    C->ph.flux = ph->flux;
    C->ph.ws_umin = ph->flux == 2 ? ph->ws_umin : 1.0;
    int rc = upload_tables();
    for (int l = 0; rc == FR_OK && l < m->nlevels; ++l) rc = setup_level(C, l, m->plevels[l], m);
    for (int F = 0; F < m->nfaces; ++F)
        if (m->faces[6 * F + 2] == m->faces[6 * F]) C->self_face = 1;
    if (rc == FR_OK) {
        std::vector<int> col(C->E);
        C->ncolor = frh_color(C->E, m->nfaces, m->faces, col.data());
        rc = dalloc_t(C, &C->color, C->E);
        if (rc == FR_OK && cudaMemcpy(C->color, col.data(), sizeof(int) * C->E, cudaMemcpyHostToDevice) != cudaSuccess)
            rc = fail(FR_ERR_CUDA, "copying colours");
    }
    if (rc == FR_OK) {
        int nf = 2 * C->d;
        std::vector<int> nb((size_t)C->E * nf), c2(C->E);
        if (frh_neighbours(C->E, nf, m->nfaces, m->faces, nb.data()) != 0)
            rc = fail(FR_ERR_INVALID_ARG, "a face names a local face index outside 0..%d", nf - 1);
        else if ((C->ncolor2 = frh_color2(C->E, nf, nb.data(), c2.data())) < 0)
            rc = fail(FR_ERR_INVALID_ARG, "the distance-2 colouring needs more than 1024 colours");
        if (rc == FR_OK) rc = dalloc_t(C, &C->nbr, nb.size());
        if (rc == FR_OK) rc = dalloc_t(C, &C->color2, c2.size());
        if (rc == FR_OK && (cudaMemcpy(C->nbr, nb.data(), sizeof(int) * nb.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
                            cudaMemcpy(C->color2, c2.data(), sizeof(int) * c2.size(), cudaMemcpyHostToDevice) != cudaSuccess))
            rc = fail(FR_ERR_CUDA, "copying the neighbour table");
    }
    long long n0 = C->L[0].ndof;
    if (rc == FR_OK) rc = dalloc_t(C, &C->info, 1);
    if (rc == FR_OK) rc = dalloc_t(C, &C->dots, 520);   // Krylov dimensions up to 512: j + 1 <= 512 sums
    if (rc == FR_OK) rc = dalloc_t(C, &C->partial, (size_t)frk64_multidot_scratch(C->L[0].ndof));
    C->ndof_rms = (double)C->L[0].ndof;
    if (rc == FR_OK) rc = dalloc_t(C, &C->jv_qp, n0);
    if (rc == FR_OK) rc = dalloc_t(C, &C->jv_Rp, n0);
    if (rc != FR_OK) { fr_destroy(C); return rc; }
    apply_cached_tiles(C, 0);
    frk64_lu_solve_prepare();
    frk32_lu_solve_prepare();
    *out = C;
    return FR_OK;
}

extern "C" int fr_kernel_timeouts(int clear) {
    return frk64_lu_solve_error(clear) | frk32_lu_solve_error(clear) | frktc_lu_error(clear);
}

extern "C" int fr_selftest_wait_timeout(void) {
    frk32_wait_selftest(1 << 12, 0);
    CKLAUNCH();
    CK(cudaDeviceSynchronize());
    return FR_OK;
}

extern "C" int fr_level_info(const fr_ctx *C, int l, int *p, int *np, long long *ndof) {
    if (!C || l < 0 || l >= C->nlev) return fail(FR_ERR_INVALID_ARG, "bad context or level");
    if (p) *p = C->L[l].p;
    if (np) *np = C->L[l].np;
    if (ndof) *ndof = C->L[l].ndof;
    return FR_OK;
}
extern "C" int fr_num_colors(const fr_ctx *C, int *n) {
    if (!C || !n) return fail(FR_ERR_INVALID_ARG, "bad argument");
    *n = C->ncolor;
    return FR_OK;
}

// read-only access to a level for other translation units of the library
int fr_internal_level(const fr_ctx *C, int l, FrLevel *out, FrPhysH *ph) {
    if (l < 0 || l >= C->nlev) return FR_ERR_INVALID_ARG;
    *out = C->L[l];
    *ph = C->ph;
    return FR_OK;
}
int fr_internal_fail(int code, const char *msg) { return fail(code, "%s", msg); }
int fr_internal_has_comm(const fr_ctx *C) { return C->has_comm; }

// ------------------------------------------------------------------ residual, Jv
// ---------------------------------------------------------- element partition
// the ghost elements of the level-l vector x take their owners' values (no-op without a
// communicator); x is the caller's state: only its ghost entries change
static int halo64(fr_ctx *C, int l, const double *x, cudaStream_t s);
static int halo32(fr_ctx *C, int l, const float *x, cudaStream_t s);

static int residual(fr_ctx *C, int l, const double *q, double *R, cudaStream_t s) {
    TRY(halo64(C, l, q, s));
    if (frk64_residual(C->L[l], C->ph, q, R, s) != 0)
        return fail(FR_ERR_UNIMPLEMENTED, "no kernel for d=%d p=%d", C->d, C->L[l].p);
    CKLAUNCH();
    return FR_OK;
}

extern "C" int fr_residual(fr_ctx *C, int l, const double *q, double *R, void *stream) {
    if (!C || l < 0 || l >= C->nlev || !q || !R) return fail(FR_ERR_INVALID_ARG, "bad argument");
    if (q == R) return fail(FR_ERR_INVALID_ARG, "q and R must not alias");
    return residual(C, l, q, R, S_(stream));
}

static int jvp(fr_ctx *C, const double *q, const double *Rq, const double *v, double eps, double shift, double *Av,
               cudaStream_t s) {
    long long n = C->L[0].ndof;
    frk64_axpy_perturb(n, q, eps, v, C->jv_qp, s);
    TRY(residual(C, 0, C->jv_qp, C->jv_Rp, s));
    frk64_jv_finish(n, shift, v, C->jv_Rp, Rq, eps, Av, s);
    CKLAUNCH();
    return FR_OK;
}

extern "C" int fr_jvp(fr_ctx *C, const double *q, const double *Rq, const double *v, double eps, double shift,
                      double *Av, void *stream) {
    if (!C || !q || !Rq || !v || !Av) return fail(FR_ERR_INVALID_ARG, "NULL argument");
    if (Av == q || Av == Rq || Av == v) return fail(FR_ERR_INVALID_ARG, "Av must not alias the inputs");
    if (!(eps != 0.0)) return fail(FR_ERR_INVALID_ARG, "eps must be non-zero");
    return jvp(C, q, Rq, v, eps, shift, Av, S_(stream));
}

// ------------------------------------------------- kernel dispatch per precision
template <typename T>
struct Kn;
#define KN_BODY(P, T)                                                                                            \
    static int residual(const FrLevelT<T> &L, const FrPhysH &ph, const T *q, T *R, cudaStream_t s) {             \
        return P##_residual(L, ph, q, R, s);                                                                     \
    }                                                                                                            \
    static void copy(long long n, const T *x, T *y, cudaStream_t s) { P##_copy(n, x, y, s); }                  \
    static void add(long long n, const T *a, const T *b, T *y, cudaStream_t s) { P##_add(n, a, b, y, s); }     \
    static void sub(long long n, const T *a, const T *b, T *y, cudaStream_t s) { P##_sub(n, a, b, y, s); }     \
    static void pmg_rhs(long long n, double c, const T *d, const T *qh, const T *b, const T *Rqh, const T *Rb,  \
                        T *r, cudaStream_t s) {                                                                  \
        P##_pmg_rhs(n, c, d, qh, b, Rqh, Rb, r, s);                                                              \
    }                                                                                                            \
    static void perturb(const FrLevelT<T> &L, const int *c, int col, int j, const T *q, T *qp, double er,      \
                        cudaStream_t s) {                                                                        \
        P##_perturb_color(L, c, col, j, q, qp, er, s);                                                           \
    }                                                                                                            \
    static void restore(const FrLevelT<T> &L, const int *c, int col, int j, const T *q, T *qp, cudaStream_t s) { \
        P##_restore_color(L, c, col, j, q, qp, s);                                                               \
    }                                                                                                            \
    static void column(const FrLevelT<T> &L, const int *c, int col, int j, const T *q, const T *R0,             \
                       const T *Rp, double shift, double er, T *M, cudaStream_t s) {                             \
        P##_block_column(L, c, col, j, q, R0, Rp, shift, er, M, s);                                              \
    }                                                                                                            \
    static int factor(const FrLevelT<T> &L, T *M, int *perm, int *info, cudaStream_t s) {                      \
        return P##_lu_factor(L, M, perm, info, s);                                                               \
    }                                                                                                            \
    static int solve(const FrLevelT<T> &L, const T *M, const int *perm, T *x, cudaStream_t s) {                \
        return P##_lu_solve(L, M, perm, x, s);                                                                   \
    }                                                                                                            \
    static int transfer(const FrLevelT<T> &Lf, const FrLevelT<T> &Lc, bool r, const T *x, T *y,               \
                        cudaStream_t s) {                                                                        \
        return P##_transfer(Lf, Lc, r, x, y, s);                                                                 \
    }
template <>
struct Kn<double> {
    KN_BODY(frk64, double)
    static constexpr double epsrel = 1e-7;   // FD step of the FP64 blocks: 1e-7 max(1, |q_j|)
};
template <>
struct Kn<float> {
    KN_BODY(frk32, float)
    static constexpr double epsrel = 3e-4;   // FP32 blocks: about the square root of FP32 unit roundoff
};

template <typename T> static FrLevelT<T> *levels(fr_ctx *C);
template <> FrLevelT<double> *levels<double>(fr_ctx *C) { return C->L; }
template <> FrLevelT<float> *levels<float>(fr_ctx *C) { return C->L32; }
template <typename T> static PmgBuf<T> &pbuf(fr_ctx *C);
template <> PmgBuf<double> &pbuf<double>(fr_ctx *C) { return C->p64; }
template <> PmgBuf<float> &pbuf<float>(fr_ctx *C) { return C->p32; }

static int halo_t(fr_ctx *C, int l, const double *x, cudaStream_t s) { return halo64(C, l, x, s); }
static int halo_t(fr_ctx *C, int l, const float *x, cudaStream_t s) { return halo32(C, l, x, s); }

// exchange = false: a finite-difference column, whose perturbation stays on this process
template <typename T>
static int residual_t(fr_ctx *C, int l, const T *q, T *R, cudaStream_t s, bool exchange = true) {
    if (exchange) TRY(halo_t(C, l, q, s));
    if (Kn<T>::residual(levels<T>(C)[l], C->ph, q, R, s) != 0)
        return fail(FR_ERR_UNIMPLEMENTED, "no kernel for d=%d p=%d", C->d, C->L[l].p);
    CKLAUNCH();
    return FR_OK;
}

template <typename T>
static int halo_impl(fr_ctx *C, int l, const T *x, int prec, cudaStream_t s,
                     void (*pack)(int, long long, int, const int *, const T *, T *, cudaStream_t),
                     void (*unpack)(int, long long, int, int, const T *, T *, cudaStream_t)) {
    if (!C->has_comm) return FR_OK;
    const FrLevel &L = C->L[l];
    int rows = L.nv * L.np, nrecv = C->E - C->comm.n_owned;
    T *xm = const_cast<T *>(x);   // only the ghost entries are written
    pack(rows, C->E, C->comm.nsend, C->send_idx_dev, x, (T *)C->comm.send_buf, s);
    CKLAUNCH();
    CK(cudaStreamSynchronize(s));
    if (C->comm.halo(C->comm.user, l, prec, (long long)rows * (long long)sizeof(T), (void *)s) != 0)
        return fail(FR_ERR_CUDA, "ghost exchange failed (level %d)", l);
    unpack(rows, C->E, C->comm.n_owned, nrecv, (const T *)C->comm.recv_buf, xm, s);
    CKLAUNCH();
    return FR_OK;
}
static int halo64(fr_ctx *C, int l, const double *x, cudaStream_t s) {
    return halo_impl<double>(C, l, x, 0, s, frk64_halo_pack, frk64_halo_unpack);
}
static int halo32(fr_ctx *C, int l, const float *x, cudaStream_t s) {
    return halo_impl<float>(C, l, x, 1, s, frk32_halo_pack, frk32_halo_unpack);
}

// maxima or sums of n device doubles over the processes (in place; no-op alone)
static int allreduce_dev(fr_ctx *C, double *dev, int n, int op, cudaStream_t s) {
    if (!C->has_comm) return FR_OK;
    double h[64];
    if (n > 64) return fail(FR_ERR_INVALID_ARG, "allreduce of more than 64 values");
    CK(cudaMemcpyAsync(h, dev, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (C->comm.allreduce(C->comm.user, h, n, op) != 0) return fail(FR_ERR_CUDA, "allreduce failed");
    CK(cudaMemcpyAsync(dev, h, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    return FR_OK;
}

extern "C" int fr_set_comm(fr_ctx *C, const fr_comm *m) {
    if (!C) return fail(FR_ERR_INVALID_ARG, "NULL context");
    if (!m) {
        C->has_comm = 0;
        C->ndof_rms = (double)C->L[0].ndof;
        return FR_OK;
    }
    int nrecv = C->E - m->n_owned;
    if (m->n_owned < 1 || m->n_owned > C->E || m->nsend < 0)
        return fail(FR_ERR_INVALID_ARG, "n_owned must be 1..E and nsend >= 0");
    if (!m->halo || !m->allreduce) return fail(FR_ERR_INVALID_ARG, "both callbacks are needed");
    if ((m->nsend > 0 && (!m->send_idx || !m->send_buf)) || (nrecv > 0 && !m->recv_buf))
        return fail(FR_ERR_INVALID_ARG, "send list or exchange buffers missing");
    for (int i = 0; i < m->nsend; ++i)
        if (m->send_idx[i] < 0 || m->send_idx[i] >= m->n_owned)
            return fail(FR_ERR_INVALID_ARG, "send_idx[%d] = %d is not an owned element", i, m->send_idx[i]);
    if (C->mbnk) return fail(FR_ERR_INVALID_ARG, "the matrix-based coarse smoother is not partitioned");
    int *dev = nullptr;
    TRY(dalloc_t(C, &dev, (size_t)(m->nsend > 0 ? m->nsend : 1)));
    if (m->nsend > 0) CK(cudaMemcpy(dev, m->send_idx, sizeof(int) * m->nsend, cudaMemcpyHostToDevice));
    if (C->send_idx_dev) dfree(C, C->send_idx_dev);
    C->send_idx_dev = dev;
    C->comm = *m;
    C->comm.send_idx = nullptr;
    if (m->n_owned_total < m->n_owned) return fail(FR_ERR_INVALID_ARG, "n_owned_total below n_owned");
    C->ndof_rms = (double)C->L[0].nv * C->L[0].np * (double)m->n_owned_total;
    C->has_comm = 1;
    return FR_OK;
}

// FP32 copies of every level: geometric factors converted on the device, own workspace
static int ensure_levels32(fr_ctx *C) {
    if (C->have32) return FR_OK;
    for (int l = 0; l < C->nlev; ++l) {
        FrLevel &L = C->L[l];
        FrLevel32 &M = C->L32[l];
        M.d = L.d; M.p = L.p; M.n = L.n; M.np = L.np; M.nf1 = L.nf1; M.nfp = L.nfp; M.nv = L.nv; M.E = L.E;
        M.ndof = L.ndof; M.nd = L.nd; M.npairs = L.npairs; M.pairs = L.pairs; M.bc = L.bc;
        M.etagL = L.etagL; M.etagR = L.etagR;
        size_t E = L.E, nsp = (size_t)L.d * L.d * L.np * E, nfpt = (size_t)L.d * L.d * L.nfp * E;
        TRY(dalloc_t(C, &M.S, nsp)); TRY(dalloc_t(C, &M.G, nsp)); TRY(dalloc_t(C, &M.invJ, (size_t)L.np * E));
        TRY(dalloc_t(C, &M.Sf, nfpt)); TRY(dalloc_t(C, &M.Gf, nfpt));
        frk32_d2f(nsp, L.S, M.S, 0); frk32_d2f(nsp, L.G, M.G, 0); frk32_d2f((long long)L.np * E, L.invJ, M.invJ, 0);
        frk32_d2f(nfpt, L.Sf, M.Sf, 0); frk32_d2f(nfpt, L.Gf, M.Gf, 0);
        size_t nfv = (size_t)L.nv * L.nfp * E, npv = (size_t)L.nv * L.np * E;
        TRY(dalloc_t(C, &M.qf, nfv)); TRY(dalloc_t(C, &M.dq, nfv)); TRY(dalloc_t(C, &M.fn, nfv));
        TRY(dalloc_t(C, &M.Ftf, nfv)); TRY(dalloc_t(C, &M.Ft, L.d * npv));
        TRY(dalloc_t(C, &M.Qf, L.d * nfv));
    }
    long long n0 = C->L[0].ndof;
    TRY(dalloc_t(C, &C->x32, n0)); TRY(dalloc_t(C, &C->q32, n0)); TRY(dalloc_t(C, &C->Rq32, n0));
    TRY(dalloc_t(C, &C->y32, n0)); TRY(dalloc_t(C, &C->xmax, 1));
    CK(cudaDeviceSynchronize());
    CKLAUNCH();
    C->have32 = 1;
    apply_cached_tiles(C, 1);
    return FR_OK;
}

// ---------------------------------------------------------------- element blocks
template <typename T>
static int ensure_blk_tmp(fr_ctx *C) {
    PmgBuf<T> &P = pbuf<T>(C);
    if (P.blk_R0) return FR_OK;
    long long n0 = C->L[0].ndof;
    TRY(dalloc_t(C, &P.blk_R0, n0));
    TRY(dalloc_t(C, &P.blk_Rp, n0));
    TRY(dalloc_t(C, &P.blk_qp, n0));
    return FR_OK;
}

static int ensure_levelsAD(fr_ctx *C) {
    if (C->haveAD) return FR_OK;
    for (int l = 0; l < C->nlev; ++l) {
        FrLevel32 &F = C->L32[l];
        FrLevelAD &A = C->LA[l];
        A.d = F.d; A.p = F.p; A.n = F.n; A.np = F.np; A.nf1 = F.nf1; A.nfp = F.nfp; A.nv = F.nv; A.E = F.E;
        A.ndof = F.ndof; A.nd = F.nd; A.npairs = F.npairs; A.pairs = F.pairs; A.bc = F.bc;
        A.etagL = F.etagL; A.etagR = F.etagR;
        A.S = F.S; A.G = F.G; A.invJ = F.invJ; A.Sf = F.Sf; A.Gf = F.Gf;
        size_t E = F.E, nfv = (size_t)F.nv * F.nfp * E, npv = (size_t)F.nv * F.np * E;
        TRY(dalloc_t(C, &A.qf, nfv)); TRY(dalloc_t(C, &A.dq, nfv)); TRY(dalloc_t(C, &A.fn, nfv));
        TRY(dalloc_t(C, &A.Ftf, nfv)); TRY(dalloc_t(C, &A.Ft, F.d * npv));
        TRY(dalloc_t(C, &A.Qf, F.d * nfv));
    }
    TRY(dalloc_t(C, &C->qd, C->L[0].ndof));
    TRY(dalloc_t(C, &C->Rd, C->L[0].ndof));
    C->haveAD = 1;
    return FR_OK;
}

// FP32 blocks of level l, element by element (fr_ad_elem.cuh): one FP32 residual at q
// leaves the traces and face gradients that the other side of every face contributes,
// then one kernel differentiates each element's residual in all its degrees of freedom
static int elem_blocks_ad_local(fr_ctx *C, int l, const float *q, double shift, float *M, cudaStream_t s) {
    TRY(ensure_levels32(C));
    TRY(ensure_blk_tmp<float>(C));
    if (!C->ad_nt) {
        TRY(dalloc_t(C, &C->ad_nt, (size_t)frkad_elem_nt_floats(C->L32[0])));
        TRY(dalloc_t(C, &C->ad_bck, (size_t)C->L32[0].nfp * C->E));
    }
    FrLevel32 &F = C->L32[l];
    TRY(residual_t<float>(C, l, q, pbuf<float>(C).blk_R0, s));
    if (frkad_elem_blocks(F, C->ph, q, F.qf, F.Qf, C->ad_nt, C->ad_bck, shift, M, s) != 0)
        return fail(FR_ERR_UNIMPLEMENTED, "no kernel for d=%d p=%d", C->d, F.p);
    CKLAUNCH();
    return FR_OK;
}

// FP32 blocks of level l by colours: one forward-mode residual of the whole level per
// (colour, batch of FR_AD_K columns), seeds in those degrees of freedom of the colour's
// elements.  The element-local kernel above gives the same blocks to FP32 rounding; this
// path serves meshes where a face joins an element to itself.
static int elem_blocks_ad_colour(fr_ctx *C, int l, const float *q, double shift, float *M, cudaStream_t s) {
    TRY(ensure_levelsAD(C));
    FrLevelAD &A = C->LA[l];
    frkad_init(A.ndof, q, C->qd, s);
    for (int col = 0; col < C->ncolor; ++col)
        for (int j0 = 0; j0 < A.nd; j0 += FR_AD_K) {
            frkad_seed(A, C->color, col, j0, C->qd, 1.f, s);
            if (frkad_residual(A, C->ph, C->qd, C->Rd, s) != 0)
                return fail(FR_ERR_UNIMPLEMENTED, "no kernel for d=%d p=%d", C->d, A.p);
            frkad_block_column(A, C->color, col, j0, C->Rd, shift, M, s);
            frkad_seed(A, C->color, col, j0, C->qd, 0.f, s);
        }
    CKLAUNCH();
    return FR_OK;
}

// blocks of level l by colours: one residual per (colour, column); in FP32 the columns
// come from forward-mode differentiation instead of differences
template <typename T>
static int elem_blocks_t(fr_ctx *C, int l, const T *q, double shift, T *M, cudaStream_t s);
static int elem_blocks_ad(fr_ctx *C, int l, const float *q, double shift, float *M, cudaStream_t s) {
    return (C->self_face || C->ad_method == 1) ? elem_blocks_ad_colour(C, l, q, shift, M, s)
                                               : elem_blocks_ad_local(C, l, q, shift, M, s);
}

extern "C" int fr_set_block_method(fr_ctx *C, int method) {
    if (!C || method < 0 || method > 1) return fail(FR_ERR_INVALID_ARG, "method must be 0 or 1");
    C->ad_method = method;
    return FR_OK;
}
template <>
int elem_blocks_t<float>(fr_ctx *C, int l, const float *q, double shift, float *M, cudaStream_t s) {
    return elem_blocks_ad(C, l, q, shift, M, s);
}

extern "C" int fr_elem_blocks_f32(fr_ctx *C, int l, const float *q, double shift, float *M, int method, void *stream) {
    if (!C || l < 0 || l >= C->nlev || !q || !M) return fail(FR_ERR_INVALID_ARG, "bad argument");
    if (method < 0 || method > 1) return fail(FR_ERR_INVALID_ARG, "method must be 0 (element-local) or 1 (colours)");
    if (method == 0 && C->self_face)
        return fail(FR_ERR_INVALID_ARG, "a face joins an element to itself: only the colouring method applies");
    cudaStream_t s = S_(stream);
    TRY(ensure_levels32(C));
    return method == 0 ? elem_blocks_ad_local(C, l, q, shift, M, s) : elem_blocks_ad_colour(C, l, q, shift, M, s);
}
template <>
int elem_blocks_t<double>(fr_ctx *C, int l, const double *q, double shift, double *M, cudaStream_t s) {
    typedef double T;
    TRY(ensure_blk_tmp<T>(C));
    PmgBuf<T> &P = pbuf<T>(C);
    FrLevelT<T> &L = levels<T>(C)[l];
    TRY(residual_t<T>(C, l, q, P.blk_R0, s));
    Kn<T>::copy(L.ndof, q, P.blk_qp, s);
    for (int col = 0; col < C->ncolor; ++col)
        for (int j = 0; j < L.nd; ++j) {
            Kn<T>::perturb(L, C->color, col, j, q, P.blk_qp, Kn<T>::epsrel, s);
            TRY(residual_t<T>(C, l, P.blk_qp, P.blk_Rp, s, false));
            Kn<T>::column(L, C->color, col, j, q, P.blk_R0, P.blk_Rp, shift, Kn<T>::epsrel, M, s);
            Kn<T>::restore(L, C->color, col, j, q, P.blk_qp, s);
        }
    CKLAUNCH();
    return FR_OK;
}

// diagonal and neighbour blocks of level l in one pass over the distance-2 colours (for
// the matrix-based smoother): the diagonal columns equal those of elem_blocks_t, since
// each element's residual sees the same single perturbation either way
template <typename T>
static int elem_blocks_mbnk_t(fr_ctx *C, int l, const T *q, double shift, T *M, T *O, cudaStream_t s);
template <>
int elem_blocks_mbnk_t<float>(fr_ctx *C, int l, const float *q, double shift, float *M, float *O, cudaStream_t s) {
    TRY(ensure_levelsAD(C));
    FrLevelAD &A = C->LA[l];
    int nf = 2 * C->d;
    CK(cudaMemsetAsync(O, 0, sizeof(float) * (size_t)A.E * nf * A.nd * A.nd, s));
    frkad_init(A.ndof, q, C->qd, s);
    for (int col = 0; col < C->ncolor2; ++col)
        for (int j0 = 0; j0 < A.nd; j0 += FR_AD_K) {
            frkad_seed(A, C->color2, col, j0, C->qd, 1.f, s);
            if (frkad_residual(A, C->ph, C->qd, C->Rd, s) != 0)
                return fail(FR_ERR_UNIMPLEMENTED, "no kernel for d=%d p=%d", C->d, A.p);
            frkad_block_column(A, C->color2, col, j0, C->Rd, shift, M, s);
            frkad_nbr_column(A, nf, C->nbr, C->color2, col, j0, C->Rd, O, s);
            frkad_seed(A, C->color2, col, j0, C->qd, 0.f, s);
        }
    CKLAUNCH();
    return FR_OK;
}
template <>
int elem_blocks_mbnk_t<double>(fr_ctx *C, int l, const double *q, double shift, double *M, double *O, cudaStream_t s) {
    typedef double T;
    TRY(ensure_blk_tmp<T>(C));
    PmgBuf<T> &P = pbuf<T>(C);
    FrLevelT<T> &L = levels<T>(C)[l];
    int nf = 2 * C->d;
    CK(cudaMemsetAsync(O, 0, sizeof(T) * (size_t)L.E * nf * L.nd * L.nd, s));
    TRY(residual_t<T>(C, l, q, P.blk_R0, s));
    Kn<T>::copy(L.ndof, q, P.blk_qp, s);
    for (int col = 0; col < C->ncolor2; ++col)
        for (int j = 0; j < L.nd; ++j) {
            Kn<T>::perturb(L, C->color2, col, j, q, P.blk_qp, Kn<T>::epsrel, s);
            TRY(residual_t<T>(C, l, P.blk_qp, P.blk_Rp, s, false));
            Kn<T>::column(L, C->color2, col, j, q, P.blk_R0, P.blk_Rp, shift, Kn<T>::epsrel, M, s);
            frmb_nbr_column(L.E, L.nd, nf, C->nbr, C->color2, col, j, q, P.blk_R0, P.blk_Rp, Kn<T>::epsrel, O, s);
            Kn<T>::restore(L, C->color2, col, j, q, P.blk_qp, s);
        }
    CKLAUNCH();
    return FR_OK;
}

extern "C" int fr_nbr_blocks(fr_ctx *C, int l, const double *q, double shift, double *M, double *O, void *stream) {
    if (!C || l < 0 || l >= C->nlev || !q || !M || !O) return fail(FR_ERR_INVALID_ARG, "bad argument");
    return elem_blocks_mbnk_t<double>(C, l, q, shift, M, O, S_(stream));
}

extern "C" int fr_neighbour_table(const fr_ctx *C, int *nbr) {
    if (!C || !nbr) return fail(FR_ERR_INVALID_ARG, "bad argument");
    CK(cudaMemcpy(nbr, C->nbr, sizeof(int) * (size_t)C->E * 2 * C->d, cudaMemcpyDeviceToHost));
    return FR_OK;
}

extern "C" int fr_elem_blocks(fr_ctx *C, int l, const double *q, double shift, double *M, void *stream) {
    if (!C || l < 0 || l >= C->nlev || !q || !M) return fail(FR_ERR_INVALID_ARG, "bad argument");
    return elem_blocks_t<double>(C, l, q, shift, M, S_(stream));
}

// FP32 blocks go to the tensor-core factorisation where its block size allows it and the
// context's LU method is 0; FP64 blocks always take the CUDA-core kernels (their fma
// order is the oracle's)
static bool use_tc_lu(fr_ctx *C, int l, const float *) { return C->lu_method == 0 && frktc_lu_supported(C->L32[l].nd); }
static bool use_tc_lu(fr_ctx *, int, const double *) { return false; }
static int tc_scratch(fr_ctx *C, int E, int nd) {
    size_t need = frktc_lu_scratch_floats(E, nd);
    if (C->lu_scr && C->lu_scr_cap >= need) return FR_OK;
    dfree(C, C->lu_scr);
    C->lu_scr = nullptr;
    C->lu_scr_cap = 0;
    TRY(dalloc_t(C, &C->lu_scr, need));
    C->lu_scr_cap = need;
    return FR_OK;
}
static int tc_factor(fr_ctx *C, int l, float *M, int *perm, cudaStream_t s) {
    TRY(tc_scratch(C, C->L32[l].E, C->L32[l].nd));
    if (frktc_lu_factor(C->L32[l].E, C->L32[l].nd, M, perm, C->info, C->lu_scr, s) != 0)
        return fail(FR_ERR_UNIMPLEMENTED, "tensor-core LU: %d blocks of %d rows exceed its launch grid",
                    C->L32[l].E, C->L32[l].nd);
    return FR_OK;
}
static int tc_factor(fr_ctx *, int, double *, int *, cudaStream_t) { return FR_OK; }

// half-width copy of level l's FP32 factors for the solves (FP64 factors: nothing)
static int half_factors(fr_ctx *C, int l, const float *M, cudaStream_t s) {
    PmgBuf<float> &P = C->p32;
    P.half_ok[l] = 0;
    const FrLevel32 &L = C->L32[l];
    if (!C->lu_half || (L.nd + 63) / 64 > 6) return FR_OK;   // blocks over 384 rows keep FP32 factors
    size_t need = (size_t)L.E * L.nd * frktc_half_ld(L.nd);
    if (!P.H[l] || P.H_cap[l] < need) {
        dfree(C, P.H[l]);
        dfree(C, P.dg[l]);
        P.H[l] = nullptr; P.dg[l] = nullptr; P.H_cap[l] = 0;
        TRY(dalloc(C, &P.H[l], 2 * need));
        TRY(dalloc_t(C, &P.dg[l], (size_t)2 * L.E * L.nd));
        P.H_cap[l] = need;
    }
    frktc_lu_to_half(L.E, L.nd, M, P.H[l], P.dg[l], s);
    P.half_ok[l] = 1;
    return FR_OK;
}
static int half_factors(fr_ctx *, int, const double *, cudaStream_t) { return FR_OK; }
// the block solve of the smoother on level l with the factors pmg_setup stored
static int smoother_solve(fr_ctx *C, int l, float *x, cudaStream_t s) {
    PmgBuf<float> &P = C->p32;
    const FrLevel32 &L = C->L32[l];
    if (P.half_ok[l]) return frktc_lu_solve_half(L.E, L.nd, L.lu_g, P.H[l], P.dg[l], P.perm[l], x, s) == 0
                                 ? FR_OK : fail(FR_ERR_UNIMPLEMENTED, "block size %d", L.nd);
    return Kn<float>::solve(L, P.M[l], P.perm[l], x, s) == 0 ? FR_OK : fail(FR_ERR_UNIMPLEMENTED, "block size %d", L.nd);
}
static int smoother_solve(fr_ctx *C, int l, double *x, cudaStream_t s) {
    PmgBuf<double> &P = C->p64;
    return Kn<double>::solve(C->L[l], P.M[l], P.perm[l], x, s) == 0 ? FR_OK
                                                                       : fail(FR_ERR_UNIMPLEMENTED, "block size %d", C->L[l].nd);
}

template <typename T>
static int block_factor_t(fr_ctx *C, int l, T *M, int *perm, cudaStream_t s) {
    CK(cudaMemsetAsync(C->info, 0, sizeof(int), s));
    if (use_tc_lu(C, l, M)) TRY(tc_factor(C, l, M, perm, s));
    else Kn<T>::factor(levels<T>(C)[l], M, perm, C->info, s);
    CKLAUNCH();
    return FR_OK;
}

extern "C" int fr_block_factor(fr_ctx *C, int l, double *M, int *perm, void *stream) {
    if (!C || l < 0 || l >= C->nlev || !M || !perm) return fail(FR_ERR_INVALID_ARG, "bad argument");
    cudaStream_t s = S_(stream);
    TRY(block_factor_t<double>(C, l, M, perm, s));
    int info = 0;
    CK(cudaMemcpyAsync(&info, C->info, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (info) return fail(FR_ERR_BREAKDOWN, "zero pivot in an element block");
    return FR_OK;
}

extern "C" int fr_set_lu_method(fr_ctx *C, int method) {
    if (!C || method < 0 || method > 1) return fail(FR_ERR_INVALID_ARG, "method must be 0 or 1");
    C->lu_method = method;
    return FR_OK;
}

// ------------------------------------------------------------- p-adaptation
extern "C" int fr_spectral_decay(fr_ctx *C, int l, const double *q, int var, double *eta, void *stream) {
    if (!C || l < 0 || l >= C->nlev || !q || !eta) return fail(FR_ERR_INVALID_ARG, "bad argument");
    if (var < 0 || var >= C->nv) return fail(FR_ERR_INVALID_ARG, "variable %d outside 0..%d", var, C->nv - 1);
    if (!C->pa_max) TRY(dalloc_t(C, &C->pa_max, 1));
    const FrLevel &L = C->L[l];
    if (frpa_spectral_decay(L.d, L.p, L.E, q, var, eta, C->pa_max, S_(stream)) != 0)
        return fail(FR_ERR_UNIMPLEMENTED, "spectral-decay indicator for d = %d, p = %d", L.d, L.p);
    CKLAUNCH();
    return FR_OK;
}

extern "C" int fr_padapt_mark(fr_ctx *C, const double *eta, const int *p_in, int p_min, int p_max, double nu_min,
                              double nu_max, int *p_out, void *stream) {
    if (!C || !eta || !p_in || !p_out) return fail(FR_ERR_INVALID_ARG, "NULL argument");
    if (p_min < 0 || p_max < p_min || !(nu_min >= 0.0) || !(nu_max >= nu_min))
        return fail(FR_ERR_INVALID_ARG, "need 0 <= p_min <= p_max and 0 <= nu_min <= nu_max");
    if (!C->pa_max) TRY(dalloc_t(C, &C->pa_max, 1));
    cudaStream_t s = S_(stream);
    // max(eta) of the given indicators (not necessarily the last fr_spectral_decay's)
    if (frk32_absmax(C->E, eta, C->pa_max, s) != 0) return fail(FR_ERR_CUDA, "max");
    frpa_mark(C->E, eta, C->pa_max, p_in, p_min, p_max, nu_min, nu_max, p_out, s);
    CKLAUNCH();
    return FR_OK;
}

extern "C" int fr_nested_hierarchy(int p_elem, int gap, int nlevels, int *degrees) {
    if (p_elem < 0 || gap < 1 || nlevels < 1 || nlevels > FRL_MAXLEV || !degrees)
        return fail(FR_ERR_INVALID_ARG, "need p >= 0, gap >= 1, 1 <= nlevels <= %d", FRL_MAXLEV);
    degrees[0] = p_elem;
    for (int l = 1; l < nlevels; ++l) {
        int a = p_elem - gap * l, b = nlevels - 1 - l, c = degrees[l - 1] - 1;
        int lo = a > b ? a : b, hi = c > 0 ? c : 0;
        degrees[l] = lo < hi ? lo : hi;
    }
    return FR_OK;
}

extern "C" int fr_set_cycle_scaling(fr_ctx *C, int on) {
    if (!C || on < 0 || on > 1) return fail(FR_ERR_INVALID_ARG, "on must be 0 or 1");
    C->scale64 = on;
    C->pmg_ready = 0;
    return FR_OK;
}

extern "C" int fr_set_precision_fallback(fr_ctx *C, int on) {
    if (!C || on < 0 || on > 1) return fail(FR_ERR_INVALID_ARG, "on must be 0 or 1");
    C->no_fallback = !on;
    return FR_OK;
}

extern "C" int fr_set_lu_storage(fr_ctx *C, int half) {
    if (!C || half < 0 || half > 1) return fail(FR_ERR_INVALID_ARG, "half must be 0 or 1");
    C->lu_half = half;
    return FR_OK;
}

extern "C" int fr_block_to_half(fr_ctx *C, int l, const float *M, void *H, float *dg, void *stream) {
    if (!C || l < 0 || l >= C->nlev || !M || !H || !dg) return fail(FR_ERR_INVALID_ARG, "bad argument");
    TRY(ensure_levels32(C));
    frktc_lu_to_half(C->L32[l].E, C->L32[l].nd, M, H, dg, S_(stream));
    CKLAUNCH();
    return FR_OK;
}

extern "C" int fr_block_solve_half(fr_ctx *C, int l, const void *H, const float *dg, const int *perm, float *x,
                                   void *stream) {
    if (!C || l < 0 || l >= C->nlev || !H || !dg || !perm || !x) return fail(FR_ERR_INVALID_ARG, "bad argument");
    TRY(ensure_levels32(C));
    const FrLevel32 &L = C->L32[l];
    if (frktc_lu_solve_half(L.E, L.nd, L.lu_g, H, dg, perm, x, S_(stream)) != 0)
        return fail(FR_ERR_UNIMPLEMENTED, "block size %d", L.nd);
    CKLAUNCH();
    return FR_OK;
}

extern "C" int fr_block_factor_f32(fr_ctx *C, int l, float *M, int *perm, int method, void *stream) {
    if (!C || l < 0 || l >= C->nlev || !M || !perm) return fail(FR_ERR_INVALID_ARG, "bad argument");
    if (method < 0 || method > 2) return fail(FR_ERR_INVALID_ARG, "method must be 0, 1 or 2");
    TRY(ensure_levels32(C));
    cudaStream_t s = S_(stream);
    const FrLevel32 &L = C->L32[l];
    bool tc = method == 2 || (method == 0 && frktc_lu_supported(L.nd));
    if (tc && !frktc_lu_supported(L.nd))
        return fail(FR_ERR_UNIMPLEMENTED, "tensor-core LU: block size %d outside 65..384", L.nd);
    if (tc) TRY(tc_scratch(C, L.E, L.nd));
    CK(cudaMemsetAsync(C->info, 0, sizeof(int), s));
    if (tc) {
        if (frktc_lu_factor(L.E, L.nd, M, perm, C->info, C->lu_scr, s) != 0)
            return fail(FR_ERR_UNIMPLEMENTED, "tensor-core LU: %d blocks of %d rows exceed its launch grid", L.E, L.nd);
    } else {
        frk32_lu_factor(L, M, perm, C->info, s);
    }
    CKLAUNCH();
    int info = 0;
    CK(cudaMemcpyAsync(&info, C->info, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (frktc_lu_error(1)) return fail(FR_ERR_CUDA, "tensor-core LU: a wait for the tensor cores ran out");
    if (info) return fail(FR_ERR_BREAKDOWN, "zero pivot in an element block");
    return FR_OK;
}

extern "C" int fr_block_solve_f32(fr_ctx *C, int l, const float *M, const int *perm, float *x, void *stream) {
    if (!C || l < 0 || l >= C->nlev || !M || !perm || !x) return fail(FR_ERR_INVALID_ARG, "bad argument");
    TRY(ensure_levels32(C));
    if (frk32_lu_solve(C->L32[l], M, perm, x, S_(stream)) != 0)
        return fail(FR_ERR_UNIMPLEMENTED, "block size %d", C->L32[l].nd);
    CKLAUNCH();
    return FR_OK;
}

extern "C" int fr_block_solve(fr_ctx *C, int l, const double *M, const int *perm, double *x, void *stream) {
    if (!C || l < 0 || l >= C->nlev || !M || !perm || !x) return fail(FR_ERR_INVALID_ARG, "bad argument");
    if (frk64_lu_solve(C->L[l], M, perm, x, S_(stream)) != 0) return fail(FR_ERR_UNIMPLEMENTED, "block size %d", C->L[l].nd);
    CKLAUNCH();
    return FR_OK;
}

template <typename T>
static int transfer_t(fr_ctx *C, int l, bool r, const T *x, T *y, cudaStream_t s) {
    if (Kn<T>::transfer(levels<T>(C)[l], levels<T>(C)[l + 1], r, x, y, s) != 0)
        return fail(FR_ERR_UNIMPLEMENTED, "no transfer kernel p%d <-> p%d", C->L[l].p, C->L[l + 1].p);
    CKLAUNCH();
    return FR_OK;
}
extern "C" int fr_restrict(fr_ctx *C, int l, const double *xf, double *xc, void *stream) {
    if (!C || l < 0 || l + 1 >= C->nlev || !xf || !xc) return fail(FR_ERR_INVALID_ARG, "bad argument");
    return transfer_t<double>(C, l, true, xf, xc, S_(stream));
}
extern "C" int fr_prolong(fr_ctx *C, int l, const double *xc, double *xf, void *stream) {
    if (!C || l < 0 || l + 1 >= C->nlev || !xf || !xc) return fail(FR_ERR_INVALID_ARG, "bad argument");
    return transfer_t<double>(C, l, false, xc, xf, S_(stream));
}

// ------------------------------------------------------------------------- pMG
template <typename T>
static int pmg_alloc_t(fr_ctx *C, int nlev) {
    PmgBuf<T> &P = pbuf<T>(C);
    for (int l = 0; l < nlev; ++l) {
        FrLevel &L = C->L[l];
        size_t need = (size_t)L.E * L.nd * L.nd;
        if (P.M_cap[l] < need) {
            dfree(C, P.M[l]);
            dfree(C, P.perm[l]);
            P.M[l] = nullptr; P.perm[l] = nullptr; P.M_cap[l] = 0;
            TRY(dalloc_t(C, &P.M[l], need));
            TRY(dalloc_t(C, &P.perm[l], (size_t)L.E * L.nd));
            P.M_cap[l] = need;
        }
        if (!P.qh[l]) {
            long long n = L.ndof;
            if (l > 0) { TRY(dalloc_t(C, &P.b[l], n)); TRY(dalloc_t(C, &P.Rb[l], n)); TRY(dalloc_t(C, &P.d[l], n)); }
            TRY(dalloc_t(C, &P.qh[l], n)); TRY(dalloc_t(C, &P.Rqh[l], n));
            TRY(dalloc_t(C, &P.rhs[l], n)); TRY(dalloc_t(C, &P.C[l], n));
        }
    }
    return FR_OK;
}

template <typename T>
static int ensure_cap(fr_ctx *C, T **p, size_t *cap, size_t need) {
    if (*p && *cap >= need) return FR_OK;
    dfree(C, *p);
    *p = nullptr;
    *cap = 0;
    TRY(dalloc_t(C, p, need));
    *cap = need;
    return FR_OK;
}

// buffers of the matrix-based smoother on level l
template <typename T>
static int mbnk_alloc_t(fr_ctx *C, int l) {
    PmgBuf<T> &P = pbuf<T>(C);
    const FrLevel &L = C->L[l];
    size_t blk = (size_t)L.nd * L.nd, N = (size_t)L.ndof;
    TRY(ensure_cap(C, &P.Md, &P.Md_cap, (size_t)L.E * blk));
    TRY(ensure_cap(C, &P.O, &P.O_cap, (size_t)L.E * 2 * C->d * blk));
    TRY(ensure_cap(C, &P.V, &P.V_cap, (size_t)(FRMB_MAXIT + 1) * N));
    size_t wc = P.w_cap;
    TRY(ensure_cap(C, &P.mz, &wc, N));
    wc = P.w_cap;
    TRY(ensure_cap(C, &P.mw, &P.w_cap, N));
    if (!C->mb_gm) {
        TRY(dalloc_t(C, &C->mb_gm, FRMB_GM));
        TRY(dalloc_t(C, &C->mb_partial, (size_t)FRMB_MAXBLK * (FRMB_MAXIT + 1)));
        CK(cudaMemset(C->mb_gm, 0, sizeof(double) * FRMB_GM));
    }
    return FR_OK;
}

// blocks (1/dtau* + c) I - J_ee at q_ref restricted level by level, and their LU factors;
// with the matrix-based smoother the coarsest level also keeps its diagonal blocks
// unfactored and its neighbour blocks
template <typename T>
static int pmg_factor_levels(fr_ctx *C, const T *q_ref, const fr_pmg_opts *o, cudaStream_t s) {
    PmgBuf<T> &P = pbuf<T>(C);
    double shift = o->inv_dtau_star + o->c;
    const T *qr = q_ref;
    for (int l = 0; l < o->nlevels; ++l) {
        if (l > 0) {
            TRY(transfer_t<T>(C, l - 1, true, qr, P.b[l], s));   // P.b[l] is free until the first cycle
            qr = P.b[l];
        }
        if (C->mbnk && l == o->nlevels - 1) {
            const FrLevel &L = C->L[l];
            TRY(mbnk_alloc_t<T>(C, l));
            TRY(elem_blocks_mbnk_t<T>(C, l, qr, shift, P.M[l], P.O, s));
            CK(cudaMemcpyAsync(P.Md, P.M[l], sizeof(T) * (size_t)L.E * L.nd * L.nd, cudaMemcpyDeviceToDevice, s));
        } else {
            TRY(elem_blocks_t<T>(C, l, qr, shift, P.M[l], s));
        }
        TRY(block_factor_t<T>(C, l, P.M[l], P.perm[l], s));
        TRY(half_factors(C, l, P.M[l], s));
    }
    return FR_OK;
}

static int pmg_setup_(fr_ctx *C, const double *q_ref, const fr_pmg_opts *o, cudaStream_t s) {
    NvtxRange nv("pmg setup");
    C->pmg_ready = 0;
    C->pmg_nlev = o->nlevels;
    for (int l = 0; l < o->nlevels; ++l) C->nsmooth[l] = o->nsmooth[l];
    C->pmg_c = o->c;
    C->pmg_ids = o->inv_dtau_star;
    C->pmg_prec = o->precision;
    if (C->has_comm && o->coarse_smoother == 1)
        return fail(FR_ERR_INVALID_ARG, "the matrix-based coarse smoother is not partitioned");
    C->mbnk = o->coarse_smoother == 1;
    C->mbnk_maxit = o->mbnk_maxit;
    C->mbnk_tol = o->mbnk_tol;
    C->pmg_gain = o->c + o->inv_dtau_star > 0.0 ? 1.0 / (o->c + o->inv_dtau_star) : 1.0;
    if (o->precision == 0 && !C->scale64) {
        TRY(pmg_alloc_t<double>(C, o->nlevels));
        TRY(pmg_factor_levels<double>(C, q_ref, o, s));
    } else {
        if (o->precision != 0) {
            TRY(ensure_levels32(C));
            TRY(pmg_alloc_t<float>(C, o->nlevels));
        } else {
            TRY(pmg_alloc_t<double>(C, o->nlevels));
            if (!C->x64s) TRY(dalloc_t(C, &C->x64s, C->L[0].ndof));
        }
        long long n = C->L[0].ndof;
        if (!C->ymax) TRY(dalloc_t(C, &C->ymax, 5));
        if (!C->xmax) TRY(dalloc_t(C, &C->xmax, 1));
        int rc_m = C->has_comm ? frk32_absmax_var_owned(C->nv, C->L[0].np, C->E, C->comm.n_owned, q_ref, C->ymax, s)
                               : frk32_absmax_var(C->nv, n / C->nv, q_ref, C->ymax, s);
        if (rc_m != 0) return fail(FR_ERR_CUDA, "absmax");
        TRY(allreduce_dev(C, C->ymax, C->nv, 1, s));
        CK(cudaMemcpyAsync(C->pmg_qref, C->ymax, sizeof(double) * C->nv, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        // per-variable magnitudes of the reference state, floored at 1e-3 of the largest
        // (a momentum component of a flow at rest); the cycle's first gain guess
        double qbig = 0.0, qsmall = INFINITY;
        for (int v = 0; v < C->nv; ++v) qbig = fmax(qbig, C->pmg_qref[v]);
        for (int v = 0; v < C->nv; ++v) {
            C->pmg_qref[v] = fmax(C->pmg_qref[v], 1e-3 * qbig);
            qsmall = fmin(qsmall, C->pmg_qref[v]);
        }
        if (!(qsmall > 0.0)) return fail(FR_ERR_INVALID_ARG, "reference state is zero");
        C->pmg_gain /= qsmall;
        if (o->precision != 0) {
            frk32_d2f(n, q_ref, C->q32, s);
            TRY(pmg_factor_levels<float>(C, C->q32, o, s));
        } else {
            TRY(pmg_factor_levels<double>(C, q_ref, o, s));
        }
    }
    int info = 0;
    CK(cudaMemcpyAsync(&info, C->info, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CKLAUNCH();
    if (info) return fail(FR_ERR_BREAKDOWN, "zero pivot in an element block");
    C->pmg_ready = 1;
    return FR_OK;
}

extern "C" int pmg_setup(fr_ctx *C, const double *q_ref, const fr_pmg_opts *o, void *stream) {
    if (!C || !q_ref || !o) return fail(FR_ERR_INVALID_ARG, "NULL argument");
    if (o->nlevels < 1 || o->nlevels > C->nlev) return fail(FR_ERR_INVALID_ARG, "nlevels %d outside 1..%d", o->nlevels, C->nlev);
    if (o->precision != 0 && o->precision != 1) return fail(FR_ERR_INVALID_ARG, "precision must be 0 (FP64) or 1 (FP32)");
    for (int l = 0; l < o->nlevels; ++l)
        if (o->nsmooth[l] < 0) return fail(FR_ERR_INVALID_ARG, "negative smoothing count");
    TRY(check_coarse_opts(o->coarse_smoother, o->mbnk_maxit, o->mbnk_tol));
    return pmg_setup_(C, q_ref, o, S_(stream));
}

// one matrix-based smoothing solve on level l, in place (x: r in, delta out): GMRES on
// A delta = r from 0, right-preconditioned by the factored diagonal blocks, at most
// mbnk_maxit iterations to the relative tolerance mbnk_tol (the stopping iteration is
// taken on the device; later iterations run and are ignored), delta = Md^{-1} V y
template <typename T>
static int mbnk_solve_t(fr_ctx *C, int l, T *x, cudaStream_t s) {
    PmgBuf<T> &P = pbuf<T>(C);
    FrLevelT<T> &L = levels<T>(C)[l];
    long long N = L.ndof;
    int m = C->mbnk_maxit, nf = 2 * C->d;
    frmb_start(N, x, P.V, C->mb_partial, C->mb_gm, s);
    for (int k = 0; k < m; ++k) {
        Kn<T>::copy(N, P.V + (size_t)k * N, P.mz, s);
        TRY(smoother_solve(C, l, P.mz, s));
        frmb_bsr_mv(L.E, L.nd, nf, C->nbr, P.Md, P.O, P.mz, P.mw, s);
        frmb_arnoldi(N, m, k, P.V, P.mw, C->mb_partial, C->mb_gm, s);
    }
    frmb_small_solve(m, C->mbnk_tol, C->mb_gm, s);
    frmb_combine(N, m, P.V, C->mb_gm, x, s);
    TRY(smoother_solve(C, l, x, s));
    return FR_OK;
}

extern "C" int fr_mbnk_operator(const fr_ctx *C, void *Md, void *O, void *stream) {
    if (!C || !Md || !O) return fail(FR_ERR_INVALID_ARG, "bad argument");
    if (!C->pmg_ready || !C->mbnk) return fail(FR_ERR_NOT_READY, "no pmg_setup with the matrix-based smoother");
    const FrLevel &L = C->L[C->pmg_nlev - 1];
    size_t nb = (size_t)L.E * L.nd * L.nd, es = C->pmg_prec ? sizeof(float) : sizeof(double);
    const void *src_M = C->pmg_prec ? (const void *)C->p32.Md : (const void *)C->p64.Md;
    const void *src_O = C->pmg_prec ? (const void *)C->p32.O : (const void *)C->p64.O;
    cudaStream_t s = S_(stream);
    CK(cudaMemcpyAsync(Md, src_M, es * nb, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(O, src_O, es * nb * 2 * C->d, cudaMemcpyDeviceToDevice, s));
    return FR_OK;
}

extern "C" int fr_mbnk_last(const fr_ctx *C, int *iters, double *relres) {
    if (!C || !C->mb_gm) return fail(FR_ERR_NOT_READY, "no matrix-based smoother has run");
    double g[2];
    CK(cudaMemcpy(g, C->mb_gm + FRMB_KUSED, sizeof(double) * 2, cudaMemcpyDeviceToHost));
    if (iters) *iters = (int)g[0];
    if (relres) *relres = g[1];
    return FR_OK;
}

// smoothing steps on level l: qh <- qh + M^{-1} (d - (c (qh - b) - (R(qh) - Rb))); on the
// coarsest level with the matrix-based smoother, M^{-1} is the GMRES solve with A
template <typename T>
static int smooth_t(fr_ctx *C, int l, int nsteps, const T *b, const T *Rb, const T *d, T *qh, bool first_is_base,
                    cudaStream_t s) {
    PmgBuf<T> &P = pbuf<T>(C);
    FrLevelT<T> &L = levels<T>(C)[l];
    for (int k = 0; k < nsteps; ++k) {
        if (k == 0 && first_is_base) Kn<T>::copy(L.ndof, d, P.rhs[l], s);
        else {
            TRY(residual_t<T>(C, l, qh, P.Rqh[l], s));
            Kn<T>::pmg_rhs(L.ndof, C->pmg_c, d, qh, b, P.Rqh[l], Rb, P.rhs[l], s);
        }
        if (C->mbnk && l == C->pmg_nlev - 1) TRY(mbnk_solve_t<T>(C, l, P.rhs[l], s));
        else TRY(smoother_solve(C, l, P.rhs[l], s));
        Kn<T>::add(L.ndof, qh, P.rhs[l], qh, s);
    }
    CKLAUNCH();
    return FR_OK;
}

template <typename T>
static int vcycle_t(fr_ctx *C, int l, const T *b, const T *Rb, const T *d, T *qh, cudaStream_t s) {
    NvtxRange nv(kVcycleRange[l]);
    PmgBuf<T> &P = pbuf<T>(C);
    int n = C->nsmooth[l];
    TRY(smooth_t<T>(C, l, n, b, Rb, d, qh, true, s));
    if (l + 1 >= C->pmg_nlev) return FR_OK;
    FrLevelT<T> &L = levels<T>(C)[l];
    FrLevelT<T> &L1 = levels<T>(C)[l + 1];
    T *r = P.rhs[l];
    if (n == 0) Kn<T>::copy(L.ndof, d, r, s);
    else {
        TRY(residual_t<T>(C, l, qh, P.Rqh[l], s));
        Kn<T>::pmg_rhs(L.ndof, C->pmg_c, d, qh, b, P.Rqh[l], Rb, r, s);
    }
    T *b1 = P.b[l + 1], *Rb1 = P.Rb[l + 1], *d1 = P.d[l + 1], *qh1 = P.qh[l + 1];
    TRY(transfer_t<T>(C, l, true, qh, b1, s));
    TRY(transfer_t<T>(C, l, true, r, d1, s));
    TRY(residual_t<T>(C, l + 1, b1, Rb1, s));
    Kn<T>::copy(L1.ndof, b1, qh1, s);
    TRY(vcycle_t<T>(C, l + 1, b1, Rb1, d1, qh1, s));
    Kn<T>::sub(L1.ndof, qh1, b1, qh1, s);
    TRY(transfer_t<T>(C, l, false, qh1, P.C[l], s));
    Kn<T>::add(L.ndof, qh, P.C[l], qh, s);
    TRY(smooth_t<T>(C, l, n, b, Rb, d, qh, false, s));
    return FR_OK;
}

// alpha: the FP32 cycle is driven with X scaled so that max_v ||Y_v||_inf / qref_v ~ alpha
// (qref_v: magnitude of variable v in the reference state).  FP32 rounding of R(qh) - R(q)
// perturbs the result by ~2.5e-5 / alpha relative (measured against the FP64 cycle at the
// same scale on stretched curved meshes); the cycle's own nonlinearity grows with alpha but
// leaves it a preconditioner (FGMRES takes a varying one).
// The scale needs the cycle's gain (relative ||Y|| per ||X||_inf): 1 / ((c + 1/dtau*) min_v
// qref_v) to start with (exact for a diagonally dominant operator), then the gain measured
// by the previous application.  If an application lands more than kMixedSlack away from
// the target (a small c, where the Jacobian and not c sets the gain), it is repeated once
// at the measured gain.
static const double kMixedAlpha = 1e-2;
static const double kMixedSlack = 30.0;

// nonlinear = true: the cycle is a nonlinear solver's update (pMG solver, pMG stage
// solver), whose X may not be scaled
static int pmg_apply(fr_ctx *C, const double *q, const double *Rq, const double *X, double *Y, cudaStream_t s,
                     bool nonlinear = false) {
    long long n = C->L[0].ndof;
    if (C->pmg_prec == 0 && (!C->scale64 || nonlinear)) {
        PmgBuf<double> &P = C->p64;
        frk64_copy(n, q, P.qh[0], s);
        TRY(vcycle_t<double>(C, 0, q, Rq, X, P.qh[0], s));
        frk64_sub(n, P.qh[0], q, Y, s);
        CKLAUNCH();
        return FR_OK;
    }
    if (C->pmg_prec == 0) {
        // the FP64 cycle driven like the FP32 one: X scaled so that the correction is about
        // kMixedAlpha of the state per variable, the result scaled back (for states whose
        // magnitude dwarfs a unit-norm Krylov vector, e.g. p ~ 1/(gamma Ma^2) at low Mach,
        // where an unscaled correction is lost in the rounding of R(q + Y) - R(q))
        PmgBuf<double> &P = C->p64;
        int rc_x = C->has_comm ? frk32_absmax_owned(n / C->E, C->E, C->comm.n_owned, X, C->xmax, s)
                               : frk32_absmax(n, X, C->xmax, s);
        if (rc_x != 0) return fail(FR_ERR_CUDA, "absmax");
        TRY(allreduce_dev(C, C->xmax, 1, 1, s));
        double xm;
        CK(cudaMemcpyAsync(&xm, C->xmax, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (!(xm > 0.0) || !isfinite(xm)) return fail(FR_ERR_NONFINITE, "preconditioner input max %g", xm);
        double want = kMixedAlpha, target = want / C->pmg_gain;
        for (int attempt = 0; attempt < 2; ++attempt) {
            if (attempt) target = want / C->pmg_gain;
            frk64_scale(n, target / xm, X, C->x64s, s);
            frk64_copy(n, q, P.qh[0], s);
            TRY(vcycle_t<double>(C, 0, q, Rq, C->x64s, P.qh[0], s));
            frk64_sub(n, P.qh[0], q, Y, s);
            int rc_y = C->has_comm ? frk32_absmax_var_owned(C->nv, C->L[0].np, C->E, C->comm.n_owned, Y, C->ymax, s)
                                   : frk32_absmax_var(C->nv, n / C->nv, Y, C->ymax, s);
            if (rc_y != 0) return fail(FR_ERR_CUDA, "absmax");
            TRY(allreduce_dev(C, C->ymax, C->nv, 1, s));
            double yv[5], ym = 0.0;
            CK(cudaMemcpyAsync(yv, C->ymax, sizeof(double) * C->nv, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            for (int v = 0; v < C->nv; ++v) ym = fmax(ym, yv[v] / C->pmg_qref[v]);
            if (!(ym > 0.0) || !isfinite(ym)) break;
            C->pmg_gain = ym / target;
            if (ym <= want * kMixedSlack && ym >= want / kMixedSlack) break;
        }
        frk64_scale(n, xm / target, Y, Y, s);
        CKLAUNCH();
        return FR_OK;
    }
    PmgBuf<float> &P = C->p32;
    int rc_x = C->has_comm ? frk32_absmax_owned(n / C->E, C->E, C->comm.n_owned, X, C->xmax, s)
                           : frk32_absmax(n, X, C->xmax, s);
    if (rc_x != 0) return fail(FR_ERR_CUDA, "absmax");
    TRY(allreduce_dev(C, C->xmax, 1, 1, s));
    if (C->q32_of != q) {
        frk32_d2f(n, q, C->q32, s);
        TRY(residual_t<float>(C, 0, C->q32, C->Rq32, s));
    }
    double want = kMixedAlpha, target = want / C->pmg_gain;
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (attempt) target = want / C->pmg_gain;
        frk32_d2f_scaled(n, X, C->xmax, target, C->x32, s);
        frk32_copy(n, C->q32, P.qh[0], s);
        TRY(vcycle_t<float>(C, 0, C->q32, C->Rq32, C->x32, P.qh[0], s));
        frk32_sub(n, P.qh[0], C->q32, C->y32, s);
        int rc_y = C->has_comm ? frk32_absmax_var_owned_f(C->nv, C->L[0].np, C->E, C->comm.n_owned, C->y32, C->ymax, s)
                               : frk32_absmax_var_f(C->nv, n / C->nv, C->y32, C->ymax, s);
        if (rc_y != 0) return fail(FR_ERR_CUDA, "absmax");
        TRY(allreduce_dev(C, C->ymax, C->nv, 1, s));
        double yv[5], ym = 0.0;
        CK(cudaMemcpyAsync(yv, C->ymax, sizeof(double) * C->nv, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int v = 0; v < C->nv; ++v) ym = fmax(ym, yv[v] / C->pmg_qref[v]);
        if (!(ym > 0.0) || !isfinite(ym)) break;
        C->pmg_gain = ym / target;
        if (ym <= want * kMixedSlack && ym >= want / kMixedSlack) break;
    }
    frk32_f2d_unscale(n, C->y32, C->xmax, target, Y, s);
    CKLAUNCH();
    return FR_OK;
}

extern "C" int pmg_precondition(fr_ctx *C, const double *q, const double *Rq, const double *X, double *Y, void *stream) {
    if (!C || !q || !Rq || !X || !Y) return fail(FR_ERR_INVALID_ARG, "NULL argument");
    if (!C->pmg_ready) return fail(FR_ERR_NOT_READY, "pmg_setup has not been called");
    if (Y == q || Y == Rq || Y == X) return fail(FR_ERR_INVALID_ARG, "Y must not alias the inputs");
    return pmg_apply(C, q, Rq, X, Y, S_(stream));
}

// ------------------------------------------------------------------------ FGMRES
// w . V_j on the finest level's [nv Np][E] vectors: over the owned elements, summed over
// the processes; the sums are left in C->dots on the device too (CGS2 reads them there)
static int dots(fr_ctx *C, long long n, int m, const double *w, const double *const *V, double *host, cudaStream_t s) {
    long long E = C->E, rows = n / E, own = C->has_comm ? C->comm.n_owned : E;
    if (frk64_multidot(rows, E, own, m, w, V, C->dots, C->partial, s) != 0) return fail(FR_ERR_OOM, "reduction");
    CKLAUNCH();
    CK(cudaMemcpyAsync(host, C->dots, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (C->has_comm) {
        if (C->comm.allreduce(C->comm.user, host, m, 0) != 0) return fail(FR_ERR_CUDA, "allreduce failed");
        CK(cudaMemcpyAsync(C->dots, host, sizeof(double) * m, cudaMemcpyHostToDevice, s));
    }
    return FR_OK;
}
static int norm2(fr_ctx *C, long long n, const double *w, double *out, cudaStream_t s) {
    const double *V[1] = {w};
    TRY(dots(C, n, 1, w, V, out, s));
    *out = sqrt(*out);
    return FR_OK;
}

static int gmres_alloc(fr_ctx *C, int kdim) {
    long long n = C->L[0].ndof;
    while ((int)C->V.size() < kdim + 1) {
        double *p;
        TRY(dalloc_t(C, &p, n));
        C->V.push_back(p);
    }
    while ((int)C->Z.size() < kdim) {
        double *p;
        TRY(dalloc_t(C, &p, n));
        C->Z.push_back(p);
    }
    if (!C->gw) { TRY(dalloc_t(C, &C->gw, n)); TRY(dalloc_t(C, &C->gr, n)); TRY(dalloc_t(C, &C->gtmp, n)); }
    return FR_OK;
}

static int gmres_(fr_ctx *C, const double *q, const double *Rq, const double *b, double *x, const fr_gmres_opts *o,
                  fr_gmres_stats *st, cudaStream_t s);

// q stays fixed through one FGMRES solve, so the FP32 cycle's copy of q and its FP32
// residual are formed by the first preconditioner application and reused by the rest
static int gmres(fr_ctx *C, const double *q, const double *Rq, const double *b, double *x, const fr_gmres_opts *o,
                 fr_gmres_stats *st, cudaStream_t s) {
    NvtxRange nv("fgmres");
    C->q32_of = nullptr;
    int rc = gmres_(C, q, Rq, b, x, o, st, s);
    C->q32_of = nullptr;
    return rc;
}

static int gmres_(fr_ctx *C, const double *q, const double *Rq, const double *b, double *x, const fr_gmres_opts *o,
                  fr_gmres_stats *st, cudaStream_t s) {
    int K = o->kdim;
    TRY(gmres_alloc(C, K));
    long long n = C->L[0].ndof;
    double *w = C->gw, *r = C->gr;
    std::vector<double> H((size_t)(K + 1) * K, 0.0), cs(K), sn(K), g(K + 1), y(K), h(K + 1), h2(K + 1);
    CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    frk64_copy(n, b, r, s);
    double bnorm, beta, est;
    TRY(norm2(C, n, b, &bnorm, s));
    beta = bnorm;
    est = bnorm;
    int total = 0, restarts = 0;
    fr_gmres_stats loc = {0, 0, 0.0};
    if (bnorm == 0.0) { if (st) *st = loc; return FR_OK; }
    if (!isfinite(bnorm)) return fail(FR_ERR_NONFINITE, "non-finite right-hand side");
    std::vector<const double *> Zp(K);
    for (;;) {
        frk64_scale(n, 1.0 / beta, r, C->V[0], s);   // FP64 division is slow: one reciprocal
        for (int j = 0; j <= K; ++j) g[j] = 0.0;
        g[0] = beta;
        int jj = 0;
        for (int j = 0; j < K; ++j) {
            const double *zj;
            if (o->use_pmg) {
                TRY(pmg_apply(C, q, Rq, C->V[j], C->Z[j], s));
                if (C->pmg_prec == 1) C->q32_of = q;
                double zn;
                TRY(norm2(C, n, C->Z[j], &zn, s));
                if (!(zn > 0.0) || !isfinite(zn)) return fail(FR_ERR_NONFINITE, "preconditioner output norm %g", zn);
                frk64_scale(n, 1.0 / zn, C->Z[j], C->Z[j], s);
                zj = C->Z[j];
            } else {
                zj = C->V[j];
            }
            Zp[j] = zj;
            TRY(jvp(C, q, Rq, zj, o->eps, o->shift, w, s));
            // CGS2
            const double *const *Vp = (const double *const *)C->V.data();
            TRY(dots(C, n, j + 1, w, Vp, h.data(), s));      // h also left in C->dots
            frk64_multi_axpy(n, j + 1, C->dots, Vp, w, s);
            TRY(dots(C, n, j + 1, w, Vp, h2.data(), s));
            frk64_multi_axpy(n, j + 1, C->dots, Vp, w, s);
            for (int i = 0; i <= j; ++i) H[(size_t)i * K + j] = h[i] + h2[i];
            double hn;
            TRY(norm2(C, n, w, &hn, s));
            if (!isfinite(hn)) return fail(FR_ERR_NONFINITE, "non-finite Arnoldi vector");
            H[(size_t)(j + 1) * K + j] = hn;
            if (hn > 0.0) frk64_scale(n, 1.0 / hn, w, C->V[j + 1], s);
            for (int i = 0; i < j; ++i) {
                double a = H[(size_t)i * K + j], bb = H[(size_t)(i + 1) * K + j];
                H[(size_t)i * K + j] = cs[i] * a + sn[i] * bb;
                H[(size_t)(i + 1) * K + j] = -sn[i] * a + cs[i] * bb;
            }
            double a = H[(size_t)j * K + j], bb = H[(size_t)(j + 1) * K + j];
            double rr = hypot(a, bb);
            cs[j] = a / rr; sn[j] = bb / rr;
            H[(size_t)j * K + j] = rr; H[(size_t)(j + 1) * K + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++total; jj = j + 1;
            est = fabs(g[j + 1]);
            if (est <= o->tol * bnorm || total >= o->maxit || hn == 0.0) break;
        }
        for (int i = jj - 1; i >= 0; --i) {
            double sacc = g[i];
            for (int k = i + 1; k < jj; ++k) sacc -= H[(size_t)i * K + k] * y[k];
            y[i] = sacc / H[(size_t)i * K + i];
        }
        frk64_update_x(n, jj, y.data(), Zp.data(), x, s);
        if (est <= o->tol * bnorm || total >= o->maxit) break;
        // restart: true residual of the current iterate starts the next cycle
        double xn;
        TRY(norm2(C, n, x, &xn, s));
        if (xn > 0.0) {
            frk64_scale(n, 1.0 / xn, x, r, s);
            TRY(jvp(C, q, Rq, r, o->eps, o->shift, w, s));
            frk64_scale(n, xn, w, C->gtmp, s);
            frk64_sub(n, b, C->gtmp, r, s);
        } else {
            frk64_copy(n, b, r, s);
        }
        TRY(norm2(C, n, r, &beta, s));
        if (!isfinite(beta)) return fail(FR_ERR_NONFINITE, "non-finite GMRES residual");
        ++restarts;
    }
    CK(cudaStreamSynchronize(s));
    loc.iters = total; loc.restarts = restarts; loc.relres = est / bnorm;
    if (st) *st = loc;
    return FR_OK;
}

extern "C" int gmres_solve(fr_ctx *C, const double *q, const double *Rq, const double *b, double *x,
                           const fr_gmres_opts *o, fr_gmres_stats *st, void *stream) {
    if (!C || !q || !Rq || !b || !x || !o) return fail(FR_ERR_INVALID_ARG, "NULL argument");
    if (o->kdim < 1 || o->kdim > 512 || o->maxit < 1) return fail(FR_ERR_INVALID_ARG, "kdim must be 1..512, maxit >= 1");
    if (o->use_pmg && !C->pmg_ready) return fail(FR_ERR_NOT_READY, "pmg_setup has not been called");
    if (x == b || x == q || x == Rq) return fail(FR_ERR_INVALID_ARG, "x must not alias the inputs");
    return gmres(C, q, Rq, b, x, o, st, S_(stream));
}

// --------------------------------------------------------------------- steppers
static int stepper_alloc(fr_ctx *C, int nvec) {
    long long n = C->L[0].ndof;
    while ((int)C->stv.size() < nvec) {
        double *p;
        TRY(dalloc_t(C, &p, n));
        C->stv.push_back(p);
    }
    return FR_OK;
}

static fr_gmres_opts gm_opts(const fr_solve_opts *o, double shift) {
    fr_gmres_opts g;
    g.kdim = o->kdim; g.maxit = o->maxit_gmres; g.use_pmg = o->use_pmg;
    g.tol = o->tol_gmres; g.eps = o->eps; g.shift = shift;
    return g;
}

static int check_solve_opts(const fr_ctx *C, const fr_solve_opts *o) {
    if (o->kdim < 1 || o->kdim > 512 || o->maxit_gmres < 1 || o->max_ptc < 0)
        return fail(FR_ERR_INVALID_ARG, "bad solver options");
    if (o->use_pmg && (o->nlevels < 1 || o->nlevels > C->nlev))
        return fail(FR_ERR_INVALID_ARG, "nlevels outside 1..%d", C->nlev);
    if (o->precision != 0 && o->precision != 1) return fail(FR_ERR_INVALID_ARG, "precision must be 0 or 1");
    if (o->use_pmg) TRY(check_coarse_opts(o->coarse_smoother, o->mbnk_maxit, o->mbnk_tol));
    if (o->nonlinear != 0 && o->nonlinear != 1) return fail(FR_ERR_INVALID_ARG, "nonlinear must be 0 (JFNK) or 1 (pMG)");
    if (o->nonlinear == 1 && (!o->use_pmg || o->precision != 0))
        return fail(FR_ERR_INVALID_ARG, "the pMG nonlinear solver needs use_pmg and the FP64 cycle (precision 0)");
    return FR_OK;
}

// --------------------------------------------------------------- initial guess
extern "C" int mlp_train_step(fr_mlp *M, int B, const unsigned short *X, const float *T, float lr, float *loss,
                              float *grads, void *stream);

static int mlp_sizes(const fr_ctx *C, int *K0, int *O) {
    const FrLevel &L = C->L[0];
    *O = L.nd;
    *K0 = ((4 * L.nd + L.np + 1) + 15) / 16 * 16;
    return FR_OK;
}

extern "C" int fr_mlp_dims(const fr_ctx *C, int *in_dim, int *out_dim) {
    if (!C || !in_dim || !out_dim) return fail(FR_ERR_INVALID_ARG, "NULL argument");
    return mlp_sizes(C, in_dim, out_dim);
}

extern "C" int fr_set_mlp(fr_ctx *C, fr_mlp *M) {
    if (!C) return fail(FR_ERR_INVALID_ARG, "NULL context");
    if (M) {
        int in, hid, out, K0, O;
        frkmlp_dims(M, &in, &hid, &out);
        mlp_sizes(C, &K0, &O);
        if (in != K0 || out != O) return fail(FR_ERR_INVALID_ARG, "network is %d -> %d, the context needs %d -> %d", in, out, K0, O);
    }
    C->mlp = M;
    C->mlp_steps = 0;
    return FR_OK;
}

extern "C" int fr_reset_history(fr_ctx *C) {
    if (!C) return fail(FR_ERR_INVALID_ARG, "NULL context");
    C->nhist = 0;
    C->hist_dt = 0.0;
    C->ring_n = 0;
    C->ring_head = 0;
    C->train_cursor = 0;
    return FR_OK;
}

static int ensure_guess_buffers(fr_ctx *C, int stages);

extern "C" int fr_guess_features(fr_ctx *C, const double *qn, const double *q1, const double *q2, const double *Rn,
                                 double dt, double c, unsigned short *X, double *scales, void *stream) {
    if (!C || !qn || !q1 || !q2 || !Rn || !X) return fail(FR_ERR_INVALID_ARG, "NULL argument");
    TRY(ensure_guess_buffers(C, 4));
    cudaStream_t s = S_(stream);
    const FrLevel &L0 = C->L[0];
    frkmlp_var_stats(L0.nv, (long long)L0.np * L0.E, qn, q1, C->qinf_dev, C->vpart, C->sdev, s);
    frkmlp_features(L0.E, L0.nv, L0.np, C->K0, qn, q1, q2, Rn, dt, L0.invJ, c, C->sdev, C->sdev + 5, C->qinf_dev, X,
                    s);
    CKLAUNCH();
    if (scales) CK(cudaMemcpyAsync(scales, C->sdev, sizeof(double) * 10, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return FR_OK;
}

static const int kRingSteps = 6;   // training ring: samples of the last six steps

static int ensure_guess_buffers(fr_ctx *C, int stages) {
    if (C->qex) return FR_OK;
    const FrLevel &L = C->L[0];
    long long n = L.ndof;
    mlp_sizes(C, &C->K0, &C->O);
    for (int k = 0; k < 3; ++k) TRY(dalloc_t(C, &C->hist[k], n));
    TRY(dalloc_t(C, &C->qex, n)); TRY(dalloc_t(C, &C->qcand, n));
    TRY(dalloc_t(C, &C->Rtmp, n)); TRY(dalloc_t(C, &C->Ftmp, n)); TRY(dalloc_t(C, &C->Fex, n));
    TRY(dalloc_t(C, &C->sdev, 16)); TRY(dalloc_t(C, &C->qinf_dev, 5)); TRY(dalloc_t(C, &C->vpart, 5 * 64 * 2));
    CK(cudaMemcpy(C->qinf_dev, C->ph.qinf, sizeof(double) * 5, cudaMemcpyHostToDevice));
    TRY(dalloc_t(C, &C->Xf, (size_t)L.E * C->K0));
    TRY(dalloc_t(C, &C->Yf, (size_t)L.E * C->O));
    TRY(dalloc_t(C, &C->Tf, (size_t)L.E * C->O));
    C->ring_cap = kRingSteps * (stages - 1) * L.E;
    TRY(dalloc_t(C, &C->ringX, (size_t)C->ring_cap * C->K0));
    TRY(dalloc_t(C, &C->ringT, (size_t)C->ring_cap * C->O));
    return FR_OK;
}

static void push_history(fr_ctx *C, const double *q, cudaStream_t s) {
    double *t = C->hist[0];
    C->hist[0] = C->hist[1];
    C->hist[1] = C->hist[2];
    C->hist[2] = t;
    frk64_copy(C->L[0].ndof, q, C->hist[2], s);
    if (C->nhist < 3) ++C->nhist;
}

// RMS(a_ii dt F(qc)) of a candidate stage state
static int stage_rms(fr_ctx *C, const double *qc, const double *sv, double adt, double *rms, cudaStream_t s) {
    long long n = C->L[0].ndof;
    TRY(residual(C, 0, qc, C->Rtmp, s));
    frk64_stage_F(n, qc, sv, adt, C->Rtmp, C->Ftmp, s);
    double fn;
    TRY(norm2(C, n, C->Ftmp, &fn, s));
    *rms = fabs(adt) * fn / sqrt(C->ndof_rms);
    if (!isfinite(*rms)) *rms = INFINITY;
    return FR_OK;
}

static void ring_append(fr_ctx *C, cudaStream_t s) {
    int E = C->L[0].E;
    for (int e0 = 0; e0 < E;) {
        int cnt = std::min(E - e0, C->ring_cap - C->ring_head);
        cudaMemcpyAsync(C->ringX + (size_t)C->ring_head * C->K0, C->Xf + (size_t)e0 * C->K0,
                        sizeof(unsigned short) * (size_t)cnt * C->K0, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(C->ringT + (size_t)C->ring_head * C->O, C->Tf + (size_t)e0 * C->O,
                        sizeof(float) * (size_t)cnt * C->O, cudaMemcpyDeviceToDevice, s);
        C->ring_head = (C->ring_head + cnt) % C->ring_cap;
        C->ring_n = std::min(C->ring_n + cnt, C->ring_cap);
        e0 += cnt;
    }
}

static int train_from_ring(fr_ctx *C, const fr_solve_opts *o, fr_step_stats *st, cudaStream_t s) {
    if (!C->mlp || C->ring_n == 0 || o->train_iters <= 0) return FR_OK;
    int B = std::min(o->train_batch > 0 ? o->train_batch : 4096, C->ring_n);
    float loss = 0.f;
    for (int it = 0; it < o->train_iters; ++it) {
        if (C->train_cursor + B > C->ring_n) C->train_cursor = 0;
        int rc = mlp_train_step(C->mlp, B, C->ringX + (size_t)C->train_cursor * C->K0,
                                C->ringT + (size_t)C->train_cursor * C->O, (float)o->lr,
                                it + 1 == o->train_iters ? &loss : nullptr, nullptr, s);
        if (rc != FR_OK) return rc;
        C->train_cursor += B;
    }
    C->mlp_steps += o->train_iters;
    if (st) st->train_loss = loss;
    return FR_OK;
}

extern "C" int esdirk_step(fr_ctx *C, const fr_esdirk_tableau *tab, double dt, double *q, const fr_solve_opts *o,
                           fr_step_stats *st, void *stream) {
    if (!C || !tab || !q || !o) return fail(FR_ERR_INVALID_ARG, "NULL argument");
    if (tab->stages < 2 || tab->stages > 6 || !(dt > 0.0)) return fail(FR_ERR_INVALID_ARG, "bad tableau or dt");
    TRY(check_solve_opts(C, o));
    if (o->guess < 0 || o->guess > 2) return fail(FR_ERR_INVALID_ARG, "guess must be 0, 1 or 2");
    if ((o->guess == 2 || o->train_iters > 0) && !C->mlp) return fail(FR_ERR_NOT_READY, "no network attached (fr_set_mlp)");
    if ((o->guess == 2 || o->train_iters > 0) && C->has_comm)
        return fail(FR_ERR_INVALID_ARG, "the network guess is not partitioned (its feature scales sum over all elements)");
    cudaStream_t s = S_(stream);
    int ns = tab->stages;
    TRY(stepper_alloc(C, ns + 5));
    long long n = C->L[0].ndof;
    const FrLevel &L0 = C->L[0];
    double *qn = C->stv[0], *sv = C->stv[1], *F = C->stv[2], *Rk = C->stv[3], *dq = C->stv[4];
    double **Rs = &C->stv[5];
    fr_step_stats loc;
    memset(&loc, 0, sizeof loc);
    loc.converged = 1;
    bool learn = o->guess > 0 || o->train_iters > 0;
    if (learn) {
        TRY(ensure_guess_buffers(C, ns));
        // the extrapolation and the network's features assume states spaced by this dt:
        // a history taken at another step (a caller that halved dt after a failed step)
        // restarts from the current state
        if (C->nhist >= 2 && C->hist_dt != 0.0 && fabs(C->hist_dt - dt) > 1e-12 * dt) C->nhist = 0;
        if (C->nhist == 0) {
            push_history(C, q, s);
            C->hist_dt = 0.0;
        }
    }
    bool have3 = learn && C->nhist >= 3;
    if (have3) frkmlp_var_stats(L0.nv, (long long)L0.np * L0.E, C->hist[2], C->hist[1], C->qinf_dev, C->vpart, C->sdev, s);
    frk64_copy(n, q, qn, s);
    TRY(residual(C, 0, qn, Rs[0], s));
    double aii = tab->A[1 * ns + 1];
    double c = 1.0 / o->dtau + 1.0 / (aii * dt);
    if (o->use_pmg) {
        fr_pmg_opts po;
        po.nlevels = o->nlevels;
        for (int l = 0; l < 4; ++l) po.nsmooth[l] = o->nsmooth[l];
        po.c = c;
        po.inv_dtau_star = o->inv_dtau_star;
        po.precision = o->precision;
        coarse_opts_copy(o, &po);
        TRY(pmg_setup_(C, qn, &po, s));
    }
    fr_gmres_opts go = gm_opts(o, c);
    int nguess_stages = 0;
    for (int i = 1; i < ns; ++i) {
        NvtxRange nv_stage("esdirk stage");
        double adt = tab->A[i * ns + i] * dt;
        double coef[6], ci = 0.0;
        for (int j = 0; j < i; ++j) coef[j] = tab->A[i * ns + j];
        for (int j = 0; j <= i; ++j) ci += tab->A[i * ns + j];
        frk64_lincomb(n, i, coef, (const double *const *)Rs, qn, dt, sv, s);
        frk64_copy(n, qn, q, s);
        if (have3) {
            // candidates judged by the FP64 stage residual: q^n (the paper's guess),
            // quadratic extrapolation in time, and the network's correction of it
            frkmlp_extrap(n, C->hist[2], C->hist[1], C->hist[0], ci, C->qex, s);
            frkmlp_features(L0.E, L0.nv, L0.np, C->K0, C->hist[2], C->hist[1], C->hist[0], Rs[0], dt, L0.invJ, ci,
                            C->sdev, C->sdev + 5, C->qinf_dev, C->Xf, s);
            if (o->guess >= 1) {
                double r[3] = {INFINITY, INFINITY, INFINITY};
                TRY(stage_rms(C, qn, sv, adt, &r[0], s));
                TRY(stage_rms(C, C->qex, sv, adt, &r[1], s));
                int best = r[1] < r[0] ? 1 : 0;
                if (o->guess == 2 && C->mlp_steps > 0) {
                    // the network's correction d = qnet - qex, scaled by the step beta that
                    // minimises the linearised ||F(qex + beta d)||: F(qnet) - F(qex) = J d
                    frk64_copy(n, C->Ftmp, C->Fex, s);
                    if (frkmlp_forward(C->mlp, L0.E, C->Xf, C->Yf, s) != 0) return fail(FR_ERR_OOM, "network activations");
                    frkmlp_guess(L0.E, L0.nv, L0.np, C->qex, C->sdev, C->Yf, C->qcand, s);
                    double rnet;
                    TRY(stage_rms(C, C->qcand, sv, adt, &rnet, s));
                    frk64_sub(n, C->Ftmp, C->Fex, C->Ftmp, s);
                    const double *V2[2] = {C->Fex, C->Ftmp};
                    double ab[2];
                    TRY(dots(C, n, 2, C->Ftmp, V2, ab, s));
                    double beta = ab[1] > 0.0 ? -ab[0] / ab[1] : 0.0;
                    beta = isfinite(beta) ? fmin(fmax(beta, -1.0), 2.0) : 0.0;
                    loc.guess_beta += beta;
                    double cf[2] = {1.0 - beta, beta};
                    const double *Xs[2] = {C->qex, C->qcand};
                    frk64_lincomb(n, 2, cf, Xs, nullptr, 1.0, C->qcand, s);
                    TRY(stage_rms(C, C->qcand, sv, adt, &r[2], s));
                    if (rnet < r[2]) {   // the linear model misjudged: keep the raw network guess
                        frkmlp_guess(L0.E, L0.nv, L0.np, C->qex, C->sdev, C->Yf, C->qcand, s);
                        r[2] = rnet;
                    }
                    if (r[2] < r[best]) best = 2;
                }
                for (int k = 0; k < 3; ++k) loc.guess_rms[k] += isfinite(r[k]) ? r[k] : 0.0;
                loc.guess_pick[best]++;
                ++nguess_stages;
                if (best == 1) frk64_copy(n, C->qex, q, s);
                else if (best == 2) frk64_copy(n, C->qcand, q, s);
            }
        }
        int conv = 0;
        double res = 0.0;
        for (int k = 0; k <= o->max_ptc; ++k) {
            TRY(residual(C, 0, q, Rk, s));
            frk64_stage_F(n, q, sv, adt, Rk, F, s);
            double fn;
            TRY(norm2(C, n, F, &fn, s));
            res = fabs(adt) * fn / sqrt(C->ndof_rms);
            if (!isfinite(res)) return fail(FR_ERR_NONFINITE, "non-finite stage residual (stage %d, iteration %d)", i, k);
            if (res <= o->tol_newton) { conv = 1; break; }
            if (k == o->max_ptc) break;
            NvtxRange nv_upd("pseudo-time update");
            frk64_neg(n, F, F, s);
            if (o->nonlinear == 1) {
                TRY(pmg_apply(C, q, Rk, F, dq, s, true));   // one V-cycle of the stage's pseudo-time equation
            } else {
                fr_gmres_stats gs;
                TRY(gmres(C, q, Rk, F, dq, &go, &gs, s));
                loc.n_gmres += gs.iters;
            }
            frk64_add(n, q, dq, q, s);
            loc.n_ptc++;
        }
        if (!conv) loc.converged = 0;
        loc.final_res = res;
        frk64_copy(n, Rk, Rs[i], s);
        if (have3 && o->train_iters > 0 && conv) {
            frkmlp_targets(L0.E, L0.nv, L0.np, q, C->qex, C->sdev, C->Tf, s);
            ring_append(C, s);
        }
    }
    for (int k = 0; k < 3 && nguess_stages; ++k) loc.guess_rms[k] /= nguess_stages;
    if (nguess_stages) loc.guess_beta /= nguess_stages;
    frk64_lincomb(n, ns, tab->b, (const double *const *)Rs, qn, dt, q, s);
    // only a converged step extends the history: a caller that undoes a failed step (and
    // retries it) finds the history as it was before the attempt
    if (learn && loc.converged) {
        push_history(C, q, s);
        C->hist_dt = dt;
    }
    if (o->train_iters > 0) TRY(train_from_ring(C, o, &loc, s));
    CKLAUNCH();
    CK(cudaStreamSynchronize(s));
    if (st) *st = loc;
    return loc.converged ? FR_OK : fail(FR_ERR_NOT_CONVERGED, "a stage did not reach the Newton tolerance");
}

extern "C" int row_step(fr_ctx *C, const fr_row_tableau *tab, double dt, double *q, const fr_solve_opts *o,
                        fr_step_stats *st, void *stream) {
    if (!C || !tab || !q || !o) return fail(FR_ERR_INVALID_ARG, "NULL argument");
    if (tab->stages < 1 || tab->stages > 6 || !(dt > 0.0) || !(tab->gamma > 0.0)) return fail(FR_ERR_INVALID_ARG, "bad tableau or dt");
    TRY(check_solve_opts(C, o));
    if (o->nonlinear != 0) return fail(FR_ERR_INVALID_ARG, "ROW stages are linear solves: nonlinear must be 0");
    cudaStream_t s = S_(stream);
    int ns = tab->stages;
    TRY(stepper_alloc(C, ns + 5));
    long long n = C->L[0].ndof;
    double *qn = C->stv[0], *Rn = C->stv[1], *qi = C->stv[2], *rhs = C->stv[3], *Ri = C->stv[4];
    double **Y = &C->stv[5];
    fr_step_stats loc;
    memset(&loc, 0, sizeof loc);
    loc.converged = 1;
    frk64_copy(n, q, qn, s);
    TRY(residual(C, 0, qn, Rn, s));
    double c = 1.0 / (tab->gamma * dt);
    if (o->use_pmg) {
        fr_pmg_opts po;
        po.nlevels = o->nlevels;
        for (int l = 0; l < 4; ++l) po.nsmooth[l] = o->nsmooth[l];
        po.c = c;
        po.inv_dtau_star = o->inv_dtau_star;
        po.precision = o->precision;
        coarse_opts_copy(o, &po);
        TRY(pmg_setup_(C, qn, &po, s));
    }
    fr_gmres_opts go = gm_opts(o, c);
    for (int i = 0; i < ns; ++i) {
        double coef[6];
        for (int j = 0; j < i; ++j) coef[j] = tab->a[i * ns + j];
        frk64_lincomb(n, i, coef, (const double *const *)Y, qn, 1.0, qi, s);
        if (i == 0) frk64_copy(n, Rn, Ri, s);
        else TRY(residual(C, 0, qi, Ri, s));
        for (int j = 0; j < i; ++j) coef[j] = tab->c[i * ns + j];
        frk64_lincomb(n, i, coef, (const double *const *)Y, nullptr, 1.0, rhs, s);
        frk64_add_div(n, Ri, rhs, dt, rhs, s);
        fr_gmres_stats gs;
        TRY(gmres(C, qn, Rn, rhs, Y[i], &go, &gs, s));
        loc.n_gmres += gs.iters;
        if (gs.relres > o->tol_gmres) loc.converged = 0;
        loc.final_res = gs.relres;
    }
    frk64_lincomb(n, ns, tab->m, (const double *const *)Y, qn, 1.0, q, s);
    CKLAUNCH();
    CK(cudaStreamSynchronize(s));
    if (st) *st = loc;
    return loc.converged ? FR_OK : fail(FR_ERR_NOT_CONVERGED, "a stage's linear solve missed its tolerance");
}

extern "C" int ptc_steady(fr_ctx *C, double *q, double dtau_init, double dtau_max, double tol_rel, int max_it,
                          const fr_solve_opts *o, fr_step_stats *st, double *hist, void *stream) {
    if (!C || !q || !o) return fail(FR_ERR_INVALID_ARG, "NULL argument");
    if (!(dtau_init > 0.0) || !(dtau_max >= dtau_init) || max_it < 0) return fail(FR_ERR_INVALID_ARG, "bad pseudo-time parameters");
    TRY(check_solve_opts(C, o));
    cudaStream_t s = S_(stream);
    TRY(stepper_alloc(C, 2));
    long long n = C->L[0].ndof;
    double *R = C->stv[0], *dq = C->stv[1];
    fr_step_stats loc;
    memset(&loc, 0, sizeof loc);
    loc.prec_switch_it = -1;
    int prec = o->precision, stall = 0;
    TRY(residual(C, 0, q, R, s));
    double r0, rk, dtau = dtau_init;
    TRY(norm2(C, n, R, &r0, s));
    rk = r0;
    if (hist) hist[0] = r0;
    for (int k = 0; k < max_it; ++k) {
        if (rk <= tol_rel * r0) break;
        double c = 1.0 / dtau;
        if (o->use_pmg) {
            fr_pmg_opts po;
            po.nlevels = o->nlevels;
            for (int l = 0; l < 4; ++l) po.nsmooth[l] = o->nsmooth[l];
            po.c = c;
            po.inv_dtau_star = o->inv_dtau_star < 0 ? c : o->inv_dtau_star;
            po.precision = prec;
            coarse_opts_copy(o, &po);
            TRY(pmg_setup_(C, q, &po, s));
        }
        fr_gmres_opts go = gm_opts(o, c);
        fr_gmres_stats gs;
        TRY(gmres(C, q, R, R, dq, &go, &gs, s));
        loc.n_gmres += gs.iters;
        frk64_add(n, q, dq, q, s);
        TRY(residual(C, 0, q, R, s));
        double rn;
        TRY(norm2(C, n, R, &rn, s));
        if (!isfinite(rn)) return fail(FR_ERR_NONFINITE, "non-finite residual at pseudo step %d", k);
        // FP32 preconditioner stalled (FGMRES used every iteration and the residual fell by
        // less than half, or five pseudo steps in a row each gained less than 10%): with
        // 1/dtau -> 0 the element blocks grow too ill-conditioned for FP32 LU, so the rest of
        // the pseudo-time march takes the FP64 cycle
        stall = rn > 0.9 * rk ? stall + 1 : 0;
        if (prec == 1 && o->use_pmg && !C->no_fallback && ((gs.iters >= o->maxit_gmres && rn > 0.5 * rk) || stall >= 5)) {
            prec = 0;
            loc.prec_switch_it = k + 1;
        }
        dtau = fmin(dtau * (rk / rn), dtau_max);
        rk = rn;
        loc.n_ptc++;
        if (hist) hist[k + 1] = rn;
    }
    loc.final_res = rk / r0;
    loc.converged = rk <= tol_rel * r0;
    if (st) *st = loc;
    return loc.converged ? FR_OK : fail(FR_ERR_NOT_CONVERGED, "steady PTC stopped at %g relative residual", loc.final_res);
}

// ------------------------------------------------------------------ checkpoints
// Library-side state of a time-stepping run: the learned guess's converged-state history
// and training ring, and the network's weights and Adam state.  Layout (host buffer):
// a header of 24 int64 (magic, version, sizes, counters), then the three history states
// (FP64), the ring's inputs (bf16) and targets (FP32), then the network (FP32 weights,
// first and second moments).
static const long long kCkMagic = 0x31504B43474D5046LL;   // "FPMGCKP1"
enum { CK_MAGIC, CK_VERSION, CK_E, CK_NV, CK_NP, CK_NDOF, CK_HAS_GUESS, CK_K0, CK_O, CK_NHIST, CK_RING_CAP,
       CK_RING_N, CK_RING_HEAD, CK_CURSOR, CK_MLP_STEPS, CK_HAS_MLP, CK_MLP_IN, CK_MLP_HID, CK_MLP_OUT, CK_MLP_T,
       CK_MLP_FLOATS, CK_HIST_DT, CK_NHEAD = 24 };

static long long ck_bytes(const fr_ctx *C, const fr_mlp *M) {
    long long b = 8LL * CK_NHEAD;
    if (C->qex) {
        b += 3LL * C->L[0].ndof * 8;
        b += (long long)C->ring_cap * C->K0 * 2 + (long long)C->ring_cap * C->O * 4;
    }
    if (M) b += frkmlp_state_floats(M) * 4;
    return b;
}

extern "C" int fr_checkpoint_size(const fr_ctx *C, const fr_mlp *M, long long *bytes) {
    if (!C || !bytes) return fail(FR_ERR_INVALID_ARG, "NULL argument");
    *bytes = ck_bytes(C, M);
    return FR_OK;
}

extern "C" int fr_checkpoint_save(const fr_ctx *C, const fr_mlp *M, void *buf, long long bytes) {
    if (!C || !buf) return fail(FR_ERR_INVALID_ARG, "NULL argument");
    if (bytes < ck_bytes(C, M)) return fail(FR_ERR_INVALID_ARG, "buffer of %lld bytes, %lld needed", bytes, ck_bytes(C, M));
    CK(cudaDeviceSynchronize());
    long long *h = (long long *)buf;
    memset(h, 0, 8 * CK_NHEAD);
    h[CK_MAGIC] = kCkMagic; h[CK_VERSION] = 1; h[CK_E] = C->E; h[CK_NV] = C->nv; h[CK_NP] = C->L[0].np;
    h[CK_NDOF] = C->L[0].ndof; h[CK_HAS_GUESS] = C->qex != nullptr; h[CK_K0] = C->K0; h[CK_O] = C->O;
    h[CK_NHIST] = C->nhist; h[CK_RING_CAP] = C->ring_cap; h[CK_RING_N] = C->ring_n; h[CK_RING_HEAD] = C->ring_head;
    h[CK_CURSOR] = C->train_cursor; h[CK_MLP_STEPS] = C->mlp_steps; h[CK_HAS_MLP] = M != nullptr;
    memcpy(&h[CK_HIST_DT], &C->hist_dt, sizeof(double));
    char *p = (char *)buf + 8 * CK_NHEAD;
    if (C->qex) {
        size_t sb = sizeof(double) * C->L[0].ndof;
        for (int k = 0; k < 3; ++k, p += sb) CK(cudaMemcpy(p, C->hist[k], sb, cudaMemcpyDeviceToHost));
        size_t xb = sizeof(unsigned short) * (size_t)C->ring_cap * C->K0, tb = sizeof(float) * (size_t)C->ring_cap * C->O;
        CK(cudaMemcpy(p, C->ringX, xb, cudaMemcpyDeviceToHost)); p += xb;
        CK(cudaMemcpy(p, C->ringT, tb, cudaMemcpyDeviceToHost)); p += tb;
    }
    if (M) {
        int d4[4];
        if (frkmlp_state_save(M, d4, (float *)p) != 0) return fail(FR_ERR_CUDA, "reading the network state");
        h[CK_MLP_IN] = d4[0]; h[CK_MLP_HID] = d4[1]; h[CK_MLP_OUT] = d4[2]; h[CK_MLP_T] = d4[3];
        h[CK_MLP_FLOATS] = frkmlp_state_floats(M);
    }
    return FR_OK;
}

extern "C" int fr_checkpoint_load(fr_ctx *C, fr_mlp *M, const void *buf, long long bytes) {
    if (!C || !buf || bytes < 8 * CK_NHEAD) return fail(FR_ERR_INVALID_ARG, "NULL or short buffer");
    const long long *h = (const long long *)buf;
    if (h[CK_MAGIC] != kCkMagic || h[CK_VERSION] != 1) return fail(FR_ERR_INVALID_ARG, "not a checkpoint of this version");
    if (h[CK_E] != C->E || h[CK_NV] != C->nv || h[CK_NP] != C->L[0].np || h[CK_NDOF] != C->L[0].ndof)
        return fail(FR_ERR_INVALID_ARG, "checkpoint of another mesh or degree");
    if (h[CK_HAS_MLP] && !M) return fail(FR_ERR_INVALID_ARG, "the checkpoint holds a network: pass one of its sizes");
    long long need = 8LL * CK_NHEAD;
    if (h[CK_HAS_GUESS])
        need += 3LL * h[CK_NDOF] * 8 + h[CK_RING_CAP] * h[CK_K0] * 2 + h[CK_RING_CAP] * h[CK_O] * 4;
    if (h[CK_HAS_MLP]) need += h[CK_MLP_FLOATS] * 4;
    if (bytes < need) return fail(FR_ERR_INVALID_ARG, "checkpoint truncated (%lld of %lld bytes)", bytes, need);
    const char *p = (const char *)buf + 8 * CK_NHEAD;
    if (h[CK_HAS_GUESS]) {
        int E = C->L[0].E;
        long long per_stage = (long long)kRingSteps * E;
        if (h[CK_RING_CAP] % per_stage) return fail(FR_ERR_INVALID_ARG, "checkpoint ring of another size");
        TRY(ensure_guess_buffers(C, (int)(h[CK_RING_CAP] / per_stage) + 1));
        if (C->ring_cap != h[CK_RING_CAP] || C->K0 != h[CK_K0] || C->O != h[CK_O])
            return fail(FR_ERR_INVALID_ARG, "checkpoint ring does not match this context's");
        size_t sb = sizeof(double) * C->L[0].ndof;
        for (int k = 0; k < 3; ++k, p += sb) CK(cudaMemcpy(C->hist[k], p, sb, cudaMemcpyHostToDevice));
        size_t xb = sizeof(unsigned short) * (size_t)C->ring_cap * C->K0, tb = sizeof(float) * (size_t)C->ring_cap * C->O;
        CK(cudaMemcpy(C->ringX, p, xb, cudaMemcpyHostToDevice)); p += xb;
        CK(cudaMemcpy(C->ringT, p, tb, cudaMemcpyHostToDevice)); p += tb;
        C->nhist = (int)h[CK_NHIST]; C->ring_n = (int)h[CK_RING_N]; C->ring_head = (int)h[CK_RING_HEAD];
        C->train_cursor = (int)h[CK_CURSOR];
        memcpy(&C->hist_dt, &h[CK_HIST_DT], sizeof(double));
    } else {
        C->nhist = 0; C->ring_n = 0; C->ring_head = 0; C->train_cursor = 0;
        C->hist_dt = 0.0;
    }
    C->mlp_steps = (int)h[CK_MLP_STEPS];
    if (h[CK_HAS_MLP]) {
        int d4[4] = {(int)h[CK_MLP_IN], (int)h[CK_MLP_HID], (int)h[CK_MLP_OUT], (int)h[CK_MLP_T]};
        if (frkmlp_state_floats(M) != h[CK_MLP_FLOATS] || frkmlp_state_load(M, d4, (const float *)p) != 0)
            return fail(FR_ERR_INVALID_ARG, "network of other sizes, or copy failed");
    }
    return FR_OK;
}

// The pMG nonlinear solver for steady problems (Sec. 3.1, Eqs. 11-16): one nonlinear
// V-cycle per iteration.  The preconditioner's cycle solves 0 = X + R(qh) - c (qh - q) -
// R(q); with X = R(q) that is the backward-Euler pseudo step R(qh) - c (qh - q) = 0, so an
// iteration is q <- q + P(q, R(q), R(q)) with c = 1/dtau and the SER rule of ptc_steady.
extern "C" int pmg_solve_steady(fr_ctx *C, double *q, double dtau_init, double dtau_max, double tol_rel, int max_it,
                                const fr_solve_opts *o, fr_step_stats *st, double *hist, void *stream) {
    if (!C || !q || !o) return fail(FR_ERR_INVALID_ARG, "NULL argument");
    if (!(dtau_init > 0.0) || !(dtau_max >= dtau_init) || max_it < 0) return fail(FR_ERR_INVALID_ARG, "bad pseudo-time parameters");
    if (o->nlevels < 1 || o->nlevels > C->nlev) return fail(FR_ERR_INVALID_ARG, "nlevels outside 1..%d", C->nlev);
    if (o->precision != 0)
        return fail(FR_ERR_UNIMPLEMENTED, "the nonlinear pMG solver runs the FP64 cycle (the FP32 cycle is scaled for "
                                          "preconditioning)");
    cudaStream_t s = S_(stream);
    TRY(stepper_alloc(C, 2));
    long long n = C->L[0].ndof;
    double *R = C->stv[0], *Y = C->stv[1];
    fr_step_stats loc;
    memset(&loc, 0, sizeof loc);
    loc.prec_switch_it = -1;
    TRY(residual(C, 0, q, R, s));
    double r0, rk, dtau = dtau_init;
    TRY(norm2(C, n, R, &r0, s));
    rk = r0;
    if (hist) hist[0] = r0;
    for (int k = 0; k < max_it; ++k) {
        if (rk <= tol_rel * r0) break;
        double c = 1.0 / dtau;
        fr_pmg_opts po;
        po.nlevels = o->nlevels;
        for (int l = 0; l < 4; ++l) po.nsmooth[l] = o->nsmooth[l];
        po.c = c;
        po.inv_dtau_star = o->inv_dtau_star < 0 ? c : o->inv_dtau_star;
        po.precision = 0;
        coarse_opts_copy(o, &po);
        TRY(pmg_setup_(C, q, &po, s));
        TRY(pmg_apply(C, q, R, R, Y, s, true));
        frk64_add(n, q, Y, q, s);
        TRY(residual(C, 0, q, R, s));
        double rn;
        TRY(norm2(C, n, R, &rn, s));
        if (!isfinite(rn)) return fail(FR_ERR_NONFINITE, "non-finite residual at iteration %d", k);
        dtau = fmin(dtau * (rk / rn), dtau_max);
        rk = rn;
        loc.n_ptc++;
        if (hist) hist[k + 1] = rn;
    }
    loc.final_res = rk / r0;
    loc.converged = rk <= tol_rel * r0;
    if (st) *st = loc;
    return loc.converged ? FR_OK : fail(FR_ERR_NOT_CONVERGED, "pMG solver stopped at %g relative residual", loc.final_res);
}

// -------------------------------------------------------------------- autotuner
// Launch shapes per (device, dimension, degree, precision, element count bucket): the CTA
// size of each of the 8 residual kernels and the columns in flight of the block solve.
// None of them changes a result bit; the autotuner times the candidates with CUDA events
// on the context's own levels and keeps the fastest (one coordinate-descent pass over the
// residual kernels, then G of the solve if that level's blocks are factored).
struct TuneKey {
    char dev[64];
    int d, p, prec, ebucket;
};
struct TuneVal {
    short tile[8];
    short lu_g;
};
static std::vector<std::pair<TuneKey, TuneVal>> g_tune;   // process-wide; guarded by g_tune_mu
static std::mutex g_tune_mu;

static int ebucket(long long E) {
    int b = 0;
    while ((1LL << (b + 1)) <= E) ++b;
    return b;
}
static TuneKey tune_key(const FrLevel &L, int prec) {
    TuneKey k;
    memset(&k, 0, sizeof k);
    cudaDeviceProp pr;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaGetDeviceProperties(&pr, dev) == cudaSuccess) snprintf(k.dev, sizeof k.dev, "%s", pr.name);
    for (char *c = k.dev; *c; ++c)
        if (*c == ' ' || *c == '|') *c = '_';
    k.d = L.d; k.p = L.p; k.prec = prec; k.ebucket = ebucket(L.E);
    return k;
}
static bool same_key(const TuneKey &a, const TuneKey &b) {
    return !strcmp(a.dev, b.dev) && a.d == b.d && a.p == b.p && a.prec == b.prec && a.ebucket == b.ebucket;
}
static bool tune_lookup(const TuneKey &k, TuneVal *out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto &x : g_tune)
        if (same_key(x.first, k)) { *out = x.second; return true; }
    return false;
}
static void tune_store(const TuneKey &k, const TuneVal &v) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto &x : g_tune)
        if (same_key(x.first, k)) { x.second = v; return; }
    g_tune.push_back({k, v});
}

template <typename T>
static int time_residual(fr_ctx *C, int l, const T *q, T *R, int reps, cudaEvent_t e0, cudaEvent_t e1, float *ms) {
    TRY(residual_t<T>(C, l, q, R, 0));
    CK(cudaEventRecord(e0, 0));
    for (int r = 0; r < reps; ++r) TRY(residual_t<T>(C, l, q, R, 0));
    CK(cudaEventRecord(e1, 0));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(ms, e0, e1));
    *ms /= reps;
    return FR_OK;
}

template <typename T>
static int tune_level(fr_ctx *C, int l, int prec, int reps, char *rep, size_t replen) {
    FrLevelT<T> &L = levels<T>(C)[l];
    const FrLevel &L64 = C->L[l];
    long long n = L64.ndof;
    // a state for timing: the free stream at every point
    std::vector<T> h((size_t)n);
    long long per = n / C->nv;
    for (int v = 0; v < C->nv; ++v)
        for (long long i = 0; i < per; ++i) h[(size_t)(v * per + i)] = (T)C->ph.qinf[v];
    T *q = nullptr, *R = nullptr;
    TRY(dalloc_t(C, &q, n));
    TRY(dalloc_t(C, &R, n));
    CK(cudaMemcpy(q, h.data(), sizeof(T) * n, cudaMemcpyHostToDevice));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    static const short cand[3] = {64, 128, 256};
    float t0 = 0.f, best = 0.f;
    int rc = time_residual<T>(C, l, q, R, reps, e0, e1, &t0);
    best = t0;
    for (int k = 0; rc == FR_OK && k < 8; ++k) {
        if (k == 5) continue;          // no kernel in this slot
        short keep = L.tile[k];
        for (short c : cand) {
            L.tile[k] = c;
            float t;
            rc = time_residual<T>(C, l, q, R, reps, e0, e1, &t);
            if (rc != FR_OK) break;
            if (t < best) { best = t; keep = c; }
        }
        L.tile[k] = keep;
    }
    // G of the block solve, on the factored blocks of this level if there are any
    float sg = -1.f;
    char gtimes[160] = "";
    PmgBuf<T> &P = pbuf<T>(C);
    if (rc == FR_OK && C->pmg_ready && C->pmg_prec == prec && l < C->pmg_nlev && P.M[l]) {
        static const short gc[4] = {1, 2, 4, 8};
        short keep = L.lu_g;
        for (short g : gc) {
            L.lu_g = g;
            CK(cudaMemset(P.rhs[l], 0, sizeof(T) * n));
            Kn<T>::solve(L, P.M[l], P.perm[l], P.rhs[l], 0);
            CK(cudaEventRecord(e0, 0));
            for (int r = 0; r < reps; ++r) Kn<T>::solve(L, P.M[l], P.perm[l], P.rhs[l], 0);
            CK(cudaEventRecord(e1, 0));
            CK(cudaEventSynchronize(e1));
            float t;
            CK(cudaEventElapsedTime(&t, e0, e1));
            t /= reps;
            size_t u = strlen(gtimes);
            snprintf(gtimes + u, sizeof gtimes - u, " %d:%.3f", g, t);
            if (sg < 0.f || t < sg) { sg = t; keep = g; }
        }
        L.lu_g = keep;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dfree(C, q);
    dfree(C, R);
    TRY(rc);
    CKLAUNCH();
    TuneKey key = tune_key(L64, prec);
    TuneVal val;
    memcpy(val.tile, L.tile, sizeof val.tile);
    val.lu_g = L.lu_g;
    tune_store(key, val);
    if (rep) {
        size_t u = strlen(rep);
        snprintf(rep + u, replen - u,
                 "d=%d p=%d %s E=%d: tiles %d %d %d %d %d %d %d %d, residual %.4f -> %.4f ms; solve G %d%s%s\n", L.d,
                 L.p, prec ? "fp32" : "fp64", L.E, L.tile[0], L.tile[1], L.tile[2], L.tile[3], L.tile[4], L.tile[5],
                 L.tile[6], L.tile[7], t0, best, L.lu_g, sg >= 0.f ? " (ms per G" : " (not tuned: no factored blocks)",
                 sg >= 0.f ? (std::string(gtimes) + ")").c_str() : "");
    }
    return FR_OK;
}

template <typename T>
static void apply_tune(fr_ctx *C, int l, const TuneVal &v) {
    FrLevelT<T> &L = levels<T>(C)[l];
    memcpy(L.tile, v.tile, sizeof v.tile);
    L.lu_g = v.lu_g;
}

// a new context (or its FP32 levels) takes the shapes already tuned for its key
static void apply_cached_tiles(fr_ctx *C, int prec) {
    for (int l = 0; l < C->nlev; ++l) {
        TuneVal v;
        if (tune_lookup(tune_key(C->L[l], prec), &v)) {
            if (prec) apply_tune<float>(C, l, v);
            else apply_tune<double>(C, l, v);
        }
    }
}

extern "C" int fr_autotune(fr_ctx *C, int flags, int reps, char *report, int report_len) {
    if (!C || reps < 1) return fail(FR_ERR_INVALID_ARG, "bad argument");
    if (report && report_len > 0) report[0] = 0;
    size_t rl = report && report_len > 0 ? (size_t)report_len : 0;
    char *rp = rl ? report : nullptr;
    for (int prec = 0; prec < 2; ++prec) {
        if (!(flags & (1 << prec))) continue;
        if (prec == 1) TRY(ensure_levels32(C));
        for (int l = 0; l < C->nlev; ++l) {
            TuneVal v;
            if (!(flags & 4) && tune_lookup(tune_key(C->L[l], prec), &v)) {
                if (prec) apply_tune<float>(C, l, v);
                else apply_tune<double>(C, l, v);
                if (rp) {
                    size_t u = strlen(rp);
                    snprintf(rp + u, rl - u, "d=%d p=%d %s E=%d: cached\n", C->L[l].d, C->L[l].p, prec ? "fp32" : "fp64",
                             C->L[l].E);
                }
                continue;
            }
            if (prec) TRY(tune_level<float>(C, l, 1, reps, rp, rl));
            else TRY(tune_level<double>(C, l, 0, reps, rp, rl));
        }
    }
    return FR_OK;
}

extern "C" int fr_get_tiles(const fr_ctx *C, int l, int prec, int *tiles) {
    if (!C || l < 0 || l >= C->nlev || !tiles || (prec != 0 && prec != 1)) return fail(FR_ERR_INVALID_ARG, "bad argument");
    const short *t = prec ? C->L32[l].tile : C->L[l].tile;
    for (int k = 0; k < 8; ++k) tiles[k] = t[k] > 0 ? t[k] : 128;
    tiles[8] = prec ? C->L32[l].lu_g : C->L[l].lu_g;
    return FR_OK;
}

extern "C" int fr_set_tiles(fr_ctx *C, int l, int prec, const int *tiles) {
    if (!C || l < 0 || l >= C->nlev || !tiles || (prec != 0 && prec != 1)) return fail(FR_ERR_INVALID_ARG, "bad argument");
    for (int k = 0; k < 8; ++k)
        if (tiles[k] != 0 && (tiles[k] < 32 || tiles[k] > 256 || tiles[k] % 32))
            return fail(FR_ERR_INVALID_ARG, "CTA size %d: a multiple of 32 in 32..256 (or 0)", tiles[k]);
    if (tiles[8] != 0 && tiles[8] != 1 && tiles[8] != 2 && tiles[8] != 4 && tiles[8] != 8)
        return fail(FR_ERR_INVALID_ARG, "solve G must be 0, 1 (bulk-copy kernel), 2, 4 or 8");
    if (prec == 1) TRY(ensure_levels32(C));
    short *t = prec ? C->L32[l].tile : C->L[l].tile;
    for (int k = 0; k < 8; ++k) t[k] = (short)tiles[k];
    (prec ? C->L32[l].lu_g : C->L[l].lu_g) = (short)tiles[8];
    return FR_OK;
}

extern "C" int fr_autotune_save(const char *path) {
    if (!path) return fail(FR_ERR_INVALID_ARG, "NULL path");
    FILE *f = fopen(path, "w");
    if (!f) return fail(FR_ERR_INVALID_ARG, "cannot write %s", path);
    fprintf(f, "# frpmg launch shapes: device d p precision log2E tile0..tile7 solveG\n");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto &x : g_tune) {
        fprintf(f, "%s %d %d %d %d", x.first.dev, x.first.d, x.first.p, x.first.prec, x.first.ebucket);
        for (int k = 0; k < 8; ++k) fprintf(f, " %d", x.second.tile[k]);
        fprintf(f, " %d\n", x.second.lu_g);
    }
    fclose(f);
    return FR_OK;
}

extern "C" int fr_autotune_load(const char *path) {
    if (!path) return fail(FR_ERR_INVALID_ARG, "NULL path");
    FILE *f = fopen(path, "r");
    if (!f) return fail(FR_ERR_INVALID_ARG, "cannot read %s", path);
    char line[512];
    int n = 0;
    while (fgets(line, sizeof line, f)) {
        if (line[0] == '#') continue;
        TuneKey k;
        TuneVal v;
        memset(&k, 0, sizeof k);
        int t[9];
        if (sscanf(line, "%63s %d %d %d %d %d %d %d %d %d %d %d %d %d", k.dev, &k.d, &k.p, &k.prec, &k.ebucket, &t[0],
                   &t[1], &t[2], &t[3], &t[4], &t[5], &t[6], &t[7], &t[8]) != 14)
            continue;
        bool ok = true;
        for (int i = 0; i < 8; ++i) ok &= t[i] == 0 || (t[i] >= 32 && t[i] <= 256 && t[i] % 32 == 0);
        ok &= t[8] == 0 || t[8] == 1 || t[8] == 2 || t[8] == 4 || t[8] == 8;
        if (!ok) continue;
        for (int i = 0; i < 8; ++i) v.tile[i] = (short)t[i];
        v.lu_g = (short)t[8];
        tune_store(k, v);
        ++n;
    }
    fclose(f);
    return FR_OK;
}

#include "batch_impl.h"
