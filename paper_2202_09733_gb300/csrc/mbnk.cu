// Matrix-based Newton-Krylov (MBNK) smoother of the coarsest pMG level (Sec. 3.2): the
// level's linearised operator A = shift I - dR/dq is assembled as element blocks (the
// diagonal blocks of the element-Jacobi smoother, kept unfactored, plus one block per
// face neighbour), and each smoothing step solves A delta = r by GMRES of at most m
// iterations to a relative tolerance, right-preconditioned by the LU-factored diagonal
// blocks.  Every scalar of the GMRES recurrence (inner products, the Hessenberg matrix,
// its Givens rotations, the stopping iteration) stays in device memory, so a smoothing
// step issues a fixed sequence of launches with no host synchronisation and can be
// captured in a CUDA graph; iterations past the stopping one are computed and ignored.
//
// Layouts: vectors [nd][E] (dof r = v Np + i, element fastest); diagonal blocks Md and
// neighbour blocks O column-major per block: Md[(e nd + j) nd + r],
// O[((e nf + f) nd + j) nd + r]; neighbour table nbr[f E + e] (-1: none).
#include <atomic>
#include <cuda_runtime.h>
#include <math.h>
#include <algorithm>
#include "fr_lib.h"

static std::atomic<unsigned long long> g_launches{0};
unsigned long long frmb_launch_count() { return g_launches; }
#define CNT() (g_launches.fetch_add(1, std::memory_order_relaxed))

#define MB_THREADS 256
#define MB_KMAX (FRMB_MAXIT + 1)

static inline int mb_blocks(long long n) {
    long long g = (n + MB_THREADS - 1) / MB_THREADS;
    return (int)std::max<long long>(1, std::min<long long>(g, FRMB_MAXBLK));
}

// ---------------------------------------------------------------- assembly (FP64)
// Column j of the neighbour blocks: for element e and slot f whose neighbour n has the
// colour col (one perturbed element at most among e and its neighbours: distance-2
// colouring), O_(e,f)[r][j] = -(Rp_e[r] - R0_e[r]) / eps_j, eps_j = epsrel max(1, |q_n,j|).
// One thread per (element, row), rows fastest across a warp for the block writes.
__global__ void k_nbr_column(int E, int nd, int nf, const int *nbr, const int *color2, int col, int j,
                             const double *q, const double *R0, const double *Rp, double epsrel, double *O) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)E * nd) return;
    int e = (int)(t / nd), r = (int)(t - (long long)e * nd);
    for (int f = 0; f < nf; ++f) {
        int n = nbr[(size_t)f * E + e];
        if (n < 0 || color2[n] != col) continue;
        double x = q[(size_t)j * E + n];
        double eps = epsrel * fmax(1.0, fabs(x));
        double m = (Rp[(size_t)r * E + e] - R0[(size_t)r * E + e]) / eps;
        O[(((size_t)e * nf + f) * nd + j) * nd + r] = -m;
    }
}
void frmb_nbr_column(int E, int nd, int nf, const int *nbr, const int *color2, int col, int j, const double *q,
                     const double *R0, const double *Rp, double epsrel, double *O, cudaStream_t s) {
    long long n = (long long)E * nd;
    CNT(); k_nbr_column<<<(unsigned)((n + MB_THREADS - 1) / MB_THREADS), MB_THREADS, 0, s>>>(E, nd, nf, nbr, color2,
                                                                                           col, j, q, R0, Rp, epsrel, O);
}

// ---------------------------------------------------------------- y = A x
// y_e[r] = sum_j Md_e[r][j] x_e[j] + sum_f sum_j O_(e,f)[r][j] x_nbr(e,f)[j]; one thread
// per (element, row), rows fastest so that a warp reads consecutive block entries
template <typename T>
__global__ void k_bsr_mv(int E, int nd, int nf, const int *nbr, const T *Md, const T *O, const T *x, T *y) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)E * nd) return;
    int e = (int)(t / nd), r = (int)(t - (long long)e * nd);
    const T *M = Md + (size_t)e * nd * nd + r;
    T acc = T(0);
    for (int j = 0; j < nd; ++j) acc = fma(M[(size_t)j * nd], x[(size_t)j * E + e], acc);
    for (int f = 0; f < nf; ++f) {
        int n = nbr[(size_t)f * E + e];
        if (n < 0) continue;
        const T *B = O + ((size_t)e * nf + f) * nd * nd + r;
        for (int j = 0; j < nd; ++j) acc = fma(B[(size_t)j * nd], x[(size_t)j * E + n], acc);
    }
    y[(size_t)r * E + e] = acc;
}
template <typename T>
static void bsr_mv(int E, int nd, int nf, const int *nbr, const T *Md, const T *O, const T *x, T *y, cudaStream_t s) {
    long long n = (long long)E * nd;
    CNT(); k_bsr_mv<T><<<(unsigned)((n + MB_THREADS - 1) / MB_THREADS), MB_THREADS, 0, s>>>(E, nd, nf, nbr, Md, O, x, y);
}
void frmb_bsr_mv(int E, int nd, int nf, const int *nbr, const double *Md, const double *O, const double *x, double *y,
                 cudaStream_t s) { bsr_mv(E, nd, nf, nbr, Md, O, x, y, s); }
void frmb_bsr_mv(int E, int nd, int nf, const int *nbr, const float *Md, const float *O, const float *x, float *y,
                 cudaStream_t s) { bsr_mv(E, nd, nf, nbr, Md, O, x, y, s); }

// ---------------------------------------------------------------- reductions
// partial[b * MB_KMAX + j] = sum over block b's grid-stride share of V_j[i] w[i], j < k
// (V_j = V + j N); FP64 accumulation for either vector type
template <typename T>
__global__ void __launch_bounds__(MB_THREADS) k_dots_partial(long long N, int k, const T *V, const T *w,
                                                             double *partial) {
    double acc[MB_KMAX];
#pragma unroll
    for (int j = 0; j < MB_KMAX; ++j) acc[j] = 0.0;
    for (long long i = blockIdx.x * (long long)MB_THREADS + threadIdx.x; i < N; i += (long long)gridDim.x * MB_THREADS) {
        double wi = (double)w[i];
#pragma unroll
        for (int j = 0; j < MB_KMAX; ++j)
            if (j < k) acc[j] = fma((double)V[(size_t)j * N + i], wi, acc[j]);
    }
    __shared__ double sh[MB_THREADS / 32][MB_KMAX];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < MB_KMAX; ++j) {
        if (j >= k) break;
        double v = acc[j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[wid][j] = v;
    }
    __syncthreads();
    if (threadIdx.x < k) {
        double t = 0.0;
        for (int q = 0; q < MB_THREADS / 32; ++q) t += sh[q][threadIdx.x];
        partial[(size_t)blockIdx.x * MB_KMAX + threadIdx.x] = t;
    }
}

// c[j] = sum_b partial[b][j] (fixed order); mode 0: h[j * ldh] = c[j]; mode 1: h[j * ldh] += c[j];
// mode 2 (a norm, k = 1): h[0] = sqrt(c[0])
__global__ void k_dots_final(int nblk, int k, const double *partial, double *c, double *h, int ldh, int mode) {
    int j = threadIdx.x;
    if (j >= k) return;
    double t = 0.0;
    for (int b = 0; b < nblk; ++b) t += partial[(size_t)b * MB_KMAX + j];
    c[j] = t;
    if (mode == 0) h[(size_t)j * ldh] = t;
    else if (mode == 1) h[(size_t)j * ldh] += t;
    else h[0] = sqrt(t);
}

// w -= sum_j c[j] V_j, j < k
template <typename T>
__global__ void k_gs_axpy(long long N, int k, const T *V, const double *c, T *w) {
    __shared__ double sc[MB_KMAX];
    if (threadIdx.x < k) sc[threadIdx.x] = c[threadIdx.x];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        double t = (double)w[i];
        for (int j = 0; j < k; ++j) t = fma(-sc[j], (double)V[(size_t)j * N + i], t);
        w[i] = (T)t;
    }
}

// v = w / h (v = 0 where h is not positive: a breakdown or a zero right-hand side)
template <typename T>
__global__ void k_scale_by(long long N, const T *w, const double *h, T *v) {
    double hv = *h;
    double inv = hv > 0.0 ? 1.0 / hv : 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        v[i] = (T)((double)w[i] * inv);
}

template <typename T>
static void gs_pass(long long N, int k, const T *V, T *w, double *partial, double *c, double *h, int ldh, int mode,
                    cudaStream_t s) {
    int nb = mb_blocks(N);
    CNT(); k_dots_partial<T><<<nb, MB_THREADS, 0, s>>>(N, k, V, w, partial);
    CNT(); k_dots_final<<<1, 32, 0, s>>>(nb, k, partial, c, h, ldh, mode);
    CNT(); k_gs_axpy<T><<<nb, MB_THREADS, 0, s>>>(N, k, V, c, w);
}
template <typename T>
static void norm_scale(long long N, const T *w, double *partial, double *c, double *h, T *v, cudaStream_t s) {
    int nb = mb_blocks(N);
    CNT(); k_dots_partial<T><<<nb, MB_THREADS, 0, s>>>(N, 1, w, w, partial);
    CNT(); k_dots_final<<<1, 32, 0, s>>>(nb, 1, partial, c, h, 1, 2);
    CNT(); k_scale_by<T><<<nb, MB_THREADS, 0, s>>>(N, w, h, v);
}

// Arnoldi step k: w = A z_k arrives in w; orthogonalise against V_0..V_k (classical
// Gram-Schmidt, two passes), h_(k+1,k) = ||w||, V_(k+1) = w / h_(k+1,k).  H[i * m + k].
void frmb_arnoldi(long long N, int m, int k, double *V, double *w, double *partial, double *gm, cudaStream_t s) {
    double *H = gm, *c = gm + FRMB_H;
    gs_pass<double>(N, k + 1, V, w, partial, c, H + k, m, 0, s);
    gs_pass<double>(N, k + 1, V, w, partial, c, H + k, m, 1, s);
    norm_scale<double>(N, w, partial, c, H + (size_t)(k + 1) * m + k, V + (size_t)(k + 1) * N, s);
}
void frmb_arnoldi(long long N, int m, int k, float *V, float *w, double *partial, double *gm, cudaStream_t s) {
    double *H = gm, *c = gm + FRMB_H;
    gs_pass<float>(N, k + 1, V, w, partial, c, H + k, m, 0, s);
    gs_pass<float>(N, k + 1, V, w, partial, c, H + k, m, 1, s);
    norm_scale<float>(N, w, partial, c, H + (size_t)(k + 1) * m + k, V + (size_t)(k + 1) * N, s);
}
// beta = ||r||, V_0 = r / beta
void frmb_start(long long N, const double *r, double *V, double *partial, double *gm, cudaStream_t s) {
    norm_scale<double>(N, r, partial, gm + FRMB_H, gm + FRMB_BETA, V, s);
}
void frmb_start(long long N, const float *r, float *V, double *partial, double *gm, cudaStream_t s) {
    norm_scale<float>(N, r, partial, gm + FRMB_H, gm + FRMB_BETA, V, s);
}

// ---------------------------------------------------------------- least squares
// One thread: Givens rotations over the m Hessenberg columns, the first k with
// |g_(k+1)| <= tol beta (else m), back substitution for y_0..y_(k-1), zeros beyond.
// Writes y, the iteration count and the residual estimate / beta.
__global__ void k_small_solve(int m, double tol, double *gm) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double *H = gm, *y = gm + FRMB_Y;
    double beta = gm[FRMB_BETA];
    double cs[FRMB_MAXIT], sn[FRMB_MAXIT], g[FRMB_MAXIT + 1], R[FRMB_MAXIT][FRMB_MAXIT];
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta;
    int kused = 0;
    for (int k = 0; k < m && beta > 0.0; ++k) {
        double col[FRMB_MAXIT + 1];
        for (int i = 0; i <= k + 1; ++i) col[i] = H[(size_t)i * m + k];
        for (int i = 0; i < k; ++i) {
            double a = col[i], b = col[i + 1];
            col[i] = cs[i] * a + sn[i] * b;
            col[i + 1] = -sn[i] * a + cs[i] * b;
        }
        double a = col[k], b = col[k + 1], rr = hypot(a, b);
        cs[k] = rr > 0.0 ? a / rr : 1.0;
        sn[k] = rr > 0.0 ? b / rr : 0.0;
        col[k] = rr;
        for (int i = 0; i <= k; ++i) R[i][k] = col[i];
        g[k + 1] = -sn[k] * g[k];
        g[k] = cs[k] * g[k];
        kused = k + 1;
        if (fabs(g[k + 1]) <= tol * beta) break;
    }
    for (int i = 0; i < m; ++i) y[i] = 0.0;
    for (int i = kused - 1; i >= 0; --i) {
        double t = g[i];
        for (int j = i + 1; j < kused; ++j) t = t - R[i][j] * y[j];
        y[i] = R[i][i] != 0.0 ? t / R[i][i] : 0.0;
    }
    gm[FRMB_KUSED] = (double)kused;
    gm[FRMB_REL] = beta > 0.0 ? fabs(g[kused]) / beta : 0.0;
}
void frmb_small_solve(int m, double tol, double *gm, cudaStream_t s) {
    CNT(); k_small_solve<<<1, 32, 0, s>>>(m, tol, gm);
}

// u = sum_j y_j V_j, j < m (the y past the stopping iteration are zero)
template <typename T>
__global__ void k_combine(long long N, int m, const T *V, const double *y, T *u) {
    __shared__ double sy[FRMB_MAXIT];
    if (threadIdx.x < m) sy[threadIdx.x] = y[threadIdx.x];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        double t = 0.0;
        for (int j = 0; j < m; ++j) t = fma(sy[j], (double)V[(size_t)j * N + i], t);
        u[i] = (T)t;
    }
}
void frmb_combine(long long N, int m, const double *V, const double *gm, double *u, cudaStream_t s) {
    CNT(); k_combine<double><<<mb_blocks(N), MB_THREADS, 0, s>>>(N, m, V, gm + FRMB_Y, u);
}
void frmb_combine(long long N, int m, const float *V, const double *gm, float *u, cudaStream_t s) {
    CNT(); k_combine<float><<<mb_blocks(N), MB_THREADS, 0, s>>>(N, m, V, gm + FRMB_Y, u);
}
