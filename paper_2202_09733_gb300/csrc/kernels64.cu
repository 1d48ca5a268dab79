// FP64 kernels of the JFNK-pMG hot path.  Compiled with -fmad=false: the only fused
// multiply-adds are the explicit fma() calls, so every result below depends only on the
// documented evaluation order (fma chains in ascending index), not on the compiler.
#include <cuda_runtime.h>
#include <stdio.h>
#include <algorithm>
#include "fr_device.cuh"
#include "fr_lib.h"

static unsigned long long g_launches = 0;
unsigned long long frk64_launch_count() { return g_launches; }
#define CNT() (++g_launches)

__constant__ FrTab<double> c_tab64[FR_MAXP + 1];
__constant__ double c_gam64[FR_MAXP + 1][FR_MAXP + 1][FR_MAXN][FR_MAXN];
__constant__ double c_pi64[FR_MAXP + 1][FR_MAXP + 1][FR_MAXN][FR_MAXN];

template <>
__device__ __forceinline__ const FrTab<double> &frtab<double>(int p) {
    return c_tab64[p];
}

int frk64_upload_tables(const FrTabH *tabs, const double *gam, const double *pi) {
    static_assert(sizeof(FrTabH) == sizeof(FrTab<double>), "table layout");
    if (cudaMemcpyToSymbol(c_tab64, tabs, sizeof(FrTab<double>) * (FR_MAXP + 1)) != cudaSuccess) return -1;
    size_t tsz = sizeof(double) * (FR_MAXP + 1) * (FR_MAXP + 1) * FR_MAXN * FR_MAXN;
    if (cudaMemcpyToSymbol(c_gam64, gam, tsz) != cudaSuccess) return -1;
    if (cudaMemcpyToSymbol(c_pi64, pi, tsz) != cudaSuccess) return -1;
    return 0;
}

static FrPhys<double> to_phys(const FrPhysH &h, const FrLevel &L) {
    FrPhys<double> p;
    p.gamma = h.gamma; p.gm1 = h.gm1; p.mu = h.mu; p.kappa = h.kappa; p.c23 = h.c23;
    for (int v = 0; v < 5; ++v) p.qinf[v] = h.qinf[v];
    p.etagL = L.etagL; p.etagR = L.etagR;
    return p;
}

// ------------------------------------------------------------------------ residual
template <int D, int P>
static void residual_t(const FrLevel &L, const FrPhys<double> &ph, const double *q, double *R, cudaStream_t s) {
    using S = Sh<D, P>;
    const int E = L.E, gx = (E + 127) / 128, gp = (L.npairs + 127) / 128;
    CNT(); k_interp<D, P, double><<<dim3(gx, S::nv * S::nfp), 128, 0, s>>>(q, L.qf, E);
    CNT(); k_pair_common<D, P, double><<<gp, 128, 0, s>>>(L.pairs, L.bc, L.npairs, L.qf, L.dq, E, ph);
    CNT(); k_grad_sp<D, P, double><<<dim3(gx, S::nv * S::np), 128, 0, s>>>(q, L.dq, L.G, L.Q, E);
    CNT(); k_grad_fp<D, P, double><<<dim3(gx, S::nv * S::nfp), 128, 0, s>>>(q, L.qf, L.dq, L.Gf, L.Qf, E, ph.etagL, ph.etagR);
    CNT(); k_pair_flux<D, P, double><<<gp, 128, 0, s>>>(L.pairs, L.bc, L.npairs, L.qf, L.Qf, L.Sf, L.fn, E, ph);
    CNT(); k_vflux<D, P, double><<<dim3(gx, S::np), 128, 0, s>>>(q, L.Q, L.S, L.Ft, E, ph);
    CNT(); k_face_ft<D, P, double><<<dim3(gx, S::nv * S::nfp), 128, 0, s>>>(L.Ft, L.Ftf, E);
    CNT(); k_div<D, P, double><<<dim3(gx, S::nv * S::np), 128, 0, s>>>(L.Ft, L.Ftf, L.fn, L.invJ, R, E);
}

int frk64_residual(const FrLevel &L, const FrPhysH &h, const double *q, double *R, cudaStream_t s) {
    FrPhys<double> ph = to_phys(h, L);
    if (L.d == 2) {
        switch (L.p) {
            case 1: residual_t<2, 1>(L, ph, q, R, s); return 0;
            case 2: residual_t<2, 2>(L, ph, q, R, s); return 0;
            case 3: residual_t<2, 3>(L, ph, q, R, s); return 0;
            case 4: residual_t<2, 4>(L, ph, q, R, s); return 0;
        }
    } else if (L.d == 3) {
        switch (L.p) {
            case 1: residual_t<3, 1>(L, ph, q, R, s); return 0;
            case 2: residual_t<3, 2>(L, ph, q, R, s); return 0;
            case 3: residual_t<3, 3>(L, ph, q, R, s); return 0;
        }
    }
    return -1;
}

// ------------------------------------------------------------------- elementwise
static inline int nblk(long long n, int b = 256) {
    long long g = (n + b - 1) / b;
    return (int)std::min<long long>(g, 152LL * 32);
}
#define GRID_STRIDE(i, n) for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

__global__ void k_axpy_perturb(long long n, const double *q, double eps, const double *v, double *qp) {
    GRID_STRIDE(i, n) qp[i] = q[i] + eps * v[i];
}
__global__ void k_jv_finish(long long n, double shift, const double *v, const double *Rp, const double *Rq, double eps,
                            double *Av) {
    GRID_STRIDE(i, n) Av[i] = shift * v[i] - (Rp[i] - Rq[i]) / eps;
}
__global__ void k_scale(long long n, double a, const double *x, double *y) { GRID_STRIDE(i, n) y[i] = x[i] * a; }
__global__ void k_div_scalar(long long n, const double *x, double a, double *y) { GRID_STRIDE(i, n) y[i] = x[i] / a; }
__global__ void k_copy(long long n, const double *x, double *y) { GRID_STRIDE(i, n) y[i] = x[i]; }
__global__ void k_add(long long n, const double *a, const double *b, double *y) { GRID_STRIDE(i, n) y[i] = a[i] + b[i]; }
__global__ void k_sub(long long n, const double *a, const double *b, double *y) { GRID_STRIDE(i, n) y[i] = a[i] - b[i]; }
__global__ void k_neg(long long n, const double *x, double *y) { GRID_STRIDE(i, n) y[i] = -x[i]; }
__global__ void k_pmg_rhs(long long n, double c, const double *d, const double *qh, const double *b, const double *Rqh,
                          const double *Rb, double *rhs) {
    GRID_STRIDE(i, n) {
        double t1 = qh[i] - b[i], t2 = Rqh[i] - Rb[i];
        rhs[i] = d[i] - (c * t1 - t2);
    }
}
__global__ void k_stage_F(long long n, const double *q, const double *sv, double adt, const double *R, double *F) {
    GRID_STRIDE(i, n) F[i] = (q[i] - sv[i]) / adt - R[i];
}
__global__ void k_add_div(long long n, const double *a, const double *acc, double dt, double *y) {
    GRID_STRIDE(i, n) y[i] = a[i] + acc[i] / dt;
}

struct Ptr8 { const double *p[8]; double c[8]; };

// y = base + scale * (sum_j coef_j X_j) ; acc as an fma chain over j (all m <= 8 in one pass)
__global__ void k_lincomb(long long n, int m, Ptr8 X, const double *base, double scale, int has_scale, double *y) {
    GRID_STRIDE(i, n) {
        double acc = 0.0;
        for (int j = 0; j < m; ++j) acc = fma(X.c[j], X.p[j][i], acc);
        double t = has_scale ? scale * acc : acc;
        y[i] = base ? base[i] + t : t;
    }
}

void frk64_axpy_perturb(long long n, const double *q, double eps, const double *v, double *qp, cudaStream_t s) {
    CNT(); k_axpy_perturb<<<nblk(n), 256, 0, s>>>(n, q, eps, v, qp);
}
void frk64_jv_finish(long long n, double shift, const double *v, const double *Rp, const double *Rq, double eps,
                     double *Av, cudaStream_t s) {
    CNT(); k_jv_finish<<<nblk(n), 256, 0, s>>>(n, shift, v, Rp, Rq, eps, Av);
}
void frk64_scale(long long n, double a, const double *x, double *y, cudaStream_t s) { CNT(); k_scale<<<nblk(n), 256, 0, s>>>(n, a, x, y); }
void frk64_div_scalar(long long n, const double *x, double a, double *y, cudaStream_t s) {
    CNT(); k_div_scalar<<<nblk(n), 256, 0, s>>>(n, x, a, y);
}
void frk64_copy(long long n, const double *x, double *y, cudaStream_t s) { CNT(); k_copy<<<nblk(n), 256, 0, s>>>(n, x, y); }
void frk64_add(long long n, const double *a, const double *b, double *y, cudaStream_t s) { CNT(); k_add<<<nblk(n), 256, 0, s>>>(n, a, b, y); }
void frk64_sub(long long n, const double *a, const double *b, double *y, cudaStream_t s) { CNT(); k_sub<<<nblk(n), 256, 0, s>>>(n, a, b, y); }
void frk64_neg(long long n, const double *x, double *y, cudaStream_t s) { CNT(); k_neg<<<nblk(n), 256, 0, s>>>(n, x, y); }
void frk64_pmg_rhs(long long n, double c, const double *d, const double *qh, const double *b, const double *Rqh,
                   const double *Rb, double *rhs, cudaStream_t s) {
    CNT(); k_pmg_rhs<<<nblk(n), 256, 0, s>>>(n, c, d, qh, b, Rqh, Rb, rhs);
}
void frk64_stage_F(long long n, const double *q, const double *sv, double adt, const double *R, double *F, cudaStream_t s) {
    CNT(); k_stage_F<<<nblk(n), 256, 0, s>>>(n, q, sv, adt, R, F);
}
void frk64_add_div(long long n, const double *a, const double *acc, double dt, double *y, cudaStream_t s) {
    CNT(); k_add_div<<<nblk(n), 256, 0, s>>>(n, a, acc, dt, y);
}
void frk64_lincomb(long long n, int m, const double *coef, const double *const *X, const double *base, double scale,
                   double *y, cudaStream_t s) {
    // m <= 8 (time-integration stages)
    Ptr8 P;
    for (int j = 0; j < 8; ++j) { P.p[j] = j < m ? X[j] : nullptr; P.c[j] = j < m ? coef[j] : 0.0; }
    CNT(); k_lincomb<<<nblk(n), 256, 0, s>>>(n, m, P, base, scale, scale != 1.0, y);
}

// ------------------------------------------------------------------- reductions
// Partial sums per block (fixed grid for a given n), then one block sums the partials in
// block order.  Block reduction: warp shuffle tree, then warp 0 over the warp sums.
#define RED_THREADS 256
static inline int red_blocks(long long n) {
    long long g = (n + RED_THREADS * 4 - 1) / (RED_THREADS * 4);
    return (int)std::max<long long>(1, std::min<long long>(g, 152LL * 8));
}

template <int M>
__global__ void __launch_bounds__(RED_THREADS) k_multidot_partial(long long n, const double *w, Ptr8 V, double *partial) {
    double acc[M];
#pragma unroll
    for (int j = 0; j < M; ++j) acc[j] = 0.0;
    GRID_STRIDE(i, n) {
        double wi = w[i];
#pragma unroll
        for (int j = 0; j < M; ++j) acc[j] = fma(wi, V.p[j][i], acc[j]);
    }
    __shared__ double sh[RED_THREADS / 32][M];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < M; ++j) {
        double v = acc[j];
        for (int o = 16; o > 0; o >>= 1) v = v + __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[wid][j] = v;
    }
    __syncthreads();
    if (threadIdx.x < M) {
        double t = 0.0;
        for (int k = 0; k < RED_THREADS / 32; ++k) t = t + sh[k][threadIdx.x];
        partial[(size_t)blockIdx.x * 8 + threadIdx.x] = t;
    }
}

__global__ void k_multidot_final(int nb, int m, const double *partial, double *out) {
    int j = threadIdx.x;
    if (j >= m) return;
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t = t + partial[(size_t)b * 8 + j];
    out[j] = t;
}

static double *g_partial = nullptr;
static int g_partial_n = 0;

int frk64_multidot(long long n, int m, const double *w, const double *const *V, double *out, cudaStream_t s) {
    int nb = red_blocks(n);
    if (g_partial_n < nb * 8) {
        if (g_partial) cudaFree(g_partial);
        if (cudaMalloc(&g_partial, sizeof(double) * nb * 8) != cudaSuccess) { g_partial = nullptr; g_partial_n = 0; return -1; }
        g_partial_n = nb * 8;
    }
    for (int j0 = 0; j0 < m; j0 += 8) {
        int mm = std::min(8, m - j0);
        Ptr8 P;
        for (int j = 0; j < 8; ++j) { P.p[j] = j < mm ? V[j0 + j] : nullptr; P.c[j] = 0.0; }
        switch (mm) {
            case 1: { CNT(); k_multidot_partial<1><<<nb, RED_THREADS, 0, s>>>(n, w, P, g_partial); break; }
            case 2: { CNT(); k_multidot_partial<2><<<nb, RED_THREADS, 0, s>>>(n, w, P, g_partial); break; }
            case 3: { CNT(); k_multidot_partial<3><<<nb, RED_THREADS, 0, s>>>(n, w, P, g_partial); break; }
            case 4: { CNT(); k_multidot_partial<4><<<nb, RED_THREADS, 0, s>>>(n, w, P, g_partial); break; }
            case 5: { CNT(); k_multidot_partial<5><<<nb, RED_THREADS, 0, s>>>(n, w, P, g_partial); break; }
            case 6: { CNT(); k_multidot_partial<6><<<nb, RED_THREADS, 0, s>>>(n, w, P, g_partial); break; }
            case 7: { CNT(); k_multidot_partial<7><<<nb, RED_THREADS, 0, s>>>(n, w, P, g_partial); break; }
            default: { CNT(); k_multidot_partial<8><<<nb, RED_THREADS, 0, s>>>(n, w, P, g_partial); break; }
        }
        CNT(); k_multidot_final<<<1, 32, 0, s>>>(nb, mm, g_partial, out + j0);
    }
    return 0;
}

__global__ void k_multi_axpy(long long n, int m, const double *h, Ptr8 V, double *w) {
    GRID_STRIDE(i, n) {
        double t = w[i];
        for (int j = 0; j < m; ++j) t = fma(-h[j], V.p[j][i], t);
        w[i] = t;
    }
}
void frk64_multi_axpy(long long n, int m, const double *h_dev, const double *const *V, double *w, cudaStream_t s) {
    for (int j0 = 0; j0 < m; j0 += 8) {
        int mm = std::min(8, m - j0);
        Ptr8 P;
        for (int j = 0; j < 8; ++j) { P.p[j] = j < mm ? V[j0 + j] : nullptr; P.c[j] = 0.0; }
        CNT(); k_multi_axpy<<<nblk(n), 256, 0, s>>>(n, mm, h_dev + j0, P, w);
    }
}
__global__ void k_update_x(long long n, int m, Ptr8 Z, double *x) {
    GRID_STRIDE(i, n) {
        double t = x[i];
        for (int j = 0; j < m; ++j) t = fma(Z.c[j], Z.p[j][i], t);
        x[i] = t;
    }
}
void frk64_update_x(long long n, int m, const double *y, const double *const *Z, double *x, cudaStream_t s) {
    for (int j0 = 0; j0 < m; j0 += 8) {
        int mm = std::min(8, m - j0);
        Ptr8 P;
        for (int j = 0; j < 8; ++j) { P.p[j] = j < mm ? Z[j0 + j] : nullptr; P.c[j] = j < mm ? y[j0 + j] : 0.0; }
        CNT(); k_update_x<<<nblk(n), 256, 0, s>>>(n, mm, P, x);
    }
}

// ------------------------------------------------------------------ element blocks
// column j of the blocks of every element of colour `col`: forward difference with the
// step 1e-7 max(1, |q_j|) on that element alone (elements of one colour share no face,
// so their perturbations do not interact in R restricted to each of them).
__global__ void k_perturb_color(int E, const int *color, int col, int j, const double *q, double *qp) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E || color[e] != col) return;
    double x = q[(size_t)j * E + e];
    double eps = 1e-7 * fmax(1.0, fabs(x));
    qp[(size_t)j * E + e] = x + eps;
}
__global__ void k_restore_color(int E, const int *color, int col, int j, const double *q, double *qp) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E || color[e] != col) return;
    qp[(size_t)j * E + e] = q[(size_t)j * E + e];
}
// tile: 32 elements x 32 rows through shared memory (coalesced on both sides)
__global__ void __launch_bounds__(256) k_block_column(int E, int nd, const int *color, int col, int j, const double *q,
                                                      const double *R0, const double *Rp, double shift, double *M) {
    __shared__ double tile[32][33];
    __shared__ int s_col[32];
    __shared__ double s_eps[32];
    int e0 = blockIdx.x * 32, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    if (threadIdx.x < 32) {
        int e = e0 + tx;
        int ok = e < E && color[e] == col;
        s_col[tx] = ok;
        double x = ok ? q[(size_t)j * E + e] : 0.0;
        s_eps[tx] = 1e-7 * fmax(1.0, fabs(x));
    }
    __syncthreads();
    for (int r0 = 0; r0 < nd; r0 += 32) {
        for (int rr = ty; rr < 32; rr += 8) {
            int r = r0 + rr, e = e0 + tx;
            double val = 0.0;
            if (r < nd && e < E && s_col[tx]) {
                double m = (Rp[(size_t)r * E + e] - R0[(size_t)r * E + e]) / s_eps[tx];
                val = (r == j) ? shift - m : -m;
            }
            tile[rr][tx] = val;
        }
        __syncthreads();
        for (int ee = ty; ee < 32; ee += 8) {
            int e = e0 + ee, r = r0 + tx;
            if (e < E && s_col[ee] && r < nd) M[((size_t)e * nd + j) * nd + r] = tile[tx][ee];
        }
        __syncthreads();
    }
}
void frk64_perturb_color(const FrLevel &L, const int *color, int col, int j, const double *q, double *qp, cudaStream_t s) {
    CNT(); k_perturb_color<<<(L.E + 255) / 256, 256, 0, s>>>(L.E, color, col, j, q, qp);
}
void frk64_restore_color(const FrLevel &L, const int *color, int col, int j, const double *q, double *qp, cudaStream_t s) {
    CNT(); k_restore_color<<<(L.E + 255) / 256, 256, 0, s>>>(L.E, color, col, j, q, qp);
}
void frk64_block_column(const FrLevel &L, const int *color, int col, int j, const double *q, const double *R0,
                        const double *Rp, double shift, double *M, cudaStream_t s) {
    CNT(); k_block_column<<<(L.E + 31) / 32, 256, 0, s>>>(L.E, L.nd, color, col, j, q, R0, Rp, shift, M);
}

// ------------------------------------------------------------------------ block LU
// One CTA per element block, column-major A(r, c) = A[c * nd + r]; right-looking
// elimination with partial pivoting (first maximal |a|, whole rows swapped),
// multipliers l = a / pivot, trailing updates a = fma(-l, u, a) in elimination order.
template <bool SMEM>
__global__ void __launch_bounds__(256) k_lu_factor(double *M, int *perm, int nd, int *info) {
    extern __shared__ double dsm[];
    __shared__ double s_best[8];
    __shared__ int s_idx[8];
    __shared__ int s_p;
    int e = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    double *Ag = M + (size_t)e * nd * nd;
    double *A = SMEM ? dsm : Ag;
    int *pv = perm + (size_t)e * nd;
    if (SMEM)
        for (int t = tid; t < nd * nd; t += nt) A[t] = Ag[t];
    for (int t = tid; t < nd; t += nt) pv[t] = t;
    __syncthreads();
    int lane = tid & 31, wid = tid >> 5;
    for (int k = 0; k < nd; ++k) {
        // pivot: largest |a(i,k)|, i >= k, smallest index among equals
        double best = -1.0;
        int bi = nd;
        for (int i = k + tid; i < nd; i += nt) {
            double a = fabs(A[(size_t)k * nd + i]);
            if (a > best) { best = a; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            double ob = __shfl_down_sync(0xffffffffu, best, o);
            int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) { s_best[wid] = best; s_idx[wid] = bi; }
        __syncthreads();
        if (tid == 0) {
            double b = s_best[0];
            int ix = s_idx[0];
            for (int w = 1; w < nt / 32; ++w)
                if (s_best[w] > b || (s_best[w] == b && s_idx[w] < ix)) { b = s_best[w]; ix = s_idx[w]; }
            if (ix >= nd) ix = k;
            s_p = ix;
            if (b == 0.0) atomicExch(info, 1);
            if (ix != k) { int t = pv[k]; pv[k] = pv[ix]; pv[ix] = t; }
        }
        __syncthreads();
        int p = s_p;
        if (p != k)
            for (int c = tid; c < nd; c += nt) {
                double t = A[(size_t)c * nd + k];
                A[(size_t)c * nd + k] = A[(size_t)c * nd + p];
                A[(size_t)c * nd + p] = t;
            }
        __syncthreads();
        double piv = A[(size_t)k * nd + k];
        for (int i = k + 1 + tid; i < nd; i += nt) A[(size_t)k * nd + i] = A[(size_t)k * nd + i] / piv;
        __syncthreads();
        int m = nd - k - 1;
        for (int t = tid; t < m * m; t += nt) {
            int c = k + 1 + t / m, i = k + 1 + t % m;
            A[(size_t)c * nd + i] = fma(-A[(size_t)k * nd + i], A[(size_t)c * nd + k], A[(size_t)c * nd + i]);
        }
        __syncthreads();
    }
    if (SMEM)
        for (int t = tid; t < nd * nd; t += nt) Ag[t] = A[t];
}

int frk64_lu_factor(const FrLevel &L, double *M, int *perm, int *info, cudaStream_t s) {
    size_t sm = sizeof(double) * (size_t)L.nd * L.nd;
    if (sm <= 200 * 1024) {
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_lu_factor<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            attr = true;
        }
        CNT(); k_lu_factor<true><<<L.E, 256, sm, s>>>(M, perm, L.nd, info);
    } else {
        CNT(); k_lu_factor<false><<<L.E, 256, 0, s>>>(M, perm, L.nd, info);
    }
    return 0;
}

// One warp per element: rows i = lane + 32 s held in registers.  Forward substitution
// with the unit lower factor applies y_k to every later row in ascending k; backward
// substitution applies x_k to every earlier row in descending k (the order the unknowns
// become known), x_k = b_k / u_kk.
template <int NR>
__global__ void __launch_bounds__(128) k_lu_solve(const double *M, const int *perm, double *x, int nd, int E) {
    int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (e >= E) return;
    const double *A = M + (size_t)e * nd * nd;
    const int *pv = perm + (size_t)e * nd;
    double b[NR];
#pragma unroll
    for (int s = 0; s < NR; ++s) {
        int i = lane + 32 * s;
        b[s] = i < nd ? x[(size_t)pv[i] * E + e] : 0.0;
    }
    for (int k = 0; k < nd; ++k) {
        int owner = k & 31, slot = k >> 5;
        double v = b[0];
#pragma unroll
        for (int s = 1; s < NR; ++s) if (s == slot) v = b[s];
        double yk = __shfl_sync(0xffffffffu, v, owner);
        const double *col = A + (size_t)k * nd;
#pragma unroll
        for (int s = 0; s < NR; ++s) {
            int i = lane + 32 * s;
            if (i > k && i < nd) b[s] = fma(-col[i], yk, b[s]);
        }
    }
    for (int k = nd - 1; k >= 0; --k) {
        int owner = k & 31, slot = k >> 5;
        const double *col = A + (size_t)k * nd;
        double v = b[0];
#pragma unroll
        for (int s = 1; s < NR; ++s) if (s == slot) v = b[s];
        double xk = 0.0;
        if (lane == owner) xk = v / col[k];
        xk = __shfl_sync(0xffffffffu, xk, owner);
#pragma unroll
        for (int s = 0; s < NR; ++s) {
            int i = lane + 32 * s;
            if (i == k) b[s] = xk;
            else if (i < k) b[s] = fma(-col[i], xk, b[s]);
        }
    }
    __syncwarp();
#pragma unroll
    for (int s = 0; s < NR; ++s) {
        int i = lane + 32 * s;
        if (i < nd) x[(size_t)i * E + e] = b[s];
    }
}

int frk64_lu_solve(const FrLevel &L, const double *M, const int *perm, double *x, cudaStream_t s) {
    int nr = (L.nd + 31) / 32;
    int grid = (L.E * 32 + 127) / 128;
    switch (nr) {
        case 1: { CNT(); k_lu_solve<1><<<grid, 128, 0, s>>>(M, perm, x, L.nd, L.E); break; }
        case 2: { CNT(); k_lu_solve<2><<<grid, 128, 0, s>>>(M, perm, x, L.nd, L.E); break; }
        case 3: { CNT(); k_lu_solve<3><<<grid, 128, 0, s>>>(M, perm, x, L.nd, L.E); break; }
        case 4: { CNT(); k_lu_solve<4><<<grid, 128, 0, s>>>(M, perm, x, L.nd, L.E); break; }
        case 5: { CNT(); k_lu_solve<5><<<grid, 128, 0, s>>>(M, perm, x, L.nd, L.E); break; }
        case 6: { CNT(); k_lu_solve<6><<<grid, 128, 0, s>>>(M, perm, x, L.nd, L.E); break; }
        case 7: { CNT(); k_lu_solve<7><<<grid, 128, 0, s>>>(M, perm, x, L.nd, L.E); break; }
        case 8: { CNT(); k_lu_solve<8><<<grid, 128, 0, s>>>(M, perm, x, L.nd, L.E); break; }
        case 10: { CNT(); k_lu_solve<10><<<grid, 128, 0, s>>>(M, perm, x, L.nd, L.E); break; }
        default: return -1;
    }
    return 0;
}

// ------------------------------------------------------------------------ transfers
// thread per (e, v); 1-D operator along direction 0, then 1, then 2 (fma chains over the
// source index); sizes at run time (ni -> no points per direction), NM = max points.
template <int D, int NM>
__global__ void __launch_bounds__(128) k_tensor(const double *__restrict__ x, double *__restrict__ y, int E, int ni,
                                                int no, int p0, int p1, int restrict_) {
    constexpr int BUF = D == 2 ? NM * NM : NM * NM * NM;
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    int v = blockIdx.y;
    int npi = D == 2 ? ni * ni : ni * ni * ni, npo = D == 2 ? no * no : no * no * no;
    double a[BUF], b[BUF];
#pragma unroll 1
    for (int i = 0; i < npi; ++i) a[i] = x[(size_t)(v * npi + i) * E + e];
    int dims[3] = {ni, ni, D == 3 ? ni : 1};
#pragma unroll 1
    for (int dir = 0; dir < D; ++dir) {
        int nd0 = dir == 0 ? no : dims[0], nd1 = dir == 1 ? no : dims[1], nd2 = dir == 2 ? no : dims[2];
#pragma unroll 1
        for (int i2 = 0; i2 < nd2; ++i2)
#pragma unroll 1
            for (int i1 = 0; i1 < nd1; ++i1)
#pragma unroll 1
                for (int i0 = 0; i0 < nd0; ++i0) {
                    int o = dir == 0 ? i0 : (dir == 1 ? i1 : i2);
                    double s = 0.0;
#pragma unroll 1
                    for (int m = 0; m < ni; ++m) {
                        int s0 = dir == 0 ? m : i0, s1 = dir == 1 ? m : i1, s2 = dir == 2 ? m : i2;
                        double op = restrict_ ? c_gam64[p0][p1][o][m] : c_pi64[p0][p1][o][m];
                        s = fma(op, a[s0 + dims[0] * (s1 + dims[1] * s2)], s);
                    }
                    b[i0 + nd0 * (i1 + nd1 * i2)] = s;
                }
        dims[0] = nd0; dims[1] = nd1; dims[2] = nd2;
        int cnt = dims[0] * dims[1] * dims[2];
#pragma unroll 1
        for (int i = 0; i < cnt; ++i) a[i] = b[i];
    }
#pragma unroll 1
    for (int i = 0; i < npo; ++i) y[(size_t)(v * npo + i) * E + e] = a[i];
}

int frk64_transfer(const FrLevel &Lf, const FrLevel &Lc, bool r, const double *x, double *y, cudaStream_t s) {
    int p0 = Lf.p, p1 = Lc.p, E = Lf.E, nv = Lf.nv;
    int ni = r ? p0 + 1 : p1 + 1, no = r ? p1 + 1 : p0 + 1;
    dim3 grid((E + 127) / 128, nv);
    if (Lf.d == 2 && p0 <= 5) { CNT(); k_tensor<2, 6><<<grid, 128, 0, s>>>(x, y, E, ni, no, p0, p1, r); }
    else if (Lf.d == 3 && p0 <= 3) { CNT(); k_tensor<3, 4><<<grid, 128, 0, s>>>(x, y, E, ni, no, p0, p1, r); }
    else return -1;
    return 0;
}
