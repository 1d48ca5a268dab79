// FP64 kernels of the JFNK-pMG hot path.  Compiled with -fmad=false: the only fused
// multiply-adds are the explicit fma() calls, so every result depends only on the
// documented evaluation order (fma chains in ascending index), not on the compiler.
#define FRT double
#define FRK(name) frk64_##name
#define FR_DOUBLE 1
#include "fr_kernels_impl.cuh"

// ------------------------------------------------- Krylov and time-stepping vectors

__global__ void k_axpy_perturb(long long n, const double *q, double eps, const double *v, double *qp) {
    GRID_STRIDE(i, n) qp[i] = q[i] + eps * v[i];
}
__global__ void k_jv_finish(long long n, double shift, const double *v, const double *Rp, const double *Rq, double eps,
                            double *Av) {
    GRID_STRIDE(i, n) Av[i] = shift * v[i] - (Rp[i] - Rq[i]) / eps;
}
__global__ void k_scale(long long n, double a, const double *x, double *y) { GRID_STRIDE(i, n) y[i] = x[i] * a; }
__global__ void k_div_scalar(long long n, const double *x, double a, double *y) { GRID_STRIDE(i, n) y[i] = x[i] / a; }
__global__ void k_neg(long long n, const double *x, double *y) { GRID_STRIDE(i, n) y[i] = -x[i]; }
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
void frk64_neg(long long n, const double *x, double *y, cudaStream_t s) { CNT(); k_neg<<<nblk(n), 256, 0, s>>>(n, x, y); }
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

// w . V_j over the owned part of level vectors: index i -> (row i / n_owned, element
// i % n_owned) of a [rows][E] vector (n_owned = E: the whole vector, in the same order)
template <int M>
__global__ void __launch_bounds__(RED_THREADS) k_multidot_partial(long long n, long long E, long long n_owned,
                                                                  const double *w, Ptr8 V, double *partial) {
    double acc[M];
#pragma unroll
    for (int j = 0; j < M; ++j) acc[j] = 0.0;
    GRID_STRIDE(t, n) {
        long long i = n_owned == E ? t : (t / n_owned) * E + t % n_owned;
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

// one CTA of RED_THREADS threads: thread t sums the partials t, t + RED_THREADS, ... of
// every column j in that order, then a fixed shuffle tree and the warp sums in warp order
// (the same order for a given nb on every call)
template <int M>
__global__ void __launch_bounds__(RED_THREADS) k_multidot_final(int nb, const double *partial, double *out) {
    double acc[M];
#pragma unroll
    for (int j = 0; j < M; ++j) acc[j] = 0.0;
    for (int b = threadIdx.x; b < nb; b += RED_THREADS)
#pragma unroll
        for (int j = 0; j < M; ++j) acc[j] = acc[j] + partial[(size_t)b * 8 + j];
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
        out[threadIdx.x] = t;
    }
}

long long frk64_multidot_scratch(long long n) { return (long long)red_blocks(n) * 8; }

// out[j] = w . V_j (j < m) over the owned elements (rows x n_owned of [rows][E] vectors;
// n_owned = E for whole vectors); partial: frk64_multidot_scratch(rows * n_owned) doubles
int frk64_multidot(long long rows, long long E, long long n_owned, int m, const double *w, const double *const *V,
                   double *out, double *partial, cudaStream_t s) {
    long long n = rows * n_owned;
    int nb = red_blocks(n);
    for (int j0 = 0; j0 < m; j0 += 8) {
        int mm = std::min(8, m - j0);
        Ptr8 P;
        for (int j = 0; j < 8; ++j) { P.p[j] = j < mm ? V[j0 + j] : nullptr; P.c[j] = 0.0; }
        switch (mm) {
            case 1: { CNT(); k_multidot_partial<1><<<nb, RED_THREADS, 0, s>>>(n, E, n_owned, w, P, partial); break; }
            case 2: { CNT(); k_multidot_partial<2><<<nb, RED_THREADS, 0, s>>>(n, E, n_owned, w, P, partial); break; }
            case 3: { CNT(); k_multidot_partial<3><<<nb, RED_THREADS, 0, s>>>(n, E, n_owned, w, P, partial); break; }
            case 4: { CNT(); k_multidot_partial<4><<<nb, RED_THREADS, 0, s>>>(n, E, n_owned, w, P, partial); break; }
            case 5: { CNT(); k_multidot_partial<5><<<nb, RED_THREADS, 0, s>>>(n, E, n_owned, w, P, partial); break; }
            case 6: { CNT(); k_multidot_partial<6><<<nb, RED_THREADS, 0, s>>>(n, E, n_owned, w, P, partial); break; }
            case 7: { CNT(); k_multidot_partial<7><<<nb, RED_THREADS, 0, s>>>(n, E, n_owned, w, P, partial); break; }
            default: { CNT(); k_multidot_partial<8><<<nb, RED_THREADS, 0, s>>>(n, E, n_owned, w, P, partial); break; }
        }
        switch (mm) {
            case 1: { CNT(); k_multidot_final<1><<<1, RED_THREADS, 0, s>>>(nb, partial, out + j0); break; }
            case 2: { CNT(); k_multidot_final<2><<<1, RED_THREADS, 0, s>>>(nb, partial, out + j0); break; }
            case 3: { CNT(); k_multidot_final<3><<<1, RED_THREADS, 0, s>>>(nb, partial, out + j0); break; }
            case 4: { CNT(); k_multidot_final<4><<<1, RED_THREADS, 0, s>>>(nb, partial, out + j0); break; }
            case 5: { CNT(); k_multidot_final<5><<<1, RED_THREADS, 0, s>>>(nb, partial, out + j0); break; }
            case 6: { CNT(); k_multidot_final<6><<<1, RED_THREADS, 0, s>>>(nb, partial, out + j0); break; }
            case 7: { CNT(); k_multidot_final<7><<<1, RED_THREADS, 0, s>>>(nb, partial, out + j0); break; }
            default: { CNT(); k_multidot_final<8><<<1, RED_THREADS, 0, s>>>(nb, partial, out + j0); break; }
        }
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

