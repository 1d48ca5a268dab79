// Segmented vector kernels of the batched solver: many independent problems share one
// [rows][E] vector (each problem owns a contiguous element range), and every reduction,
// scaling and linear combination is taken per problem.  Reductions run over work items
// (one problem's element range of at most kSegChunk elements): one block per item sums
// its share in a fixed order, then one thread per problem sums its items in item order,
// so results are reproducible run to run.
#include <atomic>
#include <cuda_runtime.h>
#include <math.h>
#include <algorithm>
#include "fr_lib.h"

static std::atomic<unsigned long long> g_launches{0};   // host-side launch counter (any thread)
unsigned long long frkb_launch_count() { return g_launches; }
#define CNT() (g_launches.fetch_add(1, std::memory_order_relaxed))

#define SEG_THREADS 256
#define GRID_STRIDE(i, n) \
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

static inline int nblk(long long n) {
    long long g = (n + 255) / 256;
    return (int)std::max<long long>(1, std::min<long long>(g, 152LL * 32));
}

struct SegPtr8 {
    const double *p[8];
};

template <int M>
__global__ void __launch_bounds__(SEG_THREADS) k_segdot_partial(int rows, int E, const int4 *items, const double *w,
                                                                SegPtr8 V, double *partial) {
    int4 it = items[blockIdx.x];   // (problem, e0, e1, unused)
    double acc[M];
#pragma unroll
    for (int j = 0; j < M; ++j) acc[j] = 0.0;
    for (int r = 0; r < rows; ++r) {
        size_t base = (size_t)r * E;
        for (int e = it.y + threadIdx.x; e < it.z; e += SEG_THREADS) {
            double wi = w[base + e];
#pragma unroll
            for (int j = 0; j < M; ++j) acc[j] = fma(wi, V.p[j][base + e], acc[j]);
        }
    }
    __shared__ double sh[SEG_THREADS / 32][M];
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
        for (int k = 0; k < SEG_THREADS / 32; ++k) t = t + sh[k][threadIdx.x];
        partial[(size_t)blockIdx.x * 8 + threadIdx.x] = t;
    }
}

// out[prob * ld + j0 + j] = sum over the problem's items (in order) of the partials
__global__ void k_segdot_final(int nprob, int m, const int *item_off, const double *partial, double *out, int ld,
                               int j0) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nprob) return;
    for (int j = 0; j < m; ++j) {
        double t = 0.0;
        for (int k = item_off[p]; k < item_off[p + 1]; ++k) t = t + partial[(size_t)k * 8 + j];
        out[(size_t)p * ld + j0 + j] = t;
    }
}

int frkb_segdots(int rows, int E, int nitems, const int4 *items, int nprob, const int *item_off, const double *w,
                 int m, const double *const *V, double *partial, double *out, int ld, cudaStream_t s) {
    for (int j0 = 0; j0 < m; j0 += 8) {
        int mm = std::min(8, m - j0);
        SegPtr8 P;
        for (int j = 0; j < 8; ++j) P.p[j] = j < mm ? V[j0 + j] : nullptr;
        switch (mm) {
            case 1: { CNT(); k_segdot_partial<1><<<nitems, SEG_THREADS, 0, s>>>(rows, E, items, w, P, partial); break; }
            case 2: { CNT(); k_segdot_partial<2><<<nitems, SEG_THREADS, 0, s>>>(rows, E, items, w, P, partial); break; }
            case 3: { CNT(); k_segdot_partial<3><<<nitems, SEG_THREADS, 0, s>>>(rows, E, items, w, P, partial); break; }
            case 4: { CNT(); k_segdot_partial<4><<<nitems, SEG_THREADS, 0, s>>>(rows, E, items, w, P, partial); break; }
            case 5: { CNT(); k_segdot_partial<5><<<nitems, SEG_THREADS, 0, s>>>(rows, E, items, w, P, partial); break; }
            case 6: { CNT(); k_segdot_partial<6><<<nitems, SEG_THREADS, 0, s>>>(rows, E, items, w, P, partial); break; }
            case 7: { CNT(); k_segdot_partial<7><<<nitems, SEG_THREADS, 0, s>>>(rows, E, items, w, P, partial); break; }
            default: { CNT(); k_segdot_partial<8><<<nitems, SEG_THREADS, 0, s>>>(rows, E, items, w, P, partial); break; }
        }
        CNT(); k_segdot_final<<<(nprob + 127) / 128, 128, 0, s>>>(nprob, mm, item_off, partial, out, ld, j0);
    }
    return 0;
}

// nrm[p] = sqrt(sq[p * ld]); inv[p] = mask[p] * 1/nrm (0 where the mask is 0 or nrm is 0)
__global__ void k_seg_invnorm(int nprob, const double *sq, int ld, const double *mask, double *nrm, double *inv) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nprob) return;
    double v = sqrt(sq[(size_t)p * ld]);
    nrm[p] = v;
    inv[p] = (mask[p] != 0.0 && v > 0.0) ? mask[p] / v : 0.0;
}
void frkb_seg_invnorm(int nprob, const double *sq, int ld, const double *mask, double *nrm, double *inv,
                      cudaStream_t s) {
    CNT(); k_seg_invnorm<<<(nprob + 127) / 128, 128, 0, s>>>(nprob, sq, ld, mask, nrm, inv);
}

// y[r][e] = x[r][e] * f[ep[e]]
__global__ void k_seg_scale(long long n, int E, const int *ep, const double *f, const double *x, double *y) {
    GRID_STRIDE(i, n) y[i] = x[i] * f[ep[i % E]];
}
void frkb_seg_scale(long long n, int E, const int *ep, const double *f, const double *x, double *y, cudaStream_t s) {
    CNT(); k_seg_scale<<<nblk(n), 256, 0, s>>>(n, E, ep, f, x, y);
}

// w[r][e] -= sum_j h[ep[e] * ld + j0 + j] V_j[r][e]
__global__ void k_seg_multi_axpy(long long n, int E, const int *ep, int m, const double *h, int ld, int j0, SegPtr8 V,
                                 double *w) {
    GRID_STRIDE(i, n) {
        const double *hp = h + (size_t)ep[i % E] * ld + j0;
        double t = w[i];
        for (int j = 0; j < m; ++j) t = fma(-hp[j], V.p[j][i], t);
        w[i] = t;
    }
}
void frkb_seg_multi_axpy(long long n, int E, const int *ep, int m, const double *h, int ld, const double *const *V,
                         double *w, cudaStream_t s) {
    for (int j0 = 0; j0 < m; j0 += 8) {
        int mm = std::min(8, m - j0);
        SegPtr8 P;
        for (int j = 0; j < 8; ++j) P.p[j] = j < mm ? V[j0 + j] : nullptr;
        CNT(); k_seg_multi_axpy<<<nblk(n), 256, 0, s>>>(n, E, ep, mm, h, ld, j0, P, w);
    }
}

// x[r][e] += sum_j y[ep[e] * ld + j0 + j] Z_j[r][e]
__global__ void k_seg_update_x(long long n, int E, const int *ep, int m, const double *y, int ld, int j0, SegPtr8 Z,
                               double *x) {
    GRID_STRIDE(i, n) {
        const double *yp = y + (size_t)ep[i % E] * ld + j0;
        double t = x[i];
        for (int j = 0; j < m; ++j) t = fma(yp[j], Z.p[j][i], t);
        x[i] = t;
    }
}
void frkb_seg_update_x(long long n, int E, const int *ep, int m, const double *y, int ld, const double *const *Z,
                       double *x, cudaStream_t s) {
    for (int j0 = 0; j0 < m; j0 += 8) {
        int mm = std::min(8, m - j0);
        SegPtr8 P;
        for (int j = 0; j < 8; ++j) P.p[j] = j < mm ? Z[j0 + j] : nullptr;
        CNT(); k_seg_update_x<<<nblk(n), 256, 0, s>>>(n, E, ep, mm, y, ld, j0, P, x);
    }
}

// gather / scatter between a problem's own [rows][Ei] vector and its element range of the
// group's [rows][E] vector
__global__ void k_seg_copy(long long n, int Ei, const double *src, long long ss, double *dst, long long ds) {
    GRID_STRIDE(i, n) {
        long long r = i / Ei, e = i - r * Ei;
        dst[r * ds + e] = src[r * ss + e];
    }
}
void frkb_gather(int rows, int Ei, const double *qi, double *Q, int E, int off, cudaStream_t s) {
    long long n = (long long)rows * Ei;
    CNT(); k_seg_copy<<<nblk(n), 256, 0, s>>>(n, Ei, qi, Ei, Q + off, E);
}
void frkb_scatter(int rows, int Ei, const double *Q, int E, int off, double *qi, cudaStream_t s) {
    long long n = (long long)rows * Ei;
    CNT(); k_seg_copy<<<nblk(n), 256, 0, s>>>(n, Ei, Q + off, E, qi, Ei);
}
