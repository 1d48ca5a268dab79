// Per-element MLP for the Newton initial guess (an addition to the method; the paper's guess is
// q^n): forward, backward and Adam, BF16 operands with FP32 accumulation on the tensor
// cores (mma.sync m16n8k16), plus the per-element feature / target / guess assembly.
//
//   h1 = tanh(W1 x + b1),  h2 = tanh(W2 h1 + b2),  y = W3 h2 + b3,  loss = mean (y - t)^2
//
// x, h1, h2, the output-side gradients and the weights enter every matrix product
// rounded to bfloat16 (nearest, ties to even); sums run in FP32; master weights and Adam
// moments are FP32.
#include <atomic>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <algorithm>
#include <vector>
#include "../../include/frpmg.h"
#include "fr_lib.h"

static std::atomic<unsigned long long> g_launches{0};   // host-side launch counter (any thread)
unsigned long long frkmlp_launch_count() { return g_launches; }
#define CNT() (g_launches.fetch_add(1, std::memory_order_relaxed))

typedef __nv_bfloat16 bf16;

// ----------------------------------------------------------------------- GEMM
// C[m][n] = sum_k A(m, k) B(k, n), A and B bf16 with arbitrary strides, FP32 accumulate.
// CTA tile 64 x 64, k-step 32, 4 warps of 32 x 32 (2 x 4 mma tiles of 16 x 8).
// Epilogue: + bias[n] (optional), tanh (optional), FP32 store (optional), bf16 store
// (optional).
struct GemmArgs {
    int M, N, K;
    const bf16 *A;
    long long sAm, sAk;
    const bf16 *B;
    long long sBk, sBn;
    const float *bias;
    int act;            // 0 none, 1 tanh
    float *C;           // [M][N] row-major, or NULL
    bf16 *Cb;           // [M][N] row-major bf16, or NULL
};

__device__ __forceinline__ uint32_t ld32(const bf16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

__global__ void __launch_bounds__(128) k_gemm_bf16(GemmArgs g) {
    __shared__ __align__(16) bf16 As[64][40];
    __shared__ __align__(16) bf16 Bs[64][40];   // stored [n][k]
    int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
    const bf16 zero = __float2bfloat16(0.f);
    for (int k0 = 0; k0 < g.K; k0 += 32) {
        for (int t = tid; t < 64 * 32; t += 128) {
            int r = t >> 5, kk = t & 31;
            int m = m0 + r, k = k0 + kk, n = n0 + r;
            As[r][kk] = (m < g.M && k < g.K) ? g.A[m * g.sAm + k * g.sAk] : zero;
            Bs[r][kk] = (n < g.N && k < g.K) ? g.B[k * g.sBk + n * g.sBn] : zero;
        }
        __syncthreads();
        int gq = lane >> 2, tq = lane & 3;
#pragma unroll
        for (int ks = 0; ks < 32; ks += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                int r = wm + a * 16 + gq;
                af[a][0] = ld32(&As[r][ks + 2 * tq]);
                af[a][1] = ld32(&As[r + 8][ks + 2 * tq]);
                af[a][2] = ld32(&As[r][ks + 2 * tq + 8]);
                af[a][3] = ld32(&As[r + 8][ks + 2 * tq + 8]);
            }
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                int n = wn + b * 8 + gq;
                bfr[b][0] = ld32(&Bs[n][ks + 2 * tq]);
                bfr[b][1] = ld32(&Bs[n][ks + 2 * tq + 8]);
            }
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                        "{%8,%9}, {%0,%1,%2,%3};\n"
                        : "+f"(acc[a][b][0]), "+f"(acc[a][b][1]), "+f"(acc[a][b][2]), "+f"(acc[a][b][3])
                        : "r"(af[a][0]), "r"(af[a][1]), "r"(af[a][2]), "r"(af[a][3]), "r"(bfr[b][0]),
                          "r"(bfr[b][1]));
        }
        __syncthreads();
    }
    int gq = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    int m = m0 + wm + a * 16 + gq + 8 * h, n = n0 + wn + b * 8 + 2 * tq + c;
                    if (m >= g.M || n >= g.N) continue;
                    float v = acc[a][b][2 * h + c];
                    if (g.bias) v += g.bias[n];
                    if (g.act == 1) v = tanhf(v);
                    if (g.C) g.C[(size_t)m * g.N + n] = v;
                    if (g.Cb) g.Cb[(size_t)m * g.N + n] = __float2bfloat16(v);
                }
}

static void gemm(const GemmArgs &g, cudaStream_t s) {
    dim3 grid((g.N + 63) / 64, (g.M + 63) / 64);
    CNT(); k_gemm_bf16<<<grid, 128, 0, s>>>(g);
}

// ----------------------------------------------------------------- elementwise
#define GS(i, n) for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)
static int nb(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 16); }

__global__ void k_to_bf16(long long n, const float *x, bf16 *y) { GS(i, n) y[i] = __float2bfloat16(x[i]); }
// g3 = 2 (y - t) / (B O); loss partial sums
__global__ void k_out_grad(long long n, const float *y, const float *t, float scale, float *g, bf16 *gb, float *lsum) {
    float acc = 0.f;
    GS(i, n) {
        float d = y[i] - t[i];
        acc += d * d;
        float gi = scale * d;
        g[i] = gi;
        gb[i] = __float2bfloat16(gi);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(lsum, acc);
}
// g = gh * (1 - h^2)
__global__ void k_tanh_back(long long n, const float *gh, const float *h, float *g, bf16 *gb) {
    GS(i, n) {
        float v = gh[i] * (1.f - h[i] * h[i]);
        g[i] = v;
        gb[i] = __float2bfloat16(v);
    }
}
// column sums of g [B][N] (bias gradients): one thread per column, fixed order
__global__ void k_colsum(int B, int N, const float *g, float *out) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += g[(size_t)b * N + n];
    out[n] = s;
}
__global__ void k_adam(long long n, float *p, const float *g, float *m, float *v, bf16 *pb, float lr, float b1,
                       float b2, float c1, float c2, float eps) {
    GS(i, n) {
        float gi = g[i];
        float mi = b1 * m[i] + (1.f - b1) * gi;
        float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        pb[i] = __float2bfloat16(pi);
    }
}

// ------------------------------------------------------------------- the network
struct fr_mlp {
    int in, hid, out;
    size_t np;                 // parameter count
    float *p, *g, *m, *v;      // master params, grads, Adam moments (FP32)
    bf16 *pb;                  // bf16 copy of the params
    int t;                     // Adam step
    // activations for the largest batch seen
    int cap;
    float *h1, *h2, *y, *gy, *g2, *g1, *gh, *lsum;
    bf16 *h1b, *h2b, *gyb, *g2b, *g1b;
    std::vector<void *> allocs;
};

// parameter offsets: W1[h][in], b1[h], W2[h][h], b2[h], W3[out][h], b3[out]
static size_t oW1(const fr_mlp *M) { return 0; }
static size_t ob1(const fr_mlp *M) { return (size_t)M->hid * M->in; }
static size_t oW2(const fr_mlp *M) { return ob1(M) + M->hid; }
static size_t ob2(const fr_mlp *M) { return oW2(M) + (size_t)M->hid * M->hid; }
static size_t oW3(const fr_mlp *M) { return ob2(M) + M->hid; }
static size_t ob3(const fr_mlp *M) { return oW3(M) + (size_t)M->out * M->hid; }

template <typename T>
static int malloc_t(fr_mlp *M, T **p, size_t n) {
    if (cudaMalloc((void **)p, sizeof(T) * (n ? n : 1)) != cudaSuccess) { cudaGetLastError(); *p = nullptr; return -1; }
    M->allocs.push_back(*p);
    return 0;
}

int fr_internal_fail(int code, const char *msg);

extern "C" int mlp_destroy(fr_mlp *M) {
    if (!M) return FR_OK;
    for (void *p : M->allocs) cudaFree(p);
    delete M;
    return FR_OK;
}

extern "C" int mlp_create(fr_mlp **out, int in_dim, int hidden, int out_dim, const float *params) {
    if (!out) return fr_internal_fail(FR_ERR_INVALID_ARG, "mlp_create: out is NULL");
    *out = nullptr;
    if (in_dim < 1 || hidden < 1 || out_dim < 1 || !params)
        return fr_internal_fail(FR_ERR_INVALID_ARG, "mlp_create: bad sizes or NULL parameters");
    if (in_dim % 2 || hidden % 2 || out_dim % 2)
        return fr_internal_fail(FR_ERR_INVALID_ARG, "mlp_create: sizes must be even (bf16 pairs)");
    fr_mlp *M = new fr_mlp();
    M->in = in_dim; M->hid = hidden; M->out = out_dim;
    M->np = ob3(M) + out_dim;
    if (malloc_t(M, &M->p, M->np) || malloc_t(M, &M->g, M->np) || malloc_t(M, &M->m, M->np) ||
        malloc_t(M, &M->v, M->np) || malloc_t(M, &M->pb, M->np) || malloc_t(M, &M->lsum, 1)) {
        mlp_destroy(M);
        return fr_internal_fail(FR_ERR_OOM, "mlp_create: out of device memory");
    }
    cudaMemcpy(M->p, params, sizeof(float) * M->np, cudaMemcpyHostToDevice);
    cudaMemset(M->m, 0, sizeof(float) * M->np);
    cudaMemset(M->v, 0, sizeof(float) * M->np);
    CNT(); k_to_bf16<<<nb(M->np), 256>>>(M->np, M->p, M->pb);
    if (cudaDeviceSynchronize() != cudaSuccess) { mlp_destroy(M); return fr_internal_fail(FR_ERR_CUDA, "mlp_create"); }
    *out = M;
    return FR_OK;
}

extern "C" int mlp_get_params(const fr_mlp *M, float *params) {
    if (!M || !params) return fr_internal_fail(FR_ERR_INVALID_ARG, "mlp_get_params: NULL argument");
    if (cudaMemcpy(params, M->p, sizeof(float) * M->np, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fr_internal_fail(FR_ERR_CUDA, "mlp_get_params");
    return FR_OK;
}

static int ensure_cap(fr_mlp *M, int B) {
    if (B <= M->cap) return 0;
    // activations are kept for the largest batch; earlier buffers stay until destroy
    size_t H = (size_t)B * M->hid, O = (size_t)B * M->out;
    if (malloc_t(M, &M->h1, H) || malloc_t(M, &M->h2, H) || malloc_t(M, &M->y, O) || malloc_t(M, &M->gy, O) ||
        malloc_t(M, &M->g2, H) || malloc_t(M, &M->g1, H) || malloc_t(M, &M->gh, H) || malloc_t(M, &M->h1b, H) ||
        malloc_t(M, &M->h2b, H) || malloc_t(M, &M->gyb, O) || malloc_t(M, &M->g2b, H) || malloc_t(M, &M->g1b, H))
        return -1;
    M->cap = B;
    return 0;
}

static void forward(fr_mlp *M, int B, const bf16 *X, float *Y, cudaStream_t s) {
    GemmArgs g;
    g = {B, M->hid, M->in, X, M->in, 1, M->pb + oW1(M), 1, M->in, M->p + ob1(M), 1, M->h1, M->h1b};
    gemm(g, s);
    g = {B, M->hid, M->hid, M->h1b, M->hid, 1, M->pb + oW2(M), 1, M->hid, M->p + ob2(M), 1, M->h2, M->h2b};
    gemm(g, s);
    g = {B, M->out, M->hid, M->h2b, M->hid, 1, M->pb + oW3(M), 1, M->hid, M->p + ob3(M), 0, Y, nullptr};
    gemm(g, s);
}

extern "C" int mlp_forward(fr_mlp *M, int B, const unsigned short *X, float *Y, void *stream) {
    if (!M || !X || !Y || B < 1) return fr_internal_fail(FR_ERR_INVALID_ARG, "mlp_forward: bad argument");
    if (ensure_cap(M, B)) return fr_internal_fail(FR_ERR_OOM, "mlp_forward: out of device memory");
    forward(M, B, (const bf16 *)X, Y, (cudaStream_t)stream);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FR_OK : fr_internal_fail(FR_ERR_CUDA, cudaGetErrorString(e));
}

// backward of the mean-squared loss into M->g (FP32, parameter layout); returns the loss
static void backward(fr_mlp *M, int B, const bf16 *X, const float *T, cudaStream_t s) {
    long long nO = (long long)B * M->out, nH = (long long)B * M->hid;
    cudaMemsetAsync(M->lsum, 0, sizeof(float), s);
    CNT(); k_out_grad<<<nb(nO), 256, 0, s>>>(nO, M->y, T, 2.f / (float)nO, M->gy, M->gyb, M->lsum);
    GemmArgs g;
    // dW3[o][h] = sum_b gy[b][o] h2[b][h]
    g = {M->out, M->hid, B, M->gyb, 1, M->out, M->h2b, M->hid, 1, nullptr, 0, M->g + oW3(M), nullptr};
    gemm(g, s);
    CNT(); k_colsum<<<(M->out + 127) / 128, 128, 0, s>>>(B, M->out, M->gy, M->g + ob3(M));
    // gh2[b][h] = sum_o gy[b][o] W3[o][h]
    g = {B, M->hid, M->out, M->gyb, M->out, 1, M->pb + oW3(M), M->hid, 1, nullptr, 0, M->gh, nullptr};
    gemm(g, s);
    CNT(); k_tanh_back<<<nb(nH), 256, 0, s>>>(nH, M->gh, M->h2, M->g2, M->g2b);
    g = {M->hid, M->hid, B, M->g2b, 1, M->hid, M->h1b, M->hid, 1, nullptr, 0, M->g + oW2(M), nullptr};
    gemm(g, s);
    CNT(); k_colsum<<<(M->hid + 127) / 128, 128, 0, s>>>(B, M->hid, M->g2, M->g + ob2(M));
    g = {B, M->hid, M->hid, M->g2b, M->hid, 1, M->pb + oW2(M), M->hid, 1, nullptr, 0, M->gh, nullptr};
    gemm(g, s);
    CNT(); k_tanh_back<<<nb(nH), 256, 0, s>>>(nH, M->gh, M->h1, M->g1, M->g1b);
    g = {M->hid, M->in, B, M->g1b, 1, M->hid, X, M->in, 1, nullptr, 0, M->g + oW1(M), nullptr};
    gemm(g, s);
    CNT(); k_colsum<<<(M->hid + 127) / 128, 128, 0, s>>>(B, M->hid, M->g1, M->g + ob1(M));
}

extern "C" int mlp_train_step(fr_mlp *M, int B, const unsigned short *X, const float *T, float lr, float *loss,
                              float *grads, void *stream) {
    if (!M || !X || !T || B < 1 || !(lr >= 0.f)) return fr_internal_fail(FR_ERR_INVALID_ARG, "mlp_train_step: bad argument");
    if (ensure_cap(M, B)) return fr_internal_fail(FR_ERR_OOM, "mlp_train_step: out of device memory");
    cudaStream_t s = (cudaStream_t)stream;
    forward(M, B, (const bf16 *)X, M->y, s);
    backward(M, B, (const bf16 *)X, T, s);
    if (grads) cudaMemcpyAsync(grads, M->g, sizeof(float) * M->np, cudaMemcpyDeviceToDevice, s);
    M->t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = 1.f - powf(b1, (float)M->t), c2 = 1.f - powf(b2, (float)M->t);
    CNT(); k_adam<<<nb(M->np), 256, 0, s>>>(M->np, M->p, M->g, M->m, M->v, M->pb, lr, b1, b2, c1, c2, 1e-8f);
    if (loss) {
        float l = 0.f;
        cudaMemcpyAsync(&l, M->lsum, sizeof(float), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        *loss = l / (float)((long long)B * M->out);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FR_OK : fr_internal_fail(FR_ERR_CUDA, cudaGetErrorString(e));
}

// ------------------------------------------------------ features, targets, guesses
// x = [(q^n - q^{n-1})/s_v, (q^{n-1} - q^{n-2})/s_v, (q^n - qinf_v)/sig_v, dt R(q^n)/s_v,
//      log J / 10, c, 0...], each rounded FP64 -> FP32 -> bf16
__global__ void k_features(int E, int nv, int Np, int K0, const double *qn, const double *q1, const double *q2,
                           const double *Rn, double dt, const double *invJ, double c, const double *s,
                           const double *sig, const double *qinf, bf16 *X) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    int nd = nv * Np;
    bf16 *x = X + (size_t)e * K0;
    for (int r = 0; r < nd; ++r) {
        int v = r / Np;
        size_t k = (size_t)r * E + e;
        double a = qn[k], b = q1[k], d = q2[k];
        x[r] = __float2bfloat16((float)((a - b) / s[v]));
        x[nd + r] = __float2bfloat16((float)((b - d) / s[v]));
        x[2 * nd + r] = __float2bfloat16((float)((a - qinf[v]) / sig[v]));
        x[3 * nd + r] = __float2bfloat16((float)(dt * Rn[k] / s[v]));
    }
    for (int i = 0; i < Np; ++i) x[4 * nd + i] = __float2bfloat16((float)(-log(fabs(invJ[(size_t)i * E + e])) / 10.0));
    x[4 * nd + Np] = __float2bfloat16((float)c);
    for (int k = 4 * nd + Np + 1; k < K0; ++k) x[k] = __float2bfloat16(0.f);
}
// qex = w0 q^{n-2} + w1 q^{n-1} + w2 q^n
__global__ void k_extrap(long long n, const double *qn, const double *q1, const double *q2, double w0, double w1,
                         double w2, double *qex) {
    GS(i, n) qex[i] = w0 * q2[i] + w1 * q1[i] + w2 * qn[i];
}
// t[e][r] = (qstage - qex)/s_v  (sample-major)
__global__ void k_targets(int E, int nv, int Np, const double *qs, const double *qex, const double *s, float *T) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    int nd = nv * Np;
    for (int r = 0; r < nd; ++r)
        T[(size_t)e * nd + r] = (float)((qs[(size_t)r * E + e] - qex[(size_t)r * E + e]) / s[r / Np]);
}
// guess = qex + s_v y
__global__ void k_guess(int E, int nv, int Np, const double *qex, const double *s, const float *Y, double *g) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    int nd = nv * Np;
    for (int r = 0; r < nd; ++r)
        g[(size_t)r * E + e] = qex[(size_t)r * E + e] + s[r / Np] * (double)Y[(size_t)e * nd + r];
}

void frkmlp_features(int E, int nv, int Np, int K0, const double *qn, const double *q1, const double *q2,
                     const double *Rn, double dt, const double *invJ, double c, const double *s_dev,
                     const double *sig_dev, const double *qinf_dev, unsigned short *X, cudaStream_t st) {
    CNT(); k_features<<<(E + 127) / 128, 128, 0, st>>>(E, nv, Np, K0, qn, q1, q2, Rn, dt, invJ, c, s_dev, sig_dev,
                                                      qinf_dev, (bf16 *)X);
}
void frkmlp_extrap(long long n, const double *qn, const double *q1, const double *q2, double c, double *qex,
                   cudaStream_t st) {
    double tau = 2.0 + c;
    double w0 = (tau - 1.0) * (tau - 2.0) / 2.0, w1 = -tau * (tau - 2.0), w2 = tau * (tau - 1.0) / 2.0;
    CNT(); k_extrap<<<nb(n), 256, 0, st>>>(n, qn, q1, q2, w0, w1, w2, qex);
}
void frkmlp_targets(int E, int nv, int Np, const double *qs, const double *qex, const double *s_dev, float *T,
                    cudaStream_t st) {
    CNT(); k_targets<<<(E + 127) / 128, 128, 0, st>>>(E, nv, Np, qs, qex, s_dev, T);
}
void frkmlp_guess(int E, int nv, int Np, const double *qex, const double *s_dev, const float *Y, double *g,
                  cudaStream_t st) {
    CNT(); k_guess<<<(E + 127) / 128, 128, 0, st>>>(E, nv, Np, qex, s_dev, Y, g);
}
int frkmlp_forward(fr_mlp *M, int B, const unsigned short *X, float *Y, cudaStream_t s) {
    if (ensure_cap(M, B)) return -1;
    forward(M, B, (const bf16 *)X, Y, s);
    return 0;
}
int frkmlp_dims(const fr_mlp *M, int *in, int *hid, int *out) {
    *in = M->in; *hid = M->hid; *out = M->out;
    return 0;
}

// per-variable sums of squares of (a - b) and of (a - qinf_v) over a [nv][Np][E] state,
// block partials then a fixed-order sum (deterministic)
#define VS_BLOCKS 64
__global__ void k_var_partials(long long per, const double *a, const double *b, const double *qinf, double *part) {
    int v = blockIdx.y;
    const double *av = a + (size_t)v * per, *bv = b + (size_t)v * per;
    double s1 = 0.0, s2 = 0.0, qi = qinf[v];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < per; i += (long long)gridDim.x * blockDim.x) {
        double d = av[i] - bv[i], f = av[i] - qi;
        s1 = fma(d, d, s1);
        s2 = fma(f, f, s2);
    }
    __shared__ double sh1[8], sh2[8];
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { sh1[w] = s1; sh2[w] = s2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { t1 += sh1[k]; t2 += sh2[k]; }
        part[((size_t)v * VS_BLOCKS + blockIdx.x) * 2] = t1;
        part[((size_t)v * VS_BLOCKS + blockIdx.x) * 2 + 1] = t2;
    }
}
// out[v] = RMS(a - b), out[5 + v] = RMS(a - qinf_v); both floored at 1e-8 max_v |qinf_v|
// so that a state at rest does not divide by zero
__global__ void k_var_final(int nv, long long per, const double *part, const double *qinf, double *out) {
    int v = threadIdx.x;
    if (v >= nv) return;
    double qmax = 0.0;
    for (int w = 0; w < nv; ++w) qmax = fmax(qmax, fabs(qinf[w]));
    double fl = fmax(1e-8 * qmax, 1e-300);
    double t1 = 0.0, t2 = 0.0;
    for (int b = 0; b < VS_BLOCKS; ++b) { t1 += part[((size_t)v * VS_BLOCKS + b) * 2]; t2 += part[((size_t)v * VS_BLOCKS + b) * 2 + 1]; }
    out[v] = fmax(sqrt(t1 / (double)per), fl);
    out[5 + v] = fmax(sqrt(t2 / (double)per), fl);
}
int frkmlp_var_stats(int nv, long long per, const double *a, const double *b, const double *qinf_dev, double *part,
                     double *out_dev, cudaStream_t s) {
    CNT(); k_var_partials<<<dim3(VS_BLOCKS, nv), 256, 0, s>>>(per, a, b, qinf_dev, part);
    CNT(); k_var_final<<<1, 32, 0, s>>>(nv, per, part, qinf_dev, out_dev);
    return 0;
}

// network state for checkpoints: sizes, Adam step, FP32 weights and moments (host copies)
long long frkmlp_state_floats(const fr_mlp *M) { return 3LL * (long long)M->np; }
int frkmlp_state_save(const fr_mlp *M, int *dims4, float *buf) {
    dims4[0] = M->in; dims4[1] = M->hid; dims4[2] = M->out; dims4[3] = M->t;
    if (cudaMemcpy(buf, M->p, sizeof(float) * M->np, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    if (cudaMemcpy(buf + M->np, M->m, sizeof(float) * M->np, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    if (cudaMemcpy(buf + 2 * M->np, M->v, sizeof(float) * M->np, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    return 0;
}
int frkmlp_state_load(fr_mlp *M, const int *dims4, const float *buf) {
    if (dims4[0] != M->in || dims4[1] != M->hid || dims4[2] != M->out) return -1;
    M->t = dims4[3];
    if (cudaMemcpy(M->p, buf, sizeof(float) * M->np, cudaMemcpyHostToDevice) != cudaSuccess) return -1;
    if (cudaMemcpy(M->m, buf + M->np, sizeof(float) * M->np, cudaMemcpyHostToDevice) != cudaSuccess) return -1;
    if (cudaMemcpy(M->v, buf + 2 * M->np, sizeof(float) * M->np, cudaMemcpyHostToDevice) != cudaSuccess) return -1;
    CNT(); k_to_bf16<<<nb(M->np), 256>>>(M->np, M->p, M->pb);
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : -1;
}
