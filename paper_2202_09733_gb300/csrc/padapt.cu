// p-adaptation indicator and marking (Sec. 3.3), FP64.
//
// The spectral-decay indicator of element e, eta_e = ||s_p - s_{p-1}||_L2 / ||s_p||_L2 of
// one variable s of the state: the element's nodal values on the tensor Gauss-Legendre
// points are expanded in tensor products of orthonormal Legendre polynomials (one 1-D
// transform per direction, M[a][i] = w_i phi_a(x_i)); s_{p-1} keeps the modes whose
// largest index is below p (the p - 1 level's tensor space), and by Parseval on the
// reference element eta_e^2 = (energy of the other modes) / (energy of all modes).  The
// marking rule raises an element's degree by one where eta_e > nu_max max(eta), lowers it
// by one where eta_e < nu_min max(eta), within [p_min, p_max].
#include <atomic>
#include "fr_lib.h"

static std::atomic<unsigned long long> g_launches{0};   // host-side launch counter (any thread)
unsigned long long frpa_launch_count() { return g_launches; }
#define CNT() (g_launches.fetch_add(1, std::memory_order_relaxed))

static __constant__ double c_modal[6][6][6];   // [p][a][i]

int frpa_upload(const double *modal /* [6][6][6] */) {
    return cudaMemcpyToSymbol(c_modal, modal, sizeof(double) * 216) == cudaSuccess ? 0 : -1;
}

namespace {

// one thread per element; s in registers, x index fastest
template <int D, int N>
__global__ void __launch_bounds__(128) k_spectral_decay(const double *__restrict__ q, int var, int E,
                                                        double *__restrict__ eta, unsigned long long *emax) {
    constexpr int NP = D == 2 ? N * N : N * N * N;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const double (*M)[6] = c_modal[N - 1];
    double s[NP], t[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) s[i] = q[(size_t)(var * NP + i) * E + e];
    // along x (stride 1), then y (stride N), then z (stride N^2)
#pragma unroll
    for (int dir = 0; dir < D; ++dir) {
        const int st = dir == 0 ? 1 : dir == 1 ? N : N * N;
#pragma unroll
        for (int o = 0; o < NP; ++o) {
            const int a = (o / st) % N, base = o - a * st;
            double acc = 0.0;
#pragma unroll
            for (int i = 0; i < N; ++i) acc = fma(M[a][i], s[base + i * st], acc);
            t[o] = acc;
        }
#pragma unroll
        for (int o = 0; o < NP; ++o) s[o] = t[o];
    }
    double all = 0.0, top = 0.0;
#pragma unroll
    for (int o = 0; o < NP; ++o) {
        const int a = o % N, b = (o / N) % N, c = D == 3 ? o / (N * N) : 0;
        const double v2 = s[o] * s[o];
        all += v2;
        if (a == N - 1 || b == N - 1 || (D == 3 && c == N - 1)) top += v2;
    }
    const double r = all > 0.0 ? sqrt(top / all) : 0.0;
    eta[e] = r;
    atomicMax(emax, (unsigned long long)__double_as_longlong(r));   // r >= 0: the bits order as the values
}

__global__ void k_padapt_mark(int E, const double *__restrict__ eta, const unsigned long long *emax,
                              const int *__restrict__ p_in, int p_min, int p_max, double nu_min, double nu_max,
                              int *__restrict__ p_out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const double m = __longlong_as_double((long long)*emax);
    int p = p_in[e];
    if (eta[e] > nu_max * m && p < p_max) ++p;
    else if (eta[e] < nu_min * m && p > p_min) --p;
    p_out[e] = p;
}

template <int D, int N>
void launch_decay(const double *q, int var, int E, double *eta, unsigned long long *emax, cudaStream_t s) {
    CNT();
    k_spectral_decay<D, N><<<(E + 127) / 128, 128, 0, s>>>(q, var, E, eta, emax);
}

}  // namespace

// eta[E] of variable var of the level state q ([nv][(p+1)^d][E]); emax_dev (one double,
// zeroed here) receives max(eta).  Returns -1 for an unsupported (d, p).
int frpa_spectral_decay(int d, int p, int E, const double *q, int var, double *eta, double *emax_dev,
                        cudaStream_t s) {
    if (cudaMemsetAsync(emax_dev, 0, sizeof(double), s) != cudaSuccess) return -1;
    unsigned long long *m = reinterpret_cast<unsigned long long *>(emax_dev);
    if (d == 2) {
        switch (p) {
            case 1: launch_decay<2, 2>(q, var, E, eta, m, s); return 0;
            case 2: launch_decay<2, 3>(q, var, E, eta, m, s); return 0;
            case 3: launch_decay<2, 4>(q, var, E, eta, m, s); return 0;
            case 4: launch_decay<2, 5>(q, var, E, eta, m, s); return 0;
            case 5: launch_decay<2, 6>(q, var, E, eta, m, s); return 0;
            default: return -1;
        }
    }
    if (d == 3) {
        switch (p) {
            case 1: launch_decay<3, 2>(q, var, E, eta, m, s); return 0;
            case 2: launch_decay<3, 3>(q, var, E, eta, m, s); return 0;
            case 3: launch_decay<3, 4>(q, var, E, eta, m, s); return 0;
            case 4: launch_decay<3, 5>(q, var, E, eta, m, s); return 0;
            default: return -1;
        }
    }
    return -1;
}

void frpa_mark(int E, const double *eta, const double *emax_dev, const int *p_in, int p_min, int p_max,
               double nu_min, double nu_max, int *p_out, cudaStream_t s) {
    CNT();
    k_padapt_mark<<<(E + 255) / 256, 256, 0, s>>>(E, eta, reinterpret_cast<const unsigned long long *>(emax_dev),
                                                  p_in, p_min, p_max, nu_min, nu_max, p_out);
}
