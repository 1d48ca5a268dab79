// FP32 element-diagonal Jacobian blocks by forward-mode differentiation: the residual
// kernels run on DualT (FR_AD_K tangents) with tangent t seeded 1 in degree of freedom
// j0 + t of every element of one colour (elements of a colour share no face), so R.d[t]
// restricted to each of those elements is column j0 + t of its block dR_e/dq_e, exact up
// to FP32 rounding of each term.  One residual evaluation gives FR_AD_K columns.
#include <atomic>
#include <algorithm>
#include "fr_device.cuh"
#include "fr_lib.h"

static std::atomic<unsigned long long> g_launches{0};   // host-side launch counter (any thread)
unsigned long long frkad_launch_count() { return g_launches; }
#define CNT() (g_launches.fetch_add(1, std::memory_order_relaxed))

__constant__ FrTab<float> c_tab_ad[FR_MAXP + 1];
template <>
__device__ __forceinline__ const FrTab<float> &frtab<float>(int p) {
    return c_tab_ad[p];
}

int frkad_upload_tables(const FrTabH *tabs) {
    static FrTab<float> t[FR_MAXP + 1];
    for (int k = 0; k <= FR_MAXP; ++k)
        for (int i = 0; i < FR_MAXN; ++i) {
            for (int m = 0; m < FR_MAXN; ++m) t[k].D[i][m] = (float)tabs[k].D[i][m];
            t[k].lm[i] = (float)tabs[k].lm[i]; t[k].lp[i] = (float)tabs[k].lp[i];
            t[k].dlm[i] = (float)tabs[k].dlm[i]; t[k].dlp[i] = (float)tabs[k].dlp[i];
            t[k].gLd[i] = (float)tabs[k].gLd[i]; t[k].gRd[i] = (float)tabs[k].gRd[i];
        }
    return cudaMemcpyToSymbol(c_tab_ad, t, sizeof t) == cudaSuccess ? 0 : -1;
}

template <int D, int P>
static void residual_ad(const FrLevelAD &L, const FrPhys<float> &ph, const DualT *q, DualT *R, cudaStream_t s) {
    using S = Sh<D, P>;
    const int E = L.E, gx = (E + 127) / 128, gp = (L.npairs + 127) / 128;
    CNT(); k_interp<D, P, DualT><<<dim3(S::nfp, gx), 128, 0, s>>>(q, L.qf, E);
    CNT(); k_pair_common<D, P, DualT><<<gp, 128, 0, s>>>(L.pairs, L.bc, L.npairs, L.qf, L.dq, E, ph);
    CNT(); k_grad_fp<D, P, DualT><<<dim3(S::nfp, gx), 128, 0, s>>>(q, L.qf, L.dq, L.Gf, L.Qf, E, ph.etagL, ph.etagR);
    CNT(); k_pair_flux<D, P, DualT><<<gp, 128, 0, s>>>(L.pairs, L.bc, L.npairs, L.qf, L.Qf, L.Sf, L.fn, E, ph);
    CNT(); k_grad_vflux<D, P, DualT><<<dim3(S::np, gx), 128, 0, s>>>(q, L.dq, L.G, L.S, L.Ft, E, ph);
    CNT(); k_face_ft<D, P, DualT><<<dim3(S::nfp, gx), 128, 0, s>>>(L.Ft, L.Ftf, E);
    CNT(); k_div<D, P, DualT><<<dim3(S::np, gx), 128, 0, s>>>(L.Ft, L.Ftf, L.fn, L.invJ, R, E);
}

int frkad_residual(const FrLevelAD &L, const FrPhysH &h, const DualT *q, DualT *R, cudaStream_t s) {
    FrPhys<float> ph;
    ph.gamma = (float)h.gamma; ph.gm1 = (float)h.gm1; ph.mu = (float)h.mu; ph.kappa = (float)h.kappa;
    ph.c23 = (float)h.c23;
    for (int v = 0; v < 5; ++v) ph.qinf[v] = (float)h.qinf[v];
    ph.etagL = (float)L.etagL; ph.etagR = (float)L.etagR;
    ph.flux = h.flux;
    ph.ws_umin = (float)h.ws_umin;
    if (L.d == 2) {
        switch (L.p) {
            case 1: residual_ad<2, 1>(L, ph, q, R, s); return 0;
            case 2: residual_ad<2, 2>(L, ph, q, R, s); return 0;
            case 3: residual_ad<2, 3>(L, ph, q, R, s); return 0;
            case 4: residual_ad<2, 4>(L, ph, q, R, s); return 0;
        }
    } else if (L.d == 3) {
        switch (L.p) {
            case 1: residual_ad<3, 1>(L, ph, q, R, s); return 0;
            case 2: residual_ad<3, 2>(L, ph, q, R, s); return 0;
            case 3: residual_ad<3, 3>(L, ph, q, R, s); return 0;
        }
    }
    return -1;
}

__global__ void k_ad_init(long long n, const float *q, DualT *qd) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        qd[i] = DualT(q[i]);
}
void frkad_init(long long n, const float *q, DualT *qd, cudaStream_t s) {
    int g = (int)std::min<long long>((n + 255) / 256, 152LL * 32);
    CNT(); k_ad_init<<<g, 256, 0, s>>>(n, q, qd);
}
// tangent t of dof j0 + t (< nd) of every element of the colour: seed (1) or clear (0)
__global__ void k_ad_seed(int E, int nd, const int *color, int col, int j0, DualT *qd, float seed) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E || color[e] != col) return;
#pragma unroll
    for (int t = 0; t < FR_AD_K; ++t)
        if (j0 + t < nd) qd[(size_t)(j0 + t) * E + e].d[t] = seed;
}
void frkad_seed(const FrLevelAD &L, const int *color, int col, int j0, DualT *qd, float seed, cudaStream_t s) {
    CNT(); k_ad_seed<<<(L.E + 255) / 256, 256, 0, s>>>(L.E, L.nd, color, col, j0, qd, seed);
}
// M[e][j][r] = (r == j ? shift : 0) - dR_r/dq_j for j = j0 + t, t < FR_AD_K (tiled)
__global__ void __launch_bounds__(256) k_ad_column(int E, int nd, const int *color, int col, int j0, const DualT *Rd,
                                                   float shift, float *M) {
    __shared__ float tile[32][33];
    __shared__ int s_col[32];
    int e0 = blockIdx.x * 32, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    if (threadIdx.x < 32) {
        int e = e0 + tx;
        s_col[tx] = e < E && color[e] == col;
    }
    __syncthreads();
    for (int t = 0; t < FR_AD_K; ++t) {
        int j = j0 + t;
        if (j >= nd) break;
        for (int r0 = 0; r0 < nd; r0 += 32) {
            for (int rr = ty; rr < 32; rr += 8) {
                int r = r0 + rr, e = e0 + tx;
                float val = 0.f;
                if (r < nd && e < E && s_col[tx]) {
                    float dr = Rd[(size_t)r * E + e].d[t];
                    val = (r == j) ? shift - dr : -dr;
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
}
void frkad_block_column(const FrLevelAD &L, const int *color, int col, int j0, const DualT *Rd, double shift,
                        float *M, cudaStream_t s) {
    CNT(); k_ad_column<<<(L.E + 31) / 32, 256, 0, s>>>(L.E, L.nd, color, col, j0, Rd, (float)shift, M);
}

// O_(e,f)[j][r] (column-major blocks) = -dR_e[r]/dq_n[j] for the face neighbour
// n = nbr[f E + e] of colour col, j = j0 + t, t < FR_AD_K (distance-2 colours: at most one
// seeded element among e and its neighbours); one thread per (element, row)
__global__ void k_ad_nbr_column(int E, int nd, int nf, const int *nbr, const int *color2, int col, int j0,
                                const DualT *Rd, float *O) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)E * nd) return;
    int e = (int)(t / nd), r = (int)(t - (long long)e * nd);
    for (int f = 0; f < nf; ++f) {
        int n = nbr[(size_t)f * E + e];
        if (n < 0 || color2[n] != col) continue;
        DualT R = Rd[(size_t)r * E + e];
#pragma unroll
        for (int k = 0; k < FR_AD_K; ++k)
            if (j0 + k < nd) O[(((size_t)e * nf + f) * nd + j0 + k) * nd + r] = -R.d[k];
    }
}
void frkad_nbr_column(const FrLevelAD &L, int nf, const int *nbr, const int *color2, int col, int j0,
                      const DualT *Rd, float *O, cudaStream_t s) {
    long long n = (long long)L.E * L.nd;
    CNT(); k_ad_nbr_column<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(L.E, L.nd, nf, nbr, color2, col, j0, Rd, O);
}

// ------------------------------------------- element-local blocks (fr_ad_elem.cuh)
#include "fr_ad_elem.cuh"

static FrPhys<float> ad_phys(const FrPhysH &h, const FrLevel32 &L) {
    FrPhys<float> ph;
    ph.gamma = (float)h.gamma; ph.gm1 = (float)h.gm1; ph.mu = (float)h.mu; ph.kappa = (float)h.kappa;
    ph.c23 = (float)h.c23;
    for (int v = 0; v < 5; ++v) ph.qinf[v] = (float)h.qinf[v];
    ph.etagL = (float)L.etagL; ph.etagR = (float)L.etagR;
    ph.flux = h.flux;
    ph.ws_umin = (float)h.ws_umin;
    return ph;
}

// elements per CTA: two CTAs of 128 threads per SM within about 100 KB of shared memory each
template <int D, int P>
static int ad_elem_te() {
    int te = (int)((100 * 1024) / AdElem<D, P>::bytes_per_elem);
    return te < 1 ? 1 : (te > 32 ? 32 : te);
}

template <int D, int P>
static void ad_elem_t(const FrLevel32 &L, const FrPhys<float> &ph, const float *q, const float *qf, const float *Qf,
                      float *NT, signed char *BCk, double shift, float *M, cudaStream_t s) {
    const int E = L.E, TE = ad_elem_te<D, P>();
    const size_t smem = (size_t)TE * AdElem<D, P>::bytes_per_elem;
    static bool attr_done = false;   // per instantiation; set before the first launch
    if (!attr_done) {
        cudaFuncSetAttribute(k_ad_elem_blocks<D, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_done = true;
    }
    CNT(); k_ad_traces<D, P><<<(L.npairs + 255) / 256, 256, 0, s>>>(L.pairs, L.bc, L.npairs, qf, Qf, L.Gf,
                                                                    ph.etagL, ph.etagR, E, NT, BCk);
    CNT(); k_ad_elem_blocks<D, P><<<(E + TE - 1) / TE, 128, smem, s>>>(q, L.G, L.S, L.invJ, L.Gf, L.Sf, NT, BCk, E, TE,
                                                                        ph, (float)shift, M);
}

long long frkad_elem_nt_floats(const FrLevel32 &L) { return (long long)(L.nv + L.d * L.nv + L.d) * L.nfp * L.E; }

int frkad_elem_blocks(const FrLevel32 &L, const FrPhysH &h, const float *q, const float *qf, const float *Qf,
                      float *NT, signed char *BCk, double shift, float *M, cudaStream_t s) {
    FrPhys<float> ph = ad_phys(h, L);
    if (L.d == 2) {
        switch (L.p) {
            case 1: ad_elem_t<2, 1>(L, ph, q, qf, Qf, NT, BCk, shift, M, s); return 0;
            case 2: ad_elem_t<2, 2>(L, ph, q, qf, Qf, NT, BCk, shift, M, s); return 0;
            case 3: ad_elem_t<2, 3>(L, ph, q, qf, Qf, NT, BCk, shift, M, s); return 0;
            case 4: ad_elem_t<2, 4>(L, ph, q, qf, Qf, NT, BCk, shift, M, s); return 0;
        }
    } else if (L.d == 3) {
        switch (L.p) {
            case 1: ad_elem_t<3, 1>(L, ph, q, qf, Qf, NT, BCk, shift, M, s); return 0;
            case 2: ad_elem_t<3, 2>(L, ph, q, qf, Qf, NT, BCk, shift, M, s); return 0;
            case 3: ad_elem_t<3, 3>(L, ph, q, qf, Qf, NT, BCk, shift, M, s); return 0;
        }
    }
    return -1;
}
