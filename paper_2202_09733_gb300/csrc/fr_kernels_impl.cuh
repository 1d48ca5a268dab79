// Kernels and launchers of the hot path, generic in the scalar type.  Included once per
// precision by a translation unit that defines
//   FRT            scalar type (double or float)
//   FRK(name)      launcher prefix (frk64_name / frk32_name)
//   FR_DOUBLE      1 for the FP64 unit (adds the Krylov/time-stepping vector kernels)
// The FP64 unit is compiled with -fmad=false, so there the only fused multiply-adds are
// the explicit fma() calls and every result follows the documented evaluation order.
#include <atomic>
#include <cuda_runtime.h>
#include <algorithm>
#include "fr_device.cuh"
#include "fr_lib.h"

static std::atomic<unsigned long long> g_launches{0};   // host-side launch counter (any thread)
unsigned long long FRK(launch_count)() { return g_launches; }
#define CNT() (g_launches.fetch_add(1, std::memory_order_relaxed))

__constant__ FrTab<FRT> c_tab[FR_MAXP + 1];
__constant__ FRT c_gam[FR_MAXP + 1][FR_MAXP + 1][FR_MAXN][FR_MAXN];
__constant__ FRT c_pi[FR_MAXP + 1][FR_MAXP + 1][FR_MAXN][FR_MAXN];

template <>
__device__ __forceinline__ const FrTab<FRT> &frtab<FRT>(int p) {
    return c_tab[p];
}

int FRK(upload_tables)(const FrTabH *tabs, const double *gam, const double *pi) {
    static FrTab<FRT> t[FR_MAXP + 1];
    static FRT g[(FR_MAXP + 1) * (FR_MAXP + 1) * FR_MAXN * FR_MAXN], p[(FR_MAXP + 1) * (FR_MAXP + 1) * FR_MAXN * FR_MAXN];
    for (int k = 0; k <= FR_MAXP; ++k)
        for (int i = 0; i < FR_MAXN; ++i) {
            for (int m = 0; m < FR_MAXN; ++m) t[k].D[i][m] = (FRT)tabs[k].D[i][m];
            t[k].lm[i] = (FRT)tabs[k].lm[i]; t[k].lp[i] = (FRT)tabs[k].lp[i];
            t[k].dlm[i] = (FRT)tabs[k].dlm[i]; t[k].dlp[i] = (FRT)tabs[k].dlp[i];
            t[k].gLd[i] = (FRT)tabs[k].gLd[i]; t[k].gRd[i] = (FRT)tabs[k].gRd[i];
        }
    for (size_t i = 0; i < sizeof(g) / sizeof(g[0]); ++i) { g[i] = (FRT)gam[i]; p[i] = (FRT)pi[i]; }
    if (cudaMemcpyToSymbol(c_tab, t, sizeof t) != cudaSuccess) return -1;
    if (cudaMemcpyToSymbol(c_gam, g, sizeof g) != cudaSuccess) return -1;
    if (cudaMemcpyToSymbol(c_pi, p, sizeof p) != cudaSuccess) return -1;
    return 0;
}

static FrPhys<FRT> to_phys(const FrPhysH &h, const FrLevelT<FRT> &L) {
    FrPhys<FRT> p;
    p.gamma = (FRT)h.gamma; p.gm1 = (FRT)h.gm1; p.mu = (FRT)h.mu; p.kappa = (FRT)h.kappa; p.c23 = (FRT)h.c23;
    for (int v = 0; v < 5; ++v) p.qinf[v] = (FRT)h.qinf[v];
    p.etagL = (FRT)L.etagL; p.etagR = (FRT)L.etagR;
    p.flux = h.flux;
    p.ws_umin = (FRT)h.ws_umin;
    return p;
}

// ------------------------------------------------------------------------ residual
template <int D, int P>
static void residual_t(const FrLevelT<FRT> &L, const FrPhys<FRT> &ph, const FRT *q, FRT *R, cudaStream_t s) {
    using S = Sh<D, P>;
    const int E = L.E;
    int b[8];
    for (int k = 0; k < 8; ++k) b[k] = L.tile[k] > 0 ? L.tile[k] : 128;
    auto gx = [&](int k) { return (E + b[k] - 1) / b[k]; };
    auto gp = [&](int k) { return (L.npairs + b[k] - 1) / b[k]; };
    CNT(); k_interp<D, P, FRT><<<dim3(S::nfp, gx(0)), b[0], 0, s>>>(q, L.qf, E);
    CNT(); k_pair_common<D, P, FRT><<<gp(1), b[1], 0, s>>>(L.pairs, L.bc, L.npairs, L.qf, L.dq, E, ph);
    CNT(); k_grad_fp<D, P, FRT><<<dim3(S::nfp, gx(3)), b[3], 0, s>>>(q, L.qf, L.dq, L.Gf, L.Qf, E, ph.etagL, ph.etagR);
    CNT(); k_pair_flux<D, P, FRT><<<gp(4), b[4], 0, s>>>(L.pairs, L.bc, L.npairs, L.qf, L.Qf, L.Sf, L.fn, E, ph);
    CNT(); k_grad_vflux<D, P, FRT><<<dim3(S::np, gx(2)), b[2], 0, s>>>(q, L.dq, L.G, L.S, L.Ft, E, ph);
    CNT(); k_face_ft<D, P, FRT><<<dim3(S::nfp, gx(6)), b[6], 0, s>>>(L.Ft, L.Ftf, E);
    CNT(); k_div<D, P, FRT><<<dim3(S::np, gx(7)), b[7], 0, s>>>(L.Ft, L.Ftf, L.fn, L.invJ, R, E);
}

int FRK(residual)(const FrLevelT<FRT> &L, const FrPhysH &h, const FRT *q, FRT *R, cudaStream_t s) {
    FrPhys<FRT> ph = to_phys(h, L);
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

// -------------------------------------------------------------- element partition
// Ghost exchange of a [rows][E] level vector: pack the owned elements idx[0..nsend) into
// buf[slot][rows] (slot-major, so every peer's slots are one contiguous chunk), and unpack
// buf[j][rows] into the ghost elements n_owned + j (j < nrecv).
__global__ void k_halo_pack(int rows, long long E, int nsend, const int *idx, const FRT *x, FRT *buf) {
    long long n = (long long)rows * nsend;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        int slot = (int)(t / rows), r = (int)(t - (long long)slot * rows);
        buf[t] = x[(size_t)r * E + idx[slot]];
    }
}
__global__ void k_halo_unpack(int rows, long long E, int n_owned, int nrecv, const FRT *buf, FRT *x) {
    long long n = (long long)rows * nrecv;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        int j = (int)(t / rows), r = (int)(t - (long long)j * rows);
        x[(size_t)r * E + n_owned + j] = buf[t];
    }
}
void FRK(halo_pack)(int rows, long long E, int nsend, const int *idx, const FRT *x, FRT *buf, cudaStream_t s) {
    long long n = (long long)rows * nsend;
    if (n == 0) return;
    CNT(); k_halo_pack<<<(int)std::min<long long>((n + 255) / 256, 152LL * 16), 256, 0, s>>>(rows, E, nsend, idx, x, buf);
}
void FRK(halo_unpack)(int rows, long long E, int n_owned, int nrecv, const FRT *buf, FRT *x, cudaStream_t s) {
    long long n = (long long)rows * nrecv;
    if (n == 0) return;
    CNT(); k_halo_unpack<<<(int)std::min<long long>((n + 255) / 256, 152LL * 16), 256, 0, s>>>(rows, E, n_owned, nrecv, buf, x);
}

// ------------------------------------------------------------------- elementwise
static inline int nblk(long long n, int b = 256) {
    long long g = (n + b - 1) / b;
    return (int)std::min<long long>(g, 152LL * 32);
}
#define GRID_STRIDE(i, n) \
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

__global__ void k_copy(long long n, const FRT *x, FRT *y) { GRID_STRIDE(i, n) y[i] = x[i]; }
__global__ void k_add(long long n, const FRT *a, const FRT *b, FRT *y) { GRID_STRIDE(i, n) y[i] = a[i] + b[i]; }
__global__ void k_sub(long long n, const FRT *a, const FRT *b, FRT *y) { GRID_STRIDE(i, n) y[i] = a[i] - b[i]; }
__global__ void k_pmg_rhs(long long n, FRT c, const FRT *d, const FRT *qh, const FRT *b, const FRT *Rqh, const FRT *Rb,
                          FRT *rhs) {
    GRID_STRIDE(i, n) {
        FRT t1 = qh[i] - b[i], t2 = Rqh[i] - Rb[i];
        rhs[i] = d[i] - (c * t1 - t2);
    }
}
void FRK(copy)(long long n, const FRT *x, FRT *y, cudaStream_t s) { CNT(); k_copy<<<nblk(n), 256, 0, s>>>(n, x, y); }
void FRK(add)(long long n, const FRT *a, const FRT *b, FRT *y, cudaStream_t s) { CNT(); k_add<<<nblk(n), 256, 0, s>>>(n, a, b, y); }
void FRK(sub)(long long n, const FRT *a, const FRT *b, FRT *y, cudaStream_t s) { CNT(); k_sub<<<nblk(n), 256, 0, s>>>(n, a, b, y); }
void FRK(pmg_rhs)(long long n, double c, const FRT *d, const FRT *qh, const FRT *b, const FRT *Rqh, const FRT *Rb,
                  FRT *rhs, cudaStream_t s) {
    CNT(); k_pmg_rhs<<<nblk(n), 256, 0, s>>>(n, (FRT)c, d, qh, b, Rqh, Rb, rhs);
}

// ------------------------------------------------------------------ element blocks
// Column j of the blocks of every element of colour `col`: forward difference with the
// step epsrel * max(1, |q_j|) on that element alone (elements of one colour share no
// face, so their perturbations do not interact in R restricted to each of them).
__global__ void k_perturb_color(int E, const int *color, int col, int j, const FRT *q, FRT *qp, FRT epsrel) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E || color[e] != col) return;
    FRT x = q[(size_t)j * E + e];
    FRT eps = epsrel * fmax((FRT)1, fabs(x));
    qp[(size_t)j * E + e] = x + eps;
}
__global__ void k_restore_color(int E, const int *color, int col, int j, const FRT *q, FRT *qp) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E || color[e] != col) return;
    qp[(size_t)j * E + e] = q[(size_t)j * E + e];
}
// tile: 32 elements x 32 rows through shared memory (coalesced on both sides)
__global__ void __launch_bounds__(256) k_block_column(int E, int nd, const int *color, int col, int j, const FRT *q,
                                                      const FRT *R0, const FRT *Rp, FRT shift, FRT epsrel, FRT *M) {
    __shared__ FRT tile[32][33];
    __shared__ int s_col[32];
    __shared__ FRT s_eps[32];
    int e0 = blockIdx.x * 32, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    if (threadIdx.x < 32) {
        int e = e0 + tx;
        int ok = e < E && color[e] == col;
        s_col[tx] = ok;
        FRT x = ok ? q[(size_t)j * E + e] : (FRT)0;
        s_eps[tx] = epsrel * fmax((FRT)1, fabs(x));
    }
    __syncthreads();
    for (int r0 = 0; r0 < nd; r0 += 32) {
        for (int rr = ty; rr < 32; rr += 8) {
            int r = r0 + rr, e = e0 + tx;
            FRT val = 0;
            if (r < nd && e < E && s_col[tx]) {
                FRT m = (Rp[(size_t)r * E + e] - R0[(size_t)r * E + e]) / s_eps[tx];
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
void FRK(perturb_color)(const FrLevelT<FRT> &L, const int *color, int col, int j, const FRT *q, FRT *qp, double epsrel,
                        cudaStream_t s) {
    CNT(); k_perturb_color<<<(L.E + 255) / 256, 256, 0, s>>>(L.E, color, col, j, q, qp, (FRT)epsrel);
}
void FRK(restore_color)(const FrLevelT<FRT> &L, const int *color, int col, int j, const FRT *q, FRT *qp, cudaStream_t s) {
    CNT(); k_restore_color<<<(L.E + 255) / 256, 256, 0, s>>>(L.E, color, col, j, q, qp);
}
void FRK(block_column)(const FrLevelT<FRT> &L, const int *color, int col, int j, const FRT *q, const FRT *R0,
                       const FRT *Rp, double shift, double epsrel, FRT *M, cudaStream_t s) {
    CNT(); k_block_column<<<(L.E + 31) / 32, 256, 0, s>>>(L.E, L.nd, color, col, j, q, R0, Rp, (FRT)shift, (FRT)epsrel, M);
}

// ------------------------------------------------------------------------ block LU
// One CTA per element block, column-major A(r, c) = A[c * nd + r]; right-looking
// elimination with partial pivoting (first maximal |a|, whole rows swapped),
// multipliers l = a / pivot, trailing updates a = fma(-l, u, a) in elimination order.
template <bool SMEM>
__global__ void __launch_bounds__(256) k_lu_factor(FRT *M, int *perm, int nd, int *info) {
    extern __shared__ __align__(16) unsigned char dsm_raw[];
    FRT *dsm = reinterpret_cast<FRT *>(dsm_raw);
    __shared__ FRT s_best[8];
    __shared__ int s_idx[8];
    __shared__ int s_p;
    int e = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    FRT *Ag = M + (size_t)e * nd * nd;
    FRT *A = SMEM ? dsm : Ag;
    int *pv = perm + (size_t)e * nd;
    if (SMEM)
        for (int t = tid; t < nd * nd; t += nt) A[t] = Ag[t];
    for (int t = tid; t < nd; t += nt) pv[t] = t;
    __syncthreads();
    int lane = tid & 31, wid = tid >> 5;
    for (int k = 0; k < nd; ++k) {
        FRT best = -1;
        int bi = nd;
        for (int i = k + tid; i < nd; i += nt) {
            FRT a = fabs(A[(size_t)k * nd + i]);
            if (a > best) { best = a; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            FRT ob = __shfl_down_sync(0xffffffffu, best, o);
            int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) { s_best[wid] = best; s_idx[wid] = bi; }
        __syncthreads();
        if (tid == 0) {
            FRT b = s_best[0];
            int ix = s_idx[0];
            for (int w = 1; w < nt / 32; ++w)
                if (s_best[w] > b || (s_best[w] == b && s_idx[w] < ix)) { b = s_best[w]; ix = s_idx[w]; }
            if (ix >= nd) ix = k;
            s_p = ix;
            if (b == (FRT)0) atomicExch(info, 1);
            if (ix != k) { int t = pv[k]; pv[k] = pv[ix]; pv[ix] = t; }
        }
        __syncthreads();
        int p = s_p;
        if (p != k)
            for (int c = tid; c < nd; c += nt) {
                FRT t = A[(size_t)c * nd + k];
                A[(size_t)c * nd + k] = A[(size_t)c * nd + p];
                A[(size_t)c * nd + p] = t;
            }
        __syncthreads();
        FRT piv = A[(size_t)k * nd + k];
        for (int i = k + 1 + tid; i < nd; i += nt) A[(size_t)k * nd + i] = A[(size_t)k * nd + i] / piv;
        __syncthreads();
        int m = nd - k - 1;
        for (int t = tid; t < m * m; t += nt) {
            int c = k + 1 + t / m, i = k + 1 + t % m;
            A[(size_t)c * nd + i] = fma(-A[(size_t)k * nd + i], A[(size_t)c * nd + k], A[(size_t)c * nd + i]);
        }
        __syncthreads();
    }
    // the factor keeps 1/u_kk in place of each pivot (the solve multiplies by it)
    for (int k = tid; k < nd; k += nt) A[(size_t)k * nd + k] = (FRT)1 / A[(size_t)k * nd + k];
    __syncthreads();
    if (SMEM)
        for (int t = tid; t < nd * nd; t += nt) Ag[t] = A[t];
}

// Blocked variant for blocks larger than shared memory: panels of LU_PB columns are
// factored in shared memory, their row swaps are then applied to the other columns, the
// panel rows of the trailing columns are forward-substituted (U12) and the trailing
// matrix receives its rank-LU_PB update in place.  Every entry still receives its updates
// a_ij = fma(-l_ik, u_kj, a_ij) one k at a time in ascending k, with the same multipliers
// and pivots as the unblocked elimination, so the factors are identical bit for bit.
#define LU_PB 32
__global__ void __launch_bounds__(256) k_lu_factor_blocked(FRT *M, int *perm, int nd, int *info) {
    extern __shared__ __align__(16) unsigned char dsm_raw[];
    FRT *Pn = reinterpret_cast<FRT *>(dsm_raw);              // [LU_PB][nd] panel, column-major
    FRT *U12 = Pn + (size_t)LU_PB * nd;                         // [nd][LU_PB] panel rows of trailing columns
    __shared__ FRT s_best[8];
    __shared__ int s_idx[8];
    __shared__ int s_p;
    __shared__ int s_piv[LU_PB];
    int e = blockIdx.x, tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
    FRT *A = M + (size_t)e * nd * nd;
    int *pv = perm + (size_t)e * nd;
    for (int t = tid; t < nd; t += nt) pv[t] = t;
    __syncthreads();
    for (int k0 = 0; k0 < nd; k0 += LU_PB) {
        int kb = min(LU_PB, nd - k0);
        // 1. panel to shared memory (rows k0..nd-1)
        for (int t = tid; t < kb * nd; t += nt) {
            int c = t / nd, i = t - c * nd;
            if (i >= k0) Pn[(size_t)c * nd + i] = A[(size_t)(k0 + c) * nd + i];
        }
        __syncthreads();
        // 2. unblocked elimination of the panel
        for (int c = 0; c < kb; ++c) {
            int k = k0 + c;
            FRT best = -1;
            int bi = nd;
            for (int i = k + tid; i < nd; i += nt) {
                FRT a = fabs(Pn[(size_t)c * nd + i]);
                if (a > best) { best = a; bi = i; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                FRT ob = __shfl_down_sync(0xffffffffu, best, o);
                int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (lane == 0) { s_best[wid] = best; s_idx[wid] = bi; }
            __syncthreads();
            if (tid == 0) {
                FRT b = s_best[0];
                int ix = s_idx[0];
                for (int w = 1; w < nt / 32; ++w)
                    if (s_best[w] > b || (s_best[w] == b && s_idx[w] < ix)) { b = s_best[w]; ix = s_idx[w]; }
                if (ix >= nd) ix = k;
                s_p = ix;
                s_piv[c] = ix;
                if (b == (FRT)0) atomicExch(info, 1);
                if (ix != k) { int t = pv[k]; pv[k] = pv[ix]; pv[ix] = t; }
            }
            __syncthreads();
            int p = s_p;
            if (p != k)
                for (int cc = tid; cc < kb; cc += nt) {
                    FRT t = Pn[(size_t)cc * nd + k];
                    Pn[(size_t)cc * nd + k] = Pn[(size_t)cc * nd + p];
                    Pn[(size_t)cc * nd + p] = t;
                }
            __syncthreads();
            FRT piv = Pn[(size_t)c * nd + k];
            for (int i = k + 1 + tid; i < nd; i += nt) Pn[(size_t)c * nd + i] = Pn[(size_t)c * nd + i] / piv;
            __syncthreads();
            int m = nd - k - 1, w = kb - c - 1;
            for (int t = tid; t < m * w; t += nt) {
                int cc = c + 1 + t / m, i = k + 1 + t % m;
                Pn[(size_t)cc * nd + i] = fma(-Pn[(size_t)c * nd + i], Pn[(size_t)cc * nd + k], Pn[(size_t)cc * nd + i]);
            }
            __syncthreads();
        }
        // 3. panel back to global memory
        for (int t = tid; t < kb * nd; t += nt) {
            int c = t / nd, i = t - c * nd;
            if (i >= k0) A[(size_t)(k0 + c) * nd + i] = Pn[(size_t)c * nd + i];
        }
        // 4. the panel's row swaps, in order, on every other column
        for (int j = tid; j < nd; j += nt) {
            if (j >= k0 && j < k0 + kb) continue;
            FRT *col = A + (size_t)j * nd;
            for (int c = 0; c < kb; ++c) {
                int p = s_piv[c], k = k0 + c;
                if (p != k) { FRT t = col[k]; col[k] = col[p]; col[p] = t; }
            }
        }
        __syncthreads();
        int r0 = k0 + kb, mt = nd - r0;
        if (mt > 0) {
            // 5. U12: forward substitution of the panel rows of every trailing column
            for (int j = r0 + tid; j < nd; j += nt) {
                FRT u[LU_PB];
                FRT *col = A + (size_t)j * nd + k0;
#pragma unroll
                for (int c = 0; c < LU_PB; ++c) u[c] = c < kb ? col[c] : (FRT)0;
#pragma unroll
                for (int cp = 0; cp < LU_PB; ++cp)
#pragma unroll
                    for (int c = cp + 1; c < LU_PB; ++c)
                        if (c < kb) u[c] = fma(-Pn[(size_t)cp * nd + k0 + c], u[cp], u[c]);
#pragma unroll
                for (int c = 0; c < LU_PB; ++c)
                    if (c < kb) { col[c] = u[c]; U12[(size_t)(j - r0) * LU_PB + c] = u[c]; }
            }
            __syncthreads();
            // 6. trailing update in place, one k at a time.  Register tiles of 4 rows x 4
            //    columns: consecutive threads take consecutive row tiles of one column
            //    tile, so the multipliers come as one 4-wide shared load per k and the
            //    U12 values are broadcasts; each entry still takes its fmas in ascending k.
            if (mt % 4 == 0 && nd % 4 == 0 && r0 % 4 == 0) {
                int ntr = mt / 4, ntile = ntr * ntr;
                for (int t = tid; t < ntile; t += nt) {
                    int tc = t / ntr, i0 = r0 + 4 * (t - tc * ntr), j0 = 4 * tc;
                    FRT acc[4][4];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
#pragma unroll
                        for (int r = 0; r < 4; ++r) acc[q][r] = A[(size_t)(r0 + j0 + q) * nd + i0 + r];
                    for (int c = 0; c < kb; ++c) {
                        const FRT *lc = Pn + (size_t)c * nd + i0;
                        FRT l[4], u[4];
                        if (sizeof(FRT) == 4) {
                            float4 v = *reinterpret_cast<const float4 *>(lc);
                            l[0] = v.x; l[1] = v.y; l[2] = v.z; l[3] = v.w;
                        } else {
#pragma unroll
                            for (int r = 0; r < 4; ++r) l[r] = lc[r];
                        }
#pragma unroll
                        for (int q = 0; q < 4; ++q) u[q] = U12[(size_t)(j0 + q) * LU_PB + c];
#pragma unroll
                        for (int q = 0; q < 4; ++q)
#pragma unroll
                            for (int r = 0; r < 4; ++r) acc[q][r] = fma(-l[r], u[q], acc[q][r]);
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q)
#pragma unroll
                        for (int r = 0; r < 4; ++r) A[(size_t)(r0 + j0 + q) * nd + i0 + r] = acc[q][r];
                }
            } else {
                for (int t = tid; t < mt * mt; t += nt) {
                    int jj = t / mt, i = r0 + (t - jj * mt);
                    FRT *pa = A + (size_t)(r0 + jj) * nd + i;
                    FRT a = *pa;
                    const FRT *uj = U12 + (size_t)jj * LU_PB;
                    for (int c = 0; c < kb; ++c) a = fma(-Pn[(size_t)c * nd + i], uj[c], a);
                    *pa = a;
                }
            }
        }
        __syncthreads();
    }
    // the factor keeps 1/u_kk in place of each pivot (the solve multiplies by it)
    for (int k = tid; k < nd; k += nt) A[(size_t)k * nd + k] = (FRT)1 / A[(size_t)k * nd + k];
}

int FRK(lu_factor)(const FrLevelT<FRT> &L, FRT *M, int *perm, int *info, cudaStream_t s) {
    size_t sm = sizeof(FRT) * (size_t)L.nd * L.nd;
    if (sm <= 200 * 1024) {
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_lu_factor<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            attr = true;
        }
        CNT(); k_lu_factor<true><<<L.E, 256, sm, s>>>(M, perm, L.nd, info);
        return 0;
    }
    size_t smb = sizeof(FRT) * (size_t)2 * LU_PB * L.nd;
    if (smb <= 200 * 1024) {
        static bool attrb = false;
        if (!attrb) {
            cudaFuncSetAttribute(k_lu_factor_blocked, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            attrb = true;
        }
        CNT(); k_lu_factor_blocked<<<L.E, 256, smb, s>>>(M, perm, L.nd, info);
        return 0;
    }
    CNT(); k_lu_factor<false><<<L.E, 256, 0, s>>>(M, perm, L.nd, info);
    return 0;
}

// One warp per element: rows i = lane + 32 s held in registers.  Forward substitution
// with the unit lower factor applies y_k to every later row in ascending k; backward
// substitution applies x_k to every earlier row in descending k (the order the unknowns
// become known), x_k = b_k (1/u_kk) with the reciprocal the factor stored.  Columns are fetched G at a time ahead of the
// dependent fma chain so that G column loads are in flight per step.
template <int NR>
__device__ __forceinline__ FRT pick(const FRT (&b)[NR], int slot) {
    FRT v = b[0];
#pragma unroll
    for (int s = 1; s < NR; ++s)
        if (s == slot) v = b[s];
    return v;
}

template <int NR, int G>
__global__ void __launch_bounds__(128) k_lu_solve(const FRT *__restrict__ M, const int *__restrict__ perm,
                                                  FRT *__restrict__ x, int nd, int E) {
    int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (e >= E) return;
    const FRT *A = M + (size_t)e * nd * nd;
    const int *pv = perm + (size_t)e * nd;
    FRT b[NR];
#pragma unroll
    for (int s = 0; s < NR; ++s) {
        int i = lane + 32 * s;
        b[s] = i < nd ? x[(size_t)pv[i] * E + e] : (FRT)0;
    }
    // forward: column k lives in register slot sk = k / 32 (compile-time in this unrolled
    // loop), so y_k is one shuffle of b[sk] and only slots sk.. hold rows below k
#pragma unroll
    for (int sk = 0; sk < NR; ++sk) {
        const int kend = min(nd, 32 * sk + 32);
        for (int k0 = 32 * sk; k0 < kend; k0 += G) {
            FRT cv[G][NR];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                int k = k0 + g;
                const FRT *col = A + (size_t)(k < kend ? k : kend - 1) * nd;
#pragma unroll
                for (int s = sk; s < NR; ++s) {
                    int i = lane + 32 * s;
                    bool need = k < kend && i < nd && (s > sk || lane > (k & 31));
                    cv[g][s] = need ? col[i] : (FRT)0;
                }
            }
#pragma unroll
            for (int g = 0; g < G; ++g) {
                int k = k0 + g;
                if (k >= kend) break;
                FRT yk = __shfl_sync(0xffffffffu, b[sk], k & 31);
#pragma unroll
                for (int s = sk; s < NR; ++s) {
                    int i = lane + 32 * s;
                    if (i < nd && (s > sk || lane > (k & 31))) b[s] = fma(-cv[g][s], yk, b[s]);
                }
            }
        }
    }
    // backward: x_k = b_k / u_kk on the owner lane, then rows above k; slots 0..sk
#pragma unroll
    for (int sk = NR - 1; sk >= 0; --sk) {
        const int kbeg = min(nd, 32 * sk + 32) - 1;
        for (int kt = kbeg; kt >= 32 * sk; kt -= G) {
            FRT cv[G][NR];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                int k = kt - g;
                const FRT *col = A + (size_t)(k >= 32 * sk ? k : 32 * sk) * nd;
#pragma unroll
                for (int s = 0; s <= sk; ++s) {
                    int i = lane + 32 * s;
                    bool need = k >= 32 * sk && (s < sk || lane <= (k & 31));
                    cv[g][s] = need ? col[i] : (FRT)0;
                }
            }
#pragma unroll
            for (int g = 0; g < G; ++g) {
                int k = kt - g;
                if (k < 32 * sk) break;
                int owner = k & 31;
                FRT xk = (FRT)0;
                if (lane == owner) xk = b[sk] * cv[g][sk];   // the factor holds 1/u_kk
                xk = __shfl_sync(0xffffffffu, xk, owner);
#pragma unroll
                for (int s = 0; s < sk; ++s) b[s] = fma(-cv[g][s], xk, b[s]);
                if (lane == owner) b[sk] = xk;
                else if (lane < owner) b[sk] = fma(-cv[g][sk], xk, b[sk]);
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (int s = 0; s < NR; ++s) {
        int i = lane + 32 * s;
        if (i < nd) x[(size_t)i * E + e] = b[s];
    }
}

// Block solve with the factor streamed through shared memory by the bulk-copy (TMA)
// engine.  One warp per element, LUB_W warps per CTA, each warp with its own ring of
// LUB_NS stages of cg columns and one mbarrier per stage.  Lane 0 issues, per column,
// one cp.async.bulk of exactly the rows the pass needs (forward: rows below the diagonal,
// from the 16-byte boundary at or before k+1; backward: rows 0..k, to the 16-byte
// boundary at or after k+1), so the factor is read about once per solve; the warp
// computes on stage t while stages t+1, t+2 are in flight.  The arithmetic is the
// register kernel's, fma for fma, so both give the same result bits.  Every wait is
// bounded: on time-out the warp waits (bounded) for its own copies in flight, records the
// failure in g_lub_err (bit 0) and returns; if that drain wait also ran out, copies may
// still land in the CTA's shared memory after it has exited, and bit 1 is set as well:
// the device's state is then undefined and the process should not launch more work.
// Needs nd * sizeof(FRT) % 16 == 0.
#define LUB_W 6
#define LUB_NS 3
#define LUB_STAGE_BYTES 12288
static __device__ int g_lub_err;

__device__ __forceinline__ unsigned lub_smem(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void lub_bar_init(unsigned long long *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(lub_smem(bar)));
}
__device__ __forceinline__ void lub_expect(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(lub_smem(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void lub_copy(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(lub_smem(dst)), "l"(src), "r"(bytes), "r"(lub_smem(bar)) : "memory");
}
__device__ __forceinline__ bool lub_wait(unsigned long long *bar, unsigned parity, int limit = 1 << 22) {
    for (int it = 0; it < limit; ++it) {
        unsigned done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(lub_smem(bar)), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// chunk t of the sequence: forward chunks (columns k0 .. k0+cg-1 ascending), then backward
// chunks (columns kt, kt-1, ... descending); returns the number of columns
__device__ __forceinline__ int lub_chunk(int t, int nf, int cg, int nd, bool *fwd, int *k0) {
    if (t < nf) {
        *fwd = true;
        *k0 = t * cg;
        return min(cg, nd - *k0);
    }
    *fwd = false;
    *k0 = nd - 1 - (t - nf) * cg;
    return min(cg, *k0 + 1);
}

// lane 0: stage the needed rows of the chunk's columns and arm the stage barrier
__device__ __forceinline__ void lub_issue(const FRT *A, FRT *stage, unsigned long long *bar, int t, int nf, int cg,
                                          int nd) {
    const int AL = 16 / (int)sizeof(FRT);
    bool fwd;
    int k0;
    int nc = lub_chunk(t, nf, cg, nd, &fwd, &k0);
    unsigned total = 0;
    for (int g = 0; g < nc; ++g) {
        int k = fwd ? k0 + g : k0 - g;
        int r0 = fwd ? ((k + 1) / AL) * AL : 0;
        int r1 = fwd ? nd : min(nd, ((k + 1 + AL - 1) / AL) * AL);
        total += (unsigned)((r1 - r0) * (int)sizeof(FRT));
    }
    lub_expect(bar, total);
    for (int g = 0; g < nc; ++g) {
        int k = fwd ? k0 + g : k0 - g;
        int r0 = fwd ? ((k + 1) / AL) * AL : 0;
        int r1 = fwd ? nd : min(nd, ((k + 1 + AL - 1) / AL) * AL);
        if (r1 > r0)
            lub_copy(stage + (size_t)g * nd + r0, A + (size_t)k * nd + r0, (unsigned)((r1 - r0) * (int)sizeof(FRT)), bar);
    }
}

template <int NR>
__global__ void __launch_bounds__(32 * LUB_W) k_lu_solve_bulk(const FRT *__restrict__ M, const int *__restrict__ perm,
                                                              FRT *__restrict__ x, int nd, int E, int cg) {
    extern __shared__ __align__(16) unsigned char lub_raw[];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(lub_raw) + warp * LUB_NS;
    FRT *ring = reinterpret_cast<FRT *>(lub_raw + 16 * ((LUB_W * LUB_NS * 8 + 15) / 16)) +
                (size_t)warp * LUB_NS * cg * nd;
    int e = blockIdx.x * LUB_W + warp;
    if (e >= E) return;   // warp-uniform: this warp has no element
    const FRT *A = M + (size_t)e * nd * nd;
    const int *pv = perm + (size_t)e * nd;
    if (lane == 0)
        for (int st = 0; st < LUB_NS; ++st) lub_bar_init(&bars[st]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncwarp();
    int nf = (nd + cg - 1) / cg, nt = 2 * nf;
    if (lane == 0)
        for (int t = 0; t < LUB_NS && t < nt; ++t) lub_issue(A, ring + (size_t)t * cg * nd, &bars[t], t, nf, cg, nd);
    FRT b[NR];
#pragma unroll
    for (int s = 0; s < NR; ++s) {
        int i = lane + 32 * s;
        b[s] = i < nd ? x[(size_t)pv[i] * E + e] : (FRT)0;
    }
    unsigned phase = 0;   // bit st: parity of stage st's next completion
    for (int t = 0; t < nt; ++t) {
        int st = t % LUB_NS;
        bool ok = lub_wait(&bars[st], (phase >> st) & 1u);
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) {
                int code = 1;
                // copies still in flight (issued for chunks t .. min(nt, t + LUB_NS) - 1)
                for (int u = t; u < nt && u < t + LUB_NS; ++u) {
                    int su = u % LUB_NS;
                    if (!lub_wait(&bars[su], (phase >> su) & 1u)) code = 3;
                    phase ^= 1u << su;
                }
                atomicOr(&g_lub_err, code);
            }
            __syncwarp();
            return;
        }
        phase ^= 1u << st;
        const FRT *stage = ring + (size_t)st * cg * nd;
        bool fwd;
        int k0;
        int nc = lub_chunk(t, nf, cg, nd, &fwd, &k0);
        if (fwd) {
            for (int g = 0; g < nc; ++g) {
                int k = k0 + g;
                const FRT *col = stage + (size_t)g * nd;
                FRT yk = __shfl_sync(0xffffffffu, pick<NR>(b, k >> 5), k & 31);
#pragma unroll
                for (int s = 0; s < NR; ++s) {
                    int i = lane + 32 * s;
                    if (i > k && i < nd) b[s] = fma(-col[i], yk, b[s]);
                }
            }
        } else {
            for (int g = 0; g < nc; ++g) {
                int k = k0 - g;
                const FRT *col = stage + (size_t)g * nd;
                int owner = k & 31, slot = k >> 5;
                FRT xk = (FRT)0;
                if (lane == owner) xk = pick<NR>(b, slot) * col[k];   // the factor holds 1/u_kk
                xk = __shfl_sync(0xffffffffu, xk, owner);
#pragma unroll
                for (int s = 0; s < NR; ++s) {
                    int i = lane + 32 * s;
                    if (i == k) b[s] = xk;
                    else if (i < k) b[s] = fma(-col[i], xk, b[s]);
                }
            }
        }
        __syncwarp();   // every lane is done with this stage before it is refilled
        if (lane == 0 && t + LUB_NS < nt) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic reads before the async writes
            lub_issue(A, ring + (size_t)st * cg * nd, &bars[st], t + LUB_NS, nf, cg, nd);
        }
    }
#pragma unroll
    for (int s = 0; s < NR; ++s) {
        int i = lane + 32 * s;
        if (i < nd) x[(size_t)i * E + e] = b[s];
    }
}

static int lub_cg(int nd) {
    int cg = LUB_STAGE_BYTES / (nd * (int)sizeof(FRT));
    return cg < 1 ? 1 : cg > 32 ? 32 : cg;
}
static size_t lub_smem_bytes(int nd) {
    return 16 * (size_t)((LUB_W * LUB_NS * 8 + 15) / 16) + (size_t)LUB_W * LUB_NS * lub_cg(nd) * nd * sizeof(FRT);
}

// shared-memory limits of the bulk kernel, set before any launch (and before any stream
// capture that may contain one)
void FRK(lu_solve_prepare)() {
    static bool done = false;
    if (done) return;
    int lim = 227 * 1024;
    cudaFuncSetAttribute(k_lu_solve_bulk<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_lu_solve_bulk<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_lu_solve_bulk<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_lu_solve_bulk<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_lu_solve_bulk<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_lu_solve_bulk<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    done = true;
}
// The time-out path of the bounded stage waits, exercised on purpose: one warp arms a
// barrier for 16 bytes that no copy will deliver, waits `limit` polls, records the
// failure and returns (nothing is in flight, so nothing is left behind).
static __global__ void k_wait_selftest(int limit) {
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) lub_bar_init(&bar);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncwarp();
    if (threadIdx.x == 0) lub_expect(&bar, 16);
    __syncwarp();
    bool ok = lub_wait(&bar, 0, limit);
    if (!__all_sync(0xffffffffu, ok) && threadIdx.x == 0) atomicOr(&g_lub_err, 1);
}
void FRK(wait_selftest)(int limit, cudaStream_t s) { CNT(); k_wait_selftest<<<1, 32, 0, s>>>(limit); }

int FRK(lu_solve_error)(int clear) {
    int h = 0;
    cudaMemcpyFromSymbol(&h, g_lub_err, sizeof(int));
    if (clear) {
        int z = 0;
        cudaMemcpyToSymbol(g_lub_err, &z, sizeof(int));
    }
    return h;
}

static bool lub_usable(int nd) {
    return (nd * (int)sizeof(FRT)) % 16 == 0 && lub_smem_bytes(nd) <= 227 * 1024;
}

template <int NR>
static void lub_launch(const FrLevelT<FRT> &L, const FRT *M, const int *perm, FRT *x, cudaStream_t s) {
    int grid = (L.E + LUB_W - 1) / LUB_W;
    CNT(); k_lu_solve_bulk<NR><<<grid, 32 * LUB_W, lub_smem_bytes(L.nd), s>>>(M, perm, x, L.nd, L.E, lub_cg(L.nd));
}

// G (columns in flight) is a launch-shape choice: 2, 4 or 8 where G x NR <= 40 registers
// of column data, else the largest allowed; every G gives the same result bits
template <int NR>
static int lu_solve_nr(int g, int grid, const FRT *M, const int *perm, FRT *x, int nd, int E, cudaStream_t s) {
    if (g >= 8 && 8 * NR <= 40) { CNT(); k_lu_solve<NR, 8><<<grid, 128, 0, s>>>(M, perm, x, nd, E); return 8; }
    if (g >= 4 && 4 * NR <= 40) { CNT(); k_lu_solve<NR, 4><<<grid, 128, 0, s>>>(M, perm, x, nd, E); return 4; }
    CNT(); k_lu_solve<NR, 2><<<grid, 128, 0, s>>>(M, perm, x, nd, E);
    return 2;
}

int FRK(lu_solve)(const FrLevelT<FRT> &L, const FRT *M, const int *perm, FRT *x, cudaStream_t s) {
    int nr = (L.nd + 31) / 32;
    int grid = (L.E * 32 + 127) / 128;
    // lu_g 1 selects the bulk-copy (TMA) kernel where the layout allows it
    if (L.lu_g == 1 && lub_usable(L.nd)) {
        switch (nr) {
            case 1: lub_launch<1>(L, M, perm, x, s); return 0;
            case 2: lub_launch<2>(L, M, perm, x, s); return 0;
            case 3: lub_launch<3>(L, M, perm, x, s); return 0;
            case 4: lub_launch<4>(L, M, perm, x, s); return 0;
            case 5: lub_launch<5>(L, M, perm, x, s); return 0;
            case 10: lub_launch<10>(L, M, perm, x, s); return 0;
            default: break;
        }
    }
    // default G: the choice measured best before tuning existed
    int g = L.lu_g > 1 ? L.lu_g : (nr <= 2 ? 8 : nr <= 5 ? 4 : (nr == 10 && sizeof(FRT) == 4) ? 4 : 2);
    switch (nr) {
        case 1: lu_solve_nr<1>(g, grid, M, perm, x, L.nd, L.E, s); break;
        case 2: lu_solve_nr<2>(g, grid, M, perm, x, L.nd, L.E, s); break;
        case 3: lu_solve_nr<3>(g, grid, M, perm, x, L.nd, L.E, s); break;
        case 4: lu_solve_nr<4>(g, grid, M, perm, x, L.nd, L.E, s); break;
        case 5: lu_solve_nr<5>(g, grid, M, perm, x, L.nd, L.E, s); break;
        case 6: lu_solve_nr<6>(g, grid, M, perm, x, L.nd, L.E, s); break;
        case 7: lu_solve_nr<7>(g, grid, M, perm, x, L.nd, L.E, s); break;
        case 8: lu_solve_nr<8>(g, grid, M, perm, x, L.nd, L.E, s); break;
        case 10: lu_solve_nr<10>(g, grid, M, perm, x, L.nd, L.E, s); break;
        default: return -1;
    }
    return 0;
}

// ------------------------------------------------------------------------ transfers
// thread per (e, v); 1-D operator along direction 0, then 1, then 2 (fma chains over the
// source index); sizes at run time (ni -> no points per direction), NM = max points.
template <int D, int NM>
__global__ void __launch_bounds__(128) k_tensor(const FRT *__restrict__ x, FRT *__restrict__ y, int E, int ni, int no,
                                                int p0, int p1, int restrict_) {
    constexpr int BUF = D == 2 ? NM * NM : NM * NM * NM;
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    int v = blockIdx.y;
    int npi = D == 2 ? ni * ni : ni * ni * ni, npo = D == 2 ? no * no : no * no * no;
    FRT a[BUF], b[BUF];
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
                    FRT acc = 0;
#pragma unroll 1
                    for (int m = 0; m < ni; ++m) {
                        int s0 = dir == 0 ? m : i0, s1 = dir == 1 ? m : i1, s2 = dir == 2 ? m : i2;
                        FRT op = restrict_ ? c_gam[p0][p1][o][m] : c_pi[p0][p1][o][m];
                        acc = fma(op, a[s0 + dims[0] * (s1 + dims[1] * s2)], acc);
                    }
                    b[i0 + nd0 * (i1 + nd1 * i2)] = acc;
                }
        dims[0] = nd0; dims[1] = nd1; dims[2] = nd2;
        int cnt = dims[0] * dims[1] * dims[2];
#pragma unroll 1
        for (int i = 0; i < cnt; ++i) a[i] = b[i];
    }
#pragma unroll 1
    for (int i = 0; i < npo; ++i) y[(size_t)(v * npo + i) * E + e] = a[i];
}

int FRK(transfer)(const FrLevelT<FRT> &Lf, const FrLevelT<FRT> &Lc, bool r, const FRT *x, FRT *y, cudaStream_t s) {
    int p0 = Lf.p, p1 = Lc.p, E = Lf.E, nv = Lf.nv;
    int ni = r ? p0 + 1 : p1 + 1, no = r ? p1 + 1 : p0 + 1;
    dim3 grid((E + 127) / 128, nv);
    if (Lf.d == 2 && p0 <= 5) { CNT(); k_tensor<2, 6><<<grid, 128, 0, s>>>(x, y, E, ni, no, p0, p1, r); }
    else if (Lf.d == 3 && p0 <= 3) { CNT(); k_tensor<3, 4><<<grid, 128, 0, s>>>(x, y, E, ni, no, p0, p1, r); }
    else return -1;
    return 0;
}
