// Batched LU factorisation with partial pivoting of the FP32 element blocks of the
// mixed-precision preconditioner (the element-Jacobi blocks M_e = shift I - dR_e/dq_e of
// Eq. 9 and the block-Jacobi smoothing of Sec. 3.2), with the trailing updates on the
// fifth-generation tensor cores.
//
// The elimination is the right-looking blocked one, run as phases over the whole batch
// (tens of thousands of independent blocks), so that every phase has enough independent
// work to hide its latencies:
//   panel phase j     one CTA per block factors the panel (columns k0 .. k0+31, rows
//                     k0 .. nd-1) in shared memory: partial pivoting (first maximal |a|),
//                     whole panel rows interchanged, multipliers a / pivot, 1/u_kk left
//                     on the diagonal; the pivot rows go to ipiv (the perm array);
//   trailing phase j  one CTA per (block, 32-column tile of the trailing columns) takes
//                     the tile's rows k0 .. nd-1 in the panel's interchange order, solves
//                     U12 = L11^-1 A12 (unit lower L11), and forms A22 - L21 U12 with the
//                     product on the tensor cores: tcgen05.mma kind::tf32, M = 128 rows of
//                     L21, N = 32 columns, K = 32, each operand split into a TF32 head and
//                     a TF32 tail (x = hi + lo), hi*hi + hi*lo + lo*hi accumulated in FP32
//                     in tensor memory, which keeps the product at FP32 accuracy;
//   final             the interchanges of later panels are applied to the columns of L
//                     (the trailing phases leave the columns left of the panel alone) and
//                     the pivot sequence becomes the row permutation the block solve
//                     gathers with (perm[i] = row of the unfactored block now at row i).
// The factors have the layout of the CUDA-core kernels (column-major per block, unit L
// below the diagonal, U above it, 1/u_kk on it) and differ from them in the rounding of
// the trailing sums only.  Operands are staged in shared memory in the no-swizzle K-major
// core-matrix layout: 8 rows x 16 bytes per core matrix, K chunks 128 bytes apart, 8-row
// groups 32 * 32 bytes apart.  Every wait on a tensor-core completion is bounded; on
// time-out the CTA records it in g_lutc_err, frees its tensor memory and returns.
#include <atomic>
#include <cstdint>
#include <cuda_fp16.h>
#include "fr_lib.h"

static std::atomic<unsigned long long> g_launches{0};   // host-side launch counter (any thread)
unsigned long long frktc_launch_count() { return g_launches; }
#define CNT() (g_launches.fetch_add(1, std::memory_order_relaxed))

#define TC_NB 32       // panel width = K of the trailing product
#define TC_NT 32       // trailing columns per CTA = N of the product
#define TC_MAXND 384   // largest block handled here (three 128-row slots per thread)
static __device__ int g_lutc_err;

namespace {

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor: start address, leading (K-chunk) and stride
// (8-row group) byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major
__host__ __device__ constexpr unsigned umma_idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}
__device__ __forceinline__ float tf32_round(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
// offset (in floats) of element (row r, k) of a K-major operand with TC_NB k per row
__device__ __forceinline__ int core_off(int r, int k) {
    return (r >> 3) * (TC_NB * 8) + (k >> 2) * 32 + (r & 7) * 4 + (k & 3);
}
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, int limit = 1 << 24) {
    for (int it = 0; it < limit; ++it) {
        unsigned done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// position x after the row interchanges tau_t = (k0 + t, piv[t]), t = 0 .. n-1, applied
// in order to an array read as a gather: new[x] = old[tau_0(tau_1(... tau_{n-1}(x)))]
__device__ __forceinline__ int compose_swaps(const int *piv, int k0, int n, int x) {
    for (int t = n - 1; t >= 0; --t) {
        int a = k0 + t, b = piv[t];
        x = x == a ? b : (x == b ? a : x);
    }
    return x;
}

// ------------------------------------------------------------------------- panel
// The panel (rows k0 .. nd-1 of columns k0 .. k0+31) in shared memory, column-major
// P[c * R + i] = A(k0 + i, k0 + c); thread tid owns rows tid, tid + 128, ...  Per column:
// the pivot search (first maximal |a| below the diagonal), the interchange of the two rows
// across the panel (thread t swaps column t), then the multipliers a / pivot and the
// rank-1 update of the columns to the right; 1/u_kk replaces the pivots at the end.
__global__ void __launch_bounds__(128) k_lutc_panel(float *__restrict__ M, int *__restrict__ ipiv, int nd, int k0,
                                                    int *info) {
    extern __shared__ __align__(16) unsigned char pn_raw[];
    float *P = reinterpret_cast<float *>(pn_raw);
    __shared__ float wbest[4];
    __shared__ int widx[4];
    const int e = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float *A = M + (size_t)e * nd * nd;
    const int R = nd - k0, kb = min(TC_NB, R);
    for (int c = 0; c < kb; ++c) {
        const float *gc = A + (size_t)(k0 + c) * nd + k0;
        for (int i = tid; i < R; i += 128)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(P + c * R + i)), "l"(gc + i) : "memory");
    }
    asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
#pragma unroll 1
    for (int c = 0; c < kb; ++c) {
        float *pc = P + c * R;
        float best = -1.f;
        int bi = R;
        for (int i = c + tid; i < R; i += 128) {
            float v = fabsf(pc[i]);
            if (v > best) { best = v; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float ob = __shfl_xor_sync(0xffffffffu, best, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) { wbest[warp] = best; widx[warp] = bi; }
        __syncthreads();
        best = wbest[0];
        bi = widx[0];
#pragma unroll
        for (int w = 1; w < 4; ++w)
            if (wbest[w] > best || (wbest[w] == best && widx[w] < bi)) { best = wbest[w]; bi = widx[w]; }
        const int p = bi >= R ? c : bi;
        if (tid == 0) {
            ipiv[(size_t)e * nd + k0 + c] = k0 + p;
            if (best == 0.f) atomicExch(info, 1);
        }
        if (p != c && tid < kb) {
            float t = P[tid * R + c];
            P[tid * R + c] = P[tid * R + p];
            P[tid * R + p] = t;
        }
        __syncthreads();
        const float piv = pc[c];
        for (int i = c + 1 + tid; i < R; i += 128) {
            float l = pc[i] / piv;
            pc[i] = l;
            for (int c2 = c + 1; c2 < kb; ++c2) P[c2 * R + i] = fmaf(-l, P[c2 * R + c], P[c2 * R + i]);
        }
        __syncthreads();
    }
    // the factor keeps 1/u_kk (the solve multiplies by it)
    if (tid < kb) P[tid * R + tid] = 1.f / P[tid * R + tid];
    __syncthreads();
    for (int c = 0; c < kb; ++c) {
        float *gc = A + (size_t)(k0 + c) * nd + k0;
        for (int i = tid; i < R; i += 128) gc[i] = P[c * R + i];
    }
}

// ---------------------------------------------------------------------- trailing
// Shared memory: A operand head/tail (2 x 128 x TC_NB), B operand head/tail
// (2 x TC_NT x TC_NB), L11 and the tile's panel rows (TC_NB x TC_NB each), 48 KB in all,
// so four CTAs share an SM; each holds 32 tensor-memory columns (one 128 x 32 product).
//
// The panel's interchanges move rows only between the panel rows k0 .. k0+31 and the rows
// below: row i >= k0+32 of the tile ends up holding either itself or one of the panel rows
// (a transposition (k, p), p >= k, puts into position p what position k held, and
// position k only ever holds panel rows or the pivot row just brought there).  So the
// rows below can be read back where they are in the epilogue, each thread reading and then
// writing its own row, provided the panel rows are rewritten (as U12) only after every
// thread has read its sources; the panel rows' sources, which may be rows below, are read
// before any write.
#define TC_SMEM_FLOATS (2 * 128 * TC_NB + 2 * TC_NT * TC_NB + 2 * TC_NB * TC_NB)

__global__ void __launch_bounds__(128, 4) k_lutc_trail(float *__restrict__ M, const int *__restrict__ ipiv, int nd,
                                                    int k0, int ntiles) {
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    float *sAh = reinterpret_cast<float *>(tc_raw);
    float *sAl = sAh + 128 * TC_NB;
    float *sBh = sAl + 128 * TC_NB;
    float *sBl = sBh + TC_NT * TC_NB;
    float *L11 = sBl + TC_NT * TC_NB;    // column-major: L11[c' * TC_NB + c] = L(k0 + c, k0 + c')
    float *U = L11 + TC_NB * TC_NB;      // U[n * TC_NB + c]: tile column n, panel row c
    __shared__ int src[TC_MAXND];
    __shared__ int pv[TC_NB];
    __shared__ unsigned tmem_base;
    __shared__ int s_ok;
    __shared__ __align__(8) unsigned long long mbar;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int e = blockIdx.x / ntiles, tile = blockIdx.x - e * ntiles;
    float *A = M + (size_t)e * nd * nd;
    const int r0 = k0 + TC_NB, mt = nd - r0, R = nd - k0;
    const int j0 = r0 + tile * TC_NT, nt = min(TC_NT, nd - j0);
    const int mtiles = (mt + 127) / 128;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < TC_NB) pv[tid] = ipiv[(size_t)e * nd + k0 + tid];
    for (int i = tid; i < R; i += 128) src[i] = k0 + i;
    __syncthreads();
    // the panel's interchanges tau_c = (k0 + c, pv[c]), applied in order, as a gather:
    // tile row i <- matrix row src[i] = tau_0(tau_1(... tau_31(k0 + i))); only the panel
    // rows and the pivot rows move, so warp 0 composes just those (lane c: row k0 + c and
    // row pv[c]; a row named twice gets the same value twice)
    if (warp == 0) {
        int x0 = k0 + lane, x1 = pv[lane];
        int y0 = compose_swaps(pv, k0, TC_NB, x0), y1 = compose_swaps(pv, k0, TC_NB, x1);
        __syncwarp();
        src[x0 - k0] = y0;
        src[x1 - k0] = y1;
    }
    __syncthreads();
    // the panel rows of the tile (gathered) and L11, eight values per thread each
    {
        float u[TC_NB * TC_NT / 128], l[TC_NB * TC_NB / 128];
#pragma unroll
        for (int s = 0; s < TC_NB * TC_NT / 128; ++s) {
            int t = tid + 128 * s, n = t / TC_NB, c = t - n * TC_NB;
            u[s] = n < nt ? A[(size_t)(j0 + n) * nd + src[c]] : 0.f;
        }
#pragma unroll
        for (int s = 0; s < TC_NB * TC_NB / 128; ++s) {
            int t = tid + 128 * s, c = t / TC_NB, i = t - c * TC_NB;
            l[s] = A[(size_t)(k0 + c) * nd + k0 + i];
        }
#pragma unroll
        for (int s = 0; s < TC_NB * TC_NT / 128; ++s) U[tid + 128 * s] = u[s];
#pragma unroll
        for (int s = 0; s < TC_NB * TC_NB / 128; ++s) L11[tid + 128 * s] = l[s];
    }
    __syncthreads();
    // U12 = L11^-1 (panel rows): lane n takes column n; B operand row n, k = c
    if (warp == 0) {
        float u[TC_NB];
#pragma unroll
        for (int c = 0; c < TC_NB; ++c) u[c] = U[lane * TC_NB + c];
#pragma unroll
        for (int cp = 0; cp < TC_NB; ++cp)
#pragma unroll
            for (int c = cp + 1; c < TC_NB; ++c) u[c] = fmaf(-L11[cp * TC_NB + c], u[cp], u[c]);
#pragma unroll
        for (int c = 0; c < TC_NB; ++c) {
            U[lane * TC_NB + c] = u[c];
            float h = tf32_round(u[c]);
            sBh[core_off(lane, c)] = h;
            sBl[core_off(lane, c)] = tf32_round(u[c] - h);
        }
    }
    const unsigned tmem = tmem_base;
    constexpr unsigned idesc = umma_idesc_tf32(128, TC_NT);
    const unsigned LBO = 128, SBO = TC_NB * 32;
    bool ok = true;
    // per 128-row slab m of the trailing rows: thread tid owns row i = 128 m + tid, for which
    // it loads the L21 row (the product's A row) and the tile's source values, stages the
    // A row, and after the product takes its D row back: A22 row = sources - D row
    for (int m = 0; m < mtiles; ++m) {
        const int i = 128 * m + tid, row = r0 + i;
        const bool live = i < mt;
        const int sr = live ? src[TC_NB + i] : 0;
        float x[TC_NB], a[TC_NT];
#pragma unroll
        for (int c = 0; c < TC_NB; ++c) x[c] = live ? A[(size_t)(k0 + c) * nd + row] : 0.f;
#pragma unroll
        for (int n = 0; n < TC_NT; ++n) a[n] = (live && n < nt) ? A[(size_t)(j0 + n) * nd + sr] : 0.f;
#pragma unroll
        for (int q = 0; q < TC_NB / 4; ++q) {
            float h[4], lo[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) { h[j] = tf32_round(x[4 * q + j]); lo[j] = tf32_round(x[4 * q + j] - h[j]); }
            *reinterpret_cast<float4 *>(sAh + core_off(tid, 4 * q)) = make_float4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<float4 *>(sAl + core_off(tid, 4 * q)) = make_float4(lo[0], lo[1], lo[2], lo[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0 && ok) {
            const float *As[3] = {sAh, sAh, sAl};
            const float *Bs[3] = {sBh, sBl, sBh};
            for (int pass = 0; pass < 3; ++pass)
                for (int s = 0; s < TC_NB / 8; ++s) {
                    uint64_t ad = umma_desc(smem_u32(As[pass]) + 256u * s, LBO, SBO);
                    uint64_t bd = umma_desc(smem_u32(Bs[pass]) + 256u * s, LBO, SBO);
                    unsigned acc = (pass > 0 || s > 0) ? 1u : 0u;
                    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                                 ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(smem_u32(&mbar)) : "memory");
        }
        // one thread polls the barrier; the others wait at the CTA barrier (no issue slots)
        if (tid == 0) s_ok = ok && mbar_wait(&mbar, (unsigned)m & 1u);
        __syncthreads();              // also: sA is free for the next slab once every thread is here
        ok = s_ok;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!ok) break;
        unsigned d[32];
        unsigned ta = tmem + ((unsigned)(32 * warp) << 16);
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                     "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                     : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]),
                       "=r"(d[7]), "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]),
                       "=r"(d[14]), "=r"(d[15]), "=r"(d[16]), "=r"(d[17]), "=r"(d[18]), "=r"(d[19]), "=r"(d[20]),
                       "=r"(d[21]), "=r"(d[22]), "=r"(d[23]), "=r"(d[24]), "=r"(d[25]), "=r"(d[26]), "=r"(d[27]),
                       "=r"(d[28]), "=r"(d[29]), "=r"(d[30]), "=r"(d[31])
                     : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (live)
#pragma unroll
            for (int n = 0; n < TC_NT; ++n)
                if (n < nt) A[(size_t)(j0 + n) * nd + row] = a[n] - __uint_as_float(d[n]);
        // the next slab's product overwrites these tensor-memory columns: every warp's
        // tcgen05.ld has completed (wait::ld) before it passes the next slab's barrier
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    if (ok) {
        __syncthreads();   // every source read before the panel rows are rewritten
#pragma unroll
        for (int s = 0; s < TC_NB * TC_NT / 128; ++s) {
            int t = tid + 128 * s, n = t / TC_NB, c = t - n * TC_NB;
            if (n < nt) A[(size_t)(j0 + n) * nd + k0 + c] = U[t];
        }
    } else if (tid == 0) {
        atomicOr(&g_lutc_err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
}

// ------------------------------------------------------------------------- final
// One CTA per block.  For every position x (in parallel), the interchanges of panels
// j+1, j+2, ... composed as a gather give pi_j(x) (the rows of panel j's L columns below
// the next panel move by pi_j: new L(x, c) = L(pi_j(x), c)), and all of them give
// perm(x) = pi_{-1}(x).  Dynamic shared memory: the L columns of one panel
// (TC_NB x nd floats) and pi_j for every panel ((nd / TC_NB + 1) x nd ints).
__global__ void __launch_bounds__(128) k_lutc_final(float *__restrict__ M, int *__restrict__ perm, int nd) {
    extern __shared__ __align__(16) unsigned char fin_raw[];
    float *col = reinterpret_cast<float *>(fin_raw);
    int *pit = reinterpret_cast<int *>(col + (size_t)TC_NB * nd);   // pit[j * nd + x], j = panel
    __shared__ int piv[TC_MAXND];
    __shared__ int moved[TC_MAXND / TC_NB + 1];
    const int e = blockIdx.x, tid = threadIdx.x;
    const int np = (nd + TC_NB - 1) / TC_NB;
    float *A = M + (size_t)e * nd * nd;
    int *pg = perm + (size_t)e * nd;
    for (int i = tid; i < nd; i += 128) piv[i] = pg[i];
    if (tid < np) moved[tid] = 0;
    __syncthreads();
    for (int x = tid; x < nd; x += 128) {
        int y = x;
        for (int j = np - 1; j >= 0; --j) {
            // y = composite of the panels after j, applied to x
            if (j < np - 1 && x >= (j + 1) * TC_NB) {
                pit[j * nd + x] = y;
                if (y != x) moved[j] = 1;
            }
            const int k0 = j * TC_NB, n = min(TC_NB, nd - k0);
            for (int t = n - 1; t >= 0; --t) {
                int a = k0 + t, b = piv[k0 + t];
                y = y == a ? b : (y == b ? a : y);
            }
        }
        pg[x] = y;
    }
    __syncthreads();
    for (int j = 0; j + 1 < np; ++j) {
        if (!moved[j]) continue;   // uniform
        const int k0 = j * TC_NB, r1 = k0 + TC_NB, R = nd - r1;
        for (int c = 0; c < TC_NB; ++c) {
            const float *gc = A + (size_t)(k0 + c) * nd + r1;
            for (int i = tid; i < R; i += 128)
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(col + c * R + i)), "l"(gc + i)
                             : "memory");
        }
        asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        for (int c = 0; c < TC_NB; ++c)
            for (int i = tid; i < R; i += 128) A[(size_t)(k0 + c) * nd + r1 + i] = col[c * R + pit[j * nd + r1 + i] - r1];
        __syncthreads();
    }
}

static size_t final_smem(int nd) {
    return sizeof(float) * (size_t)TC_NB * nd + sizeof(int) * (size_t)(nd / TC_NB + 1) * nd;
}

// ---------------------------------------------------- factors stored at half width
// For the block solves of the smoother, the factors of a block at half the bytes: L
// (unit, |l| <= 1 under partial pivoting) as binary16; column k of U (rows < k) divided by
// its largest magnitude g_k, as binary16 (entries in [-1, 1]); per column, in FP32,
// (1/u_kk, g_k).  binary16 keeps 10 mantissa bits, the precision of TF32.  One CTA per
// block, one warp per column.
__global__ void __launch_bounds__(256) k_lutc_to_half(const float *__restrict__ M, __half *__restrict__ H,
                                                      float2 *__restrict__ dg, int nd) {
    const int e = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float *Ab = M + (size_t)e * nd * nd;
    __half *Hb = H + (size_t)e * nd * nd;
    for (int k = warp; k < nd; k += 8) {
        const float *col = Ab + (size_t)k * nd;
        float m = 0.f;
        for (int i = lane; i < k; i += 32) m = fmaxf(m, fabsf(col[i]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        const float g = m > 0.f ? m : 1.f, ig = 1.f / g;
        for (int i = lane; i < nd; i += 32) {
            float v = col[i];
            Hb[(size_t)k * nd + i] = __float2half_rn(i < k ? v * ig : (i > k ? v : 0.f));
        }
        if (lane == 0) dg[(size_t)e * nd + k] = make_float2(col[k], g);
    }
}

// x <- M_e^{-1} x with the half-width factors: the register solve of the FP32 factors
// (one warp per element, rows lane + 32 s in registers, G columns fetched ahead), with
// x_k = b_k (1/u_kk) and the rows above updated by the scaled column times g_k x_k.
template <int NR, int G>
__global__ void __launch_bounds__(128) k_lu_solve_half(const __half *__restrict__ H, const float2 *__restrict__ dg,
                                                       const int *__restrict__ perm, float *__restrict__ x, int nd,
                                                       int E) {
    int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (e >= E) return;
    const __half *A = H + (size_t)e * nd * nd;
    const float2 *D = dg + (size_t)e * nd;
    const int *pv = perm + (size_t)e * nd;
    float b[NR];
#pragma unroll
    for (int s = 0; s < NR; ++s) {
        int i = lane + 32 * s;
        b[s] = i < nd ? x[(size_t)pv[i] * E + e] : 0.f;
    }
#pragma unroll
    for (int sk = 0; sk < NR; ++sk) {
        const int kend = min(nd, 32 * sk + 32);
        for (int k0 = 32 * sk; k0 < kend; k0 += G) {
            float cv[G][NR];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                int k = k0 + g;
                const __half *col = A + (size_t)(k < kend ? k : kend - 1) * nd;
#pragma unroll
                for (int s = sk; s < NR; ++s) {
                    int i = lane + 32 * s;
                    bool need = k < kend && i < nd && (s > sk || lane > (k & 31));
                    cv[g][s] = need ? __half2float(col[i]) : 0.f;
                }
            }
#pragma unroll
            for (int g = 0; g < G; ++g) {
                int k = k0 + g;
                if (k >= kend) break;
                float yk = __shfl_sync(0xffffffffu, b[sk], k & 31);
#pragma unroll
                for (int s = sk; s < NR; ++s) {
                    int i = lane + 32 * s;
                    if (i < nd && (s > sk || lane > (k & 31))) b[s] = fmaf(-cv[g][s], yk, b[s]);
                }
            }
        }
    }
#pragma unroll
    for (int sk = NR - 1; sk >= 0; --sk) {
        const int kbeg = min(nd, 32 * sk + 32) - 1;
        for (int kt = kbeg; kt >= 32 * sk; kt -= G) {
            float cv[G][NR];
            float2 dk[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                int k = kt - g;
                int kk = k >= 32 * sk ? k : 32 * sk;
                const __half *col = A + (size_t)kk * nd;
                dk[g] = D[kk];
#pragma unroll
                for (int s = 0; s <= sk; ++s) {
                    int i = lane + 32 * s;
                    bool need = k >= 32 * sk && (s < sk || lane < (k & 31));
                    cv[g][s] = need ? __half2float(col[i]) : 0.f;
                }
            }
#pragma unroll
            for (int g = 0; g < G; ++g) {
                int k = kt - g;
                if (k < 32 * sk) break;
                int owner = k & 31;
                float xk = __shfl_sync(0xffffffffu, b[sk], owner) * dk[g].x;
                float xs = xk * dk[g].y;
#pragma unroll
                for (int s = 0; s < sk; ++s) b[s] = fmaf(-cv[g][s], xs, b[s]);
                if (lane == owner) b[sk] = xk;
                else if (lane < owner) b[sk] = fmaf(-cv[g][sk], xs, b[sk]);
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

template <int NR>
static void solve_half_nr(int g, int grid, const __half *H, const float2 *dg, const int *perm, float *x, int nd,
                          int E, cudaStream_t s) {
    if (g >= 8) k_lu_solve_half<NR, 8><<<grid, 128, 0, s>>>(H, dg, perm, x, nd, E);
    else if (g >= 4) k_lu_solve_half<NR, 4><<<grid, 128, 0, s>>>(H, dg, perm, x, nd, E);
    else k_lu_solve_half<NR, 2><<<grid, 128, 0, s>>>(H, dg, perm, x, nd, E);
}

}  // namespace

// the tensor-core factorisation handles blocks with TC_NB < nd <= TC_MAXND
int frktc_lu_supported(int nd) { return nd > 2 * TC_NB && nd <= TC_MAXND; }

int frktc_lu_factor(int E, int nd, float *M, int *perm, int *info, cudaStream_t s) {
    if (!frktc_lu_supported(nd) || E <= 0) return 1;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_lutc_trail, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(float) * TC_SMEM_FLOATS));
        cudaFuncSetAttribute(k_lutc_final, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)final_smem(TC_MAXND));
        cudaFuncSetAttribute(k_lutc_panel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(float) * TC_NB * TC_MAXND));
        attr = true;
    }
    for (int k0 = 0; k0 < nd; k0 += TC_NB) {
        int rows = nd - k0;
        CNT();
        k_lutc_panel<<<E, 128, sizeof(float) * TC_NB * rows, s>>>(M, perm, nd, k0, info);
        if (k0 + TC_NB < nd) {
            int ntiles = (nd - k0 - TC_NB + TC_NT - 1) / TC_NT;
            long long grid = (long long)ntiles * E;
            if (grid > 0x7fffffffLL) return 1;
            CNT();
            k_lutc_trail<<<(unsigned)grid, 128, sizeof(float) * TC_SMEM_FLOATS, s>>>(M, perm, nd, k0, ntiles);
        }
    }
    CNT();
    k_lutc_final<<<E, 128, final_smem(nd), s>>>(M, perm, nd);
    return 0;
}

int frktc_lu_error(int clear) {
    int h = 0;
    cudaMemcpyFromSymbol(&h, g_lutc_err, sizeof(int));
    if (clear && h) {
        int z = 0;
        cudaMemcpyToSymbol(g_lutc_err, &z, sizeof(int));
    }
    return h ? 4 : 0;
}

int frktc_lu_to_half(int E, int nd, const float *M, void *H, float *dg, cudaStream_t s) {
    if (E <= 0 || nd <= 0) return 1;
    CNT();
    k_lutc_to_half<<<E, 256, 0, s>>>(M, (__half *)H, (float2 *)dg, nd);
    return 0;
}

int frktc_lu_solve_half(int E, int nd, int g, const void *H, const float *dg, const int *perm, float *x,
                        cudaStream_t s) {
    int nr = (nd + 31) / 32, grid = (E * 32 + 127) / 128;
    const __half *h = (const __half *)H;
    const float2 *d = (const float2 *)dg;
    CNT();
    switch (nr) {
        case 1: solve_half_nr<1>(g, grid, h, d, perm, x, nd, E, s); break;
        case 2: solve_half_nr<2>(g, grid, h, d, perm, x, nd, E, s); break;
        case 3: solve_half_nr<3>(g, grid, h, d, perm, x, nd, E, s); break;
        case 4: solve_half_nr<4>(g, grid, h, d, perm, x, nd, E, s); break;
        case 5: solve_half_nr<5>(g, grid, h, d, perm, x, nd, E, s); break;
        case 6: solve_half_nr<6>(g, grid, h, d, perm, x, nd, E, s); break;
        case 7: solve_half_nr<7>(g, grid, h, d, perm, x, nd, E, s); break;
        case 8: solve_half_nr<8>(g, grid, h, d, perm, x, nd, E, s); break;
        case 10: solve_half_nr<10>(g, grid, h, d, perm, x, nd, E, s); break;
        default: return -1;
    }
    return 0;
}
