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
//                     on the diagonal; the pivot rows go to ipiv (the perm array) and L21,
//                     split into TF32 head and tail, to a scratch buffer;
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
#define TC_PF 16       // half-width solve: columns prefetched ahead into L2
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
// Block e (A its matrix), panel k0; P: (nd - k0) x TC_NB floats of shared memory; 128
// threads.  Also writes the trailing phase's split L21 operand into l21 (block e's slabs).
__device__ __forceinline__ void factor_panel(float *__restrict__ A, int *__restrict__ ipiv, int nd, int k0, int *info,
                                          float *__restrict__ l21, int mtiles, float *P, int e) {
    __shared__ float wbest[4];
    __shared__ int widx[4];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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
    // the trailing phase's A operand, once per block: L21 (rows k0+32 .. nd-1 of the panel)
    // split into TF32 head and tail, in the K-major core-matrix layout of 128-row slabs
    // ([slab][head, tail][128 x TC_NB]), rows past the block zero
    if (mtiles > 0) {
        float *out = l21 + (size_t)e * mtiles * 2 * 128 * TC_NB;
        for (int m = 0; m < mtiles; ++m) {
            const int i = TC_NB + 128 * m + tid;   // panel row
            const bool live = i < R;
            float *oh = out + (size_t)(2 * m) * 128 * TC_NB, *ol = oh + 128 * TC_NB;
#pragma unroll
            for (int q = 0; q < TC_NB / 4; ++q) {
                float h[4], lo[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float x = live ? P[(4 * q + j) * R + i] : 0.f;
                    h[j] = tf32_round(x);
                    lo[j] = tf32_round(x - h[j]);
                }
                *reinterpret_cast<float4 *>(oh + core_off(tid, 4 * q)) = make_float4(h[0], h[1], h[2], h[3]);
                *reinterpret_cast<float4 *>(ol + core_off(tid, 4 * q)) = make_float4(lo[0], lo[1], lo[2], lo[3]);
            }
        }
    }
}

// the first panel: one CTA per block
__global__ void __launch_bounds__(128) k_lutc_panel(float *__restrict__ M, int *__restrict__ ipiv, int nd, int k0,
                                                    int *info, float *__restrict__ l21, int mtiles) {
    extern __shared__ __align__(16) unsigned char pn_raw[];
    const int e = blockIdx.x;
    factor_panel(M + (size_t)e * nd * nd, ipiv, nd, k0, info, l21, mtiles, reinterpret_cast<float *>(pn_raw), e);
}

// ---------------------------------------------------------------------- trailing
// Shared memory: A operand head/tail (2 x 128 x TC_NB), B operand head/tail
// (2 x TC_NT x TC_NB), L11 and the tile's panel rows (TC_NB x TC_NB each), 48 KB in all,
// so four CTAs share an SM; each holds 64 tensor-memory columns (two 128 x 32 products).
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
                                                       int k0, int ntiles, const float *__restrict__ l21) {
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
    __shared__ __align__(8) unsigned long long mbar, cbar;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int e = blockIdx.x / ntiles, tile = blockIdx.x - e * ntiles;
    float *A = M + (size_t)e * nd * nd;
    const int r0 = k0 + TC_NB, mt = nd - r0, R = nd - k0;
    const int j0 = r0 + tile * TC_NT, nt = min(TC_NT, nd - j0);
    const int mtiles = (mt + 127) / 128;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_u32(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&cbar)));
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
    // per 128-row slab m of the trailing rows: the slab's A operand (the panel kernel's
    // split L21) comes by two bulk copies while thread tid loads the tile's source values
    // of its row i = 128 m + tid; after the product, A22 row = sources - D row
    const float *slabs = l21 + (size_t)e * mtiles * 2 * 128 * TC_NB;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // B (generic stores) before the products
    __syncthreads();
    for (int m = 0; m < mtiles; ++m) {
        const int i = 128 * m + tid, row = r0 + i;
        const bool live = i < mt;
        const int sr = live ? src[TC_NB + i] : 0;
        if (tid == 0 && ok) {
            // sA is free: the previous slab's product has completed (waited below)
            const unsigned bytes = 2u * 128u * TC_NB * 4u;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&cbar)), "r"(bytes)
                         : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         ::"r"(smem_u32(sAh)), "l"(slabs + (size_t)(2 * m) * 128 * TC_NB), "r"(bytes),
                           "r"(smem_u32(&cbar)) : "memory");
        }
        float a[TC_NT];
#pragma unroll
        for (int n = 0; n < TC_NT; ++n) a[n] = (live && n < nt) ? A[(size_t)(j0 + n) * nd + sr] : 0.f;
        if (tid == 0) {
            bool okk = ok && mbar_wait(&cbar, (unsigned)m & 1u);
            if (ok && !okk && !mbar_wait(&cbar, (unsigned)m & 1u))
                atomicOr(&g_lutc_err, 2);   // the slab's copy is still in flight: shared memory undefined
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (okk) {
                const float *As[3] = {sAh, sAh, sAl};
                const float *Bs[3] = {sBh, sBl, sBh};
                for (int pass = 0; pass < 3; ++pass)
                    for (int s = 0; s < TC_NB / 8; ++s) {
                        uint64_t ad = umma_desc(smem_u32(As[pass]) + 256u * s, LBO, SBO);
                        uint64_t bd = umma_desc(smem_u32(Bs[pass]) + 256u * s, LBO, SBO);
                        unsigned acc = (pass > 0 || s > 0) ? 1u : 0u;
                        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                     " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                                     ::"r"(tmem + 32u * (m & 1)), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                    }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(smem_u32(&mbar)) : "memory");
                okk = mbar_wait(&mbar, (unsigned)m & 1u);
            }
            s_ok = okk;
        }
        // the others wait at the CTA barrier (no issue slots) while thread 0 polls
        __syncthreads();
        ok = s_ok;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!ok) break;
        unsigned d[32];
        unsigned ta = tmem + ((unsigned)(32 * warp) << 16) + 32u * (m & 1);
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
        // the products alternate between two 32-column halves of tensor memory: slab m+1's
        // product is issued after the barrier of slab m, which every warp reaches only
        // after its tcgen05.ld of slab m-1 (the same half) has completed
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
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem));
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
// (1/u_kk, g_k).  binary16 keeps 10 mantissa bits, the precision of TF32.  Columns are
// ldh = nd rounded up to even halves apart (so that two rows load as one 4-byte word).
// One CTA per block, one warp per column.
__global__ void __launch_bounds__(256) k_lutc_to_half(const float *__restrict__ M, __half *__restrict__ H,
                                                      float2 *__restrict__ dg, int nd, int ldh) {
    const int e = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float *Ab = M + (size_t)e * nd * nd;
    __half *Hb = H + (size_t)e * nd * ldh;
    for (int k = warp; k < nd; k += 8) {
        const float *col = Ab + (size_t)k * nd;
        float m = 0.f;
        for (int i = lane; i < k; i += 32) m = fmaxf(m, fabsf(col[i]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        const float g = m > 0.f ? m : 1.f, ig = 1.f / g;
        for (int i = lane; i < nd; i += 32) {
            float v = col[i];
            Hb[(size_t)k * ldh + i] = __float2half_rn(i < k ? v * ig : (i > k ? v : 0.f));
        }
        if (lane == 0) {
            dg[(size_t)e * nd + k] = make_float2(col[k], g);
            if (ldh > nd) Hb[(size_t)k * ldh + nd] = __float2half_rn(0.f);   // the pad row
        }
    }
}

// x <- M_e^{-1} x with the half-width factors.  One warp per element; lane l holds rows
// 64 s + 2 l and 64 s + 2 l + 1 (s < NR2) in registers, so one 4-byte load per lane
// brings two rows of a column and a warp reads 128 bytes of it at once; G columns are
// fetched ahead of the dependent fma chain.  Forward: rows below k take y_k (unit L);
// backward: x_k = b_k (1/u_kk), then the rows above k take the scaled column times
// g_k x_k.
template <int NR2, int G>
__global__ void __launch_bounds__(128) k_lu_solve_half(const __half *__restrict__ H, const float2 *__restrict__ dg,
                                                       const int *__restrict__ perm, float *__restrict__ x, int nd,
                                                       int ldh, int E) {
    int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (e >= E) return;
    const __half *A = H + (size_t)e * nd * ldh;
    const float2 *D = dg + (size_t)e * nd;
    const int *pv = perm + (size_t)e * nd;
    float2 b[NR2];
#pragma unroll
    for (int s = 0; s < NR2; ++s) {
        int r = 64 * s + 2 * lane;
        b[s].x = r < nd ? x[(size_t)pv[r] * E + e] : 0.f;
        b[s].y = r + 1 < nd ? x[(size_t)pv[r + 1] * E + e] : 0.f;
    }
#pragma unroll
    for (int sk = 0; sk < NR2; ++sk) {
        const int kend = min(nd, 64 * sk + 64);
        for (int k0 = 64 * sk; k0 < kend; k0 += G) {
            float2 cv[G][NR2];
            // on blocks of more than 192 rows, the columns TC_PF ahead go to L2 now (no
            // registers held for them): 1.73 against 1.81 ms on the 320-row level, while the
            // 135-row level measured 8% slower with it
#pragma unroll
            for (int g = 0; g < G; ++g) {
                int kp = k0 + TC_PF + g;
                if (NR2 >= 4 && kp < nd)
#pragma unroll
                    for (int s = sk; s < NR2; ++s) {
                        int r = 64 * s + 2 * lane;
                        if (r < nd) asm volatile("prefetch.global.L2 [%0];" ::"l"(A + (size_t)kp * ldh + r));
                    }
            }
#pragma unroll
            for (int g = 0; g < G; ++g) {
                int k = k0 + g;
                const __half *col = A + (size_t)(k < kend ? k : kend - 1) * ldh;
#pragma unroll
                for (int s = sk; s < NR2; ++s) {
                    int r = 64 * s + 2 * lane;
                    bool need = k < kend && r < nd && (s > sk || r + 1 > (k & 63) + 64 * sk);
                    cv[g][s] = need ? __half22float2(*reinterpret_cast<const __half2 *>(col + r)) : make_float2(0.f, 0.f);
                }
            }
#pragma unroll
            for (int g = 0; g < G; ++g) {
                int k = k0 + g;
                if (k >= kend) break;
                int kl = k & 63, owner = kl >> 1;
                float yk = __shfl_sync(0xffffffffu, (kl & 1) ? b[sk].y : b[sk].x, owner);
#pragma unroll
                for (int s = sk; s < NR2; ++s) {
                    int r = 64 * s + 2 * lane;
                    if (s > sk || r > k) b[s].x = fmaf(-cv[g][s].x, yk, b[s].x);
                    if (s > sk || r + 1 > k) b[s].y = fmaf(-cv[g][s].y, yk, b[s].y);
                }
            }
        }
    }
#pragma unroll
    for (int sk = NR2 - 1; sk >= 0; --sk) {
        const int kbeg = min(nd, 64 * sk + 64) - 1;
        for (int kt = kbeg; kt >= 64 * sk; kt -= G) {
            float2 cv[G][NR2];
            float2 dk[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                int kp = kt - TC_PF - g;
                if (NR2 >= 4 && kp >= 0)
#pragma unroll
                    for (int s = 0; s <= sk; ++s) {
                        int r = 64 * s + 2 * lane;
                        if (r < kp) asm volatile("prefetch.global.L2 [%0];" ::"l"(A + (size_t)kp * ldh + r));
                    }
            }
#pragma unroll
            for (int g = 0; g < G; ++g) {
                int k = kt - g;
                int kk = k >= 64 * sk ? k : 64 * sk;
                const __half *col = A + (size_t)kk * ldh;
                dk[g] = D[kk];
#pragma unroll
                for (int s = 0; s <= sk; ++s) {
                    int r = 64 * s + 2 * lane;
                    bool need = k >= 64 * sk && (s < sk || r < k);
                    cv[g][s] = need ? __half22float2(*reinterpret_cast<const __half2 *>(col + r)) : make_float2(0.f, 0.f);
                }
            }
#pragma unroll
            for (int g = 0; g < G; ++g) {
                int k = kt - g;
                if (k < 64 * sk) break;
                int kl = k & 63, owner = kl >> 1;
                float xk = __shfl_sync(0xffffffffu, (kl & 1) ? b[sk].y : b[sk].x, owner) * dk[g].x;
                float xs = xk * dk[g].y;
#pragma unroll
                for (int s = 0; s < sk; ++s) {
                    b[s].x = fmaf(-cv[g][s].x, xs, b[s].x);
                    b[s].y = fmaf(-cv[g][s].y, xs, b[s].y);
                }
                int r = 64 * sk + 2 * lane;
                if (r == k) b[sk].x = xk;
                else if (r < k) b[sk].x = fmaf(-cv[g][sk].x, xs, b[sk].x);
                if (r + 1 == k) b[sk].y = xk;
                else if (r + 1 < k) b[sk].y = fmaf(-cv[g][sk].y, xs, b[sk].y);
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (int s = 0; s < NR2; ++s) {
        int r = 64 * s + 2 * lane;
        if (r < nd) x[(size_t)r * E + e] = b[s].x;
        if (r + 1 < nd) x[(size_t)(r + 1) * E + e] = b[s].y;
    }
}

template <int NR2>
static void solve_half_nr(int g, int grid, const __half *H, const float2 *dg, const int *perm, float *x, int nd,
                          int ldh, int E, cudaStream_t s) {
    // 8 columns in flight is the slowest on every level measured (register pressure):
    // the FP32 solve's choice 8 becomes 4 here
    if (g >= 4) k_lu_solve_half<NR2, 4><<<grid, 128, 0, s>>>(H, dg, perm, x, nd, ldh, E);
    else k_lu_solve_half<NR2, 2><<<grid, 128, 0, s>>>(H, dg, perm, x, nd, ldh, E);
}

}  // namespace

// the tensor-core factorisation handles blocks with TC_NB < nd <= TC_MAXND
int frktc_lu_supported(int nd) { return nd > 2 * TC_NB && nd <= TC_MAXND; }

// each phase's split L21 operand (the panel kernel writes it, the trailing kernel reads it)
size_t frktc_lu_scratch_floats(int E, int nd) {
    int mt0 = nd - TC_NB, mtiles = mt0 > 0 ? (mt0 + 127) / 128 : 0;
    return (size_t)E * mtiles * 2 * 128 * TC_NB;
}

int frktc_lu_factor(int E, int nd, float *M, int *perm, int *info, float *l21, cudaStream_t s) {
    if (!frktc_lu_supported(nd) || E <= 0 || !l21) return 1;
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
        int rows = nd - k0, mt = rows - TC_NB, mtiles = mt > 0 ? (mt + 127) / 128 : 0;
        CNT();
        k_lutc_panel<<<E, 128, sizeof(float) * TC_NB * rows, s>>>(M, perm, nd, k0, info, l21, mtiles);
        if (mt > 0) {
            int ntiles = (mt + TC_NT - 1) / TC_NT;
            long long grid = (long long)ntiles * E;
            if (grid > 0x7fffffffLL) return 1;
            CNT();
            k_lutc_trail<<<(unsigned)grid, 128, sizeof(float) * TC_SMEM_FLOATS, s>>>(M, perm, nd, k0, ntiles, l21);
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
    return (h & 1 ? 4 : 0) | (h & 2 ? 2 : 0);
}

int frktc_half_ld(int nd) { return (nd + 1) & ~1; }

int frktc_lu_to_half(int E, int nd, const float *M, void *H, float *dg, cudaStream_t s) {
    if (E <= 0 || nd <= 0) return 1;
    CNT();
    k_lutc_to_half<<<E, 256, 0, s>>>(M, (__half *)H, (float2 *)dg, nd, frktc_half_ld(nd));
    return 0;
}

// g: columns in flight (2 or 4; 8 is taken as 4; 0 or 1: the default, 4)
int frktc_lu_solve_half(int E, int nd, int g, const void *H, const float *dg, const int *perm, float *x,
                        cudaStream_t s) {
    int nr2 = (nd + 63) / 64, grid = (E * 32 + 127) / 128, ldh = frktc_half_ld(nd);
    const __half *h = (const __half *)H;
    const float2 *d = (const float2 *)dg;
    if (g < 2) g = 4;
    CNT();
    switch (nr2) {
        case 1: solve_half_nr<1>(g, grid, h, d, perm, x, nd, ldh, E, s); break;
        case 2: solve_half_nr<2>(g, grid, h, d, perm, x, nd, ldh, E, s); break;
        case 3: solve_half_nr<3>(g, grid, h, d, perm, x, nd, ldh, E, s); break;
        case 4: solve_half_nr<4>(g, grid, h, d, perm, x, nd, ldh, E, s); break;
        case 5: solve_half_nr<5>(g, grid, h, d, perm, x, nd, ldh, E, s); break;
        case 6: solve_half_nr<6>(g, grid, h, d, perm, x, nd, ldh, E, s); break;
        default: return -1;
    }
    return 0;
}
