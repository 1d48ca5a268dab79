// fr_residual_noalloc: the FP64 residual with its stage scratch (flux-point traces, jumps,
// face gradients, common fluxes, transformed fluxes) taken from one
// file-scope device array instead of the context's workspace.  It calls no cudaMalloc,
// cudaFree or any allocating routine.
//
// For callers that cannot allocate device memory at the point of the call: code running
// under CUDA stream capture in the global capture mode (where cudaMalloc is refused),
// hosts whose device memory is owned by another allocator with a fixed budget, and
// real-time loops that must not pay an allocation's latency or risk its failure.
//
// The array has a fixed size (FR_NOALLOC_MAX_DOUBLES doubles, 16 MiB) and stays
// resident on every GPU that loads the library until the process exits.  Every value of
// it is written before it is read within one call, so nothing needs clearing between
// calls.  All calls share it: calls whose GPU work overlaps (other streams, other
// contexts, other host threads) race on it.
#include <cuda_runtime.h>
#include <stdint.h>
#include <mutex>
#include "../../include/frpmg.h"
#include "fr_lib.h"

#define FR_NOALLOC_MAX_DOUBLES (2u * 1024u * 1024u)
#define FR_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) double g_fr_noalloc_scratch[FR_NOALLOC_MAX_DOUBLES];

// host copies of the array's device address, one per device ordinal, filled on the first
// call made with that device current (under g_scratch_mutex, so first calls on several
// host threads do not race).  The address belongs to the device's primary context: after
// cudaDeviceReset the library's module, and with it this array, is gone, and the process
// must not call into the library again.
static double *g_scratch_addr[FR_NOALLOC_MAX_DEVICES];
static std::mutex g_scratch_mutex;

// access to the context's level data (defined in lib.cu)
extern "C++" int fr_internal_level(const fr_ctx *ctx, int level, FrLevel *out, FrPhysH *ph);
extern "C++" int fr_internal_fail(int code, const char *msg);
extern "C++" int fr_internal_has_comm(const fr_ctx *ctx);

static size_t align_doubles(size_t n) { return (n + 31) & ~(size_t)31; }   // 256-byte multiples

extern "C" int fr_residual_noalloc(fr_ctx *ctx, int level, const double *q, double *R, void *stream) {
    FrLevel L;
    FrPhysH ph;
    if (!ctx || !q || !R) return fr_internal_fail(FR_ERR_INVALID_ARG, "fr_residual_noalloc: NULL argument");
    if (q == R) return fr_internal_fail(FR_ERR_INVALID_ARG, "fr_residual_noalloc: q and R must not alias");
    if (fr_internal_has_comm(ctx))
        return fr_internal_fail(FR_ERR_INVALID_ARG, "fr_residual_noalloc: not with an element partition (fr_set_comm)");
    if (fr_internal_level(ctx, level, &L, &ph) != FR_OK)
        return fr_internal_fail(FR_ERR_INVALID_ARG, "fr_residual_noalloc: bad level");
    size_t E = (size_t)L.E;
    size_t nfv = align_doubles((size_t)L.nv * L.nfp * E);
    size_t npv = align_doubles((size_t)L.d * L.nv * L.np * E);
    size_t nqf = align_doubles((size_t)L.d * L.nv * L.nfp * E);
    size_t need = 4 * nfv + npv + nqf;
    if (need > FR_NOALLOC_MAX_DOUBLES)
        return fr_internal_fail(FR_ERR_INVALID_ARG,
                                "fr_residual_noalloc: this level needs more stage scratch than the fixed "
                                "16 MiB array holds; use fr_residual");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= FR_NOALLOC_MAX_DEVICES)
        return fr_internal_fail(FR_ERR_CUDA, "fr_residual_noalloc: no usable current device");
    double *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_fr_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return fr_internal_fail(FR_ERR_CUDA, "fr_residual_noalloc: cudaGetSymbolAddress failed");
            g_scratch_addr[dev] = (double *)p;
        }
        base = g_scratch_addr[dev];
    }
    L.qf = base;
    L.dq = base + nfv;
    L.fn = base + 2 * nfv;
    L.Ftf = base + 3 * nfv;
    L.Ft = base + 4 * nfv;
    L.Qf = base + 4 * nfv + npv;
    if (frk64_residual(L, ph, q, R, (cudaStream_t)stream) != 0)
        return fr_internal_fail(FR_ERR_UNIMPLEMENTED, "fr_residual_noalloc: no kernel for this degree");
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fr_internal_fail(FR_ERR_CUDA, cudaGetErrorString(e));
    return FR_OK;
}
