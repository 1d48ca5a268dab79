#include <algorithm>
// FP32 kernels of the mixed-precision preconditioner (residuals on every p-level,
// element blocks, block LU and solves, transfers), plus the FP64 <-> FP32 conversions at
// the preconditioner's boundary.  Contraction is allowed in this unit.
#define FRT float
#define FRK(name) frk32_##name
#define FR_DOUBLE 0
#include "fr_kernels_impl.cuh"

// --------------------------------------------------------- precision boundary
__global__ void k_d2f(long long n, const double *x, float *y) { GRID_STRIDE(i, n) y[i] = (float)x[i]; }
// y = float(x * s), s = target / max|x| read from the device (no host round trip)
__global__ void k_d2f_scaled(long long n, const double *x, const double *xmax, double target, float *y) {
    double m = *xmax;
    double s = m > 0.0 ? target / m : 1.0;
    GRID_STRIDE(i, n) y[i] = (float)(x[i] * s);
}
__global__ void k_absmax(long long n, const double *x, unsigned long long *out) {
    double m = 0.0;
    GRID_STRIDE(i, n) m = fmax(m, fabs(x[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

void frk32_d2f(long long n, const double *x, float *y, cudaStream_t s) { CNT(); k_d2f<<<nblk(n), 256, 0, s>>>(n, x, y); }
void frk32_d2f_scaled(long long n, const double *x, const double *xmax_dev, double target, float *y, cudaStream_t s) {
    CNT(); k_d2f_scaled<<<nblk(n), 256, 0, s>>>(n, x, xmax_dev, target, y);
}
int frk32_absmax(long long n, const double *x, double *out_dev, cudaStream_t s) {
    if (cudaMemsetAsync(out_dev, 0, sizeof(double), s) != cudaSuccess) return -1;
    CNT(); k_absmax<<<nblk(n), 256, 0, s>>>(n, x, (unsigned long long *)out_dev);
    return 0;
}
// per-variable max |x| of a [nv][per] vector: blockIdx.y = variable
template <typename S>
__global__ void k_absmax_var(long long per, const S *x, unsigned long long *out) {
    const S *xv = x + (size_t)blockIdx.y * per;
    double m = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < per; i += (long long)gridDim.x * blockDim.x)
        m = fmax(m, fabs((double)xv[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out + blockIdx.y, (unsigned long long)__double_as_longlong(m));
}
template <typename S>
static int absmax_var(int nv, long long per, const S *x, double *out_dev, cudaStream_t s) {
    if (cudaMemsetAsync(out_dev, 0, sizeof(double) * nv, s) != cudaSuccess) return -1;
    int gx = (int)std::min<long long>((per + 255) / 256, 152LL * 4);
    CNT(); k_absmax_var<S><<<dim3(gx, nv), 256, 0, s>>>(per, x, (unsigned long long *)out_dev);
    return 0;
}
int frk32_absmax_var(int nv, long long per, const double *x, double *out_dev, cudaStream_t s) {
    return absmax_var<double>(nv, per, x, out_dev, s);
}
int frk32_absmax_var_f(int nv, long long per, const float *x, double *out_dev, cudaStream_t s) {
    return absmax_var<float>(nv, per, x, out_dev, s);
}
// the same maxima over the owned elements only (index t -> row t / n_owned, element
// t % n_owned of a [rows][E] vector); per variable: rows = np per variable
template <typename S>
__global__ void k_absmax_owned(long long n, long long E, long long n_owned, long long rows_per_out, const S *x,
                               unsigned long long *out) {
    int v = blockIdx.y;
    const S *xv = x + (size_t)v * rows_per_out * E;
    double m = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        m = fmax(m, fabs((double)xv[(t / n_owned) * E + t % n_owned]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out + v, (unsigned long long)__double_as_longlong(m));
}
template <typename S>
static int absmax_owned(int nout, long long rows_per_out, long long E, long long n_owned, const S *x, double *out_dev,
                        cudaStream_t s) {
    if (cudaMemsetAsync(out_dev, 0, sizeof(double) * nout, s) != cudaSuccess) return -1;
    long long n = rows_per_out * n_owned;
    int gx = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 4));
    CNT(); k_absmax_owned<S><<<dim3(gx, nout), 256, 0, s>>>(n, E, n_owned, rows_per_out, x, (unsigned long long *)out_dev);
    return 0;
}
int frk32_absmax_owned(long long rows, long long E, long long n_owned, const double *x, double *out_dev, cudaStream_t s) {
    return absmax_owned<double>(1, rows, E, n_owned, x, out_dev, s);
}
int frk32_absmax_var_owned(int nv, long long np, long long E, long long n_owned, const double *x, double *out_dev,
                           cudaStream_t s) {
    return absmax_owned<double>(nv, np, E, n_owned, x, out_dev, s);
}
int frk32_absmax_var_owned_f(int nv, long long np, long long E, long long n_owned, const float *x, double *out_dev,
                             cudaStream_t s) {
    return absmax_owned<float>(nv, np, E, n_owned, x, out_dev, s);
}

// y = double(x) * (max / target): undoes the input scaling of the FP32 cycle
__global__ void k_f2d_unscale(long long n, const float *x, const double *xmax, double target, double *y) {
    double m = *xmax;
    double inv_s = m > 0.0 ? m / target : 1.0;
    GRID_STRIDE(i, n) y[i] = (double)x[i] * inv_s;
}
void frk32_f2d_unscale(long long n, const float *x, const double *xmax_dev, double target, double *y, cudaStream_t s) {
    CNT(); k_f2d_unscale<<<nblk(n), 256, 0, s>>>(n, x, xmax_dev, target, y);
}

// Scaling of the FP32 cycle with the target held on the device (no host round trip):
// x32 = X * target / max|X|, Y = y32 * max|X| / target, and after the cycle the target of
// the next application from the measured gain: ym = max_v max|y32_v| / qref_v,
// target' = want * target / ym (unchanged if ym is 0 or not finite).
__global__ void k_d2f_scaled_dev(long long n, const double *x, const double *xmax, const double *target, float *y) {
    double m = *xmax;
    double s = m > 0.0 ? *target / m : 1.0;
    GRID_STRIDE(i, n) y[i] = (float)(x[i] * s);
}
__global__ void k_f2d_unscale_dev(long long n, const float *x, const double *xmax, const double *target, double *y) {
    double m = *xmax;
    double inv_s = m > 0.0 ? m / *target : 1.0;
    GRID_STRIDE(i, n) y[i] = (double)x[i] * inv_s;
}
__global__ void k_next_target(int nv, const double *ymax, const double *qref, double want, double *target) {
    if (threadIdx.x != 0) return;
    double ym = 0.0;
    for (int v = 0; v < nv; ++v) ym = fmax(ym, ymax[v] / qref[v]);
    if (ym > 0.0 && ym < INFINITY) *target = want * *target / ym;
}
void frk32_d2f_scaled_dev(long long n, const double *x, const double *xmax_dev, const double *target_dev, float *y,
                          cudaStream_t s) {
    CNT(); k_d2f_scaled_dev<<<nblk(n), 256, 0, s>>>(n, x, xmax_dev, target_dev, y);
}
void frk32_f2d_unscale_dev(long long n, const float *x, const double *xmax_dev, const double *target_dev, double *y,
                           cudaStream_t s) {
    CNT(); k_f2d_unscale_dev<<<nblk(n), 256, 0, s>>>(n, x, xmax_dev, target_dev, y);
}
void frk32_next_target(int nv, const double *ymax_dev, const double *qref_dev, double want, double *target_dev,
                       cudaStream_t s) {
    CNT(); k_next_target<<<1, 32, 0, s>>>(nv, ymax_dev, qref_dev, want, target_dev);
}
