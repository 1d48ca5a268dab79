// Device building blocks of the flux-reconstruction residual (templated on dimension D,
// degree P and scalar type T).  Included by the FP64 translation unit (compiled with
// -fmad=false: the only contractions are the explicit fma() calls, so every FP64 result
// is reproducible bit for bit) and by the FP32 one (preconditioner precision).
//
// Layouts (element index e fastest everywhere, E elements):
//   state / residual      q[v][i][e]            v < nv = D+2, i < Np = n^D
//   flux-point traces     qf[v][k][e]           k = f*n^(D-1) + t, f = 2*dir + side
//   gradients             Q[c][v][i][e], Qf[c][v][k][e]
//   geometric factors     S[dd][c][i][e] = J dxi_dd/dx_c, G = S / J, invJ[i][e],
//                         Sf, Gf at flux points
// Evaluation order (fixed): every sum of products is an fma chain in ascending index
// starting from +0; everything else is evaluated as parenthesised.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "fr_dual.cuh"

// Arithmetic type T of a kernel and the base type B = FrBase<T>::type of its operator
// tables and geometric factors: B = T for double and float; float for the dual types.

#define FR_MAXN 6
#define FR_MAXP 5

template <typename T>
struct FrTab {
    T D[FR_MAXN][FR_MAXN];
    T lm[FR_MAXN], lp[FR_MAXN], dlm[FR_MAXN], dlp[FR_MAXN];
    T gLd[FR_MAXN], gRd[FR_MAXN];
};

template <typename T>
struct FrPhys {
    T gamma, gm1, mu, kappa, c23;
    T qinf[5];
    T etagL, etagR;   // eta * g_L'(-1), eta * g_R'(+1) of the level
    int flux;         // inviscid common flux: 0 Rusanov, 1 Roe, 2 Roe + Weiss-Smith
    T ws_umin;        // Weiss-Smith: floor of the reference velocity
};

template <int D, int P>
struct Sh {
    static constexpr int n = P + 1;
    static constexpr int nv = D + 2;
    static constexpr int np = D == 2 ? n * n : n * n * n;
    static constexpr int nf1 = D == 2 ? n : n * n;
    static constexpr int nfp = 2 * D * nf1;
};

template <int D, int N>
__device__ __forceinline__ int spi(int i0, int i1, int i2) {
    return D == 2 ? i0 + N * i1 : i0 + N * (i1 + N * i2);
}

// face point k -> normal direction df, side s, tangential coordinates (a, b)
template <int D, int N>
__device__ __forceinline__ void fp_decode(int k, int &df, int &s, int &a, int &b) {
    constexpr int nf1 = D == 2 ? N : N * N;
    int f = k / nf1, t = k - f * nf1;
    df = f >> 1;
    s = f & 1;
    a = t % N;
    b = D == 3 ? t / N : 0;
}

// solution point on the line normal to face direction df through tangential (a, b)
template <int D, int N>
__device__ __forceinline__ int line_pt(int df, int a, int b, int m) {
    if (D == 2) return df == 0 ? m + N * a : a + N * m;
    if (df == 0) return m + N * (a + N * b);
    if (df == 1) return a + N * (m + N * b);
    return a + N * (b + N * m);
}

// face point of face (df, s) on the df-line through the solution point (i0, i1, i2)
template <int D, int N>
__device__ __forceinline__ int fp_of(int df, int s, int i0, int i1, int i2) {
    constexpr int nf1 = D == 2 ? N : N * N;
    int t;
    if (D == 2) t = df == 0 ? i1 : i0;
    else t = df == 0 ? i1 + N * i2 : (df == 1 ? i0 + N * i2 : i0 + N * i1);
    return (2 * df + s) * nf1 + t;
}

// face point of face (df, s) whose tangential coordinates are (a, b)
template <int D, int N>
__device__ __forceinline__ int fp_at(int df, int s, int a, int b) {
    constexpr int nf1 = D == 2 ? N : N * N;
    return (2 * df + s) * nf1 + a + (D == 3 ? N * b : 0);
}

// ---------------------------------------------------------------------------- physics
template <int D, typename T, typename B>
__device__ __forceinline__ void flux_inviscid(const FrPhys<B> &ph, const T *q, T f[3][5]) {
    T rho = q[0], E = q[D + 1], rinv = T(1) / rho, u[3], ke = T(0);
#pragma unroll
    for (int j = 0; j < D; ++j) u[j] = q[1 + j] * rinv;
#pragma unroll
    for (int j = 0; j < D; ++j) ke = fma(q[1 + j], u[j], ke);
    T p = ph.gm1 * (E - T(0.5) * ke);
#pragma unroll
    for (int c = 0; c < D; ++c) {
        f[c][0] = q[1 + c];
#pragma unroll
        for (int j = 0; j < D; ++j) {
            T t = q[1 + c] * u[j];
            if (j == c) t = t + p;
            f[c][1 + j] = t;
        }
        f[c][D + 1] = (E + p) * u[c];
    }
}

template <int D, typename T, typename B>
__device__ __forceinline__ void flux_viscous(const FrPhys<B> &ph, const T *q, const T Q[3][5], bool adiabatic,
                                             T f[3][5]) {
    T rho = q[0], E = q[D + 1], rinv = T(1) / rho, Er = E * rinv, u[3];
    T du[3][3], de[3], tau[3][3];
#pragma unroll
    for (int j = 0; j < D; ++j) u[j] = q[1 + j] * rinv;
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
        for (int c = 0; c < D; ++c) du[j][c] = (Q[c][1 + j] - u[j] * Q[c][0]) * rinv;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        T s = T(0);
#pragma unroll
        for (int j = 0; j < D; ++j) s = fma(u[j], du[j][c], s);
        T t = (Q[c][D + 1] - Er * Q[c][0]) * rinv;
        de[c] = t - s;
    }
    T divu = T(0);
#pragma unroll
    for (int j = 0; j < D; ++j) divu = divu + du[j][j];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            T t = du[i][j] + du[j][i];
            if (i == j) t = t - ph.c23 * divu;
            tau[i][j] = ph.mu * t;
        }
#pragma unroll
    for (int c = 0; c < D; ++c) {
        f[c][0] = T(0);
#pragma unroll
        for (int j = 0; j < D; ++j) f[c][1 + j] = tau[j][c];
        T s = T(0);
#pragma unroll
        for (int j = 0; j < D; ++j) s = fma(u[j], tau[j][c], s);
        if (!adiabatic) s = s + ph.kappa * de[c];
        f[c][D + 1] = s;
    }
}

// Rusanov flux along the (scaled) normal n
template <int D, typename T, typename B>
__device__ __forceinline__ void rusanov(const FrPhys<B> &ph, const T *qL, const T *qR, const B *n, T *F) {
    constexpr int nv = D + 2;
    T fL[3][5], fR[3][5];
    flux_inviscid<D, T, B>(ph, qL, fL);
    flux_inviscid<D, T, B>(ph, qR, fR);
    B nn = B(0);
#pragma unroll
    for (int c = 0; c < D; ++c) nn = fma(n[c], n[c], nn);
    B nmag = sqrt(nn);
    T lam[2];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const T *q = side ? qR : qL;
        T rho = q[0], E = q[D + 1], rinv = T(1) / rho, u[3], ke = T(0), vn = T(0);
#pragma unroll
        for (int j = 0; j < D; ++j) u[j] = q[1 + j] * rinv;
#pragma unroll
        for (int j = 0; j < D; ++j) ke = fma(q[1 + j], u[j], ke);
        T p = ph.gm1 * (E - T(0.5) * ke);
        T a = sqrt((ph.gamma * p) * rinv);
#pragma unroll
        for (int c = 0; c < D; ++c) vn = fma(u[c], n[c], vn);
        lam[side] = fabs(vn) + a * nmag;
    }
    T lmax = fmax(lam[0], lam[1]);
#pragma unroll
    for (int v = 0; v < nv; ++v) {
        T FnL = T(0), FnR = T(0);
#pragma unroll
        for (int c = 0; c < D; ++c) FnL = fma(fL[c][v], n[c], FnL);
#pragma unroll
        for (int c = 0; c < D; ++c) FnR = fma(fR[c][v], n[c], FnR);
        F[v] = T(0.5) * (FnL + FnR) - T(0.5) * lmax * (qR[v] - qL[v]);
    }
}

// Roe flux along the (scaled) normal n: the mean of the two normal fluxes minus
// |A(Roe average)| (qR - qL) / 2, the wave families through the Roe-averaged state (density
// sqrt(rhoL rhoR), velocity and total enthalpy weighted by sqrt(rho)); Roe's original solver,
// without an entropy fix
template <int D, typename T, typename B>
__device__ __forceinline__ void roe(const FrPhys<B> &ph, const T *qL, const T *qR, const B *n, T *F) {
    constexpr int nv = D + 2;
    T fL[3][5], fR[3][5];
    flux_inviscid<D, T, B>(ph, qL, fL);
    flux_inviscid<D, T, B>(ph, qR, fR);
    B nn = B(0);
#pragma unroll
    for (int c = 0; c < D; ++c) nn = fma(n[c], n[c], nn);
    B nmag = sqrt(nn);
    B nh[3];
#pragma unroll
    for (int c = 0; c < D; ++c) nh[c] = n[c] / nmag;
    T rho[2], u[2][3], p[2], H[2];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const T *q = side ? qR : qL;
        T rinv = T(1) / q[0], ke = T(0);
        rho[side] = q[0];
#pragma unroll
        for (int j = 0; j < D; ++j) u[side][j] = q[1 + j] * rinv;
#pragma unroll
        for (int j = 0; j < D; ++j) ke = fma(q[1 + j], u[side][j], ke);
        p[side] = ph.gm1 * (q[D + 1] - T(0.5) * ke);
        H[side] = (q[D + 1] + p[side]) * rinv;
    }
    T sL = sqrt(rho[0]), sR = sqrt(rho[1]), wt = T(1) / (sL + sR);
    T ut[3], q2 = T(0), vn = T(0), du[3], dvn = T(0), udu = T(0);
#pragma unroll
    for (int j = 0; j < D; ++j) ut[j] = (sL * u[0][j] + sR * u[1][j]) * wt;
    T Ht = (sL * H[0] + sR * H[1]) * wt;
#pragma unroll
    for (int j = 0; j < D; ++j) q2 = fma(ut[j], ut[j], q2);
#pragma unroll
    for (int j = 0; j < D; ++j) vn = fma(ut[j], nh[j], vn);
    T c2 = ph.gm1 * (Ht - T(0.5) * q2);
    T ct = sqrt(c2);
    T rt = sL * sR;
    T drho = rho[1] - rho[0], dp = p[1] - p[0];
#pragma unroll
    for (int j = 0; j < D; ++j) du[j] = u[1][j] - u[0][j];
#pragma unroll
    for (int j = 0; j < D; ++j) dvn = fma(du[j], nh[j], dvn);
#pragma unroll
    for (int j = 0; j < D; ++j) udu = fma(ut[j], du[j], udu);
    T a1 = (dp - rt * ct * dvn) / (T(2) * c2);
    T a3 = (dp + rt * ct * dvn) / (T(2) * c2);
    T a2 = drho - dp / c2;
    T l1 = fabs(vn - ct), l2 = fabs(vn), l3 = fabs(vn + ct);
    T w1 = l1 * a1, w2 = l2 * a2, w3 = l3 * a3, ws = l2 * rt;
    T Dv[5];
    Dv[0] = w1 + w2 + w3;
#pragma unroll
    for (int j = 0; j < D; ++j)
        Dv[1 + j] = w1 * (ut[j] - ct * nh[j]) + w2 * ut[j] + ws * (du[j] - dvn * nh[j]) + w3 * (ut[j] + ct * nh[j]);
    Dv[D + 1] = w1 * (Ht - ct * vn) + w2 * (T(0.5) * q2) + ws * (udu - vn * dvn) + w3 * (Ht + ct * vn);
#pragma unroll
    for (int v = 0; v < nv; ++v) {
        T FnL = T(0), FnR = T(0);
#pragma unroll
        for (int c = 0; c < D; ++c) FnL = fma(fL[c][v], n[c], FnL);
#pragma unroll
        for (int c = 0; c < D; ++c) FnR = fma(fR[c][v], n[c], FnR);
        F[v] = T(0.5) * (FnL + FnR) - T(0.5) * nmag * Dv[v];
    }
}

// Roe's solver with the Weiss-Smith low-Mach preconditioning of its dissipation: in the
// primitive variables Q = (p, u, T) (gas constant 1, C_p = gamma/(gamma-1)) the dissipation is
// Gamma |Gamma^{-1} A_n| dQ at the Roe-averaged state, Gamma = dW/dQ with drho/dp replaced by
// theta = 1/Ur^2 - rho_T/(rho C_p), Ur = min(c, max(|u|, umin)); Gamma^{-1} A_n has the three
// distinct eigenvalues vn, u' +- c' (u' = vn (1 - alpha), c' = sqrt(alpha^2 vn^2 + Ur^2),
// alpha = (1 - Ur^2/c^2)/2), so |Gamma^{-1} A_n| is the quadratic through |lambda| at them:
// D = a0 Gamma dQ + a1 A_n dQ + a2 A_n Gamma^{-1} A_n dQ.
template <int D, typename T, typename B>
struct WsState {
    T rho, u[3], H, T_, rp, rT, cp, theta, vn;
    B nh[3];
};
template <int D, typename T, typename B>
__device__ __forceinline__ void ws_apply_A(const WsState<D, T, B> &S, const T *x, T *y) {
    T nx = T(0), ux = T(0);
#pragma unroll
    for (int j = 0; j < D; ++j) nx = fma(S.nh[j], x[1 + j], nx);
#pragma unroll
    for (int j = 0; j < D; ++j) ux = fma(S.u[j], x[1 + j], ux);
    T r = S.rp * S.vn * x[0] + S.rho * nx + S.rT * S.vn * x[D + 1];
    y[0] = r;
#pragma unroll
    for (int i = 0; i < D; ++i) y[1 + i] = S.u[i] * r + S.nh[i] * x[0] + S.rho * S.vn * x[1 + i];
    y[D + 1] = S.H * r + S.rho * S.vn * ux + S.rho * S.cp * S.vn * x[D + 1];
}
template <int D, typename T, typename B>
__device__ __forceinline__ void ws_apply_G(const WsState<D, T, B> &S, const T *x, T *y) {
    T ux = T(0);
#pragma unroll
    for (int j = 0; j < D; ++j) ux = fma(S.u[j], x[1 + j], ux);
    T r = S.theta * x[0] + S.rT * x[D + 1];
    y[0] = r;
#pragma unroll
    for (int i = 0; i < D; ++i) y[1 + i] = S.u[i] * r + S.rho * x[1 + i];
    y[D + 1] = S.H * r - x[0] + S.rho * ux + S.rho * S.cp * x[D + 1];
}
// z = Gamma^{-1} y (the velocity rows, then the 2 x 2 system of the first and energy rows)
template <int D, typename T, typename B>
__device__ __forceinline__ void ws_solve_G(const WsState<D, T, B> &S, const T *y, T *z) {
    T r0 = y[0], sum = T(0);
#pragma unroll
    for (int i = 0; i < D; ++i) {
        T t = y[1 + i] - S.u[i] * r0;
        z[1 + i] = t / S.rho;
        sum = fma(S.u[i], t, sum);
    }
    T s = y[D + 1] - S.H * r0 - sum;
    T det = S.theta * S.rho * S.cp + S.rT;
    z[0] = (r0 * S.rho * S.cp - S.rT * s) / det;
    z[D + 1] = (S.theta * s + r0) / det;
}

template <int D, typename T, typename B>
__device__ __forceinline__ void weiss_smith(const FrPhys<B> &ph, const T *qL, const T *qR, const B *n, T *F) {
    constexpr int nv = D + 2;
    T fL[3][5], fR[3][5];
    flux_inviscid<D, T, B>(ph, qL, fL);
    flux_inviscid<D, T, B>(ph, qR, fR);
    B nn = B(0);
#pragma unroll
    for (int c = 0; c < D; ++c) nn = fma(n[c], n[c], nn);
    B nmag = sqrt(nn);
    WsState<D, T, B> S;
#pragma unroll
    for (int c = 0; c < D; ++c) S.nh[c] = n[c] / nmag;
    T rho[2], u[2][3], p[2], H[2], Tt[2];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const T *q = side ? qR : qL;
        T rinv = T(1) / q[0], ke = T(0);
        rho[side] = q[0];
#pragma unroll
        for (int j = 0; j < D; ++j) u[side][j] = q[1 + j] * rinv;
#pragma unroll
        for (int j = 0; j < D; ++j) ke = fma(q[1 + j], u[side][j], ke);
        p[side] = ph.gm1 * (q[D + 1] - T(0.5) * ke);
        H[side] = (q[D + 1] + p[side]) * rinv;
        Tt[side] = p[side] * rinv;
    }
    T sL = sqrt(rho[0]), sR = sqrt(rho[1]), wt = T(1) / (sL + sR), q2 = T(0);
#pragma unroll
    for (int j = 0; j < D; ++j) S.u[j] = (sL * u[0][j] + sR * u[1][j]) * wt;
    S.H = (sL * H[0] + sR * H[1]) * wt;
#pragma unroll
    for (int j = 0; j < D; ++j) q2 = fma(S.u[j], S.u[j], q2);
    S.vn = T(0);
#pragma unroll
    for (int j = 0; j < D; ++j) S.vn = fma(S.u[j], S.nh[j], S.vn);
    T c2 = ph.gm1 * (S.H - T(0.5) * q2);
    S.rho = sL * sR;
    S.cp = T(ph.gamma / ph.gm1);
    S.T_ = c2 / T(ph.gamma);
    S.rp = T(1) / S.T_;
    S.rT = -S.rho / S.T_;
    T ur = fmin(sqrt(c2), fmax(sqrt(q2), T(ph.ws_umin)));
    S.theta = T(1) / (ur * ur) - S.rT / (S.rho * S.cp);
    T alpha = T(0.5) * (T(1) - (ur * ur) / c2);
    T up = S.vn * (T(1) - alpha), cq = sqrt(alpha * alpha * S.vn * S.vn + ur * ur);
    T l1 = S.vn, l2 = up + cq, l3 = up - cq;
    T f1 = fabs(l1), f2 = fabs(l2), f3 = fabs(l3);
    T s21 = (f2 - f1) / (l2 - l1), s31 = (f3 - f1) / (l3 - l1);
    T a2 = (s31 - s21) / (l3 - l2);
    T a1 = s21 - a2 * (l1 + l2);
    T a0 = f1 - a1 * l1 - a2 * (l1 * l1);
    T dQ[5], g[5], y1[5], z[5], y2[5];
    dQ[0] = p[1] - p[0];
#pragma unroll
    for (int j = 0; j < D; ++j) dQ[1 + j] = u[1][j] - u[0][j];
    dQ[D + 1] = Tt[1] - Tt[0];
    ws_apply_G<D, T, B>(S, dQ, g);
    ws_apply_A<D, T, B>(S, dQ, y1);
    ws_solve_G<D, T, B>(S, y1, z);
    ws_apply_A<D, T, B>(S, z, y2);
#pragma unroll
    for (int v = 0; v < nv; ++v) {
        T Dv = a0 * g[v] + a1 * y1[v] + a2 * y2[v];
        T FnL = T(0), FnR = T(0);
#pragma unroll
        for (int c = 0; c < D; ++c) FnL = fma(fL[c][v], n[c], FnL);
#pragma unroll
        for (int c = 0; c < D; ++c) FnR = fma(fR[c][v], n[c], FnR);
        F[v] = T(0.5) * (FnL + FnR) - T(0.5) * nmag * Dv;
    }
}

template <int D, typename T, typename B>
__device__ __forceinline__ void ghost_state(const FrPhys<B> &ph, int bc, const T *qL, T *qR) {
    if (bc == 1) {
#pragma unroll
        for (int v = 0; v < D + 2; ++v) qR[v] = T(ph.qinf[v]);
    } else {
        qR[0] = qL[0];
#pragma unroll
        for (int j = 0; j < D; ++j) qR[1 + j] = -qL[1 + j];
        qR[D + 1] = qL[D + 1];
    }
}

// ---------------------------------------------------------------- residual kernels
// Tables live in constant memory, indexed by degree; each including translation unit
// defines the specialisation of frtab<T> for its scalar type.
template <typename T>
__device__ const FrTab<T> &frtab(int p);

// stage 1: qf[v][k][e] = sum_m l_side[m] q[v][line(k, m)][e]; one thread per (k, e), all v
template <int D, int P, typename T>
__global__ void __launch_bounds__(256) k_interp(const T *__restrict__ q, T *__restrict__ qf, int E) {
    using S = Sh<D, P>;
    constexpr int N = S::n;
    int e = blockIdx.y * blockDim.x + threadIdx.x;   // the points of an element chunk run side by side
    if (e >= E) return;
    int k = blockIdx.x;
    int df, s, a, b;
    fp_decode<D, N>(k, df, s, a, b);
    typedef typename FrBase<T>::type B;
    const FrTab<B> &tb = frtab<B>(P);
#pragma unroll
    for (int v = 0; v < S::nv; ++v) {
        T acc = T(0);
#pragma unroll
        for (int m = 0; m < N; ++m) {
            T l = s ? tb.lp[m] : tb.lm[m];
            acc = fma(l, q[(size_t)(v * S::np + line_pt<D, N>(df, a, b, m)) * E + e], acc);
        }
        qf[(size_t)(v * S::nfp + k) * E + e] = acc;
    }
}

// stage 2: common solution, jumps dq = qs - q_side on both sides
template <int D, int P, typename T>
__global__ void __launch_bounds__(256) k_pair_common(const int4 *__restrict__ pairs, const int *__restrict__ bcs,
                                                     int npairs, const T *__restrict__ qf, T *__restrict__ dq, int E,
                                                     FrPhys<typename FrBase<T>::type> ph) {
    using S = Sh<D, P>;
    int P_ = blockIdx.x * blockDim.x + threadIdx.x;
    if (P_ >= npairs) return;
    int4 pr = pairs[P_];
    int bc = bcs[P_];
    T qL[5], qR[5];
#pragma unroll
    for (int v = 0; v < S::nv; ++v) qL[v] = qf[(size_t)(v * S::nfp + pr.y) * E + pr.x];
    if (bc == 0) {
#pragma unroll
        for (int v = 0; v < S::nv; ++v) qR[v] = qf[(size_t)(v * S::nfp + pr.w) * E + pr.z];
    } else {
        ghost_state<D, T, typename FrBase<T>::type>(ph, bc, qL, qR);
    }
#pragma unroll
    for (int v = 0; v < S::nv; ++v) {
        T qs = T(0.5) * (qL[v] + qR[v]);
        dq[(size_t)(v * S::nfp + pr.y) * E + pr.x] = qs - qL[v];
        if (bc == 0) dq[(size_t)(v * S::nfp + pr.w) * E + pr.z] = qs - qR[v];
    }
}

// stage 3: face gradient traces (uncorrected) with the BR2 lifting of the face's own jump;
// one thread per (k, e), all v (the metric terms Gf read once)
template <int D, int P, typename T>
__global__ void __launch_bounds__(256) k_grad_fp(const T *__restrict__ q, const T *__restrict__ qf,
                                                 const T *__restrict__ dq, const typename FrBase<T>::type *__restrict__ Gf,
                                                 T *__restrict__ Qf, int E, typename FrBase<T>::type etagL,
                                                 typename FrBase<T>::type etagR) {
    using S = Sh<D, P>;
    constexpr int N = S::n;
    int e = blockIdx.y * blockDim.x + threadIdx.x;   // the points of an element chunk run side by side
    if (e >= E) return;
    int k = blockIdx.x;
    int df, s, a, b;
    fp_decode<D, N>(k, df, s, a, b);
    typedef typename FrBase<T>::type B;
    const FrTab<B> &tb = frtab<B>(P);
    B g[3][3];
#pragma unroll
    for (int dd = 0; dd < D; ++dd)
#pragma unroll
        for (int c = 0; c < D; ++c) g[dd][c] = Gf[(size_t)((dd * D + c) * S::nfp + k) * E + e];
    // tangential directions in increasing order, coordinates a then b
    int td0 = df == 0 ? 1 : 0, td1 = df == 2 ? 1 : 2;
#pragma unroll
    for (int v = 0; v < S::nv; ++v) {
        T gf[3];
        {
            T t = T(0);
#pragma unroll
            for (int m = 0; m < N; ++m) {
                T dl = s ? tb.dlp[m] : tb.dlm[m];
                t = fma(dl, q[(size_t)(v * S::np + line_pt<D, N>(df, a, b, m)) * E + e], t);
            }
            gf[df] = t;
        }
        {
            T u = T(0);
#pragma unroll
            for (int m = 0; m < N; ++m)
                u = fma(tb.D[a][m], qf[(size_t)(v * S::nfp + fp_at<D, N>(df, s, m, b)) * E + e], u);
            gf[td0] = u;
        }
        if (D == 3) {
            T u = T(0);
#pragma unroll
            for (int m = 0; m < N; ++m)
                u = fma(tb.D[b][m], qf[(size_t)(v * S::nfp + fp_at<D, N>(df, s, a, m)) * E + e], u);
            gf[td1] = u;
        }
        T comp[3];
#pragma unroll
        for (int dd = 0; dd < D; ++dd) comp[dd] = gf[dd];
        comp[df] = fma(s ? etagR : etagL, dq[(size_t)(v * S::nfp + k) * E + e], gf[df]);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            T acc = T(0);
#pragma unroll
            for (int dd = 0; dd < D; ++dd) acc = fma(g[dd][c], comp[dd], acc);
            Qf[(size_t)((c * S::nv + v) * S::nfp + k) * E + e] = acc;
        }
    }
}

// stage 4: common normal flux Rusanov(qL, qR, n) - f_v(qs, Qs) . n on both sides
template <int D, int P, typename T>
__global__ void __launch_bounds__(256) k_pair_flux(const int4 *__restrict__ pairs, const int *__restrict__ bcs,
                                                   int npairs, const T *__restrict__ qf, const T *__restrict__ Qf,
                                                   const typename FrBase<T>::type *__restrict__ Sf, T *__restrict__ fn,
                                                   int E, FrPhys<typename FrBase<T>::type> ph) {
    using S = Sh<D, P>;
    typedef typename FrBase<T>::type B;
    constexpr int nv = S::nv;
    int P_ = blockIdx.x * blockDim.x + threadIdx.x;
    if (P_ >= npairs) return;
    int4 pr = pairs[P_];
    int bc = bcs[P_];
    int f = pr.y / S::nf1, df = f >> 1, side = f & 1;
    B nrm[3];
#pragma unroll
    for (int c = 0; c < D; ++c) {
        B sv = Sf[(size_t)((df * D + c) * S::nfp + pr.y) * E + pr.x];
        nrm[c] = side ? sv : -sv;
    }
    T qL[5], qR[5], qs[5], QL[3][5], Qs[3][5];
#pragma unroll
    for (int v = 0; v < nv; ++v) {
        qL[v] = qf[(size_t)(v * S::nfp + pr.y) * E + pr.x];
#pragma unroll
        for (int c = 0; c < D; ++c) QL[c][v] = Qf[(size_t)((c * nv + v) * S::nfp + pr.y) * E + pr.x];
    }
    if (bc == 0) {
#pragma unroll
        for (int v = 0; v < nv; ++v) {
            qR[v] = qf[(size_t)(v * S::nfp + pr.w) * E + pr.z];
#pragma unroll
            for (int c = 0; c < D; ++c)
                Qs[c][v] = T(0.5) * (QL[c][v] + Qf[(size_t)((c * nv + v) * S::nfp + pr.w) * E + pr.z]);
        }
    } else {
        ghost_state<D, T, B>(ph, bc, qL, qR);
#pragma unroll
        for (int v = 0; v < nv; ++v)
#pragma unroll
            for (int c = 0; c < D; ++c) Qs[c][v] = QL[c][v];
    }
#pragma unroll
    for (int v = 0; v < nv; ++v) qs[v] = T(0.5) * (qL[v] + qR[v]);
    T Fr[5], fv[3][5];
    if (ph.flux == 2) weiss_smith<D, T, B>(ph, qL, qR, nrm, Fr);
    else if (ph.flux == 1) roe<D, T, B>(ph, qL, qR, nrm, Fr);
    else rusanov<D, T, B>(ph, qL, qR, nrm, Fr);
    flux_viscous<D, T, B>(ph, qs, Qs, bc == 2, fv);
#pragma unroll
    for (int v = 0; v < nv; ++v) {
        T Fv = T(0);
#pragma unroll
        for (int c = 0; c < D; ++c) Fv = fma(fv[c][v], nrm[c], Fv);
        T F = Fr[v] - Fv;
        fn[(size_t)(v * S::nfp + pr.y) * E + pr.x] = F;
        if (bc == 0) fn[(size_t)(v * S::nfp + pr.w) * E + pr.z] = -F;
    }
}

// stage 5a: corrected gradient at the solution point (never stored), then the transformed
// volume flux Ft[dd][v][i][e] = sum_c S[dd][c] (f_inv - f_visc)_c; one thread per (i, e)
template <int D, int P, typename T>
__global__ void __launch_bounds__(256) k_grad_vflux(const T *__restrict__ q, const T *__restrict__ dq,
                                                    const typename FrBase<T>::type *__restrict__ G,
                                                    const typename FrBase<T>::type *__restrict__ Sm, T *__restrict__ Ft,
                                                    int E, FrPhys<typename FrBase<T>::type> ph) {
    using S = Sh<D, P>;
    typedef typename FrBase<T>::type B;
    constexpr int N = S::n, nv = S::nv;
    int e = blockIdx.y * blockDim.x + threadIdx.x;   // the points of an element chunk run side by side
    if (e >= E) return;
    int i = blockIdx.x;
    int ii[3] = {i % N, (i / N) % N, D == 3 ? i / (N * N) : 0};
    const FrTab<B> &tb = frtab<B>(P);
    B g[3][3];
#pragma unroll
    for (int dd = 0; dd < D; ++dd)
#pragma unroll
        for (int c = 0; c < D; ++c) g[dd][c] = G[(size_t)((dd * D + c) * S::np + i) * E + e];
    T qi[5], Qi[3][5], fi[3][5], fvi[3][5];
#pragma unroll
    for (int v = 0; v < nv; ++v) {
        qi[v] = q[(size_t)(v * S::np + i) * E + e];
        T gr[3];
#pragma unroll
        for (int dd = 0; dd < D; ++dd) {
            T t = T(0);
            int cd = ii[dd];
#pragma unroll
            for (int m = 0; m < N; ++m) {
                int jj0 = dd == 0 ? m : ii[0], jj1 = dd == 1 ? m : ii[1], jj2 = dd == 2 ? m : ii[2];
                t = fma(tb.D[cd][m], q[(size_t)(v * S::np + spi<D, N>(jj0, jj1, jj2)) * E + e], t);
            }
            int kL = fp_of<D, N>(dd, 0, ii[0], ii[1], ii[2]), kR = fp_of<D, N>(dd, 1, ii[0], ii[1], ii[2]);
            t = fma(tb.gLd[cd], dq[(size_t)(v * S::nfp + kL) * E + e], t);
            t = fma(tb.gRd[cd], dq[(size_t)(v * S::nfp + kR) * E + e], t);
            gr[dd] = t;
        }
#pragma unroll
        for (int c = 0; c < D; ++c) {
            T acc = T(0);
#pragma unroll
            for (int dd = 0; dd < D; ++dd) acc = fma(g[dd][c], gr[dd], acc);
            Qi[c][v] = acc;
        }
    }
    flux_inviscid<D, T, B>(ph, qi, fi);
    flux_viscous<D, T, B>(ph, qi, Qi, false, fvi);
#pragma unroll
    for (int dd = 0; dd < D; ++dd) {
        B sm[3];
#pragma unroll
        for (int c = 0; c < D; ++c) sm[c] = Sm[(size_t)((dd * D + c) * S::np + i) * E + e];
#pragma unroll
        for (int v = 0; v < nv; ++v) {
            T acc = T(0);
#pragma unroll
            for (int c = 0; c < D; ++c) acc = fma(sm[c], fi[c][v] - fvi[c][v], acc);
            Ft[(size_t)((dd * nv + v) * S::np + i) * E + e] = acc;
        }
    }
}

// stage 5b: transformed discontinuous flux at the face points (normal component); one
// thread per (k, e), all v
template <int D, int P, typename T>
__global__ void __launch_bounds__(256) k_face_ft(const T *__restrict__ Ft, T *__restrict__ Ftf, int E) {
    using S = Sh<D, P>;
    constexpr int N = S::n;
    int e = blockIdx.y * blockDim.x + threadIdx.x;   // the points of an element chunk run side by side
    if (e >= E) return;
    int k = blockIdx.x;
    int df, s, a, b;
    fp_decode<D, N>(k, df, s, a, b);
    typedef typename FrBase<T>::type B;
    const FrTab<B> &tb = frtab<B>(P);
#pragma unroll
    for (int v = 0; v < S::nv; ++v) {
        T acc = T(0);
#pragma unroll
        for (int m = 0; m < N; ++m) {
            T l = s ? tb.lp[m] : tb.lm[m];
            acc = fma(l, Ft[(size_t)((df * S::nv + v) * S::np + line_pt<D, N>(df, a, b, m)) * E + e], acc);
        }
        Ftf[(size_t)(v * S::nfp + k) * E + e] = acc;
    }
}

// stage 5c: divergence with FR corrections, R = -(div * invJ); one thread per (i, e), all v
template <int D, int P, typename T>
__global__ void __launch_bounds__(256) k_div(const T *__restrict__ Ft, const T *__restrict__ Ftf,
                                             const T *__restrict__ fn, const typename FrBase<T>::type *__restrict__ invJ,
                                             T *__restrict__ R, int E) {
    using S = Sh<D, P>;
    constexpr int N = S::n;
    int e = blockIdx.y * blockDim.x + threadIdx.x;   // the points of an element chunk run side by side
    if (e >= E) return;
    int i = blockIdx.x;
    int ii[3] = {i % N, (i / N) % N, D == 3 ? i / (N * N) : 0};
    typedef typename FrBase<T>::type B;
    const FrTab<B> &tb = frtab<B>(P);
    B ij = invJ[(size_t)i * E + e];
#pragma unroll
    for (int v = 0; v < S::nv; ++v) {
        T div = T(0);
#pragma unroll
        for (int dd = 0; dd < D; ++dd) {
            int cd = ii[dd];
            const T *F = Ft + (size_t)((dd * S::nv + v) * S::np) * E;
            T t = T(0);
#pragma unroll
            for (int m = 0; m < N; ++m) {
                int jj0 = dd == 0 ? m : ii[0], jj1 = dd == 1 ? m : ii[1], jj2 = dd == 2 ? m : ii[2];
                t = fma(tb.D[cd][m], F[(size_t)spi<D, N>(jj0, jj1, jj2) * E + e], t);
            }
            int kL = fp_of<D, N>(dd, 0, ii[0], ii[1], ii[2]), kR = fp_of<D, N>(dd, 1, ii[0], ii[1], ii[2]);
            T FsL = -fn[(size_t)(v * S::nfp + kL) * E + e];
            T FsR = fn[(size_t)(v * S::nfp + kR) * E + e];
            t = fma(tb.gLd[cd], FsL - Ftf[(size_t)(v * S::nfp + kL) * E + e], t);
            t = fma(tb.gRd[cd], FsR - Ftf[(size_t)(v * S::nfp + kR) * E + e], t);
            div = div + t;
        }
        R[(size_t)(v * S::np + i) * E + e] = -(div * ij);
    }
}
