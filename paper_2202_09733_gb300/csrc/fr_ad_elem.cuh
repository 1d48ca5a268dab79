// FP32 element-diagonal Jacobian blocks M_e = shift I - dR_e/dq_e (Eq. 9, Sec. 3.2) by
// forward-mode differentiation of one element's residual at a time.
//
// R_e depends on q_e through its own volume and face terms and, at each shared face
// point, through the common solution q* = (qf_e + qf_n)/2, which also enters the
// neighbour's BR2 face gradient: Qf_n = Qf_n(q) + lift_n (q* - q*(q)), lift_n[c] =
// eta g'_n Gf_n[df_n][c] (the neighbour's own lifting of its jump).  Everything else the
// neighbour contributes is frozen.  So with the neighbour's trace qf_n, its face gradient
// Qf_n and lift_n gathered once per assembly (k_ad_traces), each element's block follows
// from its own data alone: one CTA holds TE elements' state, traces and transformed
// fluxes in shared memory and runs the residual on dual numbers seeded in K degrees of
// freedom at a time, for all ceil(nd / K) seed batches, writing K columns per batch.
//
// Each face flux is evaluated with the element's own outward normal: F(qf_e, q_other, n_e),
// equal up to FP32 rounding to minus the flux the other side would form with its normal
// (n_n = -n_e on conforming faces; the Rusanov and Roe fluxes are antisymmetric under
// exchange of the states and reversal of the normal).  A face that wraps onto its own
// element (a periodic direction one element wide) couples q_e to itself through the
// "neighbour": the host uses the colouring path for such meshes.
//
// Included by kernelsad.cu (frtab<float> is its constant-memory table).
#pragma once
#include "fr_device.cuh"

// per element face point (k, e), the other side's frozen data, NT[slot][k][e]:
//   slots 0 .. nv-1                 qf_n[v]
//   slots nv + c nv + v             Qf_n[c][v]
//   slots nv + D nv + c             lift_n[c]
// and BCk[k][e]: 0 interior, 1 far field, 2 adiabatic wall
template <int D>
struct AdSlots {
    static constexpr int nv = D + 2;
    static constexpr int n = nv + D * nv + D;
};

template <int D, int P>
__global__ void __launch_bounds__(256) k_ad_traces(const int4 *__restrict__ pairs, const int *__restrict__ bcs,
                                                   int npairs, const float *__restrict__ qf,
                                                   const float *__restrict__ Qf, const float *__restrict__ Gf,
                                                   float etagL, float etagR, int E, float *__restrict__ NT,
                                                   signed char *__restrict__ BCk) {
    using S = Sh<D, P>;
    constexpr int nv = S::nv;
    int P_ = blockIdx.x * blockDim.x + threadIdx.x;
    if (P_ >= npairs) return;
    int4 pr = pairs[P_];
    int bc = bcs[P_];
    BCk[(size_t)pr.y * E + pr.x] = (signed char)bc;
    if (bc != 0) return;
    BCk[(size_t)pr.w * E + pr.z] = 0;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        int e = side ? pr.z : pr.x, k = side ? pr.w : pr.y;      // destination: this side
        int eo = side ? pr.x : pr.z, ko = side ? pr.y : pr.w;    // source: the other side
        int fo = ko / S::nf1, dfo = fo >> 1, so = fo & 1;
        float etag = so ? etagR : etagL;
        auto dst = [&](int slot) -> float & { return NT[((size_t)slot * S::nfp + k) * E + e]; };
#pragma unroll
        for (int v = 0; v < nv; ++v) dst(v) = qf[(size_t)(v * S::nfp + ko) * E + eo];
#pragma unroll
        for (int c = 0; c < D; ++c)
#pragma unroll
            for (int v = 0; v < nv; ++v)
                dst(nv + c * nv + v) = Qf[(size_t)((c * nv + v) * S::nfp + ko) * E + eo];
#pragma unroll
        for (int c = 0; c < D; ++c) dst(nv + D * nv + c) = etag * Gf[(size_t)((dfo * D + c) * S::nfp + ko) * E + eo];
    }
}

// Blocks of TE elements per CTA.  Shared memory per element (DualT values): q[nv][Np],
// qf[nv][Nfp], dq / J[nv][Nfp], Ft[D][nv][Np].  Phases of one seed batch (j0 .. j0+K-1):
//   seed   q.d[t] = (r == j0 + t)
//   A      per face point: qf (interpolation), the other side's state (frozen trace or
//          ghost), q* and the jump dq = q* - qf
//   B      per solution point: corrected gradient Q, fluxes, Ft[dd][v][i]
//   C      per face point: face gradient Qf_e (with its lifting), the other side's Qf_n,
//          common flux F along the outward normal, J = (+-F) - Ftf
//   D      per (v, i): R = -(sum_dd D Ft + gL' J_L + gR' J_R) / J, columns of M
template <int D, int P>
struct AdElem {
    using S = Sh<D, P>;
    static constexpr int nv = S::nv, np = S::np, nfp = S::nfp, nd = nv * np;
    static constexpr int per_elem = nv * np + 2 * nv * nfp + D * nv * np;   // DualT values
    static constexpr size_t bytes_per_elem = sizeof(DualT) * per_elem;
};

template <int D, int P>
__global__ void __launch_bounds__(128) k_ad_elem_blocks(const float *__restrict__ q, const float *__restrict__ Gm,
                                                        const float *__restrict__ Sm, const float *__restrict__ invJ,
                                                        const float *__restrict__ Gf, const float *__restrict__ Sf,
                                                        const float *__restrict__ NT,
                                                        const signed char *__restrict__ BCk, int E, int TE,
                                                        FrPhys<float> ph, float shift, float *__restrict__ M) {
    using S = Sh<D, P>;
    using A = AdElem<D, P>;
    constexpr int N = S::n, nv = S::nv, np = S::np, nfp = S::nfp, nd = A::nd;
    typedef DualT T;
    extern __shared__ __align__(16) unsigned char ad_raw[];
    T *sm = reinterpret_cast<T *>(ad_raw);
    const FrTab<float> &tb = frtab<float>(P);
    const int e0 = blockIdx.x * TE;
    const int te_n = min(TE, E - e0);
    const int tid = threadIdx.x, nth = blockDim.x;
    auto SQ = [&](int te) { return sm + (size_t)te * A::per_elem; };
    auto SQF = [&](int te) { return SQ(te) + nv * np; };
    auto SJ = [&](int te) { return SQF(te) + nv * nfp; };
    auto SFT = [&](int te) { return SJ(te) + nv * nfp; };

    // primal state
    for (int it = tid; it < te_n * nd; it += nth) {
        int te = it / nd, r = it - te * nd;
        SQ(te)[r] = T(q[(size_t)r * E + e0 + te]);
    }
    for (int j0 = 0; j0 < nd; j0 += FR_AD_K) {
        // ---- seeds
        for (int it = tid; it < te_n * nd; it += nth) {
            int te = it / nd, r = it - te * nd;
            T &x = SQ(te)[r];
#pragma unroll
            for (int t = 0; t < FR_AD_K; ++t) x.d[t] = (r == j0 + t) ? 1.f : 0.f;
        }
        __syncthreads();
        // ---- A: traces, common solution, jumps
        for (int it = tid; it < te_n * nfp; it += nth) {
            int te = it / nfp, k = it - te * nfp, e = e0 + te;
            int df, s, a, b;
            fp_decode<D, N>(k, df, s, a, b);
            const T *sq = SQ(te);
            T qL[5], qR[5];
#pragma unroll
            for (int v = 0; v < nv; ++v) {
                T acc = T(0);
#pragma unroll
                for (int m = 0; m < N; ++m) acc = fma(s ? tb.lp[m] : tb.lm[m], sq[v * np + line_pt<D, N>(df, a, b, m)], acc);
                qL[v] = acc;
                SQF(te)[v * nfp + k] = acc;
            }
            int bc = BCk[(size_t)k * E + e];
            if (bc == 0) {
#pragma unroll
                for (int v = 0; v < nv; ++v) qR[v] = T(NT[((size_t)v * nfp + k) * E + e]);
            } else {
                ghost_state<D, T, float>(ph, bc, qL, qR);
            }
#pragma unroll
            for (int v = 0; v < nv; ++v) {
                T qs = T(0.5f) * (qL[v] + qR[v]);
                SJ(te)[v * nfp + k] = qs - qL[v];
            }
        }
        __syncthreads();
        // ---- B: corrected gradient and transformed volume flux at the solution points
        for (int it = tid; it < te_n * np; it += nth) {
            int te = it / np, i = it - te * np, e = e0 + te;
            int ii[3] = {i % N, (i / N) % N, D == 3 ? i / (N * N) : 0};
            const T *sq = SQ(te), *sj = SJ(te);
            T qi[5], Qi[3][5], fi[3][5], fvi[3][5];
            float g[3][3];
#pragma unroll
            for (int dd = 0; dd < D; ++dd)
#pragma unroll
                for (int c = 0; c < D; ++c) g[dd][c] = Gm[(size_t)((dd * D + c) * np + i) * E + e];
#pragma unroll
            for (int v = 0; v < nv; ++v) {
                qi[v] = sq[v * np + i];
                T gr[3];
#pragma unroll
                for (int dd = 0; dd < D; ++dd) {
                    int cd = ii[dd];
                    T t = T(0);
#pragma unroll
                    for (int m = 0; m < N; ++m) {
                        int jj0 = dd == 0 ? m : ii[0], jj1 = dd == 1 ? m : ii[1], jj2 = dd == 2 ? m : ii[2];
                        t = fma(tb.D[cd][m], sq[v * np + spi<D, N>(jj0, jj1, jj2)], t);
                    }
                    int kL = fp_of<D, N>(dd, 0, ii[0], ii[1], ii[2]), kR = fp_of<D, N>(dd, 1, ii[0], ii[1], ii[2]);
                    t = fma(tb.gLd[cd], sj[v * nfp + kL], t);
                    t = fma(tb.gRd[cd], sj[v * nfp + kR], t);
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
            flux_inviscid<D, T, float>(ph, qi, fi);
            flux_viscous<D, T, float>(ph, qi, Qi, false, fvi);
#pragma unroll
            for (int dd = 0; dd < D; ++dd) {
                float sv[3];
#pragma unroll
                for (int c = 0; c < D; ++c) sv[c] = Sm[(size_t)((dd * D + c) * np + i) * E + e];
#pragma unroll
                for (int v = 0; v < nv; ++v) {
                    T acc = T(0);
#pragma unroll
                    for (int c = 0; c < D; ++c) acc = fma(sv[c], fi[c][v] - fvi[c][v], acc);
                    SFT(te)[(dd * nv + v) * np + i] = acc;
                }
            }
        }
        __syncthreads();
        // ---- C: face gradients, common flux, flux jumps
        for (int it = tid; it < te_n * nfp; it += nth) {
            int te = it / nfp, k = it - te * nfp, e = e0 + te;
            int df, s, a, b;
            fp_decode<D, N>(k, df, s, a, b);
            const T *sq = SQ(te), *sqf = SQF(te), *sft = SFT(te);
            T *sj = SJ(te);
            int bc = BCk[(size_t)k * E + e];
            float gfm[3][3], nrm[3];
#pragma unroll
            for (int dd = 0; dd < D; ++dd)
#pragma unroll
                for (int c = 0; c < D; ++c) gfm[dd][c] = Gf[(size_t)((dd * D + c) * nfp + k) * E + e];
#pragma unroll
            for (int c = 0; c < D; ++c) {
                float sv = Sf[(size_t)((df * D + c) * nfp + k) * E + e];
                nrm[c] = s ? sv : -sv;
            }
            int td0 = df == 0 ? 1 : 0, td1 = df == 2 ? 1 : 2;
            T qL[5], qR[5], qs[5], Qs[3][5];
#pragma unroll
            for (int v = 0; v < nv; ++v) {
                qL[v] = sqf[v * nfp + k];
                T gf[3];
                T t = T(0);
#pragma unroll
                for (int m = 0; m < N; ++m) t = fma(s ? tb.dlp[m] : tb.dlm[m], sq[v * np + line_pt<D, N>(df, a, b, m)], t);
                gf[df] = fma(s ? ph.etagR : ph.etagL, sj[v * nfp + k], t);
                T u = T(0);
#pragma unroll
                for (int m = 0; m < N; ++m) u = fma(tb.D[a][m], sqf[v * nfp + fp_at<D, N>(df, s, m, b)], u);
                gf[td0] = u;
                if (D == 3) {
                    T w = T(0);
#pragma unroll
                    for (int m = 0; m < N; ++m) w = fma(tb.D[b][m], sqf[v * nfp + fp_at<D, N>(df, s, a, m)], w);
                    gf[td1] = w;
                }
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    T acc = T(0);
#pragma unroll
                    for (int dd = 0; dd < D; ++dd) acc = fma(gfm[dd][c], gf[dd], acc);
                    Qs[c][v] = acc;
                }
            }
            if (bc == 0) {
#pragma unroll
                for (int v = 0; v < nv; ++v) qR[v] = T(NT[((size_t)v * nfp + k) * E + e]);
#pragma unroll
                for (int v = 0; v < nv; ++v) qs[v] = T(0.5f) * (qL[v] + qR[v]);
                float lift[3];
#pragma unroll
                for (int c = 0; c < D; ++c) lift[c] = NT[((size_t)(nv + D * nv + c) * nfp + k) * E + e];
                // the neighbour's face gradient moves with q* through its own lifting
#pragma unroll
                for (int c = 0; c < D; ++c)
#pragma unroll
                    for (int v = 0; v < nv; ++v) {
                        T Qn(NT[((size_t)(nv + c * nv + v) * nfp + k) * E + e]);
#pragma unroll
                        for (int t = 0; t < FR_AD_K; ++t) Qn.d[t] = lift[c] * qs[v].d[t];
                        Qs[c][v] = T(0.5f) * (Qs[c][v] + Qn);
                    }
            } else {
                ghost_state<D, T, float>(ph, bc, qL, qR);
#pragma unroll
                for (int v = 0; v < nv; ++v) qs[v] = T(0.5f) * (qL[v] + qR[v]);
            }
            T Fr[5], fv[3][5];
            if (ph.flux == 1) roe<D, T, float>(ph, qL, qR, nrm, Fr);
            else rusanov<D, T, float>(ph, qL, qR, nrm, Fr);
            flux_viscous<D, T, float>(ph, qs, Qs, bc == 2, fv);
#pragma unroll
            for (int v = 0; v < nv; ++v) {
                T Fv = T(0);
#pragma unroll
                for (int c = 0; c < D; ++c) Fv = fma(fv[c][v], nrm[c], Fv);
                T F = Fr[v] - Fv;
                T Ftf = T(0);
#pragma unroll
                for (int m = 0; m < N; ++m)
                    Ftf = fma(s ? tb.lp[m] : tb.lm[m], sft[(df * nv + v) * np + line_pt<D, N>(df, a, b, m)], Ftf);
                sj[v * nfp + k] = (s ? F : -F) - Ftf;
            }
        }
        __syncthreads();
        // ---- D: divergence with the FR correction, K columns of each block
        for (int it = tid; it < te_n * nd; it += nth) {
            int te = it / nd, r = it - te * nd, e = e0 + te;
            int v = r / np, i = r - v * np;
            int ii[3] = {i % N, (i / N) % N, D == 3 ? i / (N * N) : 0};
            const T *sft = SFT(te), *sj = SJ(te);
            T div = T(0);
#pragma unroll
            for (int dd = 0; dd < D; ++dd) {
                int cd = ii[dd];
                T t = T(0);
#pragma unroll
                for (int m = 0; m < N; ++m) {
                    int jj0 = dd == 0 ? m : ii[0], jj1 = dd == 1 ? m : ii[1], jj2 = dd == 2 ? m : ii[2];
                    t = fma(tb.D[cd][m], sft[(dd * nv + v) * np + spi<D, N>(jj0, jj1, jj2)], t);
                }
                int kL = fp_of<D, N>(dd, 0, ii[0], ii[1], ii[2]), kR = fp_of<D, N>(dd, 1, ii[0], ii[1], ii[2]);
                t = fma(tb.gLd[cd], sj[v * nfp + kL], t);
                t = fma(tb.gRd[cd], sj[v * nfp + kR], t);
                div = div + t;
            }
            float ij = invJ[(size_t)i * E + e];
            float *Me = M + (size_t)e * nd * nd;
#pragma unroll
            for (int t = 0; t < FR_AD_K; ++t) {
                int j = j0 + t;
                if (j < nd) {
                    float dr = -(div.d[t] * ij);
                    Me[(size_t)j * nd + r] = (r == j ? shift : 0.f) - dr;
                }
            }
        }
        __syncthreads();
    }
}
