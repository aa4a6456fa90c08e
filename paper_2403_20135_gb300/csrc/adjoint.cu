// Discrete adjoint of the explicit tendency T_E and of the sweep kernel, for
// gradients of a loss on the final state with respect to the initial state
// (reverse-mode differentiation of Algorithm 2 with the node update Eq. (7)).
//
// Every kernel is the exact transpose, with respect to the real degrees of
// freedom (Re, Im) of the stored arrays, of one forward kernel:
//   K3b^T  epilogue transpose      per extended row      T_E-bar -> Y-bar
//   K3a^T  projection transpose    per (order pair, j)   Y-bar -> W-bar     (synthesis-shaped)
//   K2^T   ring transpose          per (ring pair)       W-bar -> F1-bar    (FFTs + grid products)
//   K1a^T  synthesis transpose     per extended row      F1-bar -> Z-bar    (projection-shaped)
//   K1b^T  prep transpose          per mode, accumulate  Z-bar -> u-bar
//   K4^T   sweep transpose         per mode, all nodes
// Transposes of the building blocks: a complex constant z becomes conj(z)
// (i m -> -i m); a real matrix becomes its transpose;
// f = F_0 + 2 Re sum_{m>0} F_m e^{i m lambda} becomes Fbar_m = w_m sum_k f_k e^{-i m lambda_k}
// (w_0 = 1, w_m = 2); F_m = (1/L) sum_k f_k e^{-i m lambda_k} becomes
// fbar_k = (1/L) Re sum_m Fbar_m e^{i m lambda_k}.  The grid products need the
// base state's grid fields, recorded by the forward ring kernel during the
// retape of the step.
#include <cuda_runtime.h>

#include "async_copy.cuh"
#include "convert.cuh"
#include "fft.cuh"
#include "fft_pass.cuh"
#include "sdc_internal.h"

namespace sdc {

constexpr int kAdjThreads = 64;

// ---------------------------------------------------------------------------
// K3b^T: per extended row e = (m, n'), from the T_E adjoint (3 fields):
//   A-bar_n' = (i m/a) zeta-bar_n' - (cu/a) div-bar_{n'-1} + (cl/a) div-bar_{n'+1}
//   B-bar_n' = -(cu/a) zeta-bar_{n'-1} + (cl/a) zeta-bar_{n'+1} - (i m/a) div-bar_n'
//   C-bar_n' = (i m/a) Phi-bar_n'
//   D-bar_n' = -(cu/a) Phi-bar_{n'-1} + (cl/a) Phi-bar_{n'+1}
//   E-bar_n' = lambda_n' div-bar_n'
// with cu = (n'-1) eps_n' and cl = (n'+2) eps_{n'+1}; entries outside m..T are 0.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k3t_epilogue(const double2 *__restrict__ abar, long long astride, Dims d,
                             const double *__restrict__ eps, const int *__restrict__ row_m,
                             V2<R> *__restrict__ ybar) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (e >= d.next) return;
    const int T = d.T, nc = d.ncoef;
    const int m = row_m[e];
    const int t = e - ext_offset(T, m);
    const int n = m + t;
    const int off = order_offset(T, m);
    const double2 *ab = abar + b * astride;
    auto ld = [&](int f, int k) -> double2 {
        return (k >= m && k <= T) ? ab[f * nc + off + k - m] : make_double2(0.0, 0.0);
    };
    const double inv_a = d.inv_a;
    const double cu = (t >= 1) ? (n - 1.0) * eps[e] * inv_a : 0.0;
    const double cl = (n + 1 <= T) ? (n + 2.0) * eps[e + 1] * inv_a : 0.0;
    const double mi = double(m) * inv_a;
    const double lam = double(n) * double(n + 1) * inv_a * inv_a;
    const double2 z0 = ld(F_ZETA, n), zm = ld(F_ZETA, n - 1), zp = ld(F_ZETA, n + 1);
    const double2 d0 = ld(F_DIV, n), dm = ld(F_DIV, n - 1), dp = ld(F_DIV, n + 1);
    const double2 p0 = ld(F_PHI, n), pm = ld(F_PHI, n - 1), pp = ld(F_PHI, n + 1);
    // (i c) z = (-c z.y, c z.x); narrowed to FP32 on the integer pipe (convert.cuh)
    auto nr = [](double x) -> R {
        if constexpr (sizeof(R) == sizeof(float)) return f64_to_f32_rn(x);
        else return x;
    };
    V2<R> *o = ybar + (static_cast<size_t>(b) * d.next + e) * 5;
    o[P_A] = mk<R>(nr(-mi * z0.y - cu * dm.x + cl * dp.x), nr(mi * z0.x - cu * dm.y + cl * dp.y));
    o[P_B] = mk<R>(nr(-cu * zm.x + cl * zp.x + mi * d0.y), nr(-cu * zm.y + cl * zp.y - mi * d0.x));
    o[P_C] = mk<R>(nr(-mi * p0.y), nr(mi * p0.x));
    o[P_D] = mk<R>(nr(-cu * pm.x + cl * pp.x), nr(-cu * pm.y + cl * pp.y));
    o[P_E] = mk<R>(nr(lam * d0.x), nr(lam * d0.y));
}

// ---------------------------------------------------------------------------
// K3a^T: W-bar_g[parity][j] = sum over rows e of order m with that parity of
// Pbar_e(mu_j) Y-bar_g[e]; blocks serve orders m and T - m.  Output in the
// FP64 forward's F2 layout [b][m][g][parity][j2].
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(64) k3t_synth(const V2<R> *__restrict__ ybar, Dims d, const R *__restrict__ pbar,
                                                V2<R> *__restrict__ wbar) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V2<R> *ys = reinterpret_cast<V2<R> *>(smem_raw);   // [rows][5]
    const int T = d.T;
    const int m1 = blockIdx.x, m2 = T - blockIdx.x;
    const int b = blockIdx.y;
    const int nn1 = T + 2 - m1;
    const int nn2 = (m2 > m1) ? T + 2 - m2 : 0;
    const int rows = nn1 + nn2;
    for (int i = threadIdx.x; i < rows * 5; i += blockDim.x) {
        const int r = i / 5, g = i - r * 5;
        const int m = (r < nn1) ? m1 : m2;
        const int t = (r < nn1) ? r : r - nn1;
        ys[i] = ybar[(static_cast<size_t>(b) * d.next + ext_offset(T, m) + t) * 5 + g];
    }
    __syncthreads();
    const int j = blockIdx.z * blockDim.x + threadIdx.x;
    if (j >= d.J2) return;
    for (int half = 0; half < 2; ++half) {
        const int m = half ? m2 : m1;
        const int nn = half ? nn2 : nn1;
        if (nn == 0) break;
        const V2<R> *c = ys + (half ? nn1 : 0) * 5;
        V2<R> ae[5], ao[5];
#pragma unroll
        for (int g = 0; g < 5; ++g) { ae[g] = mk<R>(0, 0); ao[g] = mk<R>(0, 0); }
        const R *prow = pbar + static_cast<size_t>(ext_offset(T, m)) * d.J2p + j;
        int t = 0;
        for (; t + 1 < nn; t += 2) {
            const R pe = prow[static_cast<size_t>(t) * d.J2p];
            const R po = prow[static_cast<size_t>(t + 1) * d.J2p];
#pragma unroll
            for (int g = 0; g < 5; ++g) {
                const V2<R> ce = c[t * 5 + g], co = c[(t + 1) * 5 + g];
                ae[g].x = fma(pe, ce.x, ae[g].x);
                ae[g].y = fma(pe, ce.y, ae[g].y);
                ao[g].x = fma(po, co.x, ao[g].x);
                ao[g].y = fma(po, co.y, ao[g].y);
            }
        }
        if (t < nn) {
            const R pe = prow[static_cast<size_t>(t) * d.J2p];
#pragma unroll
            for (int g = 0; g < 5; ++g) {
                const V2<R> ce = c[t * 5 + g];
                ae[g].x = fma(pe, ce.x, ae[g].x);
                ae[g].y = fma(pe, ce.y, ae[g].y);
            }
        }
        V2<R> *o = wbar + (static_cast<size_t>(b) * (T + 1) + m) * 10 * d.J2 + j;
#pragma unroll
        for (int g = 0; g < 5; ++g) {
            o[(g * 2 + 0) * d.J2] = ae[g];
            o[(g * 2 + 1) * d.J2] = ao[g];
        }
    }
}

// ---------------------------------------------------------------------------
// K2^T: one block per (ring pair j2, state b), the transpose of the forward
// ring kernel: weights and north/south split, forward-DFT transpose (an
// inverse FFT of the m <= T spectrum with m > 0 halved, scaled 1/L), the
// grid products transposed with the recorded base fields, inverse-DFT
// transpose (a forward FFT, m > 0 doubled) and the parity split transposed.
// Output F1-bar[b][m][field][parity][j2] (the FP64 synthesis transpose reads
// it along the latitudes).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k2t_ring(const V2<R> *__restrict__ wbar, const V2<R> *__restrict__ gbase,
                         V2<R> *__restrict__ f1bar, Dims d, FftPlan plan, const V2<R> *__restrict__ tw,
                         const double *__restrict__ mu, const double *__restrict__ w, int nscratch) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V2<R> *X = reinterpret_cast<V2<R> *>(smem_raw);   // [5][L]
    V2<R> *S = X + 5 * plan.L;
    V2<R> *TW = S + nscratch * plan.L;                  // twiddles [L]
    const int j2 = blockIdx.x;
    const int b = blockIdx.y;
    const int T = d.T, L = plan.L, J2 = d.J2;
    for (int k = threadIdx.x; k < L; k += blockDim.x) TW[k] = tw[k];
    const double mun = mu[j2];
    const double c2 = (1.0 - mun) * (1.0 + mun);
    const R wt = R(w[j2] / c2), wp = R(w[j2]);
    const R invL = R(1.0) / R(L);

    for (int i = threadIdx.x; i < 5 * L; i += blockDim.x) {
        const int g = i / L, k = i - g * L;
        V2<R> z = mk<R>(0, 0);
        int m = -1;
        bool conj = false;
        if (k <= T) m = k;
        else if (k >= L - T) { m = L - k; conj = true; }
        if (m >= 0) {
            const V2<R> *src = wbar + ((static_cast<size_t>(b) * (T + 1) + m) * 5 + g) * 2 * J2 + j2;
            const V2<R> ws = src[0], wa = src[J2];
            const R wg = (g == P_E) ? wp : wt;
            const R sc = wg * ((m == 0) ? invL : R(0.5) * invL);
            V2<R> gn = cscale<R>(cadd<R>(ws, wa), sc), gsth = cscale<R>(csub<R>(ws, wa), sc);
            if (m == 0) { gn.y = 0; gsth.y = 0; }
            if (conj) { gn.y = -gn.y; gsth.y = -gsth.y; }
            z = mk<R>(gn.x - gsth.y, gn.y + gsth.x);   // north + i south
        }
        X[i] = z;
    }
    __syncthreads();
    fft_inplace<R>(X, S, nscratch, 5, plan, TW, true);

    const V2<R> *gb = gbase + (static_cast<size_t>(b) * J2 + j2) * 4 * L;
    const R fN = R(d.two_omega * mun);
    const R ic2 = R(1.0 / c2);
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        const V2<R> zz = gb[G_ZETA * L + k], pp = gb[G_PHI * L + k];
        const V2<R> uu = gb[G_U * L + k], vv = gb[G_V * L + k];
        const V2<R> Ab = X[P_A * L + k], Bb = X[P_B * L + k], Cb = X[P_C * L + k];
        const V2<R> Db = X[P_D * L + k], Eb = X[P_E * L + k];
        const R etaN = zz.x + fN, etaS = zz.y - fN;
        X[G_ZETA * L + k] = mk<R>(Ab.x * uu.x + Bb.x * vv.x, Ab.y * uu.y + Bb.y * vv.y);
        X[G_PHI * L + k] = mk<R>(Cb.x * uu.x + Db.x * vv.x, Cb.y * uu.y + Db.y * vv.y);
        X[G_U * L + k] = mk<R>(Ab.x * etaN + Cb.x * pp.x + Eb.x * uu.x * ic2,
                               Ab.y * etaS + Cb.y * pp.y + Eb.y * uu.y * ic2);
        X[G_V * L + k] = mk<R>(Bb.x * etaN + Db.x * pp.x + Eb.x * vv.x * ic2,
                               Bb.y * etaS + Db.y * pp.y + Eb.y * vv.y * ic2);
    }
    __syncthreads();
    fft_inplace<R>(X, S, nscratch, 4, plan, TW, false);

    V2<R> *o = f1bar + static_cast<size_t>(b) * (T + 1) * 8 * J2 + j2;   // [b][m][f][parity][j2]
    for (int i = threadIdx.x; i < 4 * (T + 1); i += blockDim.x) {
        const int f = i / (T + 1), m = i - f * (T + 1);
        const V2<R> y = X[f * L + m];
        V2<R> yc = X[f * L + (m == 0 ? 0 : L - m)];
        yc.y = -yc.y;
        const R wm = (m == 0) ? R(0.5) : R(1.0);           // w_m / 2
        const V2<R> fn = cscale<R>(cadd<R>(y, yc), wm);
        const V2<R> fs = cscale<R>(mul_mi<R>(csub<R>(y, yc)), wm);
        V2<R> se = cadd<R>(fn, fs), so = csub<R>(fn, fs);
        if (m == 0) { se.y = 0; so.y = 0; }
        o[(static_cast<size_t>(m) * 8 + f * 2 + 0) * J2] = se;
        o[(static_cast<size_t>(m) * 8 + f * 2 + 1) * J2] = so;
    }
}

// K2^T in FP32 on the padded radix-16 passes of fft_pass.cuh (as the FP32
// forward ring): LC > 0 fixes the ring length at compile time.  W-bar comes
// in the layout [b][j2][m][parity][g] (contiguous per ring pair: one bulk
// round of 16-byte copies; the synthesis transpose that writes it stores 40
// contiguous bytes per (j2, m, parity)); F1-bar leaves as [b][m][j2][f][parity]
// (64 contiguous bytes per (m, j2), read per order by the projection-shaped
// synthesis transpose).
template <int LC>
__global__ void __launch_bounds__(256) k2t_ring_f32(const float2 *__restrict__ wbar, const float2 *__restrict__ gbase,
                                                    float2 *__restrict__ f1bar, Dims d, FftPlan plan,
                                                    const float2 *__restrict__ twp, int ntw,
                                                    const float *__restrict__ rw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = LC > 0 ? LC : plan.L, Lp = fft_padded_len(L);
    float2 *X = reinterpret_cast<float2 *>(smem_raw);   // [5][Lp]
    float2 *S = X + 5 * Lp;                              // [5][Lp]
    float2 *TW = S + 5 * Lp;                             // [ntw]
    const int j2 = blockIdx.x;
    const int b = blockIdx.y;
    const int T = d.T, J2 = d.J2;
    // the block's W-bar slice (contiguous, 16-byte aligned) into the scratch
    // arrays S and the pass twiddles into TW, all copies in flight at once
    const float2 *win = wbar + (static_cast<size_t>(b) * J2 + j2) * 10 * (T + 1);
    float2 *raw = S;                                     // 10 (T + 1) <= 5 Lp elements
    if ((Lp & 1) == 0) {                                 // S starts on a 16-byte boundary
        for (int q = threadIdx.x; q < 5 * (T + 1); q += blockDim.x) cp_async16(raw + 2 * q, win + 2 * q);
    } else {
        for (int q = threadIdx.x; q < 10 * (T + 1); q += blockDim.x) cp_async8(raw + q, win + q);
    }
    for (int k = threadIdx.x; k < ntw; k += blockDim.x) cp_async8(TW + k, twp + k);
    cp_async_commit();
    const float fN = rw[4 * j2], ic2 = 2.f * rw[4 * j2 + 1], wt = rw[4 * j2 + 2], wp = rw[4 * j2 + 3];
    const float invL = 1.f / float(L);
    cp_async_wait<0>();
    __syncthreads();
    for (int i = threadIdx.x; i < 5 * L; i += blockDim.x) {
        const int g = i / L, k = i - g * L;
        float2 z = make_float2(0.f, 0.f);
        int m = -1;
        bool conj = false;
        if (k <= T) m = k;
        else if (k >= L - T) { m = L - k; conj = true; }
        if (m >= 0) {                                    // raw = W-bar[b][j2][m][parity][g]
            const float2 ws = raw[m * 10 + g], wa = raw[m * 10 + 5 + g];
            const float wg = (g == P_E) ? wp : wt;
            const float sc = wg * ((m == 0) ? invL : 0.5f * invL);
            float2 gn = cscale<float>(cadd<float>(ws, wa), sc), gsth = cscale<float>(csub<float>(ws, wa), sc);
            if (m == 0) { gn.y = 0.f; gsth.y = 0.f; }
            if (conj) { gn.y = -gn.y; gsth.y = -gsth.y; }
            z = make_float2(gn.x - gsth.y, gn.y + gsth.x);   // north + i south
        }
        X[g * Lp + fpad(k)] = z;
    }
    __syncthreads();
    const float2 *G;
    if constexpr (LC > 0) G = fft_passes_ct<LC, 5>(X, S, TW, true);
    else G = fft_passes(X, S, 5, Lp, plan, TW, true);

    const float2 *gb = gbase + (static_cast<size_t>(b) * J2 + j2) * 4 * L;
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        const int kp = fpad(k);
        const float2 zz = gb[G_ZETA * L + k], pp = gb[G_PHI * L + k];
        const float2 uu = gb[G_U * L + k], vv = gb[G_V * L + k];
        const float2 Ab = G[P_A * Lp + kp], Bb = G[P_B * Lp + kp], Cb = G[P_C * Lp + kp];
        const float2 Db = G[P_D * Lp + kp], Eb = G[P_E * Lp + kp];
        const float etaN = zz.x + fN, etaS = zz.y - fN;
        X[G_ZETA * Lp + kp] = make_float2(Ab.x * uu.x + Bb.x * vv.x, Ab.y * uu.y + Bb.y * vv.y);
        X[G_PHI * Lp + kp] = make_float2(Cb.x * uu.x + Db.x * vv.x, Cb.y * uu.y + Db.y * vv.y);
        X[G_U * Lp + kp] = make_float2(Ab.x * etaN + Cb.x * pp.x + Eb.x * uu.x * ic2,
                                       Ab.y * etaS + Cb.y * pp.y + Eb.y * uu.y * ic2);
        X[G_V * Lp + kp] = make_float2(Bb.x * etaN + Db.x * pp.x + Eb.x * vv.x * ic2,
                                       Bb.y * etaS + Db.y * pp.y + Eb.y * vv.y * ic2);
    }
    __syncthreads();
    const float2 *Y;
    if constexpr (LC > 0) Y = fft_passes_ct<LC, 4>(X, S, TW, false);
    else Y = fft_passes(X, S, 4, Lp, plan, TW, false);

    // F1-bar[b][m][j2][f][parity]: the values are staged as [m][f][parity] in
    // the free scratch array, then 64 contiguous bytes per (m, j2) are written
    // by neighbouring lanes (whole sectors instead of 8-byte pieces)
    float2 *Z = const_cast<float2 *>(Y == X ? S : X);
    const bool al16 = (reinterpret_cast<uintptr_t>(Z) & 15) == 0;   // odd padded lengths: Z on an 8-byte boundary
    for (int i = threadIdx.x; i < 4 * (T + 1); i += blockDim.x) {
        const int f = i / (T + 1), m = i - f * (T + 1);
        const float2 y = Y[f * Lp + fpad(m)];
        float2 yc = Y[f * Lp + fpad(m == 0 ? 0 : L - m)];
        yc.y = -yc.y;
        const float wm = (m == 0) ? 0.5f : 1.f;            // w_m / 2
        const float2 fn = cscale<float>(cadd<float>(y, yc), wm);
        const float2 fs = cscale<float>(mul_mi<float>(csub<float>(y, yc)), wm);
        float2 se = cadd<float>(fn, fs), so = csub<float>(fn, fs);
        if (m == 0) { se.y = 0.f; so.y = 0.f; }
        if (al16) {
            reinterpret_cast<float4 *>(Z)[m * 4 + f] = make_float4(se.x, se.y, so.x, so.y);
        } else {
            Z[(m * 4 + f) * 2] = se;
            Z[(m * 4 + f) * 2 + 1] = so;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * (T + 1); i += blockDim.x) {
        const int m = i >> 2, f = i & 3;
        const float4 v = al16 ? reinterpret_cast<const float4 *>(Z)[i]
                              : make_float4(Z[2 * i].x, Z[2 * i].y, Z[2 * i + 1].x, Z[2 * i + 1].y);
        reinterpret_cast<float4 *>(f1bar + ((static_cast<size_t>(b) * (T + 1) + m) * J2 + j2) * 8)[f] = v;
    }
}

// ---------------------------------------------------------------------------
// K1a^T (FP64): Z-bar_f[e] = sum_j Pbar_e(mu_j) F1-bar[b][m(e)][f][parity(e)][j],
// one thread per extended row; F1-bar comes from the FP64 ring transpose with
// the latitude index fastest (the forward projection's access pattern: two
// latitudes per table load, contiguous rows of F1-bar per order and parity).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(64) k1t_project(const V2<R> *__restrict__ f1bar, Dims d,
                                                  const R *__restrict__ pbar, const int *__restrict__ row_m,
                                                  V2<R> *__restrict__ zbar) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (e >= d.next) return;
    const int T = d.T, J2 = d.J2;
    const int m = row_m[e];
    const int par = (e - ext_offset(T, m)) & 1;
    const V2<R> *W = f1bar + ((static_cast<size_t>(b) * (T + 1) + m) * 8 + par) * J2;
    const R *prow = pbar + static_cast<size_t>(e) * d.J2p;
    V2<R> acc[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) acc[f] = mk<R>(0, 0);
    const int J2e = J2 & ~1;
    for (int j = 0; j < J2e; j += 2) {
        const V2<R> pp = *reinterpret_cast<const V2<R> *>(prow + j);
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const V2<R> w0 = W[f * 2 * J2 + j], w1 = W[f * 2 * J2 + j + 1];
            acc[f].x = fma(pp.x, w0.x, acc[f].x);
            acc[f].y = fma(pp.x, w0.y, acc[f].y);
            acc[f].x = fma(pp.y, w1.x, acc[f].x);
            acc[f].y = fma(pp.y, w1.y, acc[f].y);
        }
    }
    if (J2e < J2) {
        const R p = prow[J2e];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const V2<R> w0 = W[f * 2 * J2 + J2e];
            acc[f].x = fma(p, w0.x, acc[f].x);
            acc[f].y = fma(p, w0.y, acc[f].y);
        }
    }
    V2<R> *o = zbar + (static_cast<size_t>(b) * d.next + e) * 4;
#pragma unroll
    for (int f = 0; f < 4; ++f) o[f] = acc[f];
}

// ---------------------------------------------------------------------------
// K1b^T: per mode (m, n), accumulated into u-bar (the transpose of the
// synthesis prep U_n' = i c0 div_n' - c1 zeta_{n'-1} - c2 zeta_{n'+1},
// V_n' = i c0 zeta_n' + c1 div_{n'-1} + c2 div_{n'+1}):
//   zeta-bar_n += Z_zeta[n] - i c0[n] Z_V[n] - c1[n+1] Z_U[n+1] - c2[n-1] Z_U[n-1]
//   div-bar_n  += -i c0[n] Z_U[n] + c1[n+1] Z_V[n+1] + c2[n-1] Z_V[n-1]
//   Phi-bar_n  += Z_Phi[n]
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k1t_epilogue(const V2<R> *__restrict__ zbar, Dims d, const double *__restrict__ syn,
                             const int *__restrict__ coef_m, double2 *__restrict__ ubar, long long ustride) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (i >= d.ncoef) return;
    const int T = d.T;
    const int m = coef_m[i];
    const int t = i - order_offset(T, m);
    const int e = ext_offset(T, m) + t;
    const V2<R> *Z = zbar + static_cast<size_t>(b) * d.next * 4;
    auto ld = [&](int row, int f) -> double2 {       // widened on the integer pipe (convert.cuh)
        const V2<R> v = Z[static_cast<size_t>(row) * 4 + f];
        if constexpr (sizeof(R) == sizeof(float)) return make_double2(f32_to_f64(v.x), f32_to_f64(v.y));
        else return make_double2(v.x, v.y);
    };
    const double2 z0 = make_double2(0.0, 0.0);
    const double2 zz = ld(e, G_ZETA), zp = ld(e, G_PHI), zu = ld(e, G_U), zv = ld(e, G_V);
    const double2 zu_up = ld(e + 1, G_U), zv_up = ld(e + 1, G_V);
    const double2 zu_dn = t > 0 ? ld(e - 1, G_U) : z0;
    const double2 zv_dn = t > 0 ? ld(e - 1, G_V) : z0;
    const double c0 = syn[3 * e];
    const double c1u = syn[3 * (e + 1) + 1];
    const double c2d = t > 0 ? syn[3 * (e - 1) + 2] : 0.0;
    // -i c0 z = (c0 z.y, -c0 z.x)
    double2 *u = ubar + b * ustride;
    double2 a = u[F_ZETA * d.ncoef + i];
    a.x += zz.x + c0 * zv.y - c1u * zu_up.x - c2d * zu_dn.x;
    a.y += zz.y - c0 * zv.x - c1u * zu_up.y - c2d * zu_dn.y;
    u[F_ZETA * d.ncoef + i] = a;
    double2 dv = u[F_DIV * d.ncoef + i];
    dv.x += c0 * zu.y + c1u * zv_up.x + c2d * zv_dn.x;
    dv.y += -c0 * zu.x + c1u * zv_up.y + c2d * zv_dn.y;
    u[F_DIV * d.ncoef + i] = dv;
    double2 ph = u[F_PHI * d.ncoef + i];
    ph.x += zp.x;
    ph.y += zp.y;
    u[F_PHI * d.ncoef + i] = ph;
}

// ---------------------------------------------------------------------------
// K4^T: transpose of one sweep kernel.  For each updated node m:
//   s_m = (I - alpha_m L_g)^{-T} u-bar_m^{k+1}
// then u-bar_n += sum_m s_m, E-bar_j^k = dt sum_m q_{m,j} s_m and
// u-bar_j^k = L_g^T (E-bar_j^k - alpha_j s_j [j updated]), with
// L_g^T x = (lambda x_div, 0, -Phibar x_Phi) in (Phi', zeta, div).
// With `fold` (the first sweep, where every u_j^0 is u_n and every E_j^0 is
// T_E(u_n)) the node adjoints are summed into u-bar_n and E-bar_0.
// ---------------------------------------------------------------------------
constexpr int kAdjSweepThreads = 64;   // 514 blocks at T255: every SM gets work

template <int M>
__global__ void __launch_bounds__(kAdjSweepThreads) k4t_sweep(SweepAdjParams p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int nc = p.ncoef;
    if (i >= nc) return;
    const double lam = p.lam[i];
    double2 sp[M], sz[M], sd[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        sp[m] = sz[m] = sd[m] = make_double2(0.0, 0.0);
        if (m < p.m0 || m >= p.m1) continue;
        const double2 *ub = p.ubin + m * p.ustride;
        const double2 bp = ub[F_PHI * nc + i], bz = ub[F_ZETA * nc + i], bd = ub[F_DIV * nc + i];
        const double al = p.alpha[m];
        // (I - al L^T) s = b:  s_Phi - al lam s_div = b_Phi,  s_div + al Phibar s_Phi = b_div
        const double den = 1.0 / (1.0 + al * al * p.phibar * lam);
        sd[m] = make_double2((bd.x - al * p.phibar * bp.x) * den, (bd.y - al * p.phibar * bp.y) * den);
        sp[m] = make_double2(bp.x + al * lam * sd[m].x, bp.y + al * lam * sd[m].y);
        sz[m] = bz;
    }
    double2 np = make_double2(0.0, 0.0), nz = np, nd = np;     // u-bar_n increment
    double2 ep0 = np, ez0 = np, ed0 = np;                      // folded E-bar_0
#pragma unroll
    for (int m = 0; m < M; ++m) {
        np.x += sp[m].x; np.y += sp[m].y;
        nz.x += sz[m].x; nz.y += sz[m].y;
        nd.x += sd[m].x; nd.y += sd[m].y;
    }
#pragma unroll
    for (int j = 0; j < M; ++j) {
        double2 Sp = make_double2(0.0, 0.0), Sz = Sp, Sd = Sp;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const double q = p.Q[m][j];                  // dt q_{m,j}
            Sp.x = fma(q, sp[m].x, Sp.x); Sp.y = fma(q, sp[m].y, Sp.y);
            Sz.x = fma(q, sz[m].x, Sz.x); Sz.y = fma(q, sz[m].y, Sz.y);
            Sd.x = fma(q, sd[m].x, Sd.x); Sd.y = fma(q, sd[m].y, Sd.y);
        }
        // x = E-bar_j - alpha_j s_j (updated nodes only); u-bar_j = L^T x
        double2 xp = Sp, xd = Sd;
        if (j >= p.m0 && j < p.m1) {
            xp.x -= p.alpha[j] * sp[j].x; xp.y -= p.alpha[j] * sp[j].y;
            xd.x -= p.alpha[j] * sd[j].x; xd.y -= p.alpha[j] * sd[j].y;
        }
        const double2 up = make_double2(lam * xd.x, lam * xd.y);
        const double2 ud = make_double2(-p.phibar * xp.x, -p.phibar * xp.y);
        if (p.fold) {
            np.x += up.x; np.y += up.y;
            nd.x += ud.x; nd.y += ud.y;
            ep0.x += Sp.x; ep0.y += Sp.y;
            ez0.x += Sz.x; ez0.y += Sz.y;
            ed0.x += Sd.x; ed0.y += Sd.y;
        } else {
            double2 *uo = p.ubout + j * p.ostride;
            double2 *eo = p.ebout + j * p.ostride;
            uo[F_PHI * nc + i] = up;
            uo[F_ZETA * nc + i] = make_double2(0.0, 0.0);
            uo[F_DIV * nc + i] = ud;
            eo[F_PHI * nc + i] = Sp;
            eo[F_ZETA * nc + i] = Sz;
            eo[F_DIV * nc + i] = Sd;
        }
    }
    if (p.fold) {
        p.ebar0[F_PHI * nc + i] = ep0;
        p.ebar0[F_ZETA * nc + i] = ez0;
        p.ebar0[F_DIV * nc + i] = ed0;
    }
    double2 *un = p.ubn;
    if (p.init_un) {
        un[F_PHI * nc + i] = np;
        un[F_ZETA * nc + i] = nz;
        un[F_DIV * nc + i] = nd;
    } else {
        double2 a = un[F_PHI * nc + i], z = un[F_ZETA * nc + i], dd = un[F_DIV * nc + i];
        un[F_PHI * nc + i] = make_double2(a.x + np.x, a.y + np.y);
        un[F_ZETA * nc + i] = make_double2(z.x + nz.x, z.y + nz.y);
        un[F_DIV * nc + i] = make_double2(dd.x + nd.x, dd.y + nd.y);
    }
}

// ---------------------------------------------------------------------------
// Height loss 0.5 sum (H + Phi'/g - h_target)^2 on the grid and its seed
// dL/dPhi' (the transpose of the scalar spectral-to-grid transform applied to
// (h - h_target)/g).
// ---------------------------------------------------------------------------
__global__ void k_loss_residual(const double *__restrict__ phigrid, const double *__restrict__ htarget, int n,
                                double inv_g, double H, double *__restrict__ rg, double *__restrict__ part) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double r = H + phigrid[i] * inv_g - htarget[i];
        rg[i] = r * inv_g;
        acc += r * r;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_loss_finish(const double *__restrict__ part, int nblocks, double *__restrict__ loss) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += part[b];
        *loss = 0.5 * s;
    }
}

// grid (real) -> Fourier adjoint per ring pair: F-bar_m = w_m sum_k f_k e^{-i m lambda_k},
// split into parities: out[j2][par][m].
__global__ void k_scalar_ring_adjoint(const double *__restrict__ grid, double2 *__restrict__ out, Dims d,
                                      FftPlan plan, const double2 *__restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *X = reinterpret_cast<double2 *>(smem_raw);
    double2 *S = X + plan.L;
    const int j2 = blockIdx.x, T = d.T, L = plan.L;
    for (int k = threadIdx.x; k < L; k += blockDim.x)
        X[k] = make_double2(grid[static_cast<size_t>(j2) * L + k], grid[static_cast<size_t>(d.J - 1 - j2) * L + k]);
    __syncthreads();
    fft_inplace<double>(X, S, 1, 1, plan, tw, false);
    for (int m = threadIdx.x; m <= T; m += blockDim.x) {
        const double2 y = X[m];
        double2 yc = X[m == 0 ? 0 : L - m];
        yc.y = -yc.y;
        const double wm = (m == 0) ? 0.5 : 1.0;
        const double2 fn = make_double2(wm * (y.x + yc.x), wm * (y.y + yc.y));
        const double2 fs = make_double2(wm * (y.y - yc.y), -wm * (y.x - yc.x));
        double2 se = make_double2(fn.x + fs.x, fn.y + fs.y), so = make_double2(fn.x - fs.x, fn.y - fs.y);
        if (m == 0) { se.y = 0.0; so.y = 0.0; }
        out[(static_cast<size_t>(j2) * 2 + 0) * (T + 1) + m] = se;
        out[(static_cast<size_t>(j2) * 2 + 1) * (T + 1) + m] = so;
    }
}

// Fourier adjoint [j2][par][m] -> spectral adjoint of one field: sum_j Pbar_n(mu_j) X[j][par(n)][m].
__global__ void k_scalar_synth_adjoint(const double2 *__restrict__ in, Dims d, const double *__restrict__ pbar,
                                       double2 *__restrict__ spec) {
    const int m = blockIdx.x, T = d.T;
    const int off = order_offset(T, m), eoff = ext_offset(T, m);
    for (int t = threadIdx.x; t <= T - m; t += blockDim.x) {
        const double *prow = pbar + static_cast<size_t>(eoff + t) * d.J2p;
        double2 acc = make_double2(0.0, 0.0);
        for (int j = 0; j < d.J2; ++j) {
            const double2 x = in[(static_cast<size_t>(j) * 2 + (t & 1)) * (T + 1) + m];
            acc.x = fma(prow[j], x.x, acc.x);
            acc.y = fma(prow[j], x.y, acc.y);
        }
        spec[off + t] = acc;
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <typename R>
static cudaError_t configure_adj(const Dims &d, const FftPlan &plan) {
    cudaError_t e = cudaSuccess;
    if constexpr (sizeof(R) == sizeof(float)) {
        const int smr = (int)ring_f32_smem_bytes(plan.L, plan.L);
        for (const void *f : {(const void *)k2t_ring_f32<0>, (const void *)k2t_ring_f32<96>,
                              (const void *)k2t_ring_f32<192>, (const void *)k2t_ring_f32<384>,
                              (const void *)k2t_ring_f32<768>, (const void *)k2t_ring_f32<1536>}) {
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smr);
            if (e != cudaSuccess) return e;
        }
    } else {
        const size_t sm2 = ring_smem_bytes(plan.L, sizeof(V2<R>), nullptr);
        if (sm2 == 0) return cudaErrorInvalidValue;
        e = cudaFuncSetAttribute(k2t_ring<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
        if (e != cudaSuccess) return e;
    }
    return cudaFuncSetAttribute(k3t_synth<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(static_cast<size_t>(d.T + 4) * 5 * sizeof(V2<R>)));
}

cudaError_t configure_adjoint_kernels(const Dims &d, const FftPlan &plan, bool fp32) {
    cudaError_t e = fp32 ? configure_adj<float>(d, plan) : configure_adj<double>(d, plan);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_scalar_ring_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(2 * static_cast<size_t>(plan.L) * sizeof(double2)));
}

template <typename R>
static cudaError_t launch_tendency_adjoint_t(const Dims &d, const FftPlan &plan, int B, const void *grid_base,
                                             const double2 *abar, long long astride, double2 *ubar,
                                             long long ustride, const DeviceTables &tb, const Workspace &ws,
                                             cudaStream_t s, int *launches) {
    const R *pbar = static_cast<const R *>(tb.pbar);
    const V2<R> *tw = static_cast<const V2<R> *>(tb.tw);
    V2<R> *f1 = static_cast<V2<R> *>(ws.f1);
    V2<R> *f2 = static_cast<V2<R> *>(ws.f2);
    V2<R> *f3 = static_cast<V2<R> *>(ws.f3);
    const int rows_blocks = (d.next + kAdjThreads - 1) / kAdjThreads;
    k3t_epilogue<R><<<dim3(rows_blocks, B), kAdjThreads, 0, s>>>(abar, astride, d, tb.eps, tb.row_m, f3);
    if constexpr (sizeof(R) == sizeof(float)) {
        const cudaError_t e = launch_projection_transpose_f32(d, B, f3, pbar, f2, tb.err, s);
        if (e != cudaSuccess) return e;
    } else {
        k3t_synth<R><<<dim3((d.T + 2) / 2, B, (d.J2 + 63) / 64), 64,
                       static_cast<size_t>(d.T + 4) * 5 * sizeof(V2<R>), s>>>(f3, d, pbar, f2);
    }
    if constexpr (sizeof(R) == sizeof(float)) {
        const dim3 g2(d.J2, B);
        const size_t sm = ring_f32_smem_bytes(d.L, tb.ntwp);
        const float2 *gr = static_cast<const float2 *>(grid_base);
#define SDC_RING_T_F32(LC) \
    k2t_ring_f32<LC><<<g2, 256, sm, s>>>(f2, gr, f1, d, tb.plan16, tb.twp32, tb.ntwp, tb.ring32)
        switch (d.L) {
            case 96: SDC_RING_T_F32(96); break;
            case 192: SDC_RING_T_F32(192); break;
            case 384: SDC_RING_T_F32(384); break;
            case 768: SDC_RING_T_F32(768); break;
            case 1536: SDC_RING_T_F32(1536); break;
            default: SDC_RING_T_F32(0); break;
        }
#undef SDC_RING_T_F32
    } else {
        int nscratch = 0;
        const size_t sm2 = ring_smem_bytes(plan.L, sizeof(V2<R>), &nscratch);
        if (sm2 == 0) return cudaErrorInvalidValue;
        k2t_ring<R><<<dim3(d.J2, B), 256, sm2, s>>>(f2, static_cast<const V2<R> *>(grid_base), f1, d, plan, tw,
                                                   tb.mu, tb.w, nscratch);
    }
    if constexpr (sizeof(R) == sizeof(float)) {
        const cudaError_t e = launch_synthesis_transpose_f32(d, B, f1, pbar, f3, s);
        if (e != cudaSuccess) return e;
    } else {
        k1t_project<R><<<dim3(rows_blocks, B), kAdjThreads, 0, s>>>(f1, d, pbar, tb.row_m, f3);
    }
    k1t_epilogue<R><<<dim3((d.ncoef + 127) / 128, B), 128, 0, s>>>(f3, d, tb.syn, tb.coef_m, ubar, ustride);
    if (launches) *launches += 5;
    return cudaGetLastError();
}

cudaError_t launch_tendency_adjoint(const Dims &d, const FftPlan &plan, bool fp32, int B, const void *grid_base,
                                    const double2 *abar, long long astride, double2 *ubar, long long ustride,
                                    const DeviceTables &tb, const Workspace &ws, cudaStream_t s, int *launches) {
    if (fp32)
        return launch_tendency_adjoint_t<float>(d, plan, B, grid_base, abar, astride, ubar, ustride, tb, ws, s,
                                                launches);
    return launch_tendency_adjoint_t<double>(d, plan, B, grid_base, abar, astride, ubar, ustride, tb, ws, s,
                                             launches);
}

cudaError_t launch_sweep_adjoint(const SweepAdjParams &p, int M, cudaStream_t s, int *launches) {
    const int nb = (p.ncoef + kAdjSweepThreads - 1) / kAdjSweepThreads;
    constexpr int t = kAdjSweepThreads;
    switch (M) {
        case 1: k4t_sweep<1><<<nb, t, 0, s>>>(p); break;
        case 2: k4t_sweep<2><<<nb, t, 0, s>>>(p); break;
        case 3: k4t_sweep<3><<<nb, t, 0, s>>>(p); break;
        case 4: k4t_sweep<4><<<nb, t, 0, s>>>(p); break;
        case 5: k4t_sweep<5><<<nb, t, 0, s>>>(p); break;
        case 6: k4t_sweep<6><<<nb, t, 0, s>>>(p); break;
        case 7: k4t_sweep<7><<<nb, t, 0, s>>>(p); break;
        case 8: k4t_sweep<8><<<nb, t, 0, s>>>(p); break;
        default: return cudaErrorInvalidValue;
    }
    if (launches) *launches += 1;
    return cudaGetLastError();
}

int loss_blocks() { return 128; }

cudaError_t launch_height_loss(const Dims &d, const FftPlan &plan, const double *phigrid, const double *htarget,
                               double inv_g, double H, double *rgrid, double *part, double *loss,
                               double2 *seed_phi, const double *pbar64, const double2 *tw64, double2 *fbuf,
                               cudaStream_t s) {
    const int n = d.J * plan.L;
    k_loss_residual<<<loss_blocks(), 256, 0, s>>>(phigrid, htarget, n, inv_g, H, rgrid, part);
    k_loss_finish<<<1, 32, 0, s>>>(part, loss_blocks(), loss);
    if (seed_phi) {
        k_scalar_ring_adjoint<<<d.J2, 256, 2 * static_cast<size_t>(plan.L) * sizeof(double2), s>>>(rgrid, fbuf, d,
                                                                                                plan, tw64);
        k_scalar_synth_adjoint<<<d.T + 1, 128, 0, s>>>(fbuf, d, pbar64, seed_phi);
    }
    return cudaGetLastError();
}

}  // namespace sdc
