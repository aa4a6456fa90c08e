// Shared-memory Stockham FFT with radices up to 16 held in registers and a
// padded layout (one spare element after every 16) that keeps the strided
// reads and writes of every pass free of bank conflicts.  Used by the FP32
// ring kernel, where the transforms are bound by shared-memory traffic: a
// length-768 transform takes three passes (16, 16, 3) instead of five.
//
// Pass p of radix R over sequences of length L with Ns = R_0 ... R_{p-1}:
//   v_r = in[j + r L/R] * w^(r k L/(Ns R)),  k = j mod Ns,  w = e^{-2 pi i / L}
//   (v_0 .. v_{R-1}) <- R-point DFT,  out[(j - k) R + k + r Ns] = v_r.
// The twiddles of each pass after the first are stored pass by pass as
// [r - 1][k] (r = 1..R-1, k < Ns), so neighbouring threads read neighbouring
// entries.  Inverse transforms conjugate every twiddle; both are unscaled.
#pragma once

#include <cuda_runtime.h>

#include "fft.cuh"

namespace sdc {

__host__ __device__ constexpr int fft_padded_len(int L) { return L + (L - 1) / 16 + 1; }
// shared memory of an FP32 ring kernel: X[5] and S[5] padded, ntw twiddles
__host__ __device__ inline size_t ring_f32_smem_bytes(int L, int ntw) {
    return (10 * static_cast<size_t>(fft_padded_len(L)) + static_cast<size_t>(ntw)) * sizeof(float2);
}
__device__ __forceinline__ int fpad(int i) { return i + (i >> 4); }

// e^{-2 pi i e / 16} for e = 0..15 (cos, -sin)
__device__ __forceinline__ float2 w16(int e, bool inv) {
    constexpr float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f, h = 0.70710678118654752440f;
    const float cs[16] = {1.f, c1, h, s1, 0.f, -s1, -h, -c1, -1.f, -c1, -h, -s1, 0.f, s1, h, c1};
    const float sn[16] = {0.f, s1, h, c1, 1.f, c1, h, s1, 0.f, -s1, -h, -c1, -1.f, -c1, -h, -s1};
    return make_float2(cs[e & 15], inv ? sn[e & 15] : -sn[e & 15]);
}

// In-register DFT of v[0..R-1], output in natural order.
template <int R> __device__ __forceinline__ void dft(float2 *v, bool inv);

template <> __device__ __forceinline__ void dft<2>(float2 *v, bool inv) { butterfly<float, 2>(v, inv); }
template <> __device__ __forceinline__ void dft<3>(float2 *v, bool inv) { butterfly<float, 3>(v, inv); }
template <> __device__ __forceinline__ void dft<4>(float2 *v, bool inv) { butterfly<float, 4>(v, inv); }

// R = 4 R2: n = R2 n1 + n2, k = k1 + 4 k2.  4-point DFTs over n1, twiddle
// w_R^(n2 k1), R2-point DFTs over n2.
template <int R2>
__device__ __forceinline__ void dft4x(float2 *v, bool inv) {
    constexpr int R = 4 * R2;
    float2 y[R2][4];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) {
#pragma unroll
        for (int n1 = 0; n1 < 4; ++n1) y[n2][n1] = v[R2 * n1 + n2];
        dft<4>(y[n2], inv);
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1)
            if (n2 * k1 != 0) y[n2][k1] = cmul<float>(y[n2][k1], w16(n2 * k1 * (16 / R), inv));
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        float2 z[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) z[n2] = y[n2][k1];
        dft<R2>(z, inv);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) v[k1 + 4 * k2] = z[k2];
    }
}
template <> __device__ __forceinline__ void dft<8>(float2 *v, bool inv) { dft4x<2>(v, inv); }
template <> __device__ __forceinline__ void dft<16>(float2 *v, bool inv) { dft4x<4>(v, inv); }

// One pass over nb sequences (stride Lp) from src to dst.
template <int R>
__device__ __forceinline__ void fft_pass(const float2 *src, float2 *dst, int nb, int Lp, int L, int Ns,
                                         const float2 *__restrict__ twp, bool inv) {
    const int Lr = L / R;
    const int total = nb * Lr;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int bb = t / Lr, j = t - bb * Lr;
        const float2 *in = src + bb * Lp;
        float2 *out = dst + bb * Lp;
        const int k = j % Ns;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = in[fpad(j + r * Lr)];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = twp[(r - 1) * Ns + k];
                if (inv) w.y = -w.y;
                v[r] = cmul<float>(v[r], w);
            }
        }
        dft<R>(v, inv);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) out[fpad(base + r * Ns)] = v[r];
    }
}

// Transform nb padded sequences in a (scratch b, same size); returns the
// buffer holding the result (a after an even number of passes, else b).
__device__ inline float2 *fft_passes(float2 *a, float2 *b, int nb, int Lp, const FftPlan &plan,
                                     const float2 *__restrict__ twp, bool inv) {
    float2 *src = a, *dst = b;
    int Ns = 1, toff = 0;
    for (int p = 0; p < plan.nstages; ++p) {
        const int R = plan.radix[p];
        const float2 *tw = twp + toff;
        switch (R) {
            case 16: fft_pass<16>(src, dst, nb, Lp, plan.L, Ns, tw, inv); break;
            case 8: fft_pass<8>(src, dst, nb, Lp, plan.L, Ns, tw, inv); break;
            case 4: fft_pass<4>(src, dst, nb, Lp, plan.L, Ns, tw, inv); break;
            case 2: fft_pass<2>(src, dst, nb, Lp, plan.L, Ns, tw, inv); break;
            default: fft_pass<3>(src, dst, nb, Lp, plan.L, Ns, tw, inv); break;
        }
        __syncthreads();
        if (Ns > 1) toff += (R - 1) * Ns;
        Ns *= R;
        float2 *t = src; src = dst; dst = t;
    }
    return src;
}

// ---------------------------------------------------------------------------
// The same passes with the length, the pass radices and the batch fixed at
// compile time (index arithmetic by shifts and multiplies) for the common
// ring lengths.  plan16_radix reproduces the host factorisation: radix 16
// while possible, then one of 8/4/2, then 3s.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int plan16_radix(int L, int p) {
    int rest = L, q = 0;
    while (rest % 16 == 0) {
        if (q == p) return 16;
        ++q;
        rest /= 16;
    }
    const int rs[3] = {8, 4, 2};
    for (int i = 0; i < 3; ++i)
        if (rest % rs[i] == 0) {
            if (q == p) return rs[i];
            ++q;
            rest /= rs[i];
        }
    while (rest % 3 == 0) {
        if (q == p) return 3;
        ++q;
        rest /= 3;
    }
    return 0;
}
__host__ __device__ constexpr int plan16_npasses(int L) {
    int p = 0;
    while (plan16_radix(L, p) != 0) ++p;
    return p;
}

// Padded index of i + r * step: when step is a multiple of 16 the padding of
// the sum is the padding of i plus r * step / 16, so one padded base and
// compile-time offsets serve all R elements of a butterfly.
template <int STEP>
__device__ __forceinline__ int fpad_step(int base_padded, int i, int r) {
    if constexpr (STEP % 16 == 0) return base_padded + r * (STEP + STEP / 16);
    else return fpad(i + r * STEP);
}

template <int R, int L, int Ns, int NB>
__device__ __forceinline__ void fft_pass_ct(const float2 *src, float2 *dst, const float2 *__restrict__ twp,
                                            bool inv) {
    constexpr int Lr = L / R, Lp = fft_padded_len(L), total = NB * Lr;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int bb = t / Lr, j = t - bb * Lr;
        const float2 *in = src + bb * Lp;
        float2 *out = dst + bb * Lp;
        const int k = j % Ns;
        float2 v[R];
        const int jp = fpad(j);
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = in[fpad_step<Lr>(jp, j, r)];
        if constexpr (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = twp[(r - 1) * Ns + k];
                if (inv) w.y = -w.y;
                v[r] = cmul<float>(v[r], w);
            }
        }
        dft<R>(v, inv);
        const int base = (j - k) * R + k;
        const int bp = fpad(base);
        if constexpr (Ns == 1 && R == 16) {              // base = 16 j: the 16 outputs share one padding
#pragma unroll
            for (int r = 0; r < R; ++r) out[bp + r] = v[r];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) out[fpad_step<Ns>(bp, base, r)] = v[r];
        }
    }
}

// Ns and twiddle offset (in the [r - 1][k] pass-by-pass table) of pass p.
__host__ __device__ constexpr int plan16_ns(int L, int p) {
    int ns = 1;
    for (int q = 0; q < p; ++q) ns *= plan16_radix(L, q);
    return ns;
}
__host__ __device__ constexpr int plan16_toff(int L, int p) {
    int t = 0, ns = 1;
    for (int q = 0; q < p; ++q) {
        const int r = plan16_radix(L, q);
        if (ns > 1) t += (r - 1) * ns;
        ns *= r;
    }
    return t;
}

// Passes P .. PEND - 1 only (the caller does the rest); returns the buffer
// holding the result.
template <int L, int NB, int PEND, int P = 0, int Ns = 1, int TOFF = 0>
__device__ __forceinline__ float2 *fft_passes_ct_until(float2 *src, float2 *dst, const float2 *__restrict__ twp,
                                                       bool inv) {
    if constexpr (P == PEND) {
        return src;
    } else {
        constexpr int R = plan16_radix(L, P);
        fft_pass_ct<R, L, Ns, NB>(src, dst, twp + TOFF, inv);
        __syncthreads();
        return fft_passes_ct_until<L, NB, PEND, P + 1, Ns * R, (Ns > 1 ? TOFF + (R - 1) * Ns : TOFF)>(dst, src, twp,
                                                                                                        inv);
    }
}

template <int L, int NB, int P = 0, int Ns = 1, int TOFF = 0>
__device__ __forceinline__ float2 *fft_passes_ct(float2 *src, float2 *dst, const float2 *__restrict__ twp,
                                                 bool inv) {
    if constexpr (P == plan16_npasses(L)) {
        return src;
    } else {
        constexpr int R = plan16_radix(L, P);
        fft_pass_ct<R, L, Ns, NB>(src, dst, twp + TOFF, inv);
        __syncthreads();
        return fft_passes_ct<L, NB, P + 1, Ns * R, (Ns > 1 ? TOFF + (R - 1) * Ns : TOFF)>(dst, src, twp, inv);
    }
}

}  // namespace sdc
