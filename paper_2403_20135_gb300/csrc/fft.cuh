// Complex helpers and the shared-memory mixed-radix Stockham FFT used by the
// ring kernels (device code only).
#pragma once

#include <cuda_runtime.h>

#include <cstring>

#include "sdc_internal.h"

namespace sdc {

template <typename R> struct V2t;
template <> struct V2t<double> { using type = double2; };
template <> struct V2t<float> { using type = float2; };
template <typename R> using V2 = typename V2t<R>::type;

template <typename R> __device__ __forceinline__ V2<R> mk(R x, R y) { V2<R> v; v.x = x; v.y = y; return v; }
template <typename R> __device__ __forceinline__ V2<R> cadd(V2<R> a, V2<R> b) { return mk<R>(a.x + b.x, a.y + b.y); }
template <typename R> __device__ __forceinline__ V2<R> csub(V2<R> a, V2<R> b) { return mk<R>(a.x - b.x, a.y - b.y); }
template <typename R> __device__ __forceinline__ V2<R> cmul(V2<R> a, V2<R> b) {
    return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename R> __device__ __forceinline__ V2<R> cscale(V2<R> a, R s) { return mk<R>(a.x * s, a.y * s); }
// Packed FP32 pair FMA (two IEEE round-to-nearest FMAs in one instruction):
// (a.x * b.x + c.x, a.y * b.y + c.y).
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    unsigned long long ra, rb, rc, rd;
    memcpy(&ra, &a, 8);
    memcpy(&rb, &b, 8);
    memcpy(&rc, &c, 8);
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rd) : "l"(ra), "l"(rb), "l"(rc));
    float2 d;
    memcpy(&d, &rd, 8);
    return d;
}
// c + s * z for a real s and a complex z, as one packed FMA
__device__ __forceinline__ float2 caxpy(float s, float2 z, float2 c) { return ffma2(make_float2(s, s), z, c); }

// multiply by +i or -i
template <typename R> __device__ __forceinline__ V2<R> mul_i(V2<R> a) { return mk<R>(-a.y, a.x); }
template <typename R> __device__ __forceinline__ V2<R> mul_mi(V2<R> a) { return mk<R>(a.y, -a.x); }

// ---------------------------------------------------------------------------
// Mixed radix (8, 4, 2, 3) Stockham FFT of nb length-L sequences in shared
// memory, all threads of the block cooperating.  Forward: e^{-i...};
// inverse: e^{+i...}, unscaled.  Returns the buffer that holds the result.
// ---------------------------------------------------------------------------
template <typename R, int RADIX>
__device__ __forceinline__ void butterfly(V2<R> *v, bool inv) {
    if constexpr (RADIX == 4) {
        const V2<R> a0 = cadd<R>(v[0], v[2]), a1 = csub<R>(v[0], v[2]);
        const V2<R> b0 = cadd<R>(v[1], v[3]), b1 = csub<R>(v[1], v[3]);
        v[0] = cadd<R>(a0, b0);
        v[2] = csub<R>(a0, b0);
        const V2<R> ib1 = inv ? mul_i<R>(b1) : mul_mi<R>(b1);
        v[1] = cadd<R>(a1, ib1);
        v[3] = csub<R>(a1, ib1);
    } else if constexpr (RADIX == 2) {
        const V2<R> a = v[0];
        v[0] = cadd<R>(a, v[1]);
        v[1] = csub<R>(a, v[1]);
    } else if constexpr (RADIX == 8) {
        // even and odd samples: two 4-point DFTs, the odd one twiddled by
        // w_8^k1, then 2-point DFTs: out[k1] = a + w c, out[k1 + 4] = a - w c
        V2<R> a[4] = {v[0], v[2], v[4], v[6]}, c[4] = {v[1], v[3], v[5], v[7]};
        butterfly<R, 4>(a, inv);
        butterfly<R, 4>(c, inv);
        const R h = R(0.70710678118654752440);   // cos(pi/4)
        c[1] = inv ? mk<R>(h * (c[1].x - c[1].y), h * (c[1].x + c[1].y))
                   : mk<R>(h * (c[1].x + c[1].y), h * (c[1].y - c[1].x));
        c[2] = inv ? mul_i<R>(c[2]) : mul_mi<R>(c[2]);
        c[3] = inv ? mk<R>(-h * (c[3].x + c[3].y), h * (c[3].x - c[3].y))
                   : mk<R>(h * (c[3].y - c[3].x), -h * (c[3].x + c[3].y));
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = cadd<R>(a[k], c[k]);
            v[k + 4] = csub<R>(a[k], c[k]);
        }
    } else {   // 3
        const R h = R(0.86602540378443864676);   // sqrt(3)/2
        const V2<R> t1 = cadd<R>(v[1], v[2]);
        const V2<R> t2 = csub<R>(v[0], cscale<R>(t1, R(0.5)));
        const V2<R> t3 = cscale<R>(csub<R>(v[1], v[2]), inv ? h : -h);
        const V2<R> it3 = mul_i<R>(t3);
        v[0] = cadd<R>(v[0], t1);
        v[1] = cadd<R>(t2, it3);
        v[2] = csub<R>(t2, it3);
    }
}

// One Stockham stage of radix RADIX over nb sequences (compile-time radix so
// the butterfly operands stay in registers).
template <typename R, int RADIX>
__device__ __forceinline__ void fft_stage(const V2<R> *src, V2<R> *dst, int nb, int L, int Ns,
                                          const V2<R> *__restrict__ tw, bool inv) {
    const int Lr = L / RADIX;
    const int tws = L / (Ns * RADIX);
    const bool pow2 = (Ns & (Ns - 1)) == 0;
    for (int bb = 0; bb < nb; ++bb) {
        const V2<R> *in = src + bb * L;
        V2<R> *out = dst + bb * L;
        for (int j = threadIdx.x; j < Lr; j += blockDim.x) {
            const int k = pow2 ? (j & (Ns - 1)) : (j % Ns);
            V2<R> v[RADIX];
            v[0] = in[j];
            if (Ns == 1) {                       // first stage: every twiddle is 1
#pragma unroll
                for (int r = 1; r < RADIX; ++r) v[r] = in[j + r * Lr];
            } else {
#pragma unroll
                for (int r = 1; r < RADIX; ++r) {
                    V2<R> w = tw[r * k * tws];
                    if (inv) w.y = -w.y;
                    v[r] = cmul<R>(in[j + r * Lr], w);
                }
            }
            butterfly<R, RADIX>(v, inv);
            const int base = (j - k) * RADIX + k;
#pragma unroll
            for (int r = 0; r < RADIX; ++r) out[base + r * Ns] = v[r];
        }
    }
}

template <typename R>
__device__ V2<R> *fft_batch(V2<R> *x, V2<R> *y, int nb, const FftPlan &plan,
                            const V2<R> *__restrict__ tw, bool inv) {
    const int L = plan.L;
    V2<R> *src = x, *dst = y;
    int Ns = 1;
    for (int s = 0; s < plan.nstages; ++s) {
        const int radix = plan.radix[s];
        if (radix == 8) fft_stage<R, 8>(src, dst, nb, L, Ns, tw, inv);
        else if (radix == 4) fft_stage<R, 4>(src, dst, nb, L, Ns, tw, inv);
        else if (radix == 2) fft_stage<R, 2>(src, dst, nb, L, Ns, tw, inv);
        else fft_stage<R, 3>(src, dst, nb, L, Ns, tw, inv);
        __syncthreads();
        V2<R> *t = src; src = dst; dst = t;
        Ns *= radix;
    }
    return src;
}

// FFT of nb arrays starting at data (stride L) using `scratch` arrays of
// scratch space, in batches; results land back in data.
template <typename R>
__device__ void fft_inplace(V2<R> *data, V2<R> *scratch, int nscratch, int nb, const FftPlan &plan,
                            const V2<R> *__restrict__ tw, bool inv) {
    for (int b0 = 0; b0 < nb; b0 += nscratch) {
        const int cnt = min(nscratch, nb - b0);
        V2<R> *x = data + b0 * plan.L;
        V2<R> *res = fft_batch<R>(x, scratch, cnt, plan, tw, inv);
        if (res != x) {
            for (int i = threadIdx.x; i < cnt * plan.L; i += blockDim.x) x[i] = res[i];
            __syncthreads();
        }
    }
}

}  // namespace sdc
