// Explicit tendency T_E = L_c + N_a + N_r (Eq. (4)) through the spherical
// harmonic transform, for a batch of B node states (the paper's parallel
// node loop of Algorithm 2 becomes the batch dimension of each launch).
//
//   K1 synthesis  (per order m):   spectral -> Fourier coefficients on the
//                                  northern latitudes, split by the parity of
//                                  n - m (even/odd symmetry about the equator)
//   K2 ring       (per ring pair): inverse FFT -> grid products -> forward FFT
//   K3 analysis   (per order m):   Fourier -> spectral projections; the vector
//                                  (div/curl) epilogue per mode runs in
//                                  k3_epilogue for a standalone tendency and
//                                  inside the sweep kernel within a step
//
// The (1 - mu^2) d/dmu terms of the vector transforms are moved onto the
// coefficients with the recurrence
//   H_n^m = (1-mu^2) dPbar_n^m/dmu = -n eps_{n+1} Pbar_{n+1} + (n+1) eps_n Pbar_{n-1},
// so both contractions use the one table Pbar_n^m, n = m..T+1.  This is the
// same discrete operator as the direct H sums, up to rounding.
//
// Templated on the arithmetic type R (double for SDC_FP64, float for the
// FP32 mixed mode); spectral inputs and outputs are always FP64.
#include <cuda_runtime.h>

#include "fft.cuh"
#include "fft_pass.cuh"
#include "async_copy.cuh"
#include "convert.cuh"
#include "epilogue.cuh"
#include "sdc_internal.h"

namespace sdc {

// ---------------------------------------------------------------------------
// K1: synthesis.  grid ((T+2)/2 order pairs, B states, latitude chunks): a
// block serves orders m and T - m (equal work for every block).  Output
// F1[b][j][field][parity][m] in FP64, F1[b][j][m][parity][field] in FP32
// (the four fields of one (j, m, parity) fill one 32-byte sector, so the
// transposing stores of the FP32 kernels are whole sectors), fields
// (zeta, Phi', U, V).  The wind
// coefficients on degrees n' = m..T+1 come from host-computed factors
// (c0, c1, c2) = syn[e]:
//   U_n' = i c0 div_n' - c1 zeta_{n'-1} - c2 zeta_{n'+1}
//   V_n' = i c0 zeta_n' + c1 div_{n'-1} + c2 div_{n'+1}
// with c0 = (m/a) s_n', c1 = -(n'-1) eps_n' s_{n'-1} / a,
// c2 = (n'+2) eps_{n'+1} s_{n'+1} / a and s_n = -a^2 / (n(n+1)) (0 at n = 0).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(64) k1_synthesis(const double2 *__restrict__ states, long long sstride, Dims d,
                                                   const R *__restrict__ pbar, const double *__restrict__ syn,
                                                   V2<R> *__restrict__ f1) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V2<R> *cf = reinterpret_cast<V2<R> *>(smem_raw);   // [rows][4]
    const int T = d.T;
    const int m1 = blockIdx.x, m2 = T - blockIdx.x;
    const int b = blockIdx.y;
    const int nn1 = T + 2 - m1;
    const int nn2 = (m2 > m1) ? T + 2 - m2 : 0;
    const int rows = nn1 + nn2;
    const double2 *st = states + b * sstride;
    const int nc = d.ncoef;

    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
        const int m = (r < nn1) ? m1 : m2;
        const int t = (r < nn1) ? r : r - nn1;
        const int n = m + t;
        const int off = order_offset(T, m);
        const int e = ext_offset(T, m) + t;
        auto ld = [&](int f, int k) -> double2 {
            return (k >= m && k <= T) ? st[f * nc + off + k - m] : make_double2(0.0, 0.0);
        };
        const double2 z0 = ld(F_ZETA, n), zm = ld(F_ZETA, n - 1), zp = ld(F_ZETA, n + 1);
        const double2 d0 = ld(F_DIV, n), dm = ld(F_DIV, n - 1), dp = ld(F_DIV, n + 1);
        const double2 p0 = ld(F_PHI, n);
        const double c0 = syn[3 * e], c1 = syn[3 * e + 1], c2 = syn[3 * e + 2];
        const double ux = -c0 * d0.y - c1 * zm.x - c2 * zp.x;
        const double uy = c0 * d0.x - c1 * zm.y - c2 * zp.y;
        const double vx = -c0 * z0.y + c1 * dm.x + c2 * dp.x;
        const double vy = c0 * z0.x + c1 * dm.y + c2 * dp.y;
        cf[r * 4 + G_ZETA] = mk<R>(R(z0.x), R(z0.y));
        cf[r * 4 + G_PHI] = mk<R>(R(p0.x), R(p0.y));
        cf[r * 4 + G_U] = mk<R>(R(ux), R(uy));
        cf[r * 4 + G_V] = mk<R>(R(vx), R(vy));
    }
    __syncthreads();

    const int j = blockIdx.z * blockDim.x + threadIdx.x;
    if (j >= d.J2) return;
    V2<R> *o = f1 + (static_cast<size_t>(b) * d.J2 + j) * (4 * 2 * (T + 1));
    for (int half = 0; half < 2; ++half) {
        const int m = half ? m2 : m1;
        const int nn = half ? nn2 : nn1;
        if (nn == 0) break;
        const V2<R> *c = cf + (half ? nn1 : 0) * 4;
        V2<R> ae[4], ao[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) { ae[f] = mk<R>(0, 0); ao[f] = mk<R>(0, 0); }
        const R *prow = pbar + static_cast<size_t>(ext_offset(T, m)) * d.J2p + j;
        int t = 0;
        for (; t + 1 < nn; t += 2) {
            const R pe = prow[static_cast<size_t>(t) * d.J2p];
            const R po = prow[static_cast<size_t>(t + 1) * d.J2p];
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const V2<R> ce = c[t * 4 + f], co = c[(t + 1) * 4 + f];
                ae[f].x = fma(pe, ce.x, ae[f].x);
                ae[f].y = fma(pe, ce.y, ae[f].y);
                ao[f].x = fma(po, co.x, ao[f].x);
                ao[f].y = fma(po, co.y, ao[f].y);
            }
        }
        if (t < nn) {
            const R pe = prow[static_cast<size_t>(t) * d.J2p];
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const V2<R> ce = c[t * 4 + f];
                ae[f].x = fma(pe, ce.x, ae[f].x);
                ae[f].y = fma(pe, ce.y, ae[f].y);
            }
        }
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            o[(f * 2 + 0) * (T + 1) + m] = ae[f];
            o[(f * 2 + 1) * (T + 1) + m] = ao[f];
        }
    }
}

// Shared memory of one ring block: 5 field arrays, s scratch arrays and the
// twiddle table, L complex values each.  Prefer the largest s that still lets two blocks share an
// SM; fall back to one block per SM for long rings.
size_t ring_smem_bytes(int L, int elem_bytes, int *scratch_arrays) {
    const size_t per_sm = 227 * 1024;
    for (size_t cap : {per_sm / 2 - 1024, per_sm}) {
        for (int s = 5; s >= 1; --s) {
            const size_t bytes = static_cast<size_t>(5 + s + 1) * L * elem_bytes;   // + twiddles
            if (bytes <= cap) {
                if (scratch_arrays) *scratch_arrays = s;
                return bytes;
            }
        }
    }
    if (scratch_arrays) *scratch_arrays = 0;
    return 0;
}

// ---------------------------------------------------------------------------
// K2: one block per (latitude pair j2, state b).  The north ring (mu_j > 0)
// and its mirror (mu = -mu_j) travel together as the real and imaginary
// parts of one complex sequence.
// FP64 (the FP32 layouts are at k2_ring_f32 and ring_f32_output):
// input  F1[b][j2][4][2][T+1]; output F2[b][m][5][2][J2] =
//   w~_j (G_north + G_south) (parity 0), w~_j (G_north - G_south) (parity 1)
// for G in (A, B, C, D) = (eta U, eta V, Phi' U, Phi' V), weight w~ = w/(1-mu^2);
// G = E = (U^2 + V^2) / (2 (1 - mu^2)) uses the plain Gauss weight w.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k2_ring(const V2<R> *__restrict__ f1, V2<R> *__restrict__ f2, Dims d, FftPlan plan,
                        const V2<R> *__restrict__ tw, const R *__restrict__ rw, int nscratch,
                        V2<R> *__restrict__ gstore) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V2<R> *X = reinterpret_cast<V2<R> *>(smem_raw);   // [5][L]
    V2<R> *S = X + 5 * plan.L;                          // [nscratch][L]
    V2<R> *TW = S + nscratch * plan.L;                  // twiddles [L]
    const int j2 = blockIdx.x;
    const int b = blockIdx.y;
    const int T = d.T, L = plan.L;
    const V2<R> *in = f1 + (static_cast<size_t>(b) * d.J2 + j2) * (4 * 2 * (T + 1));
    // the twiddles and, where the scratch arrays hold it, the block's F1 slice
    // arrive by cp.async (16-byte pieces: V2<double> elements), all in flight at once
    const bool staged = sizeof(V2<R>) == 16 && static_cast<size_t>(nscratch) * L >= 8u * (T + 1);
    if constexpr (sizeof(V2<R>) == 16) {
        for (int k = threadIdx.x; k < L; k += blockDim.x) cp_async16(TW + k, tw + k);
        if (staged)
            for (int q = threadIdx.x; q < 8 * (T + 1); q += blockDim.x) cp_async16(S + q, in + q);
        cp_async_commit();
    } else {
        for (int k = threadIdx.x; k < L; k += blockDim.x) TW[k] = tw[k];
    }
    // Hermitian packing of north (real part) and south (imaginary part):
    // the band m <= T and its mirror L - m from one load, zeros in between.
    for (int i = threadIdx.x; i < 4 * (L - 2 * T - 1); i += blockDim.x) {
        const int f = i / (L - 2 * T - 1), k = T + 1 + (i - f * (L - 2 * T - 1));
        X[f * L + k] = mk<R>(0, 0);
    }
    if constexpr (sizeof(V2<R>) == 16) {
        cp_async_wait<0>();
        __syncthreads();
    }
    const V2<R> *src = staged ? S : in;
    for (int i = threadIdx.x; i < 4 * (T + 1); i += blockDim.x) {
        const int f = i / (T + 1), m = i - f * (T + 1);
        V2<R> e = src[(f * 2 + 0) * (T + 1) + m];
        V2<R> o = src[(f * 2 + 1) * (T + 1) + m];
        if (m == 0) { e.y = 0; o.y = 0; }
        const V2<R> n = cadd<R>(e, o), s = csub<R>(e, o);
        X[f * L + m] = mk<R>(n.x - s.y, n.y + s.x);            // n + i s
        if (m > 0) X[f * L + L - m] = mk<R>(n.x + s.y, -n.y + s.x);   // conj(n) + i conj(s)
    }
    __syncthreads();
    fft_inplace<R>(X, S, nscratch, 4, plan, TW, true);

    const R fN = rw[4 * j2], inv2c = rw[4 * j2 + 1];
    // optional record of the grid fields (north ring .x, south ring .y) for
    // the adjoint: gstore[b][j2][field][L]
    V2<R> *gs = gstore ? gstore + (static_cast<size_t>(b) * d.J2 + j2) * 4 * L : nullptr;
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        const V2<R> zz = X[G_ZETA * L + k], pp = X[G_PHI * L + k];
        const V2<R> uu = X[G_U * L + k], vv = X[G_V * L + k];
        if (gs) {
            gs[G_ZETA * L + k] = zz;
            gs[G_PHI * L + k] = pp;
            gs[G_U * L + k] = uu;
            gs[G_V * L + k] = vv;
        }
        // .x = north ring, .y = south ring (where f = -fN)
        const R etaN = zz.x + fN, etaS = zz.y - fN;
        X[P_A * L + k] = mk<R>(etaN * uu.x, etaS * uu.y);
        X[P_B * L + k] = mk<R>(etaN * vv.x, etaS * vv.y);
        X[P_C * L + k] = mk<R>(pp.x * uu.x, pp.y * uu.y);
        X[P_D * L + k] = mk<R>(pp.x * vv.x, pp.y * vv.y);
        X[P_E * L + k] = mk<R>((uu.x * uu.x + vv.x * vv.x) * inv2c, (uu.y * uu.y + vv.y * vv.y) * inv2c);
    }
    __syncthreads();
    fft_inplace<R>(X, S, nscratch, 5, plan, TW, false);

    const R wt = rw[4 * j2 + 2], wp = rw[4 * j2 + 3];
    const R invL = R(1.0) / R(L);
    for (int i = threadIdx.x; i < 5 * (T + 1); i += blockDim.x) {
        const int g = i / (T + 1), m = i - g * (T + 1);
        const V2<R> y = X[g * L + m];
        V2<R> yc = X[g * L + (m == 0 ? 0 : L - m)];
        yc.y = -yc.y;
        // north = (y + conj y_{L-m}) / 2, south = -i (y - conj y_{L-m}) / 2
        const V2<R> gn = cscale<R>(cadd<R>(y, yc), R(0.5) * invL);
        const V2<R> gs = cscale<R>(mul_mi<R>(csub<R>(y, yc)), R(0.5) * invL);
        const R wg = (g == P_E) ? wp : wt;
        V2<R> *o = f2 + ((static_cast<size_t>(b) * (T + 1) + m) * 5 + g) * 2 * d.J2 + j2;
        o[0] = cscale<R>(cadd<R>(gn, gs), wg);
        o[d.J2] = cscale<R>(csub<R>(gn, gs), wg);
    }
}

// ---------------------------------------------------------------------------
// K2 (FP32): the ring kernel of k2_ring with the padded radix-16 passes of
// fft_pass.cuh (shared-memory bound in FP32: fewer passes, no bank
// conflicts, no copy-back).  Input F1[b][j2][m][parity][field] (the block's
// slice is contiguous).  X[5] and S[5] are both resident; for the lengths
// fixed at compile time whose last pass is radix 3 that pass runs fused with
// the grid products, which land in the array the pass did not read; for the
// other lengths the grid fields land in X or S by the parity of the pass
// count and the products are written to X; the forward result again lands by
// parity and the other array stages the output.
// ---------------------------------------------------------------------------

// Unpack of the forward transforms of the north (real part) and south
// (imaginary part) rings, weighting and store of F2[b][m][j2][g][parity]
// (FP32 layout: the ten values of one (m, j2) are 80 contiguous bytes).  The
// values are staged as [m][g][parity] in the free scratch array Z, then
// written out by consecutive lanes, so that a warp's store covers whole
// sectors instead of one 8-byte piece per sector.
__device__ __forceinline__ void ring_f32_output(const float2 *Y, float2 *Z, float2 *__restrict__ f2, const Dims &d,
                                                int b, int j2, int Lp, int L, const float *__restrict__ rw) {
    const int T = d.T;
    const float wt = rw[4 * j2 + 2], wp = rw[4 * j2 + 3];
    const float half_invL = 0.5f / float(L);
    float4 *z4 = reinterpret_cast<float4 *>(Z);
    const bool al16 = (reinterpret_cast<uintptr_t>(Z) & 15) == 0;   // odd padded lengths: Z on an 8-byte boundary
    for (int i = threadIdx.x; i < 5 * (T + 1); i += blockDim.x) {
        const int g = i / (T + 1), m = i - g * (T + 1);
        const float2 y = Y[g * Lp + fpad(m)];
        float2 yc = Y[g * Lp + fpad(m == 0 ? 0 : L - m)];
        yc.y = -yc.y;
        const float2 gn = cscale<float>(cadd<float>(y, yc), half_invL);
        const float2 gsx = cscale<float>(mul_mi<float>(csub<float>(y, yc)), half_invL);
        const float wg = (g == P_E) ? wp : wt;
        const float2 ev = cscale<float>(cadd<float>(gn, gsx), wg), od = cscale<float>(csub<float>(gn, gsx), wg);
        if (al16) {
            z4[m * 5 + g] = make_float4(ev.x, ev.y, od.x, od.y);
        } else {
            Z[(m * 5 + g) * 2] = ev;
            Z[(m * 5 + g) * 2 + 1] = od;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 5 * (T + 1); i += blockDim.x) {
        const int m = i / 5, g = i - m * 5;
        const float4 v = al16 ? z4[i] : make_float4(Z[2 * i].x, Z[2 * i].y, Z[2 * i + 1].x, Z[2 * i + 1].y);
        reinterpret_cast<float4 *>(f2 + ((static_cast<size_t>(b) * (T + 1) + m) * d.J2 + j2) * 10)[g] = v;
    }
}

// LC > 0: ring length fixed at compile time (LC == plan.L); 0: any length.
template <int LC>
__global__ void __launch_bounds__(256) k2_ring_f32(const float2 *__restrict__ f1, float2 *__restrict__ f2, Dims d,
                                                   FftPlan plan, const float2 *__restrict__ twp, int ntw,
                                                   const float *__restrict__ rw, float2 *__restrict__ gstore) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = LC > 0 ? LC : plan.L, Lp = fft_padded_len(L);
    float2 *X = reinterpret_cast<float2 *>(smem_raw);   // [5][Lp]
    float2 *S = X + 5 * Lp;                              // [5][Lp]
    float2 *TW = S + 5 * Lp;                             // [ntw]
    const int j2 = blockIdx.x;
    const int b = blockIdx.y;
    const int T = d.T;
    // the block's F1 slice (contiguous, 16-byte aligned) into the scratch arrays
    // S and the pass twiddles into TW, all copies in flight at once
    const float2 *in = f1 + (static_cast<size_t>(b) * d.J2 + j2) * (4 * 2 * (T + 1));
    float2 *raw = S;                                     // 8 (T + 1) <= 5 Lp elements
    // twiddles and the zero band first: they need nothing of the synthesis
    for (int k = threadIdx.x; k < ntw; k += blockDim.x) cp_async8(TW + k, twp + k);
    const int gap = L - 2 * T - 1;
    for (int i = threadIdx.x; i < 4 * gap; i += blockDim.x) {
        const int f = i / gap, k = T + 1 + (i - f * gap);
        X[f * Lp + fpad(k)] = make_float2(0.f, 0.f);
    }
    pdl_wait();
    if ((Lp & 1) == 0) {                                 // S starts on a 16-byte boundary
        for (int q = threadIdx.x; q < 4 * (T + 1); q += blockDim.x) cp_async16(raw + 2 * q, in + 2 * q);
    } else {
        for (int q = threadIdx.x; q < 8 * (T + 1); q += blockDim.x) cp_async8(raw + q, in + q);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * (T + 1); i += blockDim.x) {
        const int m = i >> 2, f = i & 3;                 // raw = F1[b][j2][m][parity][f]
        float2 e = raw[m * 8 + f], o = raw[m * 8 + 4 + f];
        if (m == 0) { e.y = 0.f; o.y = 0.f; }
        const float2 n = cadd<float>(e, o), sv = csub<float>(e, o);
        X[f * Lp + fpad(m)] = make_float2(n.x - sv.y, n.y + sv.x);                // n + i s
        if (m > 0) X[f * Lp + fpad(L - m)] = make_float2(n.x + sv.y, -n.y + sv.x);   // conj(n) + i conj(s)
    }
    __syncthreads();
    const float fN = rw[4 * j2], inv2c = rw[4 * j2 + 1];
    float2 *gs = gstore ? gstore + (static_cast<size_t>(b) * d.J2 + j2) * 4 * L : nullptr;
    constexpr int NPASS = LC > 0 ? plan16_npasses(LC) : 0;
    if constexpr (LC > 0 && plan16_radix(LC, NPASS - 1) == 3) {
        // The last inverse pass (radix 3, Ns = L/3) fused with the grid
        // products: a thread finishes the butterflies of all four fields at
        // the grid points j, j + L/3, j + 2L/3 and writes the five products
        // there, so the four transformed fields never go back to shared memory.
        constexpr int Lr = LC / 3, TL = plan16_toff(LC, NPASS - 1);
        static_assert(plan16_ns(LC, NPASS - 1) == Lr, "the last pass spans the ring in three strides");
        float2 *A = fft_passes_ct_until<LC, 4, NPASS - 1>(X, S, TW, true);
        float2 *P2 = (A == X) ? S : X;
        for (int j = threadIdx.x; j < Lr; j += blockDim.x) {
            float2 w1 = TW[TL + j], w2 = TW[TL + Lr + j];
            w1.y = -w1.y;                                // inverse transform: conjugate twiddles
            w2.y = -w2.y;
            float2 v[4][3];
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                v[f][0] = A[f * Lp + fpad(j)];
                v[f][1] = cmul<float>(A[f * Lp + fpad(j + Lr)], w1);
                v[f][2] = cmul<float>(A[f * Lp + fpad(j + 2 * Lr)], w2);
                dft<3>(v[f], true);
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const int k = j + r * Lr, kp = fpad(k);
                const float2 zz = v[G_ZETA][r], pp = v[G_PHI][r], uu = v[G_U][r], vv = v[G_V][r];
                if (gs) {
                    gs[G_ZETA * L + k] = zz;
                    gs[G_PHI * L + k] = pp;
                    gs[G_U * L + k] = uu;
                    gs[G_V * L + k] = vv;
                }
                const float etaN = zz.x + fN, etaS = zz.y - fN;
                P2[P_A * Lp + kp] = make_float2(etaN * uu.x, etaS * uu.y);
                P2[P_B * Lp + kp] = make_float2(etaN * vv.x, etaS * vv.y);
                P2[P_C * Lp + kp] = make_float2(pp.x * uu.x, pp.y * uu.y);
                P2[P_D * Lp + kp] = make_float2(pp.x * vv.x, pp.y * vv.y);
                P2[P_E * Lp + kp] =
                    make_float2((uu.x * uu.x + vv.x * vv.x) * inv2c, (uu.y * uu.y + vv.y * vv.y) * inv2c);
            }
        }
        __syncthreads();
        const float2 *Y = fft_passes_ct<LC, 5>(P2, A, TW, false);
        ring_f32_output(Y, Y == P2 ? A : P2, f2, d, b, j2, Lp, L, rw);
        return;
    }
    const float2 *G;
    if constexpr (LC > 0) G = fft_passes_ct<LC, 4>(X, S, TW, true);
    else G = fft_passes(X, S, 4, Lp, plan, TW, true);

    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        const int kp = fpad(k);
        const float2 zz = G[G_ZETA * Lp + kp], pp = G[G_PHI * Lp + kp];
        const float2 uu = G[G_U * Lp + kp], vv = G[G_V * Lp + kp];
        if (gs) {
            gs[G_ZETA * L + k] = zz;
            gs[G_PHI * L + k] = pp;
            gs[G_U * L + k] = uu;
            gs[G_V * L + k] = vv;
        }
        const float etaN = zz.x + fN, etaS = zz.y - fN;
        X[P_A * Lp + kp] = make_float2(etaN * uu.x, etaS * uu.y);
        X[P_B * Lp + kp] = make_float2(etaN * vv.x, etaS * vv.y);
        X[P_C * Lp + kp] = make_float2(pp.x * uu.x, pp.y * uu.y);
        X[P_D * Lp + kp] = make_float2(pp.x * vv.x, pp.y * vv.y);
        X[P_E * Lp + kp] = make_float2((uu.x * uu.x + vv.x * vv.x) * inv2c, (uu.y * uu.y + vv.y * vv.y) * inv2c);
    }
    __syncthreads();
    const float2 *Y;
    if constexpr (LC > 0) Y = fft_passes_ct<LC, 5>(X, S, TW, false);
    else Y = fft_passes(X, S, 5, Lp, plan, TW, false);

    ring_f32_output(Y, Y == X ? S : X, f2, d, b, j2, Lp, L, rw);
}

// ---------------------------------------------------------------------------
// K3a: Legendre projections, one thread per extended row e = (m, n'), all
// orders flattened so that every block carries the same work:
//   Y[b][e][g] = sum_j2 Pbar_n'(mu_j) W_g[parity(n'-m)][j2],  g in (A, B, C, D, E).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(64) k3_project(const V2<R> *__restrict__ f2, Dims d, const R *__restrict__ pbar,
                                                 const int *__restrict__ row_m, V2<R> *__restrict__ y) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (e >= d.next) return;
    const int T = d.T, J2 = d.J2;
    const int m = row_m[e];
    const int par = (e - ext_offset(T, m)) & 1;
    const V2<R> *W = f2 + (static_cast<size_t>(b) * (T + 1) + m) * 10 * J2 + par * J2;
    const R *prow = pbar + static_cast<size_t>(e) * d.J2p;
    V2<R> acc[5];
#pragma unroll
    for (int g = 0; g < 5; ++g) acc[g] = mk<R>(0, 0);
    const int J2e = J2 & ~1;
    for (int j = 0; j < J2e; j += 2) {
        const V2<R> pp = *reinterpret_cast<const V2<R> *>(prow + j);
#pragma unroll
        for (int g = 0; g < 5; ++g) {
            const V2<R> w0 = W[g * 2 * J2 + j], w1 = W[g * 2 * J2 + j + 1];
            acc[g].x = fma(pp.x, w0.x, acc[g].x);
            acc[g].y = fma(pp.x, w0.y, acc[g].y);
            acc[g].x = fma(pp.y, w1.x, acc[g].x);
            acc[g].y = fma(pp.y, w1.y, acc[g].y);
        }
    }
    if (J2e < J2) {
        const R p = prow[J2e];
#pragma unroll
        for (int g = 0; g < 5; ++g) {
            const V2<R> w0 = W[g * 2 * J2 + J2e];
            acc[g].x = fma(p, w0.x, acc[g].x);
            acc[g].y = fma(p, w0.y, acc[g].y);
        }
    }
    V2<R> *o = y + (static_cast<size_t>(b) * d.next + e) * 5;
#pragma unroll
    for (int g = 0; g < 5; ++g) o[g] = acc[g];
}

// ---------------------------------------------------------------------------
// FP32 contractions, register-tiled for the FMA pipe (the FP64 kernels above
// are bound by GB300's FP64 rate; in FP32 the same loops would be bound by
// load issue and latency).
//
// K1 (FP32): one block per (state, order pair), all latitudes.  The table
// rows of the two orders (contiguous in the table) stream through a ring of
// shared-memory stages, kSynRows rows per bulk copy, issued nstages chunks
// ahead by one thread (bounded mbarrier waits; on expiry the block sets the
// error flag and stops).  A thread owns four consecutive latitudes and keeps
// the even/odd sums of the four fields for all four in registers; S
// neighbouring lanes split the row pairs of each chunk and are summed with
// shuffles at the end of each order (S = 2 or 1 keeps a block at <= 256
// threads).  The coefficients are prepared in FP32 (the precision of this
// path) while the first copies are in flight.
// ---------------------------------------------------------------------------
constexpr int kSynRows = 24;
constexpr int kMaxSynStages = 6;
constexpr size_t kSynCtrlBytes = 128;
static_assert(8 * kMaxSynStages <= static_cast<int>(kSynCtrlBytes), "mbarriers fit the control block");

__host__ inline int synthesis_f32_stages(int J2p) {
    const int per = kSynRows * J2p * static_cast<int>(sizeof(float));
    int ns = (48 * 1024) / per;
    return ns < 2 ? 2 : (ns > kMaxSynStages ? kMaxSynStages : ns);
}
__host__ inline size_t synthesis_f32_smem(const Dims &d, int nstages, int nf = 4) {
    return kSynCtrlBytes + static_cast<size_t>(nstages) * kSynRows * d.J2p * sizeof(float) +
           static_cast<size_t>(d.T + 4) * nf * sizeof(float2);
}

// NF = 4: the synthesis (coefficients prepared from the FP64 states, output
// F1[b][j][m][parity][f]).  NF = 5: the transpose of the analysis projection
// in the adjoint (coefficients = the rows Y-bar[b][e][5], output
// W-bar[b][j][m][parity][g], the layout the FP32 ring transpose reads).
template <int S, int NF>
__global__ void __launch_bounds__(256) k1_synthesis_f32(const double2 *__restrict__ states, long long sstride,
                                                        const float2 *__restrict__ ybar, Dims d,
                                                        const float *__restrict__ pbar,
                                                        const double *__restrict__ syn, float2 *__restrict__ f1,
                                                        int nstages, int *err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem_raw);                 // [kMaxSynStages]
    float *stage = reinterpret_cast<float *>(smem_raw + kSynCtrlBytes);      // [nstages][kSynRows][J2p]
    const size_t stage_elems = static_cast<size_t>(kSynRows) * d.J2p;
    float2 *cf = reinterpret_cast<float2 *>(stage + nstages * stage_elems);  // [rows][NF]
    const int T = d.T;
    const int b = blockIdx.x;
    const int m1 = blockIdx.y, m2 = T - blockIdx.y;
    const int nn1 = T + 2 - m1;
    const int nn2 = (m2 > m1) ? T + 2 - m2 : 0;
    const int rows = nn1 + nn2;
    const int nch1 = (nn1 + kSynRows - 1) / kSynRows;
    const int nch = nch1 + (nn2 + kSynRows - 1) / kSynRows;
    // chunk c: order, first row t0 within the order, row count
    auto chunk = [&](int c, int &m, int &t0, int &cnt) {
        const bool second = c >= nch1;
        m = second ? m2 : m1;
        t0 = (second ? c - nch1 : c) * kSynRows;
        cnt = min(kSynRows, (second ? nn2 : nn1) - t0);
    };
    auto issue = [&](int c) {
        int m, t0, cnt;
        chunk(c, m, t0, cnt);
        const uint32_t bytes = static_cast<uint32_t>(cnt) * d.J2p * sizeof(float);
        uint64_t *bar = &mbar[c % nstages];
        expect_tx(bar, bytes);
        bulk_copy(stage + (c % nstages) * stage_elems, pbar + static_cast<size_t>(ext_offset(T, m) + t0) * d.J2p,
                  bytes, bar);
    };
    int issued = 0;
    if (threadIdx.x == 0) {
        for (int k = 0; k < nstages; ++k) mbar_init(&mbar[k], 1);
        mbar_init_fence();
        for (; issued < min(nstages, nch); ++issued) issue(issued);
    }

    if constexpr (NF == 5) {                            // the rows of both orders, 8 bytes per piece
        for (int i = threadIdx.x; i < rows * 5; i += blockDim.x) {
            const int r = i / 5, g = i - r * 5;
            const int m = (r < nn1) ? m1 : m2;
            const int t = (r < nn1) ? r : r - nn1;
            cp_async8(cf + i, ybar + (static_cast<size_t>(b) * d.next + ext_offset(T, m) + t) * 5 + g);
        }
        cp_async_commit();
        cp_async_wait<0>();
    }
    const double2 *st = states + b * sstride;
    const int nc = d.ncoef;
    for (int r = threadIdx.x; NF == 4 && r < rows; r += blockDim.x) {
        const int m = (r < nn1) ? m1 : m2;
        const int t = (r < nn1) ? r : r - nn1;
        const int n = m + t;
        const int off = order_offset(T, m);
        const int e = ext_offset(T, m) + t;
        auto ld = [&](int f, int k) -> float2 {
            if (k < m || k > T) return make_float2(0.f, 0.f);
            const double2 v = st[f * nc + off + k - m];
            return make_float2(f64_to_f32_rn(v.x), f64_to_f32_rn(v.y));
        };
        const float2 z0 = ld(F_ZETA, n), zm = ld(F_ZETA, n - 1), zp = ld(F_ZETA, n + 1);
        const float2 d0 = ld(F_DIV, n), dm = ld(F_DIV, n - 1), dp = ld(F_DIV, n + 1);
        const float c0 = f64_to_f32_rn(syn[3 * e]), c1 = f64_to_f32_rn(syn[3 * e + 1]),
                    c2 = f64_to_f32_rn(syn[3 * e + 2]);
        cf[r * 4 + G_ZETA] = z0;
        cf[r * 4 + G_PHI] = ld(F_PHI, n);
        cf[r * 4 + G_U] = make_float2(-c0 * d0.y - c1 * zm.x - c2 * zp.x, c0 * d0.x - c1 * zm.y - c2 * zp.y);
        cf[r * 4 + G_V] = make_float2(-c0 * z0.y + c1 * dm.x + c2 * dp.x, c0 * z0.x + c1 * dm.y + c2 * dp.y);
    }
    __syncthreads();

    const int part = threadIdx.x % S;
    const int j0 = 4 * (threadIdx.x / S);
    const bool active = j0 < d.J2;
    const int jl = active ? j0 : 0;                      // idle lanes read a valid column and store nothing
    float2 ae[NF][4], ao[NF][4];                         // [field][latitude]
    auto reset = [&]() {
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
            for (int k = 0; k < 4; ++k) ae[f][k] = ao[f][k] = make_float2(0.f, 0.f);
    };
    auto accum = [&](float2 (&a)[NF][4], const float4 pv4, const float2 *c) {
        const float pv[4] = {pv4.x, pv4.y, pv4.z, pv4.w};
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const float2 cc = c[f];
#pragma unroll
            for (int k = 0; k < 4; ++k) a[f][k] = caxpy(pv[k], cc, a[f][k]);
        }
    };
    reset();
    int c = 0;
    for (; c < nch; ++c) {
        int m, t0, cnt;
        chunk(c, m, t0, cnt);
        const bool late = !mbar_wait(&mbar[c % nstages], (c / nstages) & 1);
        if (__syncthreads_or(late)) {                    // the block agrees before anyone leaves
            if (threadIdx.x == 0) atomicExch(err, 5);
            break;
        }
        const float *P = stage + (c % nstages) * stage_elems + jl;
        const float2 *cc = cf + ((c >= nch1 ? nn1 : 0) + t0) * NF;
#pragma unroll 4
        for (int u = part; 2 * u < cnt; u += S) {
            const int i0 = 2 * u;
            const float4 pe = *reinterpret_cast<const float4 *>(P + i0 * d.J2p);
            if (i0 + 1 < cnt) {
                const float4 po = *reinterpret_cast<const float4 *>(P + (i0 + 1) * d.J2p);
                accum(ae, pe, cc + i0 * NF);
                accum(ao, po, cc + (i0 + 1) * NF);
            } else {
                accum(ae, pe, cc + i0 * NF);
            }
        }
        if (c == nch1 - 1 || c == nch - 1) {             // end of an order: reduce and store
#pragma unroll
            for (int f = 0; f < NF; ++f)
#pragma unroll
                for (int k = 0; k < 4; ++k)
#pragma unroll
                    for (int o = 1; o < S; o <<= 1) {
                        ae[f][k].x += __shfl_xor_sync(0xffffffffu, ae[f][k].x, o);
                        ae[f][k].y += __shfl_xor_sync(0xffffffffu, ae[f][k].y, o);
                        ao[f][k].x += __shfl_xor_sync(0xffffffffu, ao[f][k].x, o);
                        ao[f][k].y += __shfl_xor_sync(0xffffffffu, ao[f][k].y, o);
                    }
            if (active && part == 0) {
                if constexpr (NF == 4) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (j0 + k >= d.J2) break;
                        float4 *o = reinterpret_cast<float4 *>(
                            f1 + (static_cast<size_t>(b) * d.J2 + j0 + k) * (4 * 2 * (T + 1)) + 8 * m);
                        o[0] = make_float4(ae[0][k].x, ae[0][k].y, ae[1][k].x, ae[1][k].y);
                        o[1] = make_float4(ae[2][k].x, ae[2][k].y, ae[3][k].x, ae[3][k].y);
                        o[2] = make_float4(ao[0][k].x, ao[0][k].y, ao[1][k].x, ao[1][k].y);
                        o[3] = make_float4(ao[2][k].x, ao[2][k].y, ao[3][k].x, ao[3][k].y);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (j0 + k >= d.J2) break;
                        float2 *o = f1 + (static_cast<size_t>(b) * d.J2 + j0 + k) * (5 * 2 * (T + 1)) + 10 * m;
#pragma unroll
                        for (int f = 0; f < 5; ++f) {
                            o[f] = ae[f][k];
                            o[5 + f] = ao[f][k];
                        }
                    }
                }
            }
            reset();
        }
        __syncthreads();                                 // every read of this stage is done
        if (threadIdx.x == 0 && issued < nch) issue(issued++);
    }
    if (c < nch && threadIdx.x == 0) {                   // stopped early: let issued copies land (bounded)
        for (int k = c; k < issued; ++k) mbar_wait(&mbar[k % nstages], (k / nstages) & 1);
    }
}

// K1 (FP32, NB node states per block): one block per (order pair m, T - m,
// group of NB states).  Each table row is then read from L2 once per NB
// states instead of once per state (the per-state kernel above streams the
// whole table B times per batch, more than L2 delivers to keep its FMAs busy).
// One thread issues, at the start, bulk copies of the FP64 coefficients of
// both orders (per state and field, contiguous in the state layout) and of
// the rows' FP32 wind factors, then the first table chunks of the stage ring
// (bounded waits as in the per-state kernel).  The states are converted to
// FP32 once in shared memory (integer-pipe conversions) and the coefficient
// rows formed there.  Threads split by parity (rows t = n' - m even, odd) and,
// for S = 2, by alternate rows of that parity (lane pairs, summed with a
// shuffle at the end of each order); a thread keeps two latitudes x NB states
// x 4 fields (64 accumulators at NB = 4).
constexpr int kSynNbMaxThreads = 384;
constexpr int kSynNbRowsMin = 56;          // table rows per chunk at least (even: chunks start on even t)
constexpr int kSynNbRowsMax = 128;         // and at most
static_assert(8 * (kMaxSynStages + 1) <= static_cast<int>(kSynCtrlBytes), "stage and prologue barriers fit");
constexpr size_t kSmemLimit = 227 * 1024;

// coefficient row stride in floats: NB x NF complex values rounded to 16
// bytes, plus 16 bytes of padding; two rows apart (the rows of an S = 2 lane
// pair) never start in the same bank group
__host__ __device__ constexpr int synthesis_nb_rowstride(int nb, int nf) {
    return ((nb * nf * 2 + 3) / 4 * 4 + 4) % 16 == 0 ? (nb * nf * 2 + 3) / 4 * 4 + 8 : (nb * nf * 2 + 3) / 4 * 4 + 4;
}
__host__ inline int synthesis_nb_threads(int J2, int S) { return 2 * S * (((J2 + 1) / 2 + 32 / S - 1) / (32 / S) * (32 / S)); }
__host__ inline int synthesis_nb_s(int J2) { return synthesis_nb_threads(J2, 2) <= kSynNbMaxThreads ? 2 : 1; }
// FP32 state copies of a block, in float2 (rounded up to keep 16-byte alignment)
__host__ __device__ inline int synthesis_nb_s32_elems(int T, int nb) { return (nb * 3 * (T + 2) + 1) & ~1; }
// shared memory besides the stage ring: control, coefficient rows and, for the
// synthesis (NF = 4), the FP64 states, their FP32 copies and the wind factors
__host__ inline size_t synthesis_nb_fixed(const Dims &d, int nb, int nf) {
    size_t b = kSynCtrlBytes + static_cast<size_t>(d.T + 4) * synthesis_nb_rowstride(nb, nf) * sizeof(float);
    if (nf == 4)
        b += static_cast<size_t>(nb) * 3 * (d.T + 2) * sizeof(double2) +
             static_cast<size_t>(synthesis_nb_s32_elems(d.T, nb)) * sizeof(float2) +
             static_cast<size_t>(d.T + 4) * sizeof(float4);
    return b;
}
// Rows per chunk: the largest even count (kSynNbRowsMin..kSynNbRowsMax) for
// which two stages fit beside the fixed part -- fewer, larger chunks mean
// fewer block barriers per order pair.
__host__ inline int synthesis_nb_rows(const Dims &d, int nb, int nf) {
    const size_t fixed = synthesis_nb_fixed(d, nb, nf);
    for (int r = kSynNbRowsMax; r > kSynNbRowsMin; r -= 2)
        if (fixed + 2 * static_cast<size_t>(r) * d.J2p * sizeof(float) <= kSmemLimit) return r;
    return kSynNbRowsMin;
}
__host__ inline int synthesis_nb_stages(const Dims &d, int nb, int nf) {
    const size_t per = static_cast<size_t>(synthesis_nb_rows(d, nb, nf)) * d.J2p * sizeof(float);
    const size_t fixed = synthesis_nb_fixed(d, nb, nf);
    const int ns = fixed < kSmemLimit ? static_cast<int>((kSmemLimit - fixed) / per) : 0;
    return ns > kMaxSynStages ? kMaxSynStages : ns;
}
__host__ inline size_t synthesis_nb_smem(const Dims &d, int nb, int nf) {
    return synthesis_nb_fixed(d, nb, nf) + static_cast<size_t>(synthesis_nb_stages(d, nb, nf)) *
                                               synthesis_nb_rows(d, nb, nf) * d.J2p * sizeof(float);
}
// whether the batched kernel serves these sizes (threads, at least two stages)
__host__ inline bool synthesis_nb_fits(const Dims &d, int nb, int nf) {
    return synthesis_nb_threads(d.J2, 1) <= kSynNbMaxThreads && synthesis_nb_stages(d, nb, nf) >= 2;
}

// NF = 4: the synthesis (coefficients prepared from the FP64 states, output
// F1[b][j][m][parity][f]).  NF = 5: the transpose of the analysis projection
// in the adjoint (coefficients = the rows Y-bar[b][e][5], gathered with
// cp.async; output W-bar[b][j][m][parity][g]: one store run of 40 bytes per (j, m, parity)).
// FP32-pair ("double-float") arithmetic of the on-the-fly Legendre
// recurrence: a value is hi + lo with |lo| <= ulp(hi) / 2.  The products use
// the FMA error-free transformation of the product, the sum Knuth's
// two-sum followed by a fast renormalisation (Dekker); the explicit _rn
// intrinsics keep the compiler from contracting or reordering them.
struct dfl {
    float hi, lo;
};
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float s = __fadd_rn(p, e);
    return {s, __fsub_rn(e, __fsub_rn(s, p))};
}
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) {
    const float s = __fsub_rn(a.hi, b.hi);
    const float v = __fsub_rn(s, a.hi);
    float e = __fsub_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fadd_rn(b.hi, v));
    e = __fadd_rn(e, __fsub_rn(a.lo, b.lo));
    const float r = __fadd_rn(s, e);
    return {r, __fsub_rn(e, __fsub_rn(r, s))};
}

// REC (NF = 4): the Legendre rows of every chunk are generated in shared
// memory by the three-term recurrence Pbar_n = a_n mu Pbar_{n-1} -
// b_n Pbar_{n-2} (a_n = 1 / eps_n, b_n = eps_{n-1} / eps_n) in FP32-pair
// arithmetic, one thread per latitude, from the FP64 values of Pbar_m^m and
// Pbar_{m+1}^m, instead of being copied from the FP32 table; the stored value
// is the FP32 rounding of the pair.
template <int NB, int S, int NF, bool REC = false>
__global__ void __launch_bounds__(kSynNbMaxThreads, 1)
    k1_synthesis_f32_nb(const double2 *__restrict__ states, long long sstride, const float2 *__restrict__ ybar,
                        int B, Dims d, const float *__restrict__ pbar, const float4 *__restrict__ syn32,
                        float2 *__restrict__ f1, int nstages, int crows, int *err,
                        const float4 *__restrict__ rec_ab = nullptr,
                        const float4 *__restrict__ rec_seed = nullptr, const float2 *__restrict__ rec_mu = nullptr) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem_raw);                 // [kMaxSynStages], then the prologue's
    uint64_t *mpro = mbar + kMaxSynStages;
    const int T = d.T;
    constexpr int RS = synthesis_nb_rowstride(NB, NF);                       // coefficient row stride (floats)
    float *cf = reinterpret_cast<float *>(smem_raw + kSynCtrlBytes);         // [T + 4 rows][RS]
    double2 *raw = reinterpret_cast<double2 *>(cf + static_cast<size_t>(T + 4) * RS);   // [NB][3][T + 2] (NF = 4)
    float2 *s32 = reinterpret_cast<float2 *>(raw + static_cast<size_t>(NB) * 3 * (T + 2));   // [NB][3][T + 2]
    float4 *sy = reinterpret_cast<float4 *>(s32 + synthesis_nb_s32_elems(T, NB));             // [T + 4]
    float *stage = NF == 4 ? reinterpret_cast<float *>(sy + (T + 4))        // [nstages][crows][J2p]
                           : reinterpret_cast<float *>(raw);
    const size_t stage_elems = static_cast<size_t>(crows) * d.J2p;
    const int m1 = blockIdx.x, m2 = T - blockIdx.x;
    const int b0 = blockIdx.y * NB;
    const int nbv = min(NB, B - b0);
    const bool two = m2 > m1;
    const int nn1 = T + 2 - m1;
    const int nn2 = two ? T + 2 - m2 : 0;
    const int rows = nn1 + nn2;
    const int nc1 = T + 1 - m1, ncs = nc1 + (two ? T + 1 - m2 : 0);         // state coefficients per field
    const int nch1 = (nn1 + crows - 1) / crows;
    const int nch = nch1 + (nn2 + crows - 1) / crows;
    auto chunk = [&](int c, int &m, int &t0, int &cnt) {
        const bool second = c >= nch1;
        m = second ? m2 : m1;
        t0 = (second ? c - nch1 : c) * crows;
        cnt = min(crows, (second ? nn2 : nn1) - t0);
    };
    auto issue = [&](int c) {
        int m, t0, cnt;
        chunk(c, m, t0, cnt);
        const uint32_t bytes = static_cast<uint32_t>(cnt) * d.J2p * sizeof(float);
        uint64_t *bar = &mbar[c % nstages];
        expect_tx(bar, bytes);
        bulk_copy(stage + (c % nstages) * stage_elems, pbar + static_cast<size_t>(ext_offset(T, m) + t0) * d.J2p,
                  bytes, bar);
    };
    const int nc = d.ncoef;
    int issued = 0;
    if (NF == 5 && threadIdx.x == 0) {
        for (int k = 0; k < kMaxSynStages; ++k) mbar_init(&mbar[k], 1);
        mbar_init_fence();
        for (; issued < min(nstages, nch); ++issued) issue(issued);
    }
    if (NF == 4 && threadIdx.x == 0) {
        for (int k = 0; k <= kMaxSynStages; ++k) mbar_init(&mbar[k], 1);
        mbar_init_fence();
        // the table stages need nothing of the preceding kernels: in flight
        // before the wait for the states (programmatic dependent launch)
        if (!REC)
            for (; issued < min(nstages, nch); ++issued) issue(issued);
        pdl_wait();
        const uint32_t n1b = static_cast<uint32_t>(nc1) * sizeof(double2);
        const uint32_t n2b = static_cast<uint32_t>(ncs - nc1) * sizeof(double2);
        expect_tx(mpro, static_cast<uint32_t>(nbv) * 3 * (n1b + n2b) +
                            static_cast<uint32_t>(rows) * sizeof(float4));
        for (int b = 0; b < nbv; ++b)
            for (int f = 0; f < 3; ++f) {
                const double2 *src = states + (b0 + b) * sstride + f * nc;
                double2 *dst = raw + (b * 3 + f) * ncs;
                bulk_copy(dst, src + order_offset(T, m1), n1b, mpro);
                if (two) bulk_copy(dst + nc1, src + order_offset(T, m2), n2b, mpro);
            }
        bulk_copy(sy, syn32 + ext_offset(T, m1), static_cast<uint32_t>(nn1) * sizeof(float4), mpro);
        if (two) bulk_copy(sy + nn1, syn32 + ext_offset(T, m2), static_cast<uint32_t>(nn2) * sizeof(float4), mpro);
    }
    if constexpr (NF == 5) {                             // the Y-bar rows of both orders, 8 bytes per piece
        for (int i = threadIdx.x; i < rows * NB * 5; i += blockDim.x) {
            const int r = i / (NB * 5), bg = i - r * (NB * 5), b = bg / 5;
            float2 *dst = reinterpret_cast<float2 *>(cf + static_cast<size_t>(r) * RS) + bg;
            if (b < nbv) {
                const int e = (r < nn1) ? ext_offset(T, m1) + r : ext_offset(T, m2) + r - nn1;
                cp_async8(dst, ybar + (static_cast<size_t>(b0 + b) * d.next + e) * 5 + (bg - 5 * b));
            } else {
                *dst = make_float2(0.f, 0.f);
            }
        }
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
    }
    if constexpr (NF == 4) {
    __syncthreads();                                     // the barriers are initialised
    const bool late = !mbar_wait(mpro, 0);
    if (__syncthreads_or(late)) {
        if (threadIdx.x == 0) {
            atomicExch(err, 5);
            for (int k = 0; k < issued; ++k) mbar_wait(&mbar[k % nstages], (k / nstages) & 1);
        }
        return;
    }
    for (int i = threadIdx.x; i < NB * 3 * ncs; i += blockDim.x) {
        const bool valid = i < nbv * 3 * ncs;
        const double2 x = valid ? raw[i] : make_double2(0.0, 0.0);
        s32[i] = make_float2(f64_to_f32_rn(x.x), f64_to_f32_rn(x.y));
    }
    __syncthreads();
    // coefficient rows: zeta, Phi' and the U, V combinations of n' - 1, n', n' + 1
    for (int i = threadIdx.x; i < rows * NB; i += blockDim.x) {
        const int r = i / NB, b = i - r * NB;
        const bool first = r < nn1;
        const int m = first ? m1 : m2;
        const int t = first ? r : r - nn1;
        const int n = m + t;
        const int base = first ? 0 : nc1;
        const float2 *sb = s32 + static_cast<size_t>(b) * 3 * ncs;
        auto ld = [&](int f, int k) -> float2 {
            return (k < m || k > T) ? make_float2(0.f, 0.f) : sb[f * ncs + base + k - m];
        };
        const float2 z0 = ld(F_ZETA, n), zm = ld(F_ZETA, n - 1), zp = ld(F_ZETA, n + 1);
        const float2 d0 = ld(F_DIV, n), dm = ld(F_DIV, n - 1), dp = ld(F_DIV, n + 1);
        const float4 cy = sy[r];
        const float c0 = cy.x, c1 = cy.y, c2 = cy.z;
        float2 *o = reinterpret_cast<float2 *>(cf + static_cast<size_t>(r) * RS) + b * 4;
        o[G_ZETA] = z0;
        o[G_PHI] = ld(F_PHI, n);
        o[G_U] = make_float2(-c0 * d0.y - c1 * zm.x - c2 * zp.x, c0 * d0.x - c1 * zm.y - c2 * zp.y);
        o[G_V] = make_float2(-c0 * z0.y + c1 * dm.x + c2 * dp.x, c0 * z0.x + c1 * dm.y + c2 * dp.y);
    }
    __syncthreads();
    }

    const int tq = blockDim.x / 2;
    const int par = threadIdx.x >= tq ? 1 : 0;
    const int lt = threadIdx.x - par * tq;
    const int sp = lt % S;                               // alternate rows of this parity
    const int j0 = 2 * (lt / S);
    const bool active = j0 < d.J2;
    const int jl = active ? j0 : 0;                      // idle lanes read a valid column and store nothing
    float2 a[NB][NF][2];                                 // [state][field][latitude]
    auto reset = [&]() {
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int f = 0; f < NF; ++f) a[b][f][0] = a[b][f][1] = make_float2(0.f, 0.f);
    };
    reset();
    // recurrence state of this thread's latitude (REC): rows t - 2 and t - 1
    dfl r_m2{0.f, 0.f}, r_m1{0.f, 0.f}, r_mu{0.f, 0.f};
    if (REC && threadIdx.x < d.J2p) {
        const float2 mv = rec_mu[threadIdx.x];
        r_mu = {mv.x, mv.y};
    }
    int c = 0;
    for (; c < nch; ++c) {
        int m, t0, cnt;
        chunk(c, m, t0, cnt);
        if constexpr (REC) {
            float *Pg = stage + (c % nstages) * stage_elems;
            const int j = threadIdx.x;
            if (j < d.J2p) {
                if (t0 == 0) {                           // a new order: Pbar_m^m, Pbar_{m+1}^m
                    const float4 sd = rec_seed[static_cast<size_t>(m) * d.J2p + j];
                    r_m2 = {sd.x, sd.y};
                    r_m1 = {sd.z, sd.w};
                }
                const float4 *ab = rec_ab + ext_offset(T, m);
                for (int r = 0; r < cnt; ++r) {
                    const int t = t0 + r;
                    dfl v;
                    if (t == 0) {
                        v = r_m2;
                    } else if (t == 1) {
                        v = r_m1;
                    } else {
                        const float4 k = __ldg(ab + t);
                        v = df_sub(df_mul(df_mul({k.x, k.y}, r_mu), r_m1), df_mul({k.z, k.w}, r_m2));
                        r_m2 = r_m1;
                        r_m1 = v;
                    }
                    Pg[static_cast<size_t>(r) * d.J2p + j] = v.hi;
                }
            }
            __syncthreads();
        } else {
            const bool slow = !mbar_wait(&mbar[c % nstages], (c / nstages) & 1);
            if (__syncthreads_or(slow)) {                // the block agrees before anyone leaves
                if (threadIdx.x == 0) atomicExch(err, 5);
                break;
            }
        }
        const float *P = stage + (c % nstages) * stage_elems + jl;
        const float *cc = cf + static_cast<size_t>((c >= nch1 ? nn1 : 0) + t0) * RS;
#pragma unroll 4
        for (int i = par + 2 * sp; i < cnt; i += 2 * S) {   // chunks start on even t: row i has parity i & 1
            const float2 pv = *reinterpret_cast<const float2 *>(P + i * d.J2p);
            float2 kk[NB * NF];                          // the row's coefficients, 16 bytes per load
            if constexpr ((NB * NF) % 2 == 0) {
                const float4 *ci = reinterpret_cast<const float4 *>(cc + i * RS);
#pragma unroll
                for (int q = 0; q < NB * NF / 2; ++q) {
                    const float4 v = ci[q];
                    kk[2 * q] = make_float2(v.x, v.y);
                    kk[2 * q + 1] = make_float2(v.z, v.w);
                }
            } else {
                const float2 *ci = reinterpret_cast<const float2 *>(cc + i * RS);
#pragma unroll
                for (int q = 0; q < NB * NF; ++q) kk[q] = ci[q];
            }
#pragma unroll
            for (int b = 0; b < NB; ++b)
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    a[b][f][0] = caxpy(pv.x, kk[b * NF + f], a[b][f][0]);
                    a[b][f][1] = caxpy(pv.y, kk[b * NF + f], a[b][f][1]);
                }
        }
        if (c == nch1 - 1 || c == nch - 1) {             // end of an order: sum the lane pair, store, restart
            if constexpr (S == 2) {
#pragma unroll
                for (int b = 0; b < NB; ++b)
#pragma unroll
                    for (int f = 0; f < NF; ++f)
#pragma unroll
                        for (int k = 0; k < 2; ++k) {
                            a[b][f][k].x += __shfl_xor_sync(0xffffffffu, a[b][f][k].x, 1);
                            a[b][f][k].y += __shfl_xor_sync(0xffffffffu, a[b][f][k].y, 1);
                        }
            }
            if (active && sp == 0) {
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (j0 + k >= d.J2) break;
#pragma unroll
                    for (int b = 0; b < NB; ++b) {
                        if (b >= nbv) break;
                        if constexpr (NF == 4) {         // F1[b][j][m][parity][f]: one 32-byte sector per store pair
                            float4 *o = reinterpret_cast<float4 *>(
                                f1 + (static_cast<size_t>(b0 + b) * d.J2 + j0 + k) * (8 * (T + 1)) + (2 * m + par) * 4);
                            o[0] = make_float4(a[b][0][k].x, a[b][0][k].y, a[b][1][k].x, a[b][1][k].y);
                            o[1] = make_float4(a[b][2][k].x, a[b][2][k].y, a[b][3][k].x, a[b][3][k].y);
                        } else {                         // W-bar[b][j][m][parity][g]: 40 contiguous bytes
                            float2 *o = f1 + (static_cast<size_t>(b0 + b) * d.J2 + j0 + k) * (NF * 2 * (T + 1)) +
                                        (2 * m + par) * NF;
#pragma unroll
                            for (int f = 0; f < NF; ++f) o[f] = a[b][f][k];
                        }
                    }
                }
            }
            reset();
        }
        __syncthreads();                                 // every read of this stage is done
        if (!REC && threadIdx.x == 0 && issued < nch) issue(issued++);
    }
    if (c < nch && threadIdx.x == 0) {                   // stopped early: let issued copies land (bounded)
        for (int k = c; k < issued; ++k) mbar_wait(&mbar[k % nstages], (k / nstages) & 1);
    }
}

// K3a (FP32): one block per (state, order pair m, T - m).  The W rows of
// both orders (10 x J2 complex each) are staged in shared memory; a thread
// group of kPrjParts neighbouring lanes owns a row quad (rows e, e+2, e+4,
// e+6 of one group (m, p)), each lane every kPrjParts-th 4-latitude block,
// 40 accumulators, summed with shuffles.  Per four latitudes a lane issues
// four 16-byte table loads (neighbouring lanes: neighbouring 16 bytes of the
// same row) and ten 16-byte shared loads for 160 FMAs.  VEC: J2 even, so
// every W row starts on a 16-byte boundary.
constexpr int kPrjParts = 4;
constexpr int kPrjDepth = 4;          // per-thread cp.async stages of the table rows (ASYNC)
constexpr int kPrjMaxThreads = 288;   // two blocks per SM fit the register file


// ASYNC: each lane streams its own four rows through kPrjDepth private
// shared-memory stages with cp.async (16 bytes per row and 4-latitude
// block), kPrjDepth - 1 blocks ahead of the FMAs; no block barrier is
// involved because a lane only reads what it copied.
// NF = 5: the analysis projection, W = F2[b][m][g][parity][j] (contiguous per
// order), Y[b][e][g].  NF = 4: the transpose of the synthesis in the adjoint,
// W = F1-bar[b][m][j][f][parity] (contiguous per order) staged into the same
// [f][parity][j] arrangement, Z-bar[b][e][f].
// W rows in shared memory: J2 latitudes padded by 2 (J2 even: rows stay on
// 16-byte boundaries, and the transposing stage of the FP32 F2 layout writes
// ten neighbouring values of one latitude to ten different bank groups).
__host__ __device__ inline int project_f32_wstride(int J2) { return J2 % 2 == 0 ? J2 + 2 : J2; }

template <bool VEC, bool ASYNC, int NF>
__global__ void __launch_bounds__(kPrjMaxThreads, 2) k3_project_f32(const float2 *__restrict__ src, Dims d,
                                                      const float *__restrict__ pbar, float2 *__restrict__ y) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int T = d.T, J2 = d.J2, JW = project_f32_wstride(d.J2);
    float2 *ws = reinterpret_cast<float2 *>(smem_raw);   // [2][2 NF][JW]
    float4 *pst = reinterpret_cast<float4 *>(ws + 2 * 2 * NF * JW);   // [kPrjDepth][4 rows][blockDim] (ASYNC)
    const int b = blockIdx.x;
    const int m1 = blockIdx.y, m2 = T - blockIdx.y;
    const int norders = (m2 > m1) ? 2 : 1;
    if constexpr (NF == 5) {
        pdl_wait();
    }
    for (int h = 0; h < norders; ++h) {
        float2 *dst = ws + h * 2 * NF * JW;
        const int mh = h ? m2 : m1;
        if constexpr (NF == 5) {                          // F2[b][m][j][g][parity] -> [g][parity][j]
            const float2 *w = src + (static_cast<size_t>(b) * (T + 1) + mh) * 10 * J2;
            for (int i = threadIdx.x; i < 10 * J2; i += blockDim.x) {
                const int j = i / 10, gp = i - j * 10;
                cp_async8(dst + gp * JW + j, w + i);
            }
        } else {                                          // F1-bar[b][m][j][f][parity] -> [f][parity][j]
            const float2 *w = src + (static_cast<size_t>(b) * (T + 1) + mh) * 8 * J2;
            for (int i = threadIdx.x; i < 8 * J2; i += blockDim.x) {
                const int j = i >> 3, fp = i & 7;
                cp_async8(dst + fp * JW + j, w + i);
            }
        }
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    // quads of (m1, p=0), (m1, p=1), (m2, p=0), (m2, p=1)
    auto quads_of = [&](int m, int p) { return ((T + 3 - m - p) / 2 + 3) / 4; };
    const int c1 = quads_of(m1, 0), c2 = c1 + quads_of(m1, 1);
    const int c3 = c2 + (norders == 2 ? quads_of(m2, 0) : 0);
    const int nqt = c3 + (norders == 2 ? quads_of(m2, 1) : 0);
    const int part = threadIdx.x % kPrjParts;
    const int per_pass = blockDim.x / kPrjParts;
    for (int qb = 0; qb < nqt; qb += per_pass) {
        const int qraw = qb + static_cast<int>(threadIdx.x) / kPrjParts;
        const bool active = qraw < nqt;
        const int qa = active ? qraw : nqt - 1;          // idle lanes compute a valid quad and store nothing
        const int k = (qa < c1) ? 0 : (qa < c2) ? 1 : (qa < c3) ? 2 : 3;
        const int qi = qa - ((k == 0) ? 0 : (k == 1) ? c1 : (k == 2) ? c2 : c3);
        const int m = (k < 2) ? m1 : m2, p = k & 1, h = k >> 1;
        const int R = (T + 3 - m - p) / 2;
        const int q0 = 4 * qi, nr = min(4, R - q0);
        const int e0 = ext_offset(T, m) + p + 2 * q0;
        const float *pr[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) pr[r] = pbar + static_cast<size_t>(e0 + 2 * min(r, nr - 1)) * d.J2p;
        const float2 *W = ws + h * 2 * NF * JW + p * JW;
        float2 acc[4][NF];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int g = 0; g < NF; ++g) acc[r][g] = make_float2(0.f, 0.f);
        int jt = 0;                                      // first latitude of the scalar tail
        if (VEC) {
            jt = J2 & ~3;
            const int nit = jt > 4 * part ? (jt - 4 * part + 4 * kPrjParts - 1) / (4 * kPrjParts) : 0;
            auto stage_ptr = [&](int it, int r) { return pst + ((it % kPrjDepth) * 4 + r) * blockDim.x + threadIdx.x; };
            auto issue = [&](int it) {
                if (it < nit) {
#pragma unroll
                    for (int r = 0; r < 4; ++r) cp_async16(stage_ptr(it, r), pr[r] + 4 * part + 4 * kPrjParts * it);
                }
                cp_async_commit();                       // one group per block index, possibly empty
            };
            if (ASYNC) {
#pragma unroll
                for (int it = 0; it < kPrjDepth - 1; ++it) issue(it);
            }
            for (int it = 0; it < nit; ++it) {
                const int j = 4 * part + 4 * kPrjParts * it;
                float pv[4][4];
                if (ASYNC) {
                    issue(it + kPrjDepth - 1);
                    cp_async_wait<kPrjDepth - 1>();      // block index it has landed
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const float4 v = ASYNC ? *stage_ptr(it, r) : *reinterpret_cast<const float4 *>(pr[r] + j);
                    pv[r][0] = v.x; pv[r][1] = v.y; pv[r][2] = v.z; pv[r][3] = v.w;
                }
#pragma unroll
                for (int g = 0; g < NF; ++g) {
                    const float4 wa = *reinterpret_cast<const float4 *>(W + g * 2 * JW + j);
                    const float4 wb = *reinterpret_cast<const float4 *>(W + g * 2 * JW + j + 2);
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        acc[r][g] = caxpy(pv[r][0], make_float2(wa.x, wa.y), acc[r][g]);
                        acc[r][g] = caxpy(pv[r][1], make_float2(wa.z, wa.w), acc[r][g]);
                        acc[r][g] = caxpy(pv[r][2], make_float2(wb.x, wb.y), acc[r][g]);
                        acc[r][g] = caxpy(pv[r][3], make_float2(wb.z, wb.w), acc[r][g]);
                    }
                }
            }
        }
        for (int j = jt + part; j < J2; j += kPrjParts) {
            float pv[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) pv[r] = pr[r][j];
#pragma unroll
            for (int g = 0; g < NF; ++g) {
                const float2 w = W[g * 2 * JW + j];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    acc[r][g].x = fmaf(pv[r], w.x, acc[r][g].x);
                    acc[r][g].y = fmaf(pv[r], w.y, acc[r][g].y);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int g = 0; g < NF; ++g)
#pragma unroll
                for (int o = 1; o < kPrjParts; o <<= 1) {
                    acc[r][g].x += __shfl_xor_sync(0xffffffffu, acc[r][g].x, o);
                    acc[r][g].y += __shfl_xor_sync(0xffffffffu, acc[r][g].y, o);
                }
        if (active && part == 0) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if (r >= nr) break;
                float2 *o = y + (static_cast<size_t>(b) * d.next + e0 + 2 * r) * NF;
#pragma unroll
                for (int g = 0; g < NF; ++g) o[g] = acc[r][g];
            }
        }
    }
}

// shared memory of a K3a (FP32) block; the per-lane cp.async stages are
// used when the W rows leave room for them (and J2 is even)
static bool project_f32_async(const Dims &d, int nthreads, size_t *bytes, int nf = 5) {
    const size_t w = 2 * 2 * static_cast<size_t>(nf) * project_f32_wstride(d.J2) * sizeof(float2);
    const size_t st = static_cast<size_t>(kPrjDepth) * 4 * nthreads * sizeof(float4);
    const bool async = d.J2 % 2 == 0 && w + st <= 200 * 1024;
    *bytes = async ? w + st : w;
    return async;
}

// threads of a K3a (FP32) block: all row quads of the largest order pair,
// kPrjParts lanes each, at most kPrjMaxThreads (larger pairs take several passes)
static int project_f32_threads(int T) {
    int best = 0;
    for (int m1 = 0; m1 <= T - m1; ++m1) {
        int nq = 0;
        for (int m : {m1, T - m1}) {
            if (m == T - m1 && T - m1 == m1) break;
            for (int p = 0; p < 2; ++p) nq += ((T + 3 - m - p) / 2 + 3) / 4;
        }
        best = best > nq ? best : nq;
    }
    const int t = (best * kPrjParts + 31) / 32 * 32;
    return t < kPrjMaxThreads ? t : kPrjMaxThreads;
}

// ---------------------------------------------------------------------------
// K3b: per spectral mode (n, m), the vector epilogue of epilogue.cuh.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k3_epilogue(const V2<R> *__restrict__ y, Dims d, const double *__restrict__ eps,
                            const double *__restrict__ lam, const float *__restrict__ epi32,
                            const int *__restrict__ coef_m, double2 *__restrict__ tend, long long tstride) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (i >= d.ncoef) return;
    double2 tp, tz, td;
    vector_epilogue<R>(y + static_cast<size_t>(b) * d.next * 5, d, i, coef_m[i], eps, lam, epi32, tp, tz, td);
    double2 *out = tend + b * tstride;
    out[F_PHI * d.ncoef + i] = tp;
    out[F_ZETA * d.ncoef + i] = tz;
    out[F_DIV * d.ncoef + i] = td;
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
__global__ void k_scalar_ring_inverse(const double2 *__restrict__ f1, double *__restrict__ grid, Dims d,
                                      FftPlan plan, const double2 *__restrict__ tw);
__global__ void k_scalar_ring_forward(const double *__restrict__ grid, double2 *__restrict__ f2, Dims d,
                                      FftPlan plan, const double2 *__restrict__ tw,
                                      const double *__restrict__ w);
constexpr int kK1Threads = 64;
constexpr int kK2Threads = 256;
constexpr int kK3Threads = 64;

template <typename R>
static cudaError_t configure(const Dims &d, const FftPlan &plan) {
    // the Stockham ring of this precision (used in FP64 mode) may not fit for the
    // longest rings; sdc_create refuses FP64 contexts in that case
    const size_t sm2 = ring_smem_bytes(plan.L, sizeof(V2<R>), nullptr);
    cudaError_t e = cudaSuccess;
    if (sm2 != 0) e = cudaFuncSetAttribute(k2_ring<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
    if (e != cudaSuccess) return e;

    e = cudaFuncSetAttribute(k1_synthesis<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(static_cast<size_t>(d.T + 4) * 4 * sizeof(V2<R>)));
    if (e != cudaSuccess || sizeof(R) != sizeof(float)) return e;
    const int smr = (int)ring_f32_smem_bytes(plan.L, plan.L);
    for (const void *f : {(const void *)k2_ring_f32<0>, (const void *)k2_ring_f32<96>, (const void *)k2_ring_f32<192>,
                          (const void *)k2_ring_f32<384>, (const void *)k2_ring_f32<768>,
                          (const void *)k2_ring_f32<1536>}) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smr);
        if (e != cudaSuccess) return e;
    }
    const int sms = (int)synthesis_f32_smem(d, synthesis_f32_stages(d.J2p), 4);
    const int sms5 = (int)synthesis_f32_smem(d, synthesis_f32_stages(d.J2p), 5);
    for (const void *f : {(const void *)k1_synthesis_f32<2, 4>, (const void *)k1_synthesis_f32<1, 4>}) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, sms);
        if (e != cudaSuccess) return e;
    }
    for (const void *f : {(const void *)k1_synthesis_f32<2, 5>, (const void *)k1_synthesis_f32<1, 5>}) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, sms5);
        if (e != cudaSuccess) return e;
    }
    {
        const void *fs[2][2][3] = {
            {{(const void *)k1_synthesis_f32_nb<1, 1, 4>, (const void *)k1_synthesis_f32_nb<2, 1, 4>,
              (const void *)k1_synthesis_f32_nb<4, 1, 4>},
             {(const void *)k1_synthesis_f32_nb<1, 2, 4>, (const void *)k1_synthesis_f32_nb<2, 2, 4>,
              (const void *)k1_synthesis_f32_nb<4, 2, 4>}},
            {{(const void *)k1_synthesis_f32_nb<1, 1, 5>, (const void *)k1_synthesis_f32_nb<2, 1, 5>, nullptr},
             {(const void *)k1_synthesis_f32_nb<1, 2, 5>, (const void *)k1_synthesis_f32_nb<2, 2, 5>, nullptr}}};
        // the recurrence variants of the synthesis (NF = 4) use the same shared memory
        const void *fr[2][3] = {{(const void *)k1_synthesis_f32_nb<1, 1, 4, true>,
                                 (const void *)k1_synthesis_f32_nb<2, 1, 4, true>,
                                 (const void *)k1_synthesis_f32_nb<4, 1, 4, true>},
                                {(const void *)k1_synthesis_f32_nb<1, 2, 4, true>,
                                 (const void *)k1_synthesis_f32_nb<2, 2, 4, true>,
                                 (const void *)k1_synthesis_f32_nb<4, 2, 4, true>}};
        for (int fi = 0; fi < 2; ++fi)
            for (int k = 0; k < 3 - fi; ++k) {
                if (!synthesis_nb_fits(d, 1 << k, 4 + fi)) continue;
                for (int si = 0; si < 2; ++si) {
                    const int bytes = (int)synthesis_nb_smem(d, 1 << k, 4 + fi);
                    e = cudaFuncSetAttribute(fs[fi][si][k], cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
                    if (e == cudaSuccess && fi == 0)
                        e = cudaFuncSetAttribute(fr[si][k], cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
                    if (e != cudaSuccess) return e;
                }
            }
    }
    size_t smp = 0, smq = 0;
    project_f32_async(d, project_f32_threads(d.T), &smp, 5);
    project_f32_async(d, project_f32_threads(d.T), &smq, 4);
    for (const void *f : {(const void *)k3_project_f32<true, true, 5>, (const void *)k3_project_f32<true, false, 5>,
                          (const void *)k3_project_f32<false, false, 5>}) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smp);
        if (e != cudaSuccess) return e;
    }
    for (const void *f : {(const void *)k3_project_f32<true, true, 4>, (const void *)k3_project_f32<true, false, 4>,
                          (const void *)k3_project_f32<false, false, 4>}) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smq);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Batched FP32 synthesis (NF = 4) or projection transpose (NF = 5): NB = 4
// states per block where it fits (else 2), 1 for a single state; S = 2 lane
// pairs per latitude pair where the block stays within kSynNbMaxThreads.
template <int NF>
static cudaError_t launch_synthesis_nb(const Dims &d, int B, const double2 *states, long long sstride,
                                       const float2 *ybar, const float *pbar, const float *syn32, float2 *f1,
                                       int *err, cudaStream_t s, const DeviceTables *rec = nullptr) {
    const bool pdl = NF == 4 && rec && rec->pdl;          // the adjoint's transpose (NF = 5) waits for nothing
    // NF = 5 keeps NB <= 2: four states' 40 accumulators and coefficient rows exceed the registers
    const int nb = B == 1 ? 1 : ((NF == 5 || B == 2 || !synthesis_nb_fits(d, 4, NF)) ? 2 : 4);
    const int S = synthesis_nb_s(d.J2);
    const dim3 g((d.T + 2) / 2, (B + nb - 1) / nb);
    const int nt = synthesis_nb_threads(d.J2, S), ns = synthesis_nb_stages(d, nb, NF), cr = synthesis_nb_rows(d, nb, NF);
    const size_t sm = synthesis_nb_smem(d, nb, NF);
    const float4 *sy = reinterpret_cast<const float4 *>(syn32);
    // the recurrence needs a thread per latitude (the block always has at least J2 + 1 threads)
    cudaError_t e = cudaSuccess;
    if constexpr (NF == 4) {
        if (rec && rec->rec_ab && nt >= d.J2p) {
#define SDC_SYN_REC(NBV, SV)                                                                              \
    e = launch_k(pdl, k1_synthesis_f32_nb<NBV, SV, 4, true>, g, dim3(nt), sm, s, states, sstride, ybar, B, d, \
                 pbar, sy, f1, ns, cr, err, rec->rec_ab, rec->rec_seed, rec->rec_mu)
            if (S == 2) {
                if (nb == 1) SDC_SYN_REC(1, 2);
                else if (nb == 2) SDC_SYN_REC(2, 2);
                else SDC_SYN_REC(4, 2);
            } else {
                if (nb == 1) SDC_SYN_REC(1, 1);
                else if (nb == 2) SDC_SYN_REC(2, 1);
                else SDC_SYN_REC(4, 1);
            }
#undef SDC_SYN_REC
            if (e != cudaSuccess) return e;
            return cudaGetLastError();
        }
    }
#define SDC_SYN_NB(NBV, SV)                                                                                   \
    e = launch_k(pdl, k1_synthesis_f32_nb<NBV, SV, NF, false>, g, dim3(nt), sm, s, states, sstride, ybar, B, d, pbar, \
                 sy, f1, ns, cr, err, static_cast<const float4 *>(nullptr), static_cast<const float4 *>(nullptr),   \
                 static_cast<const float2 *>(nullptr))
    if (S == 2) {
        if (nb == 1) SDC_SYN_NB(1, 2);
        else if (nb == 2) SDC_SYN_NB(2, 2);
        else if constexpr (NF == 4) SDC_SYN_NB(4, 2);
    } else {
        if (nb == 1) SDC_SYN_NB(1, 1);
        else if (nb == 2) SDC_SYN_NB(2, 1);
        else if constexpr (NF == 4) SDC_SYN_NB(4, 1);
    }
#undef SDC_SYN_NB
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <typename R>
static cudaError_t launch_tendency_t(const Dims &d, const FftPlan &plan, int B, const double2 *states,
                                     long long sstride, double2 *tend, long long tstride, const DeviceTables &tb,
                                     const Workspace &ws, cudaStream_t s, int *launches, StageTimer *timer,
                                     void *grid_store, const TcTables *tc) {
    const R *pbar = static_cast<const R *>(tb.pbar);
    const V2<R> *tw = static_cast<const V2<R> *>(tb.tw);
    V2<R> *f1 = static_cast<V2<R> *>(ws.f1);
    V2<R> *f2 = static_cast<V2<R> *>(ws.f2);
    V2<R> *f3 = static_cast<V2<R> *>(ws.f3);
    const size_t sm1 = static_cast<size_t>(d.T + 4) * 4 * sizeof(V2<R>);
    dim3 g1((d.T + 2) / 2, B, (d.J2 + kK1Threads - 1) / kK1Threads);
    int nscratch = 0;
    const size_t sm2 = ring_smem_bytes(d.L, sizeof(V2<R>), &nscratch);
    if (sm2 == 0) return cudaErrorInvalidValue;
    if (timer) timer->mark(STAGE_SYNTH);
    if constexpr (sizeof(R) == sizeof(float)) {
        if (tc) {
            cudaError_t e = launch_tc_synthesis(*tc, d, B, states, sstride, tb.syn, tb.row_m, f1, s, launches);
            if (e != cudaSuccess) return e;
        } else if (synthesis_nb_fits(d, 2, 4)) {
            const cudaError_t e =
                launch_synthesis_nb<4>(d, B, states, sstride, nullptr, pbar, tb.syn32, f1, tb.err, s, &tb);
            if (e != cudaSuccess) return e;
            if (launches) ++*launches;
        } else {
            const int g4 = (d.J2 + 3) / 4;
            const dim3 gs(B, (d.T + 2) / 2);
            const int ns = synthesis_f32_stages(d.J2p);
            const size_t smk = synthesis_f32_smem(d, ns);
            if (g4 <= 128)
                k1_synthesis_f32<2, 4><<<gs, (g4 * 2 + 31) / 32 * 32, smk, s>>>(states, sstride, nullptr, d, pbar,
                                                                              tb.syn, f1, ns, tb.err);
            else
                k1_synthesis_f32<1, 4><<<gs, (g4 + 31) / 32 * 32, smk, s>>>(states, sstride, nullptr, d, pbar, tb.syn,
                                                                          f1, ns, tb.err);
            if (launches) ++*launches;
        }
    } else {
        k1_synthesis<R><<<g1, kK1Threads, sm1, s>>>(states, sstride, d, pbar, tb.syn, f1);
        if (launches) ++*launches;
    }
    if (timer) timer->mark(STAGE_RING);
    if constexpr (sizeof(R) == sizeof(float)) {
        const dim3 g2(d.J2, B);
        const size_t sm = ring_f32_smem_bytes(d.L, tb.ntwp);
        float2 *gsr = static_cast<float2 *>(grid_store);
        cudaError_t e = cudaSuccess;
#define SDC_RING_F32(LC)                                                                                            \
    e = launch_k(tb.pdl, k2_ring_f32<LC>, g2, dim3(kK2Threads), sm, s, static_cast<const float2 *>(f1), f2, d, tb.plan16, \
                 tb.twp32, tb.ntwp, tb.ring32, gsr)
        switch (d.L) {
            case 96: SDC_RING_F32(96); break;
            case 192: SDC_RING_F32(192); break;
            case 384: SDC_RING_F32(384); break;
            case 768: SDC_RING_F32(768); break;
            case 1536: SDC_RING_F32(1536); break;
            default: SDC_RING_F32(0); break;
        }
#undef SDC_RING_F32
        if (e != cudaSuccess) return e;
    } else {
        k2_ring<R><<<dim3(d.J2, B), kK2Threads, sm2, s>>>(f1, f2, d, plan, tw, tb.ring64, nscratch,
                                                         static_cast<V2<R> *>(grid_store));
    }
    if (timer) timer->mark(STAGE_ANALYSIS);
    if constexpr (sizeof(R) == sizeof(float)) {
        if (tc) {
            cudaError_t e = launch_tc_projection(*tc, d, B, f2, f3, s, launches);
            if (e != cudaSuccess) return e;
        } else {
            const dim3 g3(B, (d.T + 2) / 2);
            const int nt = project_f32_threads(d.T);
            size_t smp = 0;
            const bool async = project_f32_async(d, nt, &smp);
            const float2 *f2c = f2;
            cudaError_t e;
            if (d.J2 % 2 != 0) e = launch_k(tb.pdl, k3_project_f32<false, false, 5>, g3, dim3(nt), smp, s, f2c, d, pbar, f3);
            else if (async) e = launch_k(tb.pdl, k3_project_f32<true, true, 5>, g3, dim3(nt), smp, s, f2c, d, pbar, f3);
            else e = launch_k(tb.pdl, k3_project_f32<true, false, 5>, g3, dim3(nt), smp, s, f2c, d, pbar, f3);
            if (e != cudaSuccess) return e;
            if (launches) ++*launches;
        }
    } else {
        k3_project<R><<<dim3((d.next + kK3Threads - 1) / kK3Threads, B), kK3Threads, 0, s>>>(f2, d, pbar, tb.row_m,
                                                                                              f3);
        if (launches) ++*launches;
    }
    if (tend) {
        if (timer) timer->mark(STAGE_EPILOGUE);
        k3_epilogue<R><<<dim3((d.ncoef + 127) / 128, B), 128, 0, s>>>(f3, d, tb.eps, tb.lam, tb.epi32, tb.coef_m,
                                                                      tend, tstride);
    }
    if (launches) *launches += tend ? 2 : 1;       // ring (+ epilogue)
    return cudaGetLastError();
}

cudaError_t configure_transform_kernels(const Dims &d, const FftPlan &plan, bool fp32) {
    cudaError_t e = fp32 ? configure<float>(d, plan) : configure<double>(d, plan);
    if (e != cudaSuccess) return e;
    const size_t sm = 2 * static_cast<size_t>(plan.L) * sizeof(double2);
    e = cudaFuncSetAttribute(k_scalar_ring_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_scalar_ring_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

cudaError_t launch_projection_transpose_f32(const Dims &d, int B, const float2 *ybar, const float *pbar,
                                            float2 *wbar, int *err, cudaStream_t s) {
    if (synthesis_nb_fits(d, 2, 5)) return launch_synthesis_nb<5>(d, B, nullptr, 0, ybar, pbar, nullptr, wbar, err, s);
    const int g4 = (d.J2 + 3) / 4;
    const dim3 gs(B, (d.T + 2) / 2);
    const int ns = synthesis_f32_stages(d.J2p);
    const size_t smk = synthesis_f32_smem(d, ns, 5);
    if (g4 <= 128)
        k1_synthesis_f32<2, 5><<<gs, (g4 * 2 + 31) / 32 * 32, smk, s>>>(nullptr, 0, ybar, d, pbar, nullptr, wbar,
                                                                      ns, err);
    else
        k1_synthesis_f32<1, 5><<<gs, (g4 + 31) / 32 * 32, smk, s>>>(nullptr, 0, ybar, d, pbar, nullptr, wbar, ns,
                                                                  err);
    return cudaGetLastError();
}

cudaError_t launch_synthesis_transpose_f32(const Dims &d, int B, const float2 *f1bar, const float *pbar, float2 *zbar,
                                           cudaStream_t s) {
    const dim3 g3(B, (d.T + 2) / 2);
    const int nt = project_f32_threads(d.T);
    size_t smp = 0;
    const bool async = project_f32_async(d, nt, &smp, 4);
    if (d.J2 % 2 != 0) k3_project_f32<false, false, 4><<<g3, nt, smp, s>>>(f1bar, d, pbar, zbar);
    else if (async) k3_project_f32<true, true, 4><<<g3, nt, smp, s>>>(f1bar, d, pbar, zbar);
    else k3_project_f32<true, false, 4><<<g3, nt, smp, s>>>(f1bar, d, pbar, zbar);
    return cudaGetLastError();
}

cudaError_t launch_tendency(const Dims &d, const FftPlan &plan, bool fp32, int B, const double2 *states,
                            long long sstride, double2 *tend, long long tstride, const DeviceTables &tb,
                            const Workspace &ws, cudaStream_t s, int *launches, StageTimer *timer,
                            void *grid_store, const TcTables *tc) {
    if (fp32)
        return launch_tendency_t<float>(d, plan, B, states, sstride, tend, tstride, tb, ws, s, launches, timer,
                                        grid_store, tc);
    return launch_tendency_t<double>(d, plan, B, states, sstride, tend, tstride, tb, ws, s, launches, timer,
                                     grid_store, nullptr);
}

// ---------------------------------------------------------------------------
// Scalar transforms (FP64), for initial states and grid diagnostics.
// ---------------------------------------------------------------------------
__global__ void k_scalar_synthesis(const double2 *__restrict__ spec, Dims d, const double *__restrict__ pbar,
                                   double2 *__restrict__ f1) {
    const int m = blockIdx.x;
    const int j = blockIdx.y * blockDim.x + threadIdx.x;
    if (j >= d.J2) return;
    const int T = d.T, nn = T + 1 - m;
    const int off = order_offset(T, m), eoff = ext_offset(T, m);
    double2 se = make_double2(0, 0), so = se;
    for (int t = 0; t < nn; ++t) {
        const double p = pbar[static_cast<size_t>(eoff + t) * d.J2p + j];
        const double2 c = spec[off + t];
        if (t & 1) { so.x = fma(p, c.x, so.x); so.y = fma(p, c.y, so.y); }
        else { se.x = fma(p, c.x, se.x); se.y = fma(p, c.y, se.y); }
    }
    f1[(static_cast<size_t>(j) * 2 + 0) * (T + 1) + m] = se;
    f1[(static_cast<size_t>(j) * 2 + 1) * (T + 1) + m] = so;
}

__global__ void k_scalar_ring_inverse(const double2 *__restrict__ f1, double *__restrict__ grid, Dims d,
                                      FftPlan plan, const double2 *__restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *X = reinterpret_cast<double2 *>(smem_raw);
    double2 *S = X + plan.L;
    const int j2 = blockIdx.x, T = d.T, L = plan.L;
    const double2 *in = f1 + static_cast<size_t>(j2) * 2 * (T + 1);
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        double2 z = make_double2(0, 0);
        int m = -1;
        bool conj = false;
        if (k <= T) m = k;
        else if (k >= L - T) { m = L - k; conj = true; }
        if (m >= 0) {
            double2 e = in[m], o = in[(T + 1) + m];
            if (m == 0) { e.y = 0; o.y = 0; }
            double2 n = make_double2(e.x + o.x, e.y + o.y), s = make_double2(e.x - o.x, e.y - o.y);
            if (conj) { n.y = -n.y; s.y = -s.y; }
            z = make_double2(n.x - s.y, n.y + s.x);
        }
        X[k] = z;
    }
    __syncthreads();
    fft_inplace<double>(X, S, 1, 1, plan, tw, true);
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        grid[static_cast<size_t>(j2) * L + k] = X[k].x;
        grid[static_cast<size_t>(d.J - 1 - j2) * L + k] = X[k].y;
    }
}

__global__ void k_scalar_ring_forward(const double *__restrict__ grid, double2 *__restrict__ f2, Dims d,
                                      FftPlan plan, const double2 *__restrict__ tw,
                                      const double *__restrict__ w) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *X = reinterpret_cast<double2 *>(smem_raw);
    double2 *S = X + plan.L;
    const int j2 = blockIdx.x, T = d.T, L = plan.L;
    for (int k = threadIdx.x; k < L; k += blockDim.x)
        X[k] = make_double2(grid[static_cast<size_t>(j2) * L + k], grid[static_cast<size_t>(d.J - 1 - j2) * L + k]);
    __syncthreads();
    fft_inplace<double>(X, S, 1, 1, plan, tw, false);
    const double wj = w[j2], invL = 1.0 / L;
    for (int m = threadIdx.x; m <= T; m += blockDim.x) {
        const double2 y = X[m];
        double2 yc = X[m == 0 ? 0 : L - m];
        yc.y = -yc.y;
        const double2 gn = make_double2(0.5 * invL * (y.x + yc.x), 0.5 * invL * (y.y + yc.y));
        const double2 gs = make_double2(0.5 * invL * (y.y - yc.y), -0.5 * invL * (y.x - yc.x));
        f2[(static_cast<size_t>(m) * 2 + 0) * d.J2 + j2] = make_double2(wj * (gn.x + gs.x), wj * (gn.y + gs.y));
        f2[(static_cast<size_t>(m) * 2 + 1) * d.J2 + j2] = make_double2(wj * (gn.x - gs.x), wj * (gn.y - gs.y));
    }
}

__global__ void k_scalar_analysis(const double2 *__restrict__ f2, Dims d, const double *__restrict__ pbar,
                                  double2 *__restrict__ spec) {
    const int m = blockIdx.x, T = d.T;
    const int off = order_offset(T, m), eoff = ext_offset(T, m);
    for (int t = threadIdx.x; t <= T - m; t += blockDim.x) {
        const double2 *W = f2 + (static_cast<size_t>(m) * 2 + (t & 1)) * d.J2;
        const double *prow = pbar + static_cast<size_t>(eoff + t) * d.J2p;
        double2 acc = make_double2(0, 0);
        for (int j = 0; j < d.J2; ++j) {
            acc.x = fma(prow[j], W[j].x, acc.x);
            acc.y = fma(prow[j], W[j].y, acc.y);
        }
        spec[off + t] = acc;
    }
}

cudaError_t launch_spec_to_grid(const Dims &d, const FftPlan &plan, const double2 *spec, double *grid,
                                const double *pbar, const double2 *tw, double2 *f1, cudaStream_t s) {
    k_scalar_synthesis<<<dim3(d.T + 1, (d.J2 + 63) / 64), 64, 0, s>>>(spec, d, pbar, f1);
    const size_t sm = 2 * static_cast<size_t>(plan.L) * sizeof(double2);
    k_scalar_ring_inverse<<<d.J2, 256, sm, s>>>(f1, grid, d, plan, tw);
    return cudaGetLastError();
}

cudaError_t launch_grid_to_spec(const Dims &d, const FftPlan &plan, const double *grid, double2 *spec,
                                const double *pbar, const double *w, const double2 *tw, double2 *f2,
                                cudaStream_t s) {
    const size_t sm = 2 * static_cast<size_t>(plan.L) * sizeof(double2);
    k_scalar_ring_forward<<<d.J2, 256, sm, s>>>(grid, f2, d, plan, tw, w);
    k_scalar_analysis<<<d.T + 1, 128, 0, s>>>(f2, d, pbar, spec);
    return cudaGetLastError();
}

}  // namespace sdc
