// The vector epilogue of the explicit tendency for one spectral mode (device
// code only), shared by the standalone epilogue kernel and the sweep kernel
// that consumes the projections directly.  For mode (n, m), n = m..T, with
// the projections A^, B^, C^, D^, E^ of the extended rows n' = n - 1, n, n + 1
// (1/a folded in here):
//   T_E(zeta)_n = -(1/a) [i m A^_n + n eps_{n+1} B^_{n+1} - (n+1) eps_n B^_{n-1}]
//   T_E(div)_n  =  (1/a) [i m B^_n - n eps_{n+1} A^_{n+1} + (n+1) eps_n A^_{n-1}] + lambda_n E^_n
//   T_E(Phi')_n = -(1/a) [i m C^_n + n eps_{n+1} D^_{n+1} - (n+1) eps_n D^_{n-1}]
// The arithmetic runs in R (FP32 in the mixed modes, with the per-mode
// factors from an FP32 table); the result is returned in FP64.
#pragma once

#include "convert.cuh"
#include "fft.cuh"
#include "sdc_internal.h"

namespace sdc {

template <typename R>
__device__ __forceinline__ void vector_epilogue(const V2<R> *__restrict__ Y, const Dims &d, int i, int m,
                                                const double *__restrict__ eps, const double *__restrict__ lam,
                                                const float *__restrict__ epi32, double2 &tp, double2 &tz,
                                                double2 &td) {
    const int t = i - order_offset(d.T, m);
    const int n = m + t;
    const int e = ext_offset(d.T, m) + t;
    auto ld = [&](int row, int g) -> V2<R> { return Y[static_cast<size_t>(row) * 5 + g]; };
    const V2<R> z0 = mk<R>(0, 0);
    const V2<R> Ah = ld(e, P_A), Bh = ld(e, P_B), Ch = ld(e, P_C), Eh = ld(e, P_E);
    const V2<R> Au = ld(e + 1, P_A), Bu = ld(e + 1, P_B), Du = ld(e + 1, P_D);
    const V2<R> Al = t > 0 ? ld(e - 1, P_A) : z0;
    const V2<R> Bl = t > 0 ? ld(e - 1, P_B) : z0;
    const V2<R> Dl = t > 0 ? ld(e - 1, P_D) : z0;
    R cu, cl, lm;
    if constexpr (sizeof(R) == sizeof(float)) {
        const float4 f = reinterpret_cast<const float4 *>(epi32)[i];
        cu = f.x;
        cl = f.y;
        lm = f.z;
    } else {
        cu = n * eps[e + 1];
        cl = t > 0 ? (n + 1.0) * eps[e] : 0.0;
        lm = lam[i];
    }
    const R inv_a = R(d.inv_a);
    const R mm = R(m);
    // i m X = (-m X.y, m X.x)
    const R tzx = -inv_a * (-mm * Ah.y + cu * Bu.x - cl * Bl.x);
    const R tzy = -inv_a * (mm * Ah.x + cu * Bu.y - cl * Bl.y);
    const R tdx = inv_a * (-mm * Bh.y - cu * Au.x + cl * Al.x) + lm * Eh.x;
    const R tdy = inv_a * (mm * Bh.x - cu * Au.y + cl * Al.y) + lm * Eh.y;
    const R tpx = -inv_a * (-mm * Ch.y + cu * Du.x - cl * Dl.x);
    const R tpy = -inv_a * (mm * Ch.x + cu * Du.y - cl * Dl.y);
    if constexpr (sizeof(R) == sizeof(float)) {       // widened on the integer pipe (convert.cuh)
        tp = make_double2(f32_to_f64(tpx), f32_to_f64(tpy));
        tz = make_double2(f32_to_f64(tzx), f32_to_f64(tzy));
        td = make_double2(f32_to_f64(tdx), f32_to_f64(tdy));
    } else {
        tp = make_double2(tpx, tpy);
        tz = make_double2(tzx, tzy);
        td = make_double2(tdx, tdy);
    }
}

}  // namespace sdc
