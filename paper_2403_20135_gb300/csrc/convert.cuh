// FP64 <-> FP32 conversions on the integer pipe (device code only).
//
// GB300 runs the conversion instructions between binary64 and binary32 on its
// FP64 pipe, which issues about one of them per SM and clock; the
// mixed-precision kernels convert thousands of values per block, so they
// re-encode the bits with integer operations instead, from the IEEE 754
// layouts (binary64: 1 sign, 11 exponent bits with bias 1023, 52 fraction
// bits; binary32: 1, 8 with bias 127, 23).
#pragma once

#include <cuda_runtime.h>

namespace sdc {

// binary64 -> binary32, round to nearest, ties to even.  Integer operations
// only (a hardware fallback, even on a rare branch, gets if-converted into
// every call).
__device__ __forceinline__ float f64_to_f32_rn(double x) {
    const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned hi = static_cast<unsigned>(u >> 32), lo = static_cast<unsigned>(u);
    const unsigned sign = hi & 0x80000000u;
    const int e = static_cast<int>((hi >> 20) & 0x7ffu);
    const int ef = e - 1023 + 127;
    unsigned r;
    if (ef > 0 && ef < 255) {                            // normal binary32 result (or a carry to the next binade)
        const unsigned frac = ((hi & 0xfffffu) << 3) | (lo >> 29);    // the top 23 of 52 fraction bits
        const unsigned rest = lo & 0x1fffffffu;                        // the 29 bits rounded away
        r = sign | (static_cast<unsigned>(ef) << 23) | frac;
        r += (rest > 0x10000000u || (rest == 0x10000000u && (frac & 1u))) ? 1u : 0u;   // carries step the exponent
    } else if (e == 0x7ff) {                             // infinity, NaN (quiet)
        r = sign | 0x7f800000u | (((u << 12) != 0) ? 0x400000u | static_cast<unsigned>((u >> 29) & 0x3fffffu) : 0u);
    } else if (ef >= 255) {                              // beyond the binary32 range: infinity
        r = sign | 0x7f800000u;
    } else {                                             // binary32 subnormal or zero: 53-bit significand shifted
        const int sh = 1 - ef + 29;                      // >= 30; significand units of 2^-149
        const unsigned long long sig = (e == 0) ? 0ull : ((u & 0xfffffffffffffull) | (1ull << 52));
        const unsigned long long q = sh < 64 ? sig >> sh : 0ull;
        const unsigned long long rem = sh < 64 ? sig & ((1ull << sh) - 1) : sig;
        const unsigned long long half = sh < 65 ? 1ull << (sh - 1) : ~0ull;
        r = sign | static_cast<unsigned>(q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull));
    }
    return __uint_as_float(r);
}

// binary32 -> binary64 (exact), integer operations only.
__device__ __forceinline__ double f32_to_f64(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xffu, frac = u & 0x7fffffu;
    unsigned hi, lo;
    if (e != 0 && e != 255) {                            // normal: rebias the exponent, widen the fraction
        hi = sign | ((e + 1023u - 127u) << 20) | (frac >> 3);
        lo = frac << 29;
    } else if (e == 255) {                               // infinity, NaN (payload and quiet bit kept)
        hi = sign | 0x7ff00000u | (frac >> 3);
        lo = frac << 29;
    } else if (frac == 0) {                              // signed zero
        hi = sign;
        lo = 0;
    } else {                                             // subnormal: frac 2^-149, normalised
        const int p = 31 - __clz(static_cast<int>(frac));   // position of the leading bit
        const unsigned long long m = (static_cast<unsigned long long>(frac) << (52 - p)) & 0xfffffffffffffull;
        hi = sign | (static_cast<unsigned>(p + 874) << 20) | static_cast<unsigned>(m >> 32);
        lo = static_cast<unsigned>(m);
    }
    return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
}

}  // namespace sdc
