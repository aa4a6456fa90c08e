// Checks the integer-pipe FP64 <-> FP32 conversions of convert.cuh against the
// hardware conversions, bit for bit: every binary32 value for the widening,
// and a seeded sample of binary64 values (concentrated on the binary32 range,
// with exact and near ties in the rounded-away bits) plus listed edge cases
// for the rounding.  Prints the mismatch counts; exit status 1 on any.
#include <cfloat>
#include <cmath>
#include <cstdio>

#include "convert.cuh"

using sdc::f32_to_f64;
using sdc::f64_to_f32_rn;

__device__ unsigned long long mix64(unsigned long long z) {    // SplitMix64 output function
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ bool same_f64(double a, double b) {
    return __double_as_longlong(a) == __double_as_longlong(b) || (isnan(a) && isnan(b));
}
__device__ bool same_f32(float a, float b) { return __float_as_uint(a) == __float_as_uint(b) || (isnan(a) && isnan(b)); }

__global__ void widen_all(unsigned long long *bad) {
    const unsigned long long stride = static_cast<unsigned long long>(gridDim.x) * blockDim.x;
    unsigned long long nbad = 0;
    for (unsigned long long i = blockIdx.x * blockDim.x + threadIdx.x; i < (1ull << 32); i += stride) {
        const float x = __uint_as_float(static_cast<unsigned>(i));
        nbad += same_f64(f32_to_f64(x), static_cast<double>(x)) ? 0 : 1;
    }
    if (nbad) atomicAdd(bad, nbad);
}

__global__ void narrow_sample(unsigned long long n, unsigned long long *bad) {
    const unsigned long long stride = static_cast<unsigned long long>(gridDim.x) * blockDim.x;
    const unsigned long long low29 = (1ull << 29) - 1, frac52 = (1ull << 52) - 1;
    unsigned long long nbad = 0;
    for (unsigned long long i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned long long r = mix64(i), s = mix64(r);
        const unsigned long long e = 1023 - 160 + s % 300;            // around the binary32 exponent range
        unsigned long long frac = r & frac52;
        switch (i & 7) {
            case 1: frac = (frac & ~low29) | (1ull << 28); break;         // exact tie
            case 2: frac = (frac & ~low29) | ((1ull << 28) - 1); break;   // just below a tie
            case 3: frac = (frac & ~low29) | ((1ull << 28) + 1); break;   // just above a tie
            case 4: frac = frac52 - (s >> 40 & 0xff); break;              // carries into the exponent
            default: break;
        }
        const double x = __longlong_as_double(static_cast<long long>(((r >> 63) << 63) | (e << 52) | frac));
        nbad += same_f32(f64_to_f32_rn(x), __double2float_rn(x)) ? 0 : 1;
    }
    if (nbad) atomicAdd(bad, nbad);
}

__global__ void narrow_list(const double *x, int n, unsigned long long *bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !same_f32(f64_to_f32_rn(x[i]), __double2float_rn(x[i]))) atomicAdd(bad, 1ull);
}

int main() {
    const double fmax = FLT_MAX;
    const double edges[] = {0.0, -0.0, 1.0, -1.0, fmax, -fmax, std::nextafter(fmax, INFINITY),
                            fmax + std::ldexp(1.0, 103), std::nextafter(fmax + std::ldexp(1.0, 103), 0.0),
                            FLT_MIN, -FLT_MIN, std::nextafter(static_cast<double>(FLT_MIN), 0.0), FLT_MIN / 2,
                            std::ldexp(1.0, -149), std::ldexp(1.0, -150), DBL_MIN, DBL_TRUE_MIN, -DBL_TRUE_MIN,
                            INFINITY, -INFINITY, NAN, 1e300, -1e-300, 3.0e38, 3.5e38};
    const int ne = sizeof(edges) / sizeof(edges[0]);
    unsigned long long *bad = nullptr;
    double *dx = nullptr;
    if (cudaMalloc(&bad, 3 * sizeof(unsigned long long)) != cudaSuccess) return 2;
    if (cudaMalloc(&dx, sizeof(edges)) != cudaSuccess) return 2;
    cudaMemset(bad, 0, 3 * sizeof(unsigned long long));
    cudaMemcpy(dx, edges, sizeof(edges), cudaMemcpyHostToDevice);
    widen_all<<<152 * 8, 256>>>(bad);
    narrow_sample<<<152 * 8, 256>>>(1ull << 28, bad + 1);
    narrow_list<<<1, 32>>>(dx, ne, bad + 2);
    unsigned long long h[3] = {0, 0, 0};
    const cudaError_t e = cudaMemcpy(h, bad, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        std::printf("cuda error %s\n", cudaGetErrorString(e));
        return 2;
    }
    std::printf("f32_to_f64 mismatches %llu\nf64_to_f32_rn mismatches %llu sample, %llu edge\n", h[0], h[1], h[2]);
    cudaFree(bad);
    cudaFree(dx);
    return (h[0] || h[1] || h[2]) ? 1 : 0;
}
