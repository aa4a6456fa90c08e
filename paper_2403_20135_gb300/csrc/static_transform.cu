// Spectral-to-grid transform of one field that allocates nothing.
//
// Some callers cannot call cudaMalloc: host applications that own every byte
// of device memory through their own allocator and forbid other code from
// allocating, latency-critical loops that cannot afford cudaMalloc/cudaFree
// (which may synchronise the device), and processes under a fixed
// device-memory budget.  They cannot create an sdc_ctx (which allocates its
// tables and workspaces), so this entry point needs no context:
// the Gauss nodes, the normalised Legendre functions and the FFT twiddles are
// computed on the fly, and the only intermediate data -- the Gauss nodes and
// the Fourier coefficients on each latitude between the Legendre stage and
// the FFT stage -- live in one file-scope static device array of fixed size.
//
// That array is shared by every call on a device and keeps the last call's
// contents; every entry a call reads is first written by the same call, so
// nothing needs clearing.  Calls whose work overlaps on the GPU (two streams,
// or two host threads) race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "fft.cuh"
#include "sdc_internal.h"

namespace sdc {

// 2 MiB of scratch, resident on every GPU that loads the library until exit.
constexpr size_t kStaticScratchBytes = size_t(2) << 20;
constexpr size_t kStaticScratchElems = kStaticScratchBytes / sizeof(double2);
static __device__ __align__(256) double2 g_static_scratch[kStaticScratchElems];

namespace {

constexpr int kMaxDevices = 64;
constexpr int kStaticRingThreads = 256;
std::mutex g_setup_mutex;
double2 *g_scratch_addr[kMaxDevices] = {};

// Newton's method in the colatitude for the northern roots of P_J (one thread
// per root), as in the host precompute.
__global__ void k_static_gauss(int J, double *mu) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= J / 2) return;
    double th = M_PI * (i + 0.75) / (J + 0.5);
    for (int it = 0; it < 40; ++it) {
        const double x = cos(th);
        double pm1 = 1.0, pn = x;
        for (int k = 2; k <= J; ++k) {
            const double pk = ((2.0 * k - 1.0) * x * pn - (k - 1.0) * pm1) / k;
            pm1 = pn;
            pn = pk;
        }
        // d/dtheta P_J(cos theta) = -J (P_{J-1} - x P_J) / sin(theta)
        const double delta = pn / (-J * (pm1 - x * pn) / sin(th));
        th -= delta;
        if (fabs(delta) <= 1e-17) break;
    }
    mu[i] = cos(th);
}

// Synthesis of one field on the northern latitudes, split by the parity of
// n - m, with Pbar_n^m(mu_j) generated by its three-term recurrence.
// Output four[j][parity][m].
__global__ void k_static_synthesis(const double2 *__restrict__ spec, int T, int J2,
                                   const double *__restrict__ mu, double2 *__restrict__ four) {
    const int m = blockIdx.x;
    const int j = blockIdx.y * blockDim.x + threadIdx.x;
    if (j >= J2) return;
    const double x = mu[j];
    const double s = sqrt((1.0 - x) * (1.0 + x));
    double pmm = 1.0 / sqrt(2.0);
    for (int k = 1; k <= m; ++k) pmm *= sqrt((2.0 * k + 1.0) / (2.0 * k)) * s;
    const int off = order_offset(T, m);
    double2 se = make_double2(0.0, 0.0), so = se;
    double p2 = 0.0, p1 = pmm, e1 = 0.0;   // Pbar_{n-2}, Pbar_{n-1}, eps_{n-1}
    for (int n = m; n <= T; ++n) {
        double p;
        if (n == m) {
            p = pmm;
        } else {
            const double e = sqrt((double(n) * n - double(m) * m) / (4.0 * n * n - 1.0));
            p = (x * p1 - e1 * p2) / e;
            p2 = p1;
            p1 = p;
            e1 = e;
        }
        const double2 c = spec[off + n - m];
        if ((n - m) & 1) { so.x = fma(p, c.x, so.x); so.y = fma(p, c.y, so.y); }
        else { se.x = fma(p, c.x, se.x); se.y = fma(p, c.y, se.y); }
    }
    four[(static_cast<size_t>(j) * 2 + 0) * (T + 1) + m] = se;
    four[(static_cast<size_t>(j) * 2 + 1) * (T + 1) + m] = so;
}

// One block per latitude pair: the northern and southern rings travel as the
// real and imaginary parts of one inverse FFT; twiddles are generated in
// shared memory.
__global__ void k_static_ring(const double2 *__restrict__ four, double *__restrict__ grid, int T, int J,
                              FftPlan plan) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = plan.L;
    double2 *X = reinterpret_cast<double2 *>(smem_raw);
    double2 *S = X + L;
    double2 *tw = S + L;
    const int j2 = blockIdx.x;
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        double sn, cs;
        sincospi(-2.0 * k / L, &sn, &cs);
        tw[k] = make_double2(cs, sn);
    }
    const double2 *in = four + static_cast<size_t>(j2) * 2 * (T + 1);
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        double2 z = make_double2(0.0, 0.0);
        int m = -1;
        bool conj = false;
        if (k <= T) m = k;
        else if (k >= L - T) { m = L - k; conj = true; }
        if (m >= 0) {
            double2 e = in[m], o = in[(T + 1) + m];
            if (m == 0) { e.y = 0.0; o.y = 0.0; }
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
        grid[static_cast<size_t>(J - 1 - j2) * L + k] = X[k].y;
    }
}

bool is_2a3b(int L) {
    if (L < 1) return false;
    while (L % 2 == 0) L /= 2;
    while (L % 3 == 0) L /= 3;
    return L == 1;
}

// Once per device, with that device current: look up the device address of
// the scratch array (host code may not use the symbol itself as a pointer)
// and raise the ring kernel's shared-memory limit.
int setup_device(double2 **addr) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SDC_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return SDC_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) return SDC_ECUDA;
        const int smem = static_cast<int>(3 * 2304 * sizeof(double2));
        if (cudaFuncSetAttribute(k_static_ring, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
            return SDC_ECUDA;
        g_scratch_addr[dev] = static_cast<double2 *>(p);
    }
    *addr = g_scratch_addr[dev];
    return SDC_OK;
}

}  // namespace
}  // namespace sdc

extern "C" int sdc_spec_to_grid_static(int T, int nlat, int nlon, const void *spec, double *grid,
                                       void *cuda_stream) {
    using namespace sdc;
    if (!spec || !grid) return SDC_EINVAL;
    if (T < 1 || T > 1023) return SDC_EINVAL;
    if (nlat % 2 != 0 || 2 * nlat < 3 * T + 1 || nlat > 2048) return SDC_EINVAL;
    if (!is_2a3b(nlon) || nlon < 3 * T + 1 || nlon > 2304) return SDC_EINVAL;
    const int J2 = nlat / 2;
    // scratch: the nlat/2 northern Gauss nodes (two doubles per double2 slot),
    // then the Fourier coefficients [nlat/2][2 parities][T+1]
    const size_t mu_slots = (static_cast<size_t>(J2) + 1) / 2;
    const size_t four_slots = static_cast<size_t>(J2) * 2 * (T + 1);
    if (mu_slots + four_slots > kStaticScratchElems) return SDC_EUNSUPPORTED;
    FftPlan plan{};
    if (!fft_plan(nlon, plan)) return SDC_EINVAL;
    // an error left pending by earlier work is the caller's: report it without
    // clearing it, so that the launches below are checked on their own
    if (cudaPeekAtLastError() != cudaSuccess) return SDC_ECUDA;
    double2 *scratch = nullptr;
    int st = setup_device(&scratch);
    if (st != SDC_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    double *mu = reinterpret_cast<double *>(scratch);
    double2 *four = scratch + mu_slots;
    k_static_gauss<<<(J2 + 127) / 128, 128, 0, s>>>(nlat, mu);
    k_static_synthesis<<<dim3(T + 1, (J2 + 63) / 64), 64, 0, s>>>(static_cast<const double2 *>(spec), T, J2, mu,
                                                                  four);
    k_static_ring<<<J2, kStaticRingThreads, 3 * static_cast<size_t>(nlon) * sizeof(double2), s>>>(four, grid, T,
                                                                                                  nlat, plan);
    if (cudaGetLastError() != cudaSuccess) return SDC_ECUDA;
    return SDC_OK;
}
