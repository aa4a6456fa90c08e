// K4: fused collocation quadrature, diagonal implicit solve and residual
// partial sums of one sweep (Eq. (7) with the solver form Eq. (8)), for every
// node of the sweep at once -- the paper's parallel node loop of Algorithm 2
// becomes G = M (rounded up to a power of two) neighbouring lanes per
// spectral mode, lane m owning node m.
//
// Per mode (n, m) with lambda_n = n(n+1)/a^2 and F_j = L_g(u_j^k) + T_E(u_j^k):
//   R_m   = u_n + dt sum_j q_{m,j} F_j                   (collocation right side)
//   rhs_m = R_m - alpha_m L_g(u_m^k),  alpha_m = dt q^Delta_{m,m}
//   (I - alpha_m L_g) u_m^{k+1} = rhs_m, in closed form (the denominators
//   1 / (1 + alpha_m^2 Phibar lambda_n) of the sweep come from a host table) for
//   L_g(Phi', zeta, div) = (-Phibar div, 0, lambda_n Phi'):
//     Phi' = (rhs_Phi - alpha Phibar rhs_div) / (1 + alpha^2 Phibar lambda_n)
//     div  = rhs_div + alpha lambda_n Phi',  zeta = rhs_zeta
//   residual R_m - u_m^k accumulated as sum w |r|^2 (w = 1 at m = 0, else 2).
// Lane j forms F_j (T_E(u_j^k) from the projections of the preceding tendency
// batch by the vector epilogue of epilogue.cuh, in the transform precision;
// on the first sweep every node's T_E is that of u_n, formed once by lane 0);
// the quadrature rows take the F_j of the group by warp shuffles.  All other
// arithmetic is FP64.  Spreading the nodes over lanes gives the FP64 pipe G
// times the warps of a thread-per-mode layout to hide its latency.
#include <cuda_runtime.h>

#include "async_copy.cuh"
#include "epilogue.cuh"
#include "sdc_internal.h"

namespace sdc {

constexpr int kSweepThreads = 128;

__host__ __device__ constexpr int sweep_lanes(int M) { return M <= 1 ? 1 : (M <= 2 ? 2 : (M <= 4 ? 4 : 8)); }

int sweep_blocks(int ncoef, int M) {
    return static_cast<int>((static_cast<long long>(ncoef) * sweep_lanes(M) + kSweepThreads - 1) / kSweepThreads);
}

__device__ __forceinline__ double2 shfl2(double2 v, int src) {
    return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

template <int M, bool RESID, typename R>
__global__ void __launch_bounds__(kSweepThreads) k4_sweep(SweepParams p) {
    // the sweep's successors (the next batch's synthesis) may be scheduled as
    // soon as every sweep block runs: they prefetch constant tables while
    // the sweep drains, and wait for its completion before reading its output
    pdl_release();
    pdl_wait();                                           // everything below reads the preceding kernels' results
    constexpr int G = sweep_lanes(M);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int nc = p.ncoef;
    const int i = t / G;                                  // spectral mode
    const int m = t - i * G;                              // node of this lane (m >= M: idle)
    const int ic = i < nc ? i : nc - 1;                   // lanes past the end compute on a valid mode, store nothing
    const int mr = m < M ? m : M - 1;
    const int lane = threadIdx.x & 31;
    const int g0 = lane - m;                              // lane of node 0 of this group
    const double lam = p.lam[ic];
    const int mo = p.coef_m[ic];
    const V2<R> *Y = static_cast<const V2<R> *>(p.y);

    // F of this lane's node
    const double2 *u = p.ubase + mr * p.ustride;
    const double2 up = u[F_PHI * nc + ic], uz = u[F_ZETA * nc + ic], ud = u[F_DIV * nc + ic];
    double2 ep = make_double2(0.0, 0.0), ez = ep, ed = ep;
    if (p.ybatch == 1) {                                  // first sweep: T_E(u_n) for every node
        if (m == 0) vector_epilogue<R>(Y, p.dims, ic, mo, p.eps, p.lam, p.epi32, ep, ez, ed);
        ep = shfl2(ep, g0);
        ez = shfl2(ez, g0);
        ed = shfl2(ed, g0);
    } else {
        vector_epilogue<R>(Y + static_cast<size_t>(mr) * p.dims.next * 5, p.dims, ic, mo, p.eps, p.lam, p.epi32,
                           ep, ez, ed);
    }
    const double2 Fp = make_double2(ep.x - p.phibar * ud.x, ep.y - p.phibar * ud.y);
    const double2 Fz = ez;
    const double2 Fd = make_double2(ed.x + lam * up.x, ed.y + lam * up.y);

    // R_m = u_n + quadrature row m over the group's F_j (p.Q holds dt q_{m,j})
    double2 Rp = p.un[F_PHI * nc + ic], Rz = p.un[F_ZETA * nc + ic], Rd = p.un[F_DIV * nc + ic];
#pragma unroll
    for (int j = 0; j < M; ++j) {
        const double q = p.Q[mr][j];
        const double2 a = shfl2(Fp, g0 + j), z = shfl2(Fz, g0 + j), dd = shfl2(Fd, g0 + j);
        Rp.x = fma(q, a.x, Rp.x); Rp.y = fma(q, a.y, Rp.y);
        Rz.x = fma(q, z.x, Rz.x); Rz.y = fma(q, z.y, Rz.y);
        Rd.x = fma(q, dd.x, Rd.x); Rd.y = fma(q, dd.y, Rd.y);
    }

    double rs[3] = {0.0, 0.0, 0.0};
    if (i < nc && m < M && m >= p.m0 && m < p.m1) {
        if (RESID) {   // residual of the current iterate
            const double wgt = (i <= p.T) ? 1.0 : 2.0;    // order m = 0 occupies indices 0..T
            const double rpx = Rp.x - up.x, rpy = Rp.y - up.y;
            const double rzx = Rz.x - uz.x, rzy = Rz.y - uz.y;
            const double rdx = Rd.x - ud.x, rdy = Rd.y - ud.y;
            rs[F_PHI] = wgt * (rpx * rpx + rpy * rpy);
            rs[F_ZETA] = wgt * (rzx * rzx + rzy * rzy);
            rs[F_DIV] = wgt * (rdx * rdx + rdy * rdy);
        }
        // rhs = R - alpha L_g(u_m^k)
        const double al = p.alpha[m];
        const double2 bp = make_double2(Rp.x + al * p.phibar * ud.x, Rp.y + al * p.phibar * ud.y);
        const double2 bd = make_double2(Rd.x - al * lam * up.x, Rd.y - al * lam * up.y);
        const double den = p.den[m * nc + i];             // 1 / (1 + alpha^2 Phibar lambda_n)
        const double2 np = make_double2((bp.x - al * p.phibar * bd.x) * den, (bp.y - al * p.phibar * bd.y) * den);
        const double2 nd = make_double2(bd.x + al * lam * np.x, bd.y + al * lam * np.y);
        double2 *o = p.out + (m - p.m0) * p.ostride;
        o[F_PHI * nc + i] = np;
        o[F_ZETA * nc + i] = Rz;
        o[F_DIV * nc + i] = nd;
    }

    if (!RESID) return;
    // block reduction of the residual partial sums: lanes of the same node
    // within a warp (stride G), then the warps through shared memory
    __shared__ double red[kSweepThreads / 32][M * 3];
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        double v = rs[f];
#pragma unroll
        for (int o = G; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane < M) red[warp][lane * 3 + f] = v;
    }
    __syncthreads();
    if (threadIdx.x < M * 3) {
        double v = 0.0;
        for (int w = 0; w < kSweepThreads / 32; ++w) v += red[w][threadIdx.x];
        p.resid_part[static_cast<size_t>(blockIdx.x) * M * 3 + threadIdx.x] = v;
    }
}

// K5: fixed-order (deterministic) sum of the block partials, square root,
// maximum over the updated nodes -> 3 doubles (Phi', zeta, div).
__global__ void k5_resid_reduce(const double *__restrict__ part, int nblocks, int M, int m0, int m1,
                                double *__restrict__ out3) {
    __shared__ double acc[kMaxNodes * 3][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;   // one warp per (m, f)
    for (int mf = warp; mf < M * 3; mf += blockDim.x / 32) {
        double v = 0.0;
        for (int b = lane; b < nblocks; b += 32) v += part[static_cast<size_t>(b) * M * 3 + mf];
        acc[mf][lane] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int f = threadIdx.x;
        double best = 0.0;
        for (int m = m0; m < m1; ++m) {
            double s = 0.0;
            for (int l = 0; l < 32; ++l) s += acc[m * 3 + f][l];
            const double r = sqrt(s);
            best = (r > best || r != r) ? r : best;
        }
        out3[f] = best;
    }
}

template <typename R>
static cudaError_t launch_sweep_t(const SweepParams &p, int M, cudaStream_t s) {
    const int nb = sweep_blocks(p.ncoef, M);
    cudaError_t e = cudaSuccess;
#define SDC_SWEEP_CASE(MM)                                                                               \
    case MM:                                                                                             \
        if (p.resid_part) e = launch_k(p.pdl != 0, k4_sweep<MM, true, R>, dim3(nb), dim3(kSweepThreads), 0, s, p); \
        else e = launch_k(p.pdl != 0, k4_sweep<MM, false, R>, dim3(nb), dim3(kSweepThreads), 0, s, p);             \
        break;
    switch (M) {
        SDC_SWEEP_CASE(1) SDC_SWEEP_CASE(2) SDC_SWEEP_CASE(3) SDC_SWEEP_CASE(4)
        SDC_SWEEP_CASE(5) SDC_SWEEP_CASE(6) SDC_SWEEP_CASE(7) SDC_SWEEP_CASE(8)
        default: return cudaErrorInvalidValue;
    }
#undef SDC_SWEEP_CASE
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_sweep(const SweepParams &p, int M, bool fp32, cudaStream_t s, int *launches, StageTimer *timer) {
    if (timer) timer->mark(STAGE_SWEEP);
    const cudaError_t e = fp32 ? launch_sweep_t<float>(p, M, s) : launch_sweep_t<double>(p, M, s);
    if (launches) *launches += 1;
    return e;
}

cudaError_t launch_resid_reduce(const double *part, int nblocks, int M, int m0, int m1, double *out3,
                                cudaStream_t s, int *launches, StageTimer *timer) {
    if (timer) timer->mark(STAGE_RESID);
    k5_resid_reduce<<<1, 32 * kMaxNodes * 3 > 1024 ? 1024 : 32 * kMaxNodes * 3, 0, s>>>(part, nblocks, M, m0, m1,
                                                                                         out3);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

}  // namespace sdc
