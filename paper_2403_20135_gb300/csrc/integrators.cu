// Per-mode kernels of the paper's two reference integrators, which reuse the
// explicit-tendency kernels of transforms.cu for T_E (all arithmetic FP64):
//
// Serial IMEX SDC, Algorithm 1 with Eq. (6), node m of sweep k+1:
//   beta = u_n + dt sum_j q_{m,j} F_j^k
//        + dt sum_{j<m} [qe_{m,j} (E_j^{k+1} - E_j^k) + qi_{m,j} L_g(u_j^{k+1} - u_j^k)]
//        - dt qi_{m,m} L_g u_m^k,
//   (I - dt qi_{m,m} L_g) u_m^{k+1} = beta  (Eq. (8), closed form as in the sweep),
// with F_j = E_j + L_g u_j, explicit weights qe_{m,j} = dtau_{j+1} and implicit
// weights qi_{m,j} = dtau_j (Eq. (6); dtau_1 = tau_1, dtau_j = tau_j - tau_{j-1})
// or the rows of the LU choice (host table).
//
// IMEX-o2 (Sec. 3.2): Strang splitting, Crank-Nicolson half steps on L_g
// around one Heun step on T_E:
//   a = CN(dt/2) u_n,  b = a + dt T_E(a),  c = a + dt/2 (T_E(a) + T_E(b)),
//   u_{n+1} = CN(dt/2) c,  CN(h) x = (I - h/2 L_g)^{-1} (I + h/2 L_g) x.
//
// L_g(Phi', zeta, div) = (-Phibar div, 0, lambda_n Phi'); the solve
// (I - alpha L_g) x = r is Phi' = (r_Phi - alpha Phibar r_div) / (1 + alpha^2
// Phibar lambda_n), div = r_div + alpha lambda_n Phi', zeta = r_zeta.
#include <cuda_runtime.h>

#include "sdc_internal.h"

namespace sdc {

namespace {

constexpr int kModeThreads = 128;

__device__ __forceinline__ void solve_mode(double alpha, double phibar, double lam, const double2 (&r)[3],
                                           double2 (&x)[3]) {
    const double den = 1.0 / (1.0 + alpha * alpha * phibar * lam);
    x[F_PHI] = make_double2((r[F_PHI].x - alpha * phibar * r[F_DIV].x) * den,
                            (r[F_PHI].y - alpha * phibar * r[F_DIV].y) * den);
    x[F_ZETA] = r[F_ZETA];
    x[F_DIV] = make_double2(r[F_DIV].x + alpha * lam * x[F_PHI].x, r[F_DIV].y + alpha * lam * x[F_PHI].y);
}

__device__ __forceinline__ void load3(const double2 *base, int nc, int i, double2 (&v)[3]) {
#pragma unroll
    for (int f = 0; f < 3; ++f) v[f] = base[f * nc + i];
}

// L_g u for one mode
__device__ __forceinline__ void lg(const double2 (&u)[3], double phibar, double lam, double2 (&o)[3]) {
    o[F_PHI] = make_double2(-phibar * u[F_DIV].x, -phibar * u[F_DIV].y);
    o[F_ZETA] = make_double2(0.0, 0.0);
    o[F_DIV] = make_double2(lam * u[F_PHI].x, lam * u[F_PHI].y);
}

template <int M>
__global__ void __launch_bounds__(kModeThreads) k4_serial_node(SerialNodeParams p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int nc = p.ncoef;
    if (i >= nc) return;
    const double lam = p.lam[i], phibar = p.phibar, dt = p.dt;
    const int m = p.m;
    double2 beta[3];
    load3(p.un, nc, i, beta);
    double2 lum[3];
#pragma unroll
    for (int j = 0; j < M; ++j) {
        double2 u[3], e[3], l[3];
        load3(p.uk + j * p.kstride, nc, i, u);
        load3(p.ek + j * p.kstride, nc, i, e);
        lg(u, phibar, lam, l);
        const double q = dt * p.Q[j];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            beta[f].x += q * (e[f].x + l[f].x);
            beta[f].y += q * (e[f].y + l[f].y);
        }
        if (j == m) {
#pragma unroll
            for (int f = 0; f < 3; ++f) lum[f] = l[f];
        }
        if (j < m) {                                 // sweep k+1 already holds node j
            double2 u1[3], e1[3], l1[3];
            load3(p.uk1 + j * p.k1stride, nc, i, u1);
            load3(p.ek1 + j * p.k1stride, nc, i, e1);
            lg(u1, phibar, lam, l1);
            const double ce = dt * p.qe[j], ci = dt * p.qi[j];
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                beta[f].x += ce * (e1[f].x - e[f].x) + ci * (l1[f].x - l[f].x);
                beta[f].y += ce * (e1[f].y - e[f].y) + ci * (l1[f].y - l[f].y);
            }
        }
    }
    const double alpha = dt * p.qi[m];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        beta[f].x -= alpha * lum[f].x;
        beta[f].y -= alpha * lum[f].y;
    }
    double2 x[3];
    solve_mode(alpha, phibar, lam, beta, x);
#pragma unroll
    for (int f = 0; f < 3; ++f) p.out[f * nc + i] = x[f];
}

// out = CN(h) (a + s1 (e1 + e2)), e2 may be null; s1 = 0 gives CN(h) a
__global__ void __launch_bounds__(kModeThreads) k_imex2_cn(const double2 *__restrict__ a,
                                                           const double2 *__restrict__ e1,
                                                           const double2 *__restrict__ e2, double s1, double h,
                                                           const double *__restrict__ lamv, double phibar, int nc,
                                                           double2 *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const double lam = lamv[i];
    double2 c[3];
    load3(a, nc, i, c);
    if (e1) {
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const double2 x = e1[f * nc + i];
            const double2 y = e2 ? e2[f * nc + i] : make_double2(0.0, 0.0);
            c[f].x += s1 * (x.x + y.x);
            c[f].y += s1 * (x.y + y.y);
        }
    }
    double2 l[3], r[3], x[3];
    lg(c, phibar, lam, l);
#pragma unroll
    for (int f = 0; f < 3; ++f) r[f] = make_double2(c[f].x + 0.5 * h * l[f].x, c[f].y + 0.5 * h * l[f].y);
    solve_mode(0.5 * h, phibar, lam, r, x);
#pragma unroll
    for (int f = 0; f < 3; ++f) out[f * nc + i] = x[f];
}

// b = a + dt e
__global__ void __launch_bounds__(kModeThreads) k_imex2_euler(const double2 *__restrict__ a,
                                                              const double2 *__restrict__ e, double dt, int n,
                                                              double2 *__restrict__ b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 x = a[i], y = e[i];
    b[i] = make_double2(x.x + dt * y.x, x.y + dt * y.y);
}

}  // namespace

cudaError_t launch_serial_node(const SerialNodeParams &p, int M, cudaStream_t s, int *launches) {
    const int nb = (p.ncoef + kModeThreads - 1) / kModeThreads;
#define SDC_NODE_CASE(MM) \
    case MM: k4_serial_node<MM><<<nb, kModeThreads, 0, s>>>(p); break;
    switch (M) {
        SDC_NODE_CASE(1) SDC_NODE_CASE(2) SDC_NODE_CASE(3) SDC_NODE_CASE(4)
        SDC_NODE_CASE(5) SDC_NODE_CASE(6) SDC_NODE_CASE(7) SDC_NODE_CASE(8)
        default: return cudaErrorInvalidValue;
    }
#undef SDC_NODE_CASE
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_imex2_cn(const double2 *a, const double2 *e1, const double2 *e2, double s1, double h,
                            const double *lam, double phibar, int ncoef, double2 *out, cudaStream_t s,
                            int *launches) {
    k_imex2_cn<<<(ncoef + kModeThreads - 1) / kModeThreads, kModeThreads, 0, s>>>(a, e1, e2, s1, h, lam, phibar,
                                                                                  ncoef, out);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_imex2_euler(const double2 *a, const double2 *e, double dt, int ncoef, double2 *b, cudaStream_t s,
                               int *launches) {
    const int n = 3 * ncoef;
    k_imex2_euler<<<(n + kModeThreads - 1) / kModeThreads, kModeThreads, 0, s>>>(a, e, dt, n, b);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

}  // namespace sdc
