// Internal declarations shared by the host driver and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/sdc.h"

namespace sdc {

constexpr int kMaxNodes = 8;
constexpr int kMaxStages = 16;
constexpr int kMaxSnapshots = 32;

// Field order of a spectral state (the paper's U-hat, Sec. 3.2).
enum { F_PHI = 0, F_ZETA = 1, F_DIV = 2 };
// Fields of the synthesis output (grid Fourier coefficients per latitude).
enum { G_ZETA = 0, G_PHI = 1, G_U = 2, G_V = 3, NSYN = 4 };
// Fields of the ring products fed to the analysis.
enum { P_A = 0, P_B = 1, P_C = 2, P_D = 3, P_E = 4, NANA = 5 };

// Offset of order m in the packed triangular layout (n = m..T).
__host__ __device__ inline int order_offset(int T, int m) { return m * (2 * T + 3 - m) / 2; }
// Offset of order m in the extended layout (n = m..T+1), which carries one
// more degree per order for the (1-mu^2) d/dmu recurrences.
__host__ __device__ inline int ext_offset(int T, int m) { return m * (2 * T + 5 - m) / 2; }

// Mixed-radix (2, 3, 4) Stockham plan of a length-L complex FFT.
struct FftPlan {
    int L;
    int nstages;
    int radix[kMaxStages];
};

// Sizes handed to every transform kernel.
constexpr int kMaxChains = 4;   // concurrent state chains of a split tendency batch (SDC_OPT_CHAINS)

struct Dims {
    int T;        // truncation
    int J;        // latitudes
    int J2;       // latitude pairs (north half)
    int J2p;      // padded row length of the Legendre table (multiple of 4)
    int L;        // longitudes
    int ncoef;    // (T+1)(T+2)/2
    int next;     // (T+1)(T+4)/2, extended packing
    double a;     // radius
    double inv_a; // 1 / radius
    double two_omega;
};

// Parameters of the fused quadrature + implicit solve + residual kernel.
// The explicit tendencies of the nodes come as the projections Y of the
// preceding tendency batch (the vector epilogue runs inside the sweep).
struct SweepParams {
    const double2 *un;            // u_n, [3][ncoef]
    const double2 *ubase;         // node j iterate at ubase + j * ustride
    long long ustride;            // 0 on the first sweep (u_j^0 = u_n)
    const void *y;                // projections [ybatch][next][5] in the transform precision
    int ybatch;                   // 1: every node takes Y[0] (the first sweep), else M
    Dims dims;
    const double *eps;            // epilogue factors (FP64 transforms)
    const float *epi32;           // epilogue factors (FP32 transforms)
    const int *coef_m;
    double2 *out;                 // node m result at out + (m - m0) * ostride
    long long ostride;
    const double *lam;            // n(n+1)/a^2 per packed coefficient
    const double *den;            // [M][ncoef] 1 / (1 + alpha_m^2 Phibar lambda_n) of this sweep
    double *resid_part;           // [gridDim.x][M][3] or nullptr
    int ncoef;
    int T;
    int m0, m1;                   // nodes updated: [m0, m1)
    double phibar;
    double Q[kMaxNodes][kMaxNodes];   // dt * q_{m,j}
    double alpha[kMaxNodes];      // dt * q^Delta_{m,m}
    int pdl;                      // launched as a programmatic dependent
};

// One node update of serial IMEX SDC (Algorithm 1, Eq. (6)).
struct SerialNodeParams {
    const double2 *un;            // u_n
    const double2 *uk, *ek;       // u_j^k, E_j^k at + j * kstride (kstride 0: every node is u_n)
    long long kstride;
    const double2 *uk1, *ek1;     // u_j^{k+1}, E_j^{k+1} for j < m at + j * k1stride
    long long k1stride;
    double2 *out;                 // u_m^{k+1}
    const double *lam;            // n(n+1)/a^2 [ncoef]
    int ncoef;
    int m;
    double dt;
    double phibar;
    double Q[kMaxNodes];          // row m of the collocation matrix
    double qe[kMaxNodes];         // row m of the explicit weights (j < m): dtau_{j+1}
    double qi[kMaxNodes];         // row m of the implicit weights (j <= m)
};

// Per-kernel CUDA-event timing of a directly launched (not graph) step:
// mark(c) records an event and tags the kernel launched next with class c.
enum {
    STAGE_SYNTH = 0, STAGE_RING = 1, STAGE_ANALYSIS = 2, STAGE_EPILOGUE = 3, STAGE_SWEEP = 4, STAGE_RESID = 5,
    NSTAGES = 6
};
struct StageTimer {
    static constexpr int kMax = 512;
    cudaEvent_t ev[kMax + 1];
    int cls[kMax];
    int n = 0;
    cudaStream_t stream = nullptr;
    void mark(int c) {
        if (n < kMax) { cudaEventRecord(ev[n], stream); cls[n] = c; ++n; }
    }
    void end() { cudaEventRecord(ev[n], stream); }
};

// Device-resident tables of one context (pbar and tw in the transform
// precision: double / double2 or float / float2).
struct DeviceTables {
    const void *pbar;      // Pbar [next][J2p]
    const void *tw;        // twiddles [L]
    const double *eps;     // eps_n^m [next]
    const double *lam;     // n(n+1)/a^2 [ncoef]
    const double *mu;      // northern Gauss nodes [J2]
    const double *w;       // northern Gauss weights [J2]
    const double *syn;     // wind synthesis factors (c0, c1, c2) [next][3]
    const int *row_m;      // order m of each extended row [next]
    const int *coef_m;     // order m of each packed coefficient [ncoef]
    const double *ring64;  // per northern latitude: 2 Omega mu, 1 / (2 (1 - mu^2)), w / (1 - mu^2), w [J2][4]
    const float *ring32;   // the same in FP32
    const float *epi32;    // FP32 epilogue factors per coefficient: n eps_{n+1}, (n+1) eps_n, lambda_n, 0 [ncoef][4]
    const float *syn32;    // FP32 wind synthesis factors c0, c1, c2, 0 [next][4]
    int *err;              // device flag set by a kernel whose bounded wait expired
    // on-the-fly Legendre recurrence of the FP32 synthesis (nullptr: table)
    const float4 *rec_ab;  // (a_hi, a_lo, b_hi, b_lo) per extended row [next]
    const float4 *rec_seed;   // (Pbar_m^m, Pbar_{m+1}^m) as FP32 pairs [T+1][J2p]
    const float2 *rec_mu;  // mu_j as an FP32 pair [J2p]
    FftPlan plan16;        // FP32 ring: passes of radix 16, then 8/4/2, then 3
    const float2 *twp32;   // FP32 ring: per-pass twiddles of plan16 (after the first pass)
    int ntwp;
    bool pdl;              // launch the FP32 synthesis, ring and projection as programmatic dependents
};

// Transform workspaces (elements of the transform precision):
// f1 [B][J2][4][2][T+1] (FP32: [B][J2][T+1][2][4]), f2 [B][T+1][5][2][J2]
// (FP32: [B][T+1][J2][5][2]), f3 [B][next][5] complex.
#ifdef __CUDACC__
// Launch of kernel k, as a programmatic dependent of the preceding kernel in
// the stream when pdl is set (the kernel must call pdl_wait() before it
// touches anything its predecessors write).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(bool pdl, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                            Args... args) {
    if (!pdl) {
        k<<<grid, block, smem, s>>>(args...);
        return cudaSuccess;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}
#endif

struct Workspace {
    void *f1, *f2, *f3;
};

// Parameters of the sweep adjoint (transpose of one sweep kernel).
struct SweepAdjParams {
    const double2 *ubin;          // node adjoints u-bar_m^{k+1} at ubin + m * ustride
    long long ustride;
    double2 *ubout;               // u-bar_j^k at ubout + j * ostride (unless fold)
    double2 *ebout;               // E-bar_j^k at ebout + j * ostride (unless fold)
    long long ostride;
    double2 *ubn;                 // u-bar_n, accumulated (or initialised with init_un)
    double2 *ebar0;               // with fold: E-bar_0 (the adjoint of T_E(u_n))
    const double *lam;
    int ncoef;
    int m0, m1;                   // nodes the sweep updated
    int fold;                     // first sweep: sum node adjoints into u-bar_n / E-bar_0
    int init_un;
    double phibar;
    double Q[kMaxNodes][kMaxNodes];   // dt * q_{m,j}
    double alpha[kMaxNodes];
};

// Tensor-core (tcgen05) Legendre contractions with split-BF16 operands.
// Rows of order m with parity p of n' - m ("group (m, p)"): n' = m + p + 2q,
// q = 0..R-1.  The static Legendre operand is stored pre-split into npieces
// BF16 pieces, tile by tile and chunk by chunk in the canonical K-major
// shared-memory layout (8 x 8 core matrices, [row block][k block][8][8]), so
// one chunk of one piece is one contiguous bulk copy.
constexpr int kTcChunkKB = 4;     // k blocks (of 8 elements) per chunk
struct TcTile3 {                  // analysis: rows q0..q0+nrows of group (m, p), K = latitudes
    int m, p, q0, nrows, nrb;
    long long aoff;               // element offset of chunk 0 in each piece table
};
struct TcTile1 {                  // synthesis: latitudes j0..j0+nj of group (m, p), K = rows (padded to KR)
    int m, p, j0, nj, njb, R, KR;
    long long aoff;
};
// The dynamic operands are split by their own kernels into the same layout,
// group by group: the projection's W^T as [group][chunk][col block < kNbc3]
// [k block][8][8], the synthesis coefficients as [group][chunk][col block <
// kNbc1][k block][8][8].  Col blocks come first inside a chunk, so the
// blocks of a batch of B states are one contiguous prefix.
constexpr int kNbc3 = (10 * kMaxNodes + 7) / 8;   // projection columns b*10 + g*2 + (re, im)
constexpr int kNbc1 = kMaxNodes;                  // synthesis columns b*8 + f*2 + (re, im)
struct TcTables {
    const uint16_t *a3;           // analysis pieces [npieces][elems3]
    const uint16_t *a1;           // synthesis pieces [npieces][elems1]
    long long elems3, elems1;
    uint16_t *wb;                 // projection B operand pieces [npieces][wb_elems]
    uint16_t *cb;                 // synthesis B operand pieces [npieces][cb_elems]
    long long wb_elems, cb_elems;
    const long long *cb_off;      // [2 (T+1)] start of group (m, p) = 2 m + p in each cb piece
    const TcTile3 *tiles3;
    const TcTile1 *tiles1;
    int ntiles3, ntiles1;
    int npieces;
    int kj;                       // latitudes padded to a multiple of 16
    int *err;                     // device flag: a bounded wait gave up
};
void build_tc_tables(int T, int J2, int J2p, const std::vector<double> &pbar, int npieces,
                     std::vector<uint16_t> &a3, std::vector<TcTile3> &tiles3, std::vector<uint16_t> &a1,
                     std::vector<TcTile1> &tiles1, int *kj_out);
// rows of group (m, p) and their count padded to a multiple of 16
__host__ __device__ inline int tc_group_rows(int T, int m, int p) { return (T + 3 - m - p) / 2; }
__host__ __device__ inline int tc_group_krows(int T, int m, int p) { return (tc_group_rows(T, m, p) + 15) / 16 * 16; }

// ---- host-side precompute (tables.cpp) ----------------------------------
void gauss_legendre(int J, std::vector<double> &mu, std::vector<double> &w);
void radau_right(int M, std::vector<double> &tau, std::vector<double> &Q);
// MIN-SR-S diagonal (increasing root of the stiff-limit nilpotency conditions); false if not reached
bool min_sr_s_diagonal(int M, const std::vector<double> &tau, const std::vector<double> &Q, std::vector<double> &d);
// Q_Delta = U^T of the Doolittle factorisation Q^T = L U (row-major M x M); false on a zero pivot
bool lu_implicit_weights(int M, const std::vector<double> &Q, std::vector<double> &qd);
// Pbar_n^m(mu_j) for the northern latitudes j < J2, extended packing, rows
// padded to J2p: table[(ext_offset(m) + n - m) * J2p + j].
void legendre_table(int T, int J2, int J2p, const std::vector<double> &mu, std::vector<double> &table);
void epsilon_table(int T, std::vector<double> &eps);   // extended packing, eps_n^m
// FP32-pair tables of the on-the-fly Legendre recurrence (tables.cpp)
void recurrence_tables(int T, int J2, int J2p, const std::vector<double> &mu, const std::vector<double> &table,
                       std::vector<float> &ab, std::vector<float> &seed, std::vector<float> &mu2);
void synthesis_factors(int T, double radius, std::vector<double> &syn);   // [next][3]
void order_maps(int T, std::vector<int> &row_m, std::vector<int> &coef_m);
bool fft_plan(int L, FftPlan &plan);
bool fft_plan16(int L, FftPlan &plan);
// twiddles of every pass after the first, pass by pass as [r - 1][k < Ns]
void pass_twiddles(const FftPlan &plan, const std::vector<double> &re, const std::vector<double> &im,
                   std::vector<double> &pre, std::vector<double> &pim);
void twiddles(int L, std::vector<double> &re, std::vector<double> &im);   // e^{-2 pi i k / L}

// ---- kernel launchers (transforms.cu, sweep.cu) -------------------------
// Explicit tendency of B states (K1 -> K2 -> K3a -> K3b).  With tc (FP32
// transforms only) the two Legendre contractions run on the tensor cores.
// With tend == nullptr the epilogue is left to the caller, which reads the
// projections from ws.f3 ([B][next][5] in the transform precision).
cudaError_t launch_tendency(const Dims &d, const FftPlan &plan, bool fp32, int B, const double2 *states,
                            long long sstride, double2 *tend, long long tstride, const DeviceTables &tb,
                            const Workspace &ws, cudaStream_t s, int *launches, StageTimer *timer = nullptr,
                            void *grid_store = nullptr, const TcTables *tc = nullptr);
// Each adds its two launches (operand split + MMA kernel) to *launches.
cudaError_t launch_tc_synthesis(const TcTables &tc, const Dims &d, int B, const double2 *states, long long sstride,
                                const double *syn, const int *row_m, float2 *f1, cudaStream_t s, int *launches);
cudaError_t launch_tc_projection(const TcTables &tc, const Dims &d, int B, const float2 *f2, float2 *y,
                                 cudaStream_t s, int *launches);
cudaError_t configure_tc_kernels();
cudaError_t launch_sweep(const SweepParams &p, int M, bool fp32, cudaStream_t s, int *launches,
                         StageTimer *timer = nullptr);
cudaError_t launch_resid_reduce(const double *part, int nblocks, int M, int m0, int m1,
                                double *out3, cudaStream_t s, int *launches,
                                StageTimer *timer = nullptr);
int sweep_blocks(int ncoef, int M);

cudaError_t launch_spec_to_grid(const Dims &d, const FftPlan &plan, const double2 *spec,
                                double *grid, const double *pbar, const double2 *tw,
                                double2 *f1, cudaStream_t s);
cudaError_t launch_grid_to_spec(const Dims &d, const FftPlan &plan, const double *grid,
                                double2 *spec, const double *pbar, const double *w,
                                const double2 *tw, double2 *f2, cudaStream_t s);

// Transpose of the FP32 synthesis (adjoint): Z-bar[b][e][4] = sum_j Pbar_e(mu_j)
// F1-bar[b][j][f][parity(e)][m(e)], with the register-tiled projection kernel.
cudaError_t launch_synthesis_transpose_f32(const Dims &d, int B, const float2 *f1bar, const float *pbar, float2 *zbar,
                                           cudaStream_t s);
// Transpose of the FP32 analysis projection (adjoint): W-bar[b][j][g][parity][m]
// = sum over rows e of order m with that parity of Pbar_e(mu_j) Y-bar[b][e][g],
// with the staged synthesis kernel (m fastest, as the FP32 ring transpose
// reads it).
cudaError_t launch_projection_transpose_f32(const Dims &d, int B, const float2 *ybar, const float *pbar,
                                            float2 *wbar, int *err, cudaStream_t s);

// ---- adjoint (adjoint.cu) ------------------------------------------------
cudaError_t configure_adjoint_kernels(const Dims &d, const FftPlan &plan, bool fp32);
// u-bar (accumulated) += J_E^T a-bar for B states whose forward ring kernel
// recorded its grid fields in grid_base [B][J2][4][L].
cudaError_t launch_tendency_adjoint(const Dims &d, const FftPlan &plan, bool fp32, int B, const void *grid_base,
                                    const double2 *abar, long long astride, double2 *ubar, long long ustride,
                                    const DeviceTables &tb, const Workspace &ws, cudaStream_t s, int *launches);
cudaError_t launch_sweep_adjoint(const SweepAdjParams &p, int M, cudaStream_t s, int *launches);
int loss_blocks();
cudaError_t launch_height_loss(const Dims &d, const FftPlan &plan, const double *phigrid, const double *htarget,
                               double inv_g, double H, double *rgrid, double *part, double *loss,
                               double2 *seed_phi, const double *pbar64, const double2 *tw64, double2 *fbuf,
                               cudaStream_t s);

// ---- reference integrators (integrators.cu) ------------------------------
cudaError_t launch_serial_node(const SerialNodeParams &p, int M, cudaStream_t s, int *launches);
// out = CN(h) (a + s1 (e1 + e2)); e1, e2 nullable
cudaError_t launch_imex2_cn(const double2 *a, const double2 *e1, const double2 *e2, double s1, double h,
                            const double *lam, double phibar, int ncoef, double2 *out, cudaStream_t s,
                            int *launches);
cudaError_t launch_imex2_euler(const double2 *a, const double2 *e, double dt, int ncoef, double2 *b, cudaStream_t s,
                               int *launches);

size_t ring_smem_bytes(int L, int elem_bytes, int *scratch_arrays);
cudaError_t configure_transform_kernels(const Dims &d, const FftPlan &plan, bool fp32);

}  // namespace sdc
