// C ABI: context life cycle and the dSDC step of Algorithm 2, captured once
// as a CUDA graph and replayed per time step.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>
#include <algorithm>

#include "sdc_internal.h"

using namespace sdc;

namespace {

thread_local std::string g_last_error;

int fail(int status, const std::string &msg) {
    g_last_error = msg;
    return status;
}

int cuda_fail(cudaError_t e, const char *where) {
    return fail(SDC_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define SDC_CUDA(call)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);     \
    } while (0)

bool is_2a3b(int L) {
    if (L < 1) return false;
    while (L % 2 == 0) L /= 2;
    while (L % 3 == 0) L /= 3;
    return L == 1;
}

}  // namespace

constexpr int kStepsPerGraph = 4;   // steps per graph of a long run (sdc_run)

struct sdc_ctx {
    int T = 0, J = 0, L = 0, M = 0, K = 0;
    int precision = SDC_FP64;
    int qdelta_rule = SDC_QDELTA_CLAMPED;
    int method = SDC_METHOD_DSDC;
    int serial_implicit = SDC_SERIAL_IMPLICIT_EULER;
    std::vector<double> qi_lu;           // LU implicit weights of serial SDC, row-major M x M
    double dt = 0.0;
    sdc_phys phys{};
    Dims d{};
    FftPlan plan{};
    cudaStream_t stream = nullptr;       // caller's stream
    cudaStream_t cap = nullptr;          // private stream used for graph capture
    cudaStream_t capx[kMaxChains - 1] = {};   // extra capture streams: the other chains of a split batch
    cudaEvent_t ev_fork = nullptr, ev_join[kMaxChains - 1] = {};
    int chains = 2;                      // SDC_OPT_CHAINS
    int pdl = 1;                         // SDC_OPT_PDL
    std::vector<double> mu, w, tau, Q;
    std::vector<double> qd_min_sr_s;     // MIN-SR-S diagonal, computed when that rule is selected

    // device tables
    double *pbar = nullptr;
    float *pbar32 = nullptr;
    // on-the-fly Legendre recurrence of the FP32 synthesis (SDC_OPT_LEGENDRE)
    int legendre = SDC_LEGENDRE_TABLE;
    float *rec_ab = nullptr, *rec_seed = nullptr, *rec_mu = nullptr;
    double *eps = nullptr, *lam = nullptr, *mu2 = nullptr, *w2 = nullptr, *syn = nullptr, *ring64 = nullptr;
    float *ring32 = nullptr, *epi32 = nullptr, *syn32 = nullptr;
    int *row_m = nullptr, *coef_m = nullptr;
    double2 *tw = nullptr;
    float2 *tw32 = nullptr;
    FftPlan plan16{};
    float2 *twp32 = nullptr;
    int ntwp = 0;
    // device workspaces
    double2 *un = nullptr, *U = nullptr, *E = nullptr, *E0 = nullptr;
    void *f1 = nullptr, *f2 = nullptr, *f3 = nullptr;
    double *resid_part = nullptr, *resid = nullptr;
    double *den = nullptr;                  // [K][M][ncoef] solve denominators per sweep
    int sweep_nblocks = 0;

    // adjoint workspaces
    void *gstore = nullptr;                 // recorded grid fields of a step's evaluations
    double2 *ub = nullptr, *eb = nullptr;   // node adjoints u-bar^k, E-bar^k [M]
    double2 *ubn = nullptr, *ubnext = nullptr, *eb0 = nullptr;
    double2 *snaps = nullptr;               // checkpoint pool [kMaxSnapshots]
    double *phigrid = nullptr, *rgrid = nullptr, *loss_part = nullptr, *loss_dev = nullptr;
    long long adj_forward_steps = 0;

    // tensor-core Legendre tables (split-BF16 modes)
    TcTables tc{};
    uint16_t *tc_a3 = nullptr, *tc_a1 = nullptr, *tc_wb = nullptr, *tc_cb = nullptr;
    long long *tc_cboff = nullptr;
    TcTile3 *tc_t3 = nullptr;
    TcTile1 *tc_t1 = nullptr;
    int *tc_err = nullptr;

    // [0] one step, [1] one step with residuals, [2] kStepsPerGraph steps
    cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};
    int graph_launches[3] = {0, 0, 0};
    double2 *alt = nullptr;              // reference integrators: extra node iterates
    cudaGraphExec_t graph_retape = nullptr, graph_adjoint = nullptr;
    int retape_launches = 0, adjoint_launches = 0;
    long long n_explicit = 0, n_solve = 0, n_launch = 0;

    long long state_elems() const { return 3LL * d.ncoef; }
};

namespace {

void free_ctx(sdc_ctx *c) {
    if (!c) return;
    for (auto &g : c->graph)
        if (g) cudaGraphExecDestroy(g);
    if (c->graph_retape) cudaGraphExecDestroy(c->graph_retape);
    if (c->graph_adjoint) cudaGraphExecDestroy(c->graph_adjoint);
    void *ptrs[] = {c->pbar, c->pbar32, c->ring64, c->ring32, c->epi32, c->syn32, c->eps, c->lam, c->mu2, c->w2, c->syn, c->row_m, c->coef_m, c->tw,
                    c->tw32, c->twp32, c->un, c->U, c->E, c->E0, c->f1, c->f2, c->f3, c->resid_part, c->resid,
                    c->gstore, c->ub, c->eb, c->ubn, c->ubnext, c->eb0, c->snaps, c->phigrid, c->rgrid,
                    c->loss_part, c->loss_dev, c->tc_a3, c->tc_a1, c->tc_t3, c->tc_t1, c->tc_err, c->den,
                    c->tc_wb, c->tc_cb, c->tc_cboff, c->alt, c->rec_ab, c->rec_seed, c->rec_mu};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->cap) cudaStreamDestroy(c->cap);
    for (auto &x : c->capx)
        if (x) cudaStreamDestroy(x);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    for (auto &x : c->ev_join)
        if (x) cudaEventDestroy(x);
    delete c;
}

template <typename T>
cudaError_t upload(T **dst, const T *src, size_t n) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(dst), n * sizeof(T));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
}

// Diagonal coefficient q^Delta_{m,m} of sweep k (1-based) for node m (0-based),
// Sec. 4.2: MIN-SR-FLEX tau_m / k (the q(k) reading for k > M selected by the
// rule), MIN-SR-NS tau_m / M, the implicit-Euler diagonal tau_m, or
// MIN-SR-S (computed once per context by min_sr_s_diagonal).
// MIN-SR-S: the increasing diagonal making the stiff-limit sweep nilpotent.
double qdelta_value(int rule, int M, const std::vector<double> &tau, const std::vector<double> &mss, int k, int m) {
    switch (rule) {
        case SDC_QDELTA_LITERAL: return tau[m] / k;
        case SDC_QDELTA_MIN_SR_NS: return tau[m] / M;
        case SDC_QDELTA_IMPLICIT_EULER: return tau[m];
        case SDC_QDELTA_MIN_SR_S: return mss[m];
        default: return tau[m] / (k < M ? k : M);
    }
}

double qdelta_coef(const sdc_ctx *c, int k, int m) {
    return qdelta_value(c->qdelta_rule, c->M, c->tau, c->qd_min_sr_s, k, m);
}

DeviceTables tables(const sdc_ctx *c) {
    const bool fp32 = c->precision != SDC_FP64;
    DeviceTables tb{};
    tb.pbar = fp32 ? static_cast<const void *>(c->pbar32) : static_cast<const void *>(c->pbar);
    tb.tw = fp32 ? static_cast<const void *>(c->tw32) : static_cast<const void *>(c->tw);
    tb.eps = c->eps;
    tb.lam = c->lam;
    tb.mu = c->mu2;
    tb.w = c->w2;
    tb.syn = c->syn;
    tb.row_m = c->row_m;
    tb.coef_m = c->coef_m;
    tb.err = c->tc_err;
    tb.ring64 = c->ring64;
    tb.ring32 = c->ring32;
    tb.epi32 = c->epi32;
    tb.syn32 = c->syn32;
    tb.plan16 = c->plan16;
    tb.twp32 = c->twp32;
    tb.ntwp = c->ntwp;
    if (c->legendre == SDC_LEGENDRE_RECURRENCE) {
        tb.rec_ab = reinterpret_cast<const float4 *>(c->rec_ab);
        tb.rec_seed = reinterpret_cast<const float4 *>(c->rec_seed);
        tb.rec_mu = reinterpret_cast<const float2 *>(c->rec_mu);
    }
    return tb;
}

size_t grid_slot_bytes(const sdc_ctx *c) {
    const size_t elem = c->precision == SDC_FP64 ? sizeof(double2) : sizeof(float2);
    return static_cast<size_t>(c->d.J2) * 4 * c->L * elem;
}

void *grid_slot(const sdc_ctx *c, int slot) {
    return static_cast<char *>(c->gstore) + grid_slot_bytes(c) * slot;
}

cudaError_t tendency(sdc_ctx *c, int B, const double2 *states, long long sstride, double2 *tend,
                     long long tstride, cudaStream_t s, int *launches, StageTimer *timer = nullptr,
                     void *grid_store = nullptr) {
    const bool fp32 = c->precision != SDC_FP64;
    DeviceTables tb = tables(c);
    tb.pdl = c->pdl != 0 && s == c->cap && !timer;        // inside a captured step or retape graph
    Workspace ws{c->f1, c->f2, c->f3};
    const bool use_tc = c->precision == SDC_MIXED_BF16X3 || c->precision == SDC_MIXED_BF16X6;
    // Chains (SDC_OPT_CHAINS): while a graph is captured, the states of the
    // batch are split into up to `chains` parts whose transforms run on as
    // many streams, so that the kernels of one part fill the SMs the others'
    // kernels leave idle (tails, order-pair grids smaller than the GPU).
    // Every kernel indexes its workspaces by the state, so part k runs on the
    // same buffers offset by its first state.  The tensor-core modes share
    // their split operands across the batch and stay on one chain.
    if (c->chains >= 2 && B >= 2 && s == c->cap && !timer && !use_tc) {
        const Dims &d = c->d;
        const int nch = c->chains < B ? c->chains : B;
        const size_t elem = fp32 ? sizeof(float2) : sizeof(double2);
        const size_t f1s = static_cast<size_t>(d.J2) * 8 * (d.T + 1) * elem;
        const size_t f2s = static_cast<size_t>(d.T + 1) * 10 * d.J2 * elem;
        const size_t f3s = static_cast<size_t>(d.next) * 5 * elem;
        const size_t gss = static_cast<size_t>(d.J2) * 4 * d.L * elem;
        cudaError_t e = cudaEventRecord(c->ev_fork, s);
        for (int k = 1; k < nch && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(c->capx[k - 1], c->ev_fork, 0);
        int b0 = 0;
        for (int k = 0; k < nch && e == cudaSuccess; ++k) {
            const int bk = B / nch + (k < B % nch ? 1 : 0);   // the larger parts first
            const Workspace wk{static_cast<char *>(c->f1) + b0 * f1s, static_cast<char *>(c->f2) + b0 * f2s,
                               static_cast<char *>(c->f3) + b0 * f3s};
            e = launch_tendency(d, c->plan, fp32, bk, states + b0 * sstride, sstride,
                                tend ? tend + b0 * tstride : nullptr, tstride, tb, wk, k ? c->capx[k - 1] : s,
                                launches, nullptr, grid_store ? static_cast<char *>(grid_store) + b0 * gss : nullptr,
                                nullptr);
            b0 += bk;
        }
        for (int k = 1; k < nch && e == cudaSuccess; ++k) {
            e = cudaEventRecord(c->ev_join[k - 1], c->capx[k - 1]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->ev_join[k - 1], 0);
        }
        return e;
    }
    return launch_tendency(c->d, c->plan, fp32, B, states, sstride, tend, tstride, tb, ws, s, launches, timer,
                           grid_store, use_tc ? &c->tc : nullptr);
}

// Serial IMEX SDC step (Algorithm 1, Eq. (6)) in place on c->un: node by
// node, each node update followed by the tendency of the new node state
// (except after the last node of the last sweep).  Iterate 0 is u_n and
// T_E(u_n) for every node; iterate k >= 1 lives in slot k % 2 (U/E, alt).
cudaError_t enqueue_serial(sdc_ctx *c, cudaStream_t s, int *launches, StageTimer *timer) {
    const long long se = c->state_elems();
    const int M = c->M, K = c->K;
    cudaError_t e = tendency(c, 1, c->un, se, c->E0, se, s, launches, timer);
    if (e != cudaSuccess) return e;
    SerialNodeParams p{};
    p.un = c->un;
    p.lam = c->lam;
    p.ncoef = c->d.ncoef;
    p.dt = c->dt;
    p.phibar = c->phys.gravity * c->phys.mean_depth;
    std::vector<double> dtau(M);
    for (int j = 0; j < M; ++j) dtau[j] = c->tau[j] - (j > 0 ? c->tau[j - 1] : 0.0);
    double2 *su[2] = {c->U, c->alt}, *sv[2] = {c->E, c->alt + M * se};
    for (int k = 0; k < K; ++k) {
        p.uk = k == 0 ? c->un : su[k % 2];
        p.ek = k == 0 ? c->E0 : sv[k % 2];
        p.kstride = k == 0 ? 0 : se;
        double2 *nu = su[(k + 1) % 2], *ne = sv[(k + 1) % 2];
        p.uk1 = nu;
        p.ek1 = ne;
        p.k1stride = se;
        for (int m = 0; m < M; ++m) {
            const bool final = (k == K - 1 && m == M - 1);
            p.m = m;
            for (int j = 0; j < M; ++j) {
                p.Q[j] = c->Q[m * M + j];
                p.qe[j] = j < m ? dtau[j + 1] : 0.0;
                p.qi[j] = j > m ? 0.0
                                : (c->serial_implicit == SDC_SERIAL_IMPLICIT_LU ? c->qi_lu[m * M + j] : dtau[j]);
            }
            p.out = final ? c->un : nu + m * se;
            if (timer) timer->mark(STAGE_SWEEP);
            e = launch_serial_node(p, M, s, launches);
            if (e != cudaSuccess) return e;
            if (!final) {
                e = tendency(c, 1, nu + m * se, se, ne + m * se, se, s, launches, timer);
                if (e != cudaSuccess) return e;
            }
        }
    }
    return cudaSuccess;
}

// IMEX-o2 step (Sec. 3.2) in place on c->un: CN half step, Heun step on
// T_E, CN half step (a, b, T_E(a), T_E(b) in alt).
cudaError_t enqueue_imex2(sdc_ctx *c, cudaStream_t s, int *launches, StageTimer *timer) {
    const long long se = c->state_elems();
    const int nc = c->d.ncoef;
    const double phibar = c->phys.gravity * c->phys.mean_depth, h = 0.5 * c->dt;
    double2 *a = c->alt, *b = c->alt + se, *ea = c->alt + 2 * se, *eb = c->alt + 3 * se;
    if (timer) timer->mark(STAGE_SWEEP);
    cudaError_t e = launch_imex2_cn(c->un, nullptr, nullptr, 0.0, h, c->lam, phibar, nc, a, s, launches);
    if (e == cudaSuccess) e = tendency(c, 1, a, se, ea, se, s, launches, timer);
    if (e == cudaSuccess && timer) timer->mark(STAGE_SWEEP);
    if (e == cudaSuccess) e = launch_imex2_euler(a, ea, c->dt, nc, b, s, launches);
    if (e == cudaSuccess) e = tendency(c, 1, b, se, eb, se, s, launches, timer);
    if (e == cudaSuccess && timer) timer->mark(STAGE_SWEEP);
    if (e == cudaSuccess) e = launch_imex2_cn(a, ea, eb, 0.5 * c->dt, h, c->lam, phibar, nc, c->un, s, launches);
    return e;
}

// tendency evaluations and implicit solves of one step of the selected method
long long evals_per_step(const sdc_ctx *c) {
    if (c->method == SDC_METHOD_SERIAL_SDC) return static_cast<long long>(c->K) * c->M;
    if (c->method == SDC_METHOD_IMEX2) return 2;
    return 1 + static_cast<long long>(c->K - 1) * c->M;
}
long long solves_per_step(const sdc_ctx *c) {
    if (c->method == SDC_METHOD_SERIAL_SDC) return static_cast<long long>(c->K) * c->M;
    if (c->method == SDC_METHOD_IMEX2) return 2;
    return static_cast<long long>(c->K - 1) * c->M + 1;
}

// Enqueue one step u_n -> u_n (in place on c->un), Algorithm 2 (or the
// selected reference integrator).
// With store_grid (the retape of the adjoint) every tendency evaluation also
// records its grid fields: slot 0 for E0, slots 1 + k M + j for sweep k+1, node j.
cudaError_t enqueue_step(sdc_ctx *c, cudaStream_t s, bool with_resid, int *launches,
                         StageTimer *timer = nullptr, bool store_grid = false) {
    if (c->method == SDC_METHOD_SERIAL_SDC) return enqueue_serial(c, s, launches, timer);
    if (c->method == SDC_METHOD_IMEX2) return enqueue_imex2(c, s, launches, timer);
    const long long se = c->state_elems();
    const int M = c->M, K = c->K;
    cudaError_t e;
    // E0 = T_E(u_n): the transforms here, the vector epilogue inside the first sweep
    e = tendency(c, 1, c->un, se, nullptr, se, s, launches, timer, store_grid ? grid_slot(c, 0) : nullptr);
    if (e != cudaSuccess) return e;

    const DeviceTables tb = tables(c);
    SweepParams p{};
    p.un = c->un;
    p.lam = c->lam;
    p.y = c->f3;
    p.dims = c->d;
    p.eps = tb.eps;
    p.epi32 = tb.epi32;
    p.coef_m = tb.coef_m;
    p.ncoef = c->d.ncoef;
    p.T = c->T;
    p.phibar = c->phys.gravity * c->phys.mean_depth;
    for (int m = 0; m < M; ++m)
        for (int j = 0; j < M; ++j) p.Q[m][j] = c->dt * c->Q[m * M + j];
    p.resid_part = with_resid ? c->resid_part : nullptr;
    p.pdl = (c->pdl != 0 && s == c->cap && !timer) ? 1 : 0;

    for (int k = 0; k < K; ++k) {             // sweep k+1
        const bool first = (k == 0), last = (k == K - 1);
        p.ubase = first ? c->un : c->U;
        p.ustride = first ? 0 : se;
        p.ybatch = first ? 1 : M;
        for (int m = 0; m < M; ++m) p.alpha[m] = c->dt * qdelta_coef(c, k + 1, m);
        p.den = c->den + static_cast<size_t>(k) * M * c->d.ncoef;
        if (last) {                           // node M only, written to u_{n+1}
            p.m0 = M - 1;
            p.m1 = M;
            p.out = c->un;
            p.ostride = 0;
        } else {
            p.m0 = 0;
            p.m1 = M;
            p.out = c->U;
            p.ostride = se;
        }
        e = launch_sweep(p, M, c->precision != SDC_FP64, s, launches, timer);
        if (e != cudaSuccess) return e;
        if (with_resid) {
            e = launch_resid_reduce(c->resid_part, c->sweep_nblocks, M, p.m0, p.m1, c->resid + 3 * k, s, launches,
                                    timer);
            if (e != cudaSuccess) return e;
        }
        if (!last) {
            e = tendency(c, M, c->U, se, nullptr, se, s, launches, timer,
                         store_grid ? grid_slot(c, 1 + k * M) : nullptr);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

// 1 / (1 + alpha^2 Phibar lambda_n) for every sweep, node and mode.
cudaError_t upload_denominators(sdc_ctx *c) {
    const int nc = c->d.ncoef, M = c->M, K = c->K;
    std::vector<double> lam(nc), den(static_cast<size_t>(K) * M * nc);
    for (int m = 0; m <= c->T; ++m)
        for (int n = m; n <= c->T; ++n)
            lam[order_offset(c->T, m) + n - m] = double(n) * double(n + 1) / (c->phys.radius * c->phys.radius);
    const double phibar = c->phys.gravity * c->phys.mean_depth;
    for (int k = 0; k < K; ++k) {
        for (int m = 0; m < M; ++m) {
            const double al = c->dt * qdelta_coef(c, k + 1, m);
            for (int i = 0; i < nc; ++i) den[(static_cast<size_t>(k) * M + m) * nc + i] = 1.0 / (1.0 + al * al * phibar * lam[i]);
        }
    }
    return cudaMemcpy(c->den, den.data(), den.size() * sizeof(double), cudaMemcpyHostToDevice);
}

// Graph v: 0 one step, 1 one step with residuals, 2 kStepsPerGraph steps in
// one graph (sdc_run's long runs: one graph launch per kStepsPerGraph steps,
// and each step's first kernel launched as a programmatic dependent of the
// previous step's last sweep).
int ensure_graph(sdc_ctx *c, bool with_resid, int v = -1) {
    if (v < 0) v = with_resid ? 1 : 0;
    if (c->graph[v]) return SDC_OK;
    cudaGraph_t g = nullptr;
    SDC_CUDA(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    int launches = 0;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < (v == 2 ? kStepsPerGraph : 1) && e == cudaSuccess; ++k)
        e = enqueue_step(c, c->cap, with_resid, &launches);
    cudaError_t e2 = cudaStreamEndCapture(c->cap, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(e, "capture of the step");
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->graph[v], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    c->graph_launches[v] = launches;
    return SDC_OK;
}

// Reverse of one step (Algorithm 2 transposed), after a retape recorded the
// grid fields: c->ubnext = u-bar_{n+1}  ->  c->ubn = u-bar_n.
cudaError_t enqueue_step_adjoint(sdc_ctx *c, cudaStream_t s, int *launches) {
    const long long se = c->state_elems();
    const int M = c->M, K = c->K;
    const bool fp32 = c->precision != SDC_FP64;
    const DeviceTables tb = tables(c);
    const Workspace ws{c->f1, c->f2, c->f3};
    SweepAdjParams p{};
    p.lam = c->lam;
    p.ncoef = c->d.ncoef;
    p.phibar = c->phys.gravity * c->phys.mean_depth;
    for (int m = 0; m < M; ++m)
        for (int j = 0; j < M; ++j) p.Q[m][j] = c->dt * c->Q[m * M + j];
    p.ubn = c->ubn;
    p.ebar0 = c->eb0;
    p.ubout = c->ub;
    p.ebout = c->eb;
    p.ostride = se;
    cudaError_t e;
    for (int k = K - 1; k >= 0; --k) {           // transpose of sweep k+1
        const bool last = (k == K - 1);
        if (!last) {
            // u-bar_j^{k+1} += J_E(u_j^{k+1})^T E-bar_j^{k+1}
            e = launch_tendency_adjoint(c->d, c->plan, fp32, M, grid_slot(c, 1 + k * M), c->eb, se, c->ub, se, tb,
                                        ws, s, launches);
            if (e != cudaSuccess) return e;
        }
        p.ubin = last ? c->ubnext : c->ub;
        p.ustride = last ? 0 : se;
        p.m0 = last ? M - 1 : 0;
        p.m1 = M;
        p.fold = (k == 0);
        p.init_un = last;
        for (int m = 0; m < M; ++m) p.alpha[m] = c->dt * qdelta_coef(c, k + 1, m);
        e = launch_sweep_adjoint(p, M, s, launches);
        if (e != cudaSuccess) return e;
    }
    // u-bar_n += J_E(u_n)^T E-bar_0
    return launch_tendency_adjoint(c->d, c->plan, fp32, 1, grid_slot(c, 0), c->eb0, se, c->ubn, se, tb, ws, s,
                                   launches);
}

int capture(sdc_ctx *c, cudaGraphExec_t *exec, int *nlaunch, int which) {
    if (*exec) return SDC_OK;
    cudaGraph_t g = nullptr;
    SDC_CUDA(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    int launches = 0;
    cudaError_t e = which == 0 ? enqueue_step(c, c->cap, false, &launches, nullptr, true)
                               : enqueue_step_adjoint(c, c->cap, &launches);
    cudaError_t e2 = cudaStreamEndCapture(c->cap, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(e, "capture");
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    *nlaunch = launches;
    return SDC_OK;
}

// One reverse step from the state in c->un: retape (c->un becomes u_{n+1}),
// optional loss seed from u_{n+1}, then the adjoint; the result u-bar_n is
// left in c->ubnext for the next step down.
int reverse_one(sdc_ctx *c, const double *h_target, bool seed) {
    int st = capture(c, &c->graph_retape, &c->retape_launches, 0);
    if (st != SDC_OK) return st;
    st = capture(c, &c->graph_adjoint, &c->adjoint_launches, 1);
    if (st != SDC_OK) return st;
    const size_t sbytes = 3ULL * c->d.ncoef * sizeof(double2);
    SDC_CUDA(cudaGraphLaunch(c->graph_retape, c->stream));
    if (seed) {
        SDC_CUDA(cudaMemsetAsync(c->ubnext, 0, sbytes, c->stream));
        SDC_CUDA(launch_spec_to_grid(c->d, c->plan, c->un, c->phigrid, c->pbar, c->tw,
                                     static_cast<double2 *>(c->f1), c->stream));
        SDC_CUDA(launch_height_loss(c->d, c->plan, c->phigrid, h_target, 1.0 / c->phys.gravity, c->phys.mean_depth,
                                    c->rgrid, c->loss_part, c->loss_dev, c->ubnext, c->pbar, c->tw,
                                    static_cast<double2 *>(c->f2), c->stream));
    }
    SDC_CUDA(cudaGraphLaunch(c->graph_adjoint, c->stream));
    SDC_CUDA(cudaMemcpyAsync(c->ubnext, c->ubn, sbytes, cudaMemcpyDeviceToDevice, c->stream));
    c->n_explicit += 2LL * (1 + (c->K - 1) * c->M);
    c->n_solve += 2LL * ((c->K - 1) * c->M + 1);
    c->n_launch += c->retape_launches + c->adjoint_launches;
    return SDC_OK;
}

// Optimal binomial checkpointing for uniform step costs: reversing n steps
// from a stored state with s free snapshot slots costs
//   C(n, s) = min_{0<m<n} [ m + C(n-m, s-1) + C(m, s) ],  C(1, s) = 0,  C(n, 0) = n(n-1)/2
// forward recomputations (advance m steps and store, reverse the right part
// with one slot less, restore and reverse the left part).
struct Schedule {
    int N = 0, S = 0;
    std::vector<long long> cost;
    std::vector<int> split;
    long long &C(int n, int s) { return cost[static_cast<size_t>(n) * (S + 1) + s]; }
    int &B(int n, int s) { return split[static_cast<size_t>(n) * (S + 1) + s]; }
    void build(int n_, int s_) {
        N = n_;
        S = s_;
        cost.assign(static_cast<size_t>(N + 1) * (S + 1), 0);
        split.assign(static_cast<size_t>(N + 1) * (S + 1), 0);
        for (int n = 1; n <= N; ++n) C(n, 0) = static_cast<long long>(n) * (n - 1) / 2;
        for (int s = 1; s <= S; ++s)
            for (int n = 2; n <= N; ++n) {
                long long best = -1;
                int arg = 1;
                for (int m = 1; m < n; ++m) {
                    const long long v = m + C(n - m, s - 1) + C(m, s);
                    if (best < 0 || v < best) { best = v; arg = m; }
                }
                C(n, s) = best;
                B(n, s) = arg;
            }
    }
};

struct Reverser {
    sdc_ctx *c;
    Schedule sched;
    std::vector<int> free_slots;
    const double *h_target;
    int N;
    size_t sbytes;

    int store(int slot) {
        SDC_CUDA(cudaMemcpyAsync(c->snaps + slot * c->state_elems(), c->un, sbytes, cudaMemcpyDeviceToDevice,
                                 c->stream));
        return SDC_OK;
    }
    int restore(int slot) {
        SDC_CUDA(cudaMemcpyAsync(c->un, c->snaps + slot * c->state_elems(), sbytes, cudaMemcpyDeviceToDevice,
                                 c->stream));
        return SDC_OK;
    }
    int advance(int n);
    int step(int i) { return reverse_one(c, h_target, h_target != nullptr && i == N - 1); }

    // reverse steps [a, b) given u_a in c->un and in slot slot_a
    int rev(int a, int b, int sfree, int slot_a) {
        int st;
        if (b - a == 1) return step(a);
        if (sfree == 0 || free_slots.empty()) {
            for (int i = b - 1; i >= a; --i) {
                if (i < b - 1 && (st = restore(slot_a)) != SDC_OK) return st;
                if ((st = advance(i - a)) != SDC_OK) return st;
                if ((st = step(i)) != SDC_OK) return st;
            }
            return SDC_OK;
        }
        const int m = a + sched.B(b - a, sfree);
        if ((st = advance(m - a)) != SDC_OK) return st;
        const int slot_m = free_slots.back();
        free_slots.pop_back();
        if ((st = store(slot_m)) != SDC_OK) return st;
        if ((st = rev(m, b, sfree - 1, slot_m)) != SDC_OK) return st;
        free_slots.push_back(slot_m);
        if ((st = restore(slot_a)) != SDC_OK) return st;
        return rev(a, m, sfree, slot_a);
    }
};

int run_steps(sdc_ctx *c, int nsteps, bool with_resid);

int Reverser::advance(int n) {
    c->adj_forward_steps += n;
    return run_steps(c, n, false);
}

int run_steps(sdc_ctx *c, int nsteps, bool with_resid) {
    int st = ensure_graph(c, with_resid);
    if (st != SDC_OK) return st;
    int i = 0;
    if (!with_resid && nsteps >= kStepsPerGraph) {
        st = ensure_graph(c, false, 2);
        if (st != SDC_OK) return st;
        for (; i + kStepsPerGraph <= nsteps; i += kStepsPerGraph) SDC_CUDA(cudaGraphLaunch(c->graph[2], c->stream));
    }
    for (; i < nsteps; ++i) SDC_CUDA(cudaGraphLaunch(c->graph[with_resid ? 1 : 0], c->stream));
    c->n_explicit += static_cast<long long>(nsteps) * evals_per_step(c);
    c->n_solve += static_cast<long long>(nsteps) * solves_per_step(c);
    c->n_launch += static_cast<long long>(nsteps) * c->graph_launches[with_resid ? 1 : 0];
    return SDC_OK;
}

}  // namespace

extern "C" {

const char *sdc_strerror(int status) {
    switch (status) {
        case SDC_OK: return "ok";
        case SDC_EINVAL: return "invalid argument";
        case SDC_ENOMEM: return "out of memory";
        case SDC_ECUDA: return "CUDA error";
        case SDC_EDIVERGED: return "residual not finite";
        case SDC_ESTATE: return "invalid state";
        case SDC_EUNSUPPORTED: return "unsupported option";
        default: return "unknown status";
    }
}

const char *sdc_last_error(void) { return g_last_error.c_str(); }

int sdc_create(sdc_ctx **out, int T, int J, int L, int M, int K, double dt, const sdc_phys *phys, int precision,
               void *cuda_stream) {
    if (!out) return fail(SDC_EINVAL, "out is NULL");
    *out = nullptr;
    if (T < 1 || T > 1023) return fail(SDC_EINVAL, "truncation must be in [1, 1023]");
    if (J % 2 != 0 || 2 * J < 3 * T + 1 || J > 2048) return fail(SDC_EINVAL, "nlat must be even, >= (3T+1)/2, <= 2048");
    if (!is_2a3b(L) || L < 3 * T + 1 || L > 2304) return fail(SDC_EINVAL, "nlon must be 2^a 3^b, >= 3T+1, <= 2304");
    if (M < 1 || M > kMaxNodes) return fail(SDC_EINVAL, "nodes must be in [1, 8]");
    if (K < 1 || K > 64) return fail(SDC_EINVAL, "sweeps must be in [1, 64]");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(SDC_EINVAL, "dt must be positive and finite");
    if (!phys || !(phys->radius > 0) || !(phys->gravity > 0) || !(phys->mean_depth > 0) || !std::isfinite(phys->omega))
        return fail(SDC_EINVAL, "physical constants invalid");
    if (precision != SDC_FP64 && precision != SDC_MIXED_FP32 && precision != SDC_MIXED_BF16X3 &&
        precision != SDC_MIXED_BF16X6)
        return fail(SDC_EINVAL, "unknown precision");

    sdc_ctx *c = new (std::nothrow) sdc_ctx();
    if (!c) return fail(SDC_ENOMEM, "host allocation");
    c->T = T; c->J = J; c->L = L; c->M = M; c->K = K;
    c->dt = dt;
    c->phys = *phys;
    c->precision = precision;
    c->stream = static_cast<cudaStream_t>(cuda_stream);

    Dims &d = c->d;
    d.T = T; d.J = J; d.J2 = J / 2; d.J2p = ((J / 2) + 3) / 4 * 4; d.L = L;
    d.ncoef = (T + 1) * (T + 2) / 2;
    d.next = (T + 1) * (T + 4) / 2;
    d.a = phys->radius;
    d.inv_a = 1.0 / phys->radius;
    d.two_omega = 2.0 * phys->omega;
    if (!fft_plan(L, c->plan)) { free_ctx(c); return fail(SDC_EINVAL, "no FFT plan for nlon"); }
    if (precision == SDC_FP64 && ring_smem_bytes(L, sizeof(double2), nullptr) == 0) {
        free_ctx(c);
        return fail(SDC_EUNSUPPORTED, "nlon too long for the FP64 ring kernel (at most 2048 longitudes in FP64)");
    }
    const int elem = precision == SDC_FP64 ? (int)sizeof(double2) : (int)sizeof(float2);
    if (ring_smem_bytes(L, elem, nullptr) == 0) { free_ctx(c); return fail(SDC_EINVAL, "nlon too large"); }

    // host precompute
    gauss_legendre(J, c->mu, c->w);
    radau_right(M, c->tau, c->Q);
    std::vector<double> table, eps, lam(d.ncoef), twr, twi, syn;
    std::vector<int> row_m, coef_m;
    legendre_table(T, d.J2, d.J2p, c->mu, table);
    epsilon_table(T, eps);
    synthesis_factors(T, phys->radius, syn);
    order_maps(T, row_m, coef_m);
    for (int m = 0; m <= T; ++m)
        for (int n = m; n <= T; ++n)
            lam[order_offset(T, m) + n - m] = double(n) * double(n + 1) / (phys->radius * phys->radius);
    twiddles(L, twr, twi);
    std::vector<double2> tw(L);
    std::vector<float2> tw32(L);
    for (int k = 0; k < L; ++k) {
        tw[k] = make_double2(twr[k], twi[k]);
        tw32[k] = make_float2(float(twr[k]), float(twi[k]));
    }

    cudaError_t e = cudaSuccess;
#define SDC_TRY(call)                                                          \
    do {                                                                       \
        e = (call);                                                            \
        if (e != cudaSuccess) {                                                \
            int st_ = (e == cudaErrorMemoryAllocation) ? SDC_ENOMEM : SDC_ECUDA; \
            std::string msg_ = std::string(#call) + ": " + cudaGetErrorString(e); \
            free_ctx(c);                                                       \
            return fail(st_, msg_);                                            \
        }                                                                      \
    } while (0)

    SDC_TRY(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
    for (auto &x : c->capx) SDC_TRY(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
    SDC_TRY(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    for (auto &x : c->ev_join) SDC_TRY(cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
    SDC_TRY(configure_transform_kernels(d, c->plan, precision != SDC_FP64));
    SDC_TRY(configure_adjoint_kernels(d, c->plan, precision != SDC_FP64));
    if (precision != SDC_FP64) SDC_TRY(configure_transform_kernels(d, c->plan, false));
    if (precision == SDC_FP64) {
        SDC_TRY(upload(&c->pbar, table.data(), table.size()));
        SDC_TRY(upload(&c->tw, tw.data(), tw.size()));
    } else {
        std::vector<float> t32(table.size());
        for (size_t i = 0; i < table.size(); ++i) t32[i] = float(table[i]);
        SDC_TRY(upload(&c->pbar32, t32.data(), t32.size()));
        SDC_TRY(upload(&c->tw32, tw32.data(), tw32.size()));
        if (!fft_plan16(L, c->plan16)) { free_ctx(c); return fail(SDC_EINVAL, "no FFT plan for nlon"); }
        std::vector<double> pre, pim;
        pass_twiddles(c->plan16, twr, twi, pre, pim);
        std::vector<float2> twp(pre.size() + 1);           // never empty
        for (size_t k = 0; k < pre.size(); ++k) twp[k] = make_float2(float(pre[k]), float(pim[k]));
        c->ntwp = static_cast<int>(pre.size());
        SDC_TRY(upload(&c->twp32, twp.data(), twp.size()));
        // the scalar helpers stay FP64
        SDC_TRY(upload(&c->pbar, table.data(), table.size()));
        SDC_TRY(upload(&c->tw, tw.data(), tw.size()));
    }
    SDC_TRY(cudaMalloc(&c->tc_err, sizeof(int)));
    SDC_TRY(cudaMemset(c->tc_err, 0, sizeof(int)));
    if (precision == SDC_MIXED_BF16X3 || precision == SDC_MIXED_BF16X6) {
        std::vector<uint16_t> a3, a1;
        std::vector<TcTile3> t3;
        std::vector<TcTile1> t1;
        int kj = 0;
        const int np = precision == SDC_MIXED_BF16X3 ? 2 : 3;
        build_tc_tables(T, d.J2, d.J2p, table, np, a3, t3, a1, t1, &kj);
        SDC_TRY(upload(&c->tc_a3, a3.data(), a3.size()));
        SDC_TRY(upload(&c->tc_a1, a1.data(), a1.size()));
        SDC_TRY(upload(&c->tc_t3, t3.data(), t3.size()));
        SDC_TRY(upload(&c->tc_t1, t1.data(), t1.size()));
        SDC_TRY(configure_tc_kernels());
        c->tc.a3 = c->tc_a3;
        c->tc.a1 = c->tc_a1;
        c->tc.elems3 = static_cast<long long>(a3.size() / np);
        c->tc.elems1 = static_cast<long long>(a1.size() / np);
        c->tc.tiles3 = c->tc_t3;
        c->tc.tiles1 = c->tc_t1;
        c->tc.ntiles3 = static_cast<int>(t3.size());
        c->tc.ntiles1 = static_cast<int>(t1.size());
        c->tc.npieces = np;
        c->tc.kj = kj;
        // dynamic operands, split per launch; zero once so that K padding
        // and never-written columns stay zero
        std::vector<long long> cboff(2 * (T + 1));
        long long ncb = 0;
        for (int m = 0; m <= T; ++m)
            for (int p = 0; p < 2; ++p) {
                cboff[2 * m + p] = ncb;
                ncb += static_cast<long long>(kNbc1) * (tc_group_krows(T, m, p) / 8) * 64;
            }
        const long long nwb = 2LL * (T + 1) * kNbc3 * (kj / 8) * 64;
        SDC_TRY(cudaMalloc(&c->tc_wb, static_cast<size_t>(nwb) * np * sizeof(uint16_t)));
        SDC_TRY(cudaMemset(c->tc_wb, 0, static_cast<size_t>(nwb) * np * sizeof(uint16_t)));
        SDC_TRY(cudaMalloc(&c->tc_cb, static_cast<size_t>(ncb) * np * sizeof(uint16_t)));
        SDC_TRY(cudaMemset(c->tc_cb, 0, static_cast<size_t>(ncb) * np * sizeof(uint16_t)));
        SDC_TRY(upload(&c->tc_cboff, cboff.data(), cboff.size()));
        c->tc.wb = c->tc_wb;
        c->tc.cb = c->tc_cb;
        c->tc.wb_elems = nwb;
        c->tc.cb_elems = ncb;
        c->tc.cb_off = c->tc_cboff;
        c->tc.err = c->tc_err;
    }
    SDC_TRY(upload(&c->eps, eps.data(), eps.size()));
    SDC_TRY(upload(&c->syn, syn.data(), syn.size()));
    SDC_TRY(upload(&c->row_m, row_m.data(), row_m.size()));
    SDC_TRY(upload(&c->coef_m, coef_m.data(), coef_m.size()));
    SDC_TRY(upload(&c->lam, lam.data(), lam.size()));
    SDC_TRY(upload(&c->mu2, c->mu.data(), d.J2));
    {
        // per-latitude ring constants and FP32 epilogue factors
        std::vector<double> r64(4 * static_cast<size_t>(d.J2));
        std::vector<float> r32(r64.size());
        for (int j = 0; j < d.J2; ++j) {
            const double mu = c->mu[j], c2 = (1.0 - mu) * (1.0 + mu);
            const double v[4] = {d.two_omega * mu, 0.5 / c2, c->w[j] / c2, c->w[j]};
            for (int k = 0; k < 4; ++k) { r64[4 * j + k] = v[k]; r32[4 * j + k] = float(v[k]); }
        }
        SDC_TRY(upload(&c->ring64, r64.data(), r64.size()));
        SDC_TRY(upload(&c->ring32, r32.data(), r32.size()));
        std::vector<float> e32(4 * static_cast<size_t>(d.ncoef));
        for (int m = 0; m <= T; ++m)
            for (int n = m; n <= T; ++n) {
                const size_t i = static_cast<size_t>(order_offset(T, m) + n - m);
                const int x = ext_offset(T, m) + n - m;
                e32[4 * i + 0] = float(n * eps[x + 1]);
                e32[4 * i + 1] = float(n > m ? (n + 1.0) * eps[x] : 0.0);
                e32[4 * i + 2] = float(lam[i]);
                e32[4 * i + 3] = 0.f;
            }
        SDC_TRY(upload(&c->epi32, e32.data(), e32.size()));
        std::vector<float> s32(4 * static_cast<size_t>(d.next));
        for (size_t r = 0; r < static_cast<size_t>(d.next); ++r)
            for (int k = 0; k < 3; ++k) s32[4 * r + k] = float(syn[3 * r + k]);
        SDC_TRY(upload(&c->syn32, s32.data(), s32.size()));
    }
    SDC_TRY(upload(&c->w2, c->w.data(), d.J2));

    const size_t sbytes = 3ULL * d.ncoef * sizeof(double2);
    SDC_TRY(cudaMalloc(&c->un, sbytes));
    SDC_TRY(cudaMalloc(&c->U, sbytes * M));
    SDC_TRY(cudaMalloc(&c->E, sbytes * M));
    SDC_TRY(cudaMalloc(&c->E0, sbytes));
    const size_t f1b = static_cast<size_t>(M) * d.J2 * 8 * (T + 1) * elem;
    const size_t f2b = static_cast<size_t>(M) * (T + 1) * 10 * d.J2 * elem;
    const size_t scal = static_cast<size_t>(d.J2) * 2 * (T + 1) * sizeof(double2);   // scalar helpers (FP64)
    SDC_TRY(cudaMalloc(&c->f1, f1b > scal ? f1b : scal));
    SDC_TRY(cudaMalloc(&c->f2, f2b > scal ? f2b : scal));
    SDC_TRY(cudaMalloc(&c->f3, static_cast<size_t>(M) * d.next * 5 * elem));
    c->sweep_nblocks = sweep_blocks(d.ncoef, M);
    SDC_TRY(cudaMalloc(&c->resid_part, static_cast<size_t>(c->sweep_nblocks) * M * 3 * sizeof(double)));
    SDC_TRY(cudaMalloc(&c->resid, static_cast<size_t>(K) * 3 * sizeof(double)));
    SDC_TRY(cudaMalloc(&c->den, static_cast<size_t>(K) * M * d.ncoef * sizeof(double)));
    SDC_TRY(upload_denominators(c));
    // adjoint: recorded grid fields of one step's evaluations, node adjoints,
    // checkpoint pool, loss buffers
    const int nslots = std::max(1 + (K - 1) * M, M);
    SDC_TRY(cudaMalloc(&c->gstore, grid_slot_bytes(c) * nslots));
    SDC_TRY(cudaMalloc(&c->ub, sbytes * M));
    SDC_TRY(cudaMalloc(&c->eb, sbytes * M));
    SDC_TRY(cudaMalloc(&c->ubn, sbytes));
    SDC_TRY(cudaMalloc(&c->ubnext, sbytes));
    SDC_TRY(cudaMalloc(&c->eb0, sbytes));
    SDC_TRY(cudaMalloc(&c->snaps, sbytes * kMaxSnapshots));
    SDC_TRY(cudaMalloc(&c->phigrid, sizeof(double) * J * L));
    SDC_TRY(cudaMalloc(&c->rgrid, sizeof(double) * J * L));
    SDC_TRY(cudaMalloc(&c->loss_part, sizeof(double) * loss_blocks()));
    SDC_TRY(cudaMalloc(&c->loss_dev, sizeof(double)));
    SDC_TRY(cudaDeviceSynchronize());
#undef SDC_TRY
    *out = c;
    return SDC_OK;
}

int sdc_destroy(sdc_ctx *c) {
    if (!c) return SDC_OK;
    cudaStreamSynchronize(c->stream);
    free_ctx(c);
    return SDC_OK;
}

int sdc_set_option(sdc_ctx *c, int key, int value) {
    if (!c) return fail(SDC_EINVAL, "ctx is NULL");
    if (key == SDC_OPT_QDELTA_RULE) {
        if (value < SDC_QDELTA_CLAMPED || value > SDC_QDELTA_MIN_SR_S) return fail(SDC_EINVAL, "bad q-delta rule");
        if (value == SDC_QDELTA_MIN_SR_S && c->qd_min_sr_s.empty()) {
            std::vector<double> dd;
            if (!min_sr_s_diagonal(c->M, c->tau, c->Q, dd))
                return fail(SDC_EUNSUPPORTED, "MIN-SR-S diagonal not reached for this node count");
            c->qd_min_sr_s = dd;
        }
        if (value != c->qdelta_rule) {
            c->qdelta_rule = value;
            SDC_CUDA(cudaStreamSynchronize(c->stream));
            SDC_CUDA(upload_denominators(c));
            for (auto &g : c->graph)
                if (g) { cudaGraphExecDestroy(g); g = nullptr; }
            if (c->graph_retape) { cudaGraphExecDestroy(c->graph_retape); c->graph_retape = nullptr; }
            if (c->graph_adjoint) { cudaGraphExecDestroy(c->graph_adjoint); c->graph_adjoint = nullptr; }
        }
        return SDC_OK;
    }
    if (key == SDC_OPT_METHOD) {
        if (value != SDC_METHOD_DSDC && value != SDC_METHOD_SERIAL_SDC && value != SDC_METHOD_IMEX2)
            return fail(SDC_EINVAL, "bad method");
        if (value != SDC_METHOD_DSDC && !c->alt) {
            const size_t n = static_cast<size_t>(c->M > 2 ? 2 * c->M : 4) * c->state_elems();
            SDC_CUDA(cudaMalloc(&c->alt, n * sizeof(double2)));
        }
        if (value != c->method) {
            SDC_CUDA(cudaStreamSynchronize(c->stream));
            c->method = value;
            for (auto &g : c->graph)
                if (g) { cudaGraphExecDestroy(g); g = nullptr; }
        }
        return SDC_OK;
    }
    if (key == SDC_OPT_LEGENDRE) {
        if (value != SDC_LEGENDRE_TABLE && value != SDC_LEGENDRE_RECURRENCE)
            return fail(SDC_EINVAL, "bad Legendre source");
        if (value == SDC_LEGENDRE_RECURRENCE && c->precision != SDC_MIXED_FP32)
            return fail(SDC_EUNSUPPORTED, "the Legendre recurrence serves the FP32 synthesis only");
        if (value == SDC_LEGENDRE_RECURRENCE && !c->rec_ab) {
            const Dims &d = c->d;
            std::vector<double> table;
            legendre_table(c->T, d.J2, d.J2p, c->mu, table);
            std::vector<float> ab, seed, mu2;
            recurrence_tables(c->T, d.J2, d.J2p, c->mu, table, ab, seed, mu2);
            auto up = [&](float **dst, const std::vector<float> &v) -> cudaError_t {
                cudaError_t e = cudaMalloc(dst, v.size() * sizeof(float));
                if (e != cudaSuccess) return e;
                return cudaMemcpy(*dst, v.data(), v.size() * sizeof(float), cudaMemcpyHostToDevice);
            };
            SDC_CUDA(up(&c->rec_ab, ab));
            SDC_CUDA(up(&c->rec_seed, seed));
            SDC_CUDA(up(&c->rec_mu, mu2));
        }
        if (value != c->legendre) {
            SDC_CUDA(cudaStreamSynchronize(c->stream));
            c->legendre = value;
            for (auto &g : c->graph)
                if (g) { cudaGraphExecDestroy(g); g = nullptr; }
            if (c->graph_retape) { cudaGraphExecDestroy(c->graph_retape); c->graph_retape = nullptr; }
        }
        return SDC_OK;
    }
    if (key == SDC_OPT_CHAINS) {
        if (value < 1 || value > kMaxChains) return fail(SDC_EINVAL, "chains must be 1 to 4");
        if (value != c->chains) {
            SDC_CUDA(cudaStreamSynchronize(c->stream));
            c->chains = value;
            for (auto &g : c->graph)
                if (g) { cudaGraphExecDestroy(g); g = nullptr; }
            if (c->graph_retape) { cudaGraphExecDestroy(c->graph_retape); c->graph_retape = nullptr; }
        }
        return SDC_OK;
    }
    if (key == SDC_OPT_PDL) {
        if (value != 0 && value != 1) return fail(SDC_EINVAL, "pdl must be 0 or 1");
        if (value != c->pdl) {
            SDC_CUDA(cudaStreamSynchronize(c->stream));
            c->pdl = value;
            for (auto &g : c->graph)
                if (g) { cudaGraphExecDestroy(g); g = nullptr; }
            if (c->graph_retape) { cudaGraphExecDestroy(c->graph_retape); c->graph_retape = nullptr; }
        }
        return SDC_OK;
    }
    if (key == SDC_OPT_SERIAL_IMPLICIT) {
        if (value != SDC_SERIAL_IMPLICIT_EULER && value != SDC_SERIAL_IMPLICIT_LU)
            return fail(SDC_EINVAL, "bad serial implicit weights");
        if (value == SDC_SERIAL_IMPLICIT_LU && c->qi_lu.empty()) {
            std::vector<double> qd;
            if (!lu_implicit_weights(c->M, c->Q, qd)) return fail(SDC_EUNSUPPORTED, "Q^T has no LU factorisation");
            c->qi_lu = qd;
        }
        if (value != c->serial_implicit) {
            SDC_CUDA(cudaStreamSynchronize(c->stream));
            c->serial_implicit = value;
            for (auto &g : c->graph)
                if (g) { cudaGraphExecDestroy(g); g = nullptr; }
        }
        return SDC_OK;
    }
    return fail(SDC_EINVAL, "unknown option");
}

int sdc_ncoef(const sdc_ctx *c) { return c ? c->d.ncoef : -1; }

int sdc_step(sdc_ctx *c, const void *in, void *out, double *resid_out) {
    if (!c || !in || !out) return fail(SDC_EINVAL, "NULL argument");
    if (resid_out && c->method != SDC_METHOD_DSDC) return fail(SDC_EUNSUPPORTED, "residuals need the dSDC method");
    const size_t sbytes = 3ULL * c->d.ncoef * sizeof(double2);
    SDC_CUDA(cudaMemcpyAsync(c->un, in, sbytes, cudaMemcpyDeviceToDevice, c->stream));
    int st = run_steps(c, 1, resid_out != nullptr);
    if (st != SDC_OK) return st;
    SDC_CUDA(cudaMemcpyAsync(out, c->un, sbytes, cudaMemcpyDeviceToDevice, c->stream));
    if (resid_out) {
        SDC_CUDA(cudaMemcpyAsync(resid_out, c->resid, sizeof(double) * 3 * c->K, cudaMemcpyDeviceToHost, c->stream));
        SDC_CUDA(cudaStreamSynchronize(c->stream));
        for (int i = 0; i < 3 * c->K; ++i)
            if (!std::isfinite(resid_out[i])) return fail(SDC_EDIVERGED, "non-finite residual norm");
    }
    return SDC_OK;
}

int sdc_run(sdc_ctx *c, void *state, int nsteps) {
    if (!c || !state) return fail(SDC_EINVAL, "NULL argument");
    if (nsteps < 0) return fail(SDC_EINVAL, "nsteps < 0");
    if (nsteps == 0) return SDC_OK;
    const size_t sbytes = 3ULL * c->d.ncoef * sizeof(double2);
    SDC_CUDA(cudaMemcpyAsync(c->un, state, sbytes, cudaMemcpyDeviceToDevice, c->stream));
    int st = run_steps(c, nsteps, false);
    if (st != SDC_OK) return st;
    SDC_CUDA(cudaMemcpyAsync(state, c->un, sbytes, cudaMemcpyDeviceToDevice, c->stream));
    return SDC_OK;
}

int sdc_tendency(sdc_ctx *c, const void *states, void *tend, int batch) {
    if (!c || !states || !tend) return fail(SDC_EINVAL, "NULL argument");
    if (batch < 1 || batch > c->M) return fail(SDC_EINVAL, "batch must be in [1, nodes]");
    int launches = 0;
    const long long se = c->state_elems();
    cudaError_t e = tendency(c, batch, static_cast<const double2 *>(states), se, static_cast<double2 *>(tend), se,
                             c->stream, &launches);
    if (e != cudaSuccess) return cuda_fail(e, "tendency");
    c->n_explicit += batch;
    c->n_launch += launches;
    return SDC_OK;
}

int sdc_spec_to_grid(sdc_ctx *c, const void *spec, double *grid) {
    if (!c || !spec || !grid) return fail(SDC_EINVAL, "NULL argument");
    cudaError_t e = launch_spec_to_grid(c->d, c->plan, static_cast<const double2 *>(spec), grid, c->pbar, c->tw,
                                        static_cast<double2 *>(c->f1), c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "spec_to_grid");
    c->n_launch += 2;
    return SDC_OK;
}

int sdc_grid_to_spec(sdc_ctx *c, const double *grid, void *spec) {
    if (!c || !spec || !grid) return fail(SDC_EINVAL, "NULL argument");
    cudaError_t e = launch_grid_to_spec(c->d, c->plan, grid, static_cast<double2 *>(spec), c->pbar, c->w2, c->tw,
                                        static_cast<double2 *>(c->f2), c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "grid_to_spec");
    c->n_launch += 2;
    return SDC_OK;
}

int sdc_grid_coords(const sdc_ctx *c, double *mu, double *w) {
    if (!c) return fail(SDC_EINVAL, "ctx is NULL");
    if (mu) std::memcpy(mu, c->mu.data(), sizeof(double) * c->J);
    if (w) std::memcpy(w, c->w.data(), sizeof(double) * c->J);
    return SDC_OK;
}

int sdc_collocation(const sdc_ctx *c, double *tau, double *Q) {
    if (!c) return fail(SDC_EINVAL, "ctx is NULL");
    if (tau) std::memcpy(tau, c->tau.data(), sizeof(double) * c->M);
    if (Q) std::memcpy(Q, c->Q.data(), sizeof(double) * c->M * c->M);
    return SDC_OK;
}

// Checkpoint file: one JSON header line, then the raw FP64 state [3][ncoef]
// (16 bytes per complex coefficient, the machine's little-endian layout).
static const char kStateFormat[] = "sdc-swe-state-1";

int sdc_save(sdc_ctx *c, const void *state, long long step, const char *path) {
    if (!c || !state || !path) return fail(SDC_EINVAL, "NULL argument");
    const size_t n = 3ULL * c->d.ncoef;
    std::vector<double2> h(n);
    SDC_CUDA(cudaMemcpyAsync(h.data(), state, n * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
    SDC_CUDA(cudaStreamSynchronize(c->stream));
    char hdr[1024];
    const int len = std::snprintf(
        hdr, sizeof(hdr),
        "{\"format\": \"%s\", \"truncation\": %d, \"nlat\": %d, \"nlon\": %d, \"nodes\": %d, "
        "\"sweeps\": %d, \"dt\": %.17g, \"radius\": %.17g, \"omega\": %.17g, \"gravity\": %.17g, "
        "\"mean_depth\": %.17g, \"step\": %lld, \"ncoef\": %d, \"fields\": [\"phi\", \"zeta\", \"div\"], "
        "\"bytes\": %zu}\n",
        kStateFormat, c->T, c->J, c->L, c->M, c->K, c->dt, c->phys.radius, c->phys.omega, c->phys.gravity,
        c->phys.mean_depth, step, c->d.ncoef, n * sizeof(double2));
    if (len <= 0 || len >= static_cast<int>(sizeof(hdr))) return fail(SDC_EINVAL, "header too long");
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(SDC_EINVAL, "cannot open the file for writing");
    const bool ok = std::fwrite(hdr, 1, static_cast<size_t>(len), f) == static_cast<size_t>(len) &&
                    std::fwrite(h.data(), sizeof(double2), n, f) == n;
    if (std::fclose(f) != 0 || !ok) return fail(SDC_EINVAL, "cannot write the file");
    return SDC_OK;
}

// value of an integer field "key": N in a one-line JSON header (false if absent)
static bool header_int(const std::string &hdr, const char *key, long long *out) {
    const std::string k = std::string("\"") + key + "\":";
    const size_t at = hdr.find(k);
    if (at == std::string::npos) return false;
    const char *p = hdr.c_str() + at + k.size();
    char *end = nullptr;
    *out = std::strtoll(p, &end, 10);
    return end != p;
}

// value of a floating-point field "key": x (printed with %.17g, so strtod
// gives back the same double) in a one-line JSON header (false if absent)
static bool header_double(const std::string &hdr, const char *key, double *out) {
    const std::string k = std::string("\"") + key + "\":";
    const size_t at = hdr.find(k);
    if (at == std::string::npos) return false;
    const char *p = hdr.c_str() + at + k.size();
    char *end = nullptr;
    *out = std::strtod(p, &end);
    return end != p;
}

int sdc_load(sdc_ctx *c, void *state, long long *step, const char *path) {
    if (!c || !state || !path) return fail(SDC_EINVAL, "NULL argument");
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(SDC_EINVAL, "cannot open the file for reading");
    std::string hdr;
    for (int ch; (ch = std::fgetc(f)) != EOF && ch != '\n' && hdr.size() < 4096;) hdr.push_back(static_cast<char>(ch));
    long long T = -1, nc = -1, st = 0, bytes = -1;
    const size_t n = 3ULL * c->d.ncoef;
    const bool hdr_ok = hdr.find(std::string("\"format\": \"") + kStateFormat + "\"") != std::string::npos &&
                        header_int(hdr, "truncation", &T) && header_int(hdr, "ncoef", &nc) &&
                        header_int(hdr, "step", &st) && header_int(hdr, "bytes", &bytes);
    if (!hdr_ok) {
        std::fclose(f);
        return fail(SDC_EINVAL, "not a state file of this library");
    }
    if (T != c->T || nc != c->d.ncoef || bytes != static_cast<long long>(n * sizeof(double2))) {
        std::fclose(f);
        return fail(SDC_EINVAL, "state file of another truncation");
    }
    // the step count only means a model time under the same grid, nodes,
    // sweeps, step size and physical constants: all must match exactly
    long long J = -1, L = -1, M = -1, K = -1;
    double dt = 0, a = 0, om = 0, g = 0, H = 0;
    const bool same = header_int(hdr, "nlat", &J) && header_int(hdr, "nlon", &L) && header_int(hdr, "nodes", &M) &&
                      header_int(hdr, "sweeps", &K) && header_double(hdr, "dt", &dt) &&
                      header_double(hdr, "radius", &a) && header_double(hdr, "omega", &om) &&
                      header_double(hdr, "gravity", &g) && header_double(hdr, "mean_depth", &H) && J == c->J &&
                      L == c->L && M == c->M && K == c->K && dt == c->dt && a == c->phys.radius &&
                      om == c->phys.omega && g == c->phys.gravity && H == c->phys.mean_depth;
    if (!same) {
        std::fclose(f);
        return fail(SDC_EINVAL, "state file of another configuration (grid, nodes, sweeps, dt or constants)");
    }
    std::vector<double2> h(n);
    const bool got = std::fread(h.data(), sizeof(double2), n, f) == n && std::fgetc(f) == EOF;
    std::fclose(f);
    if (!got) return fail(SDC_EINVAL, "state file truncated or too long");
    SDC_CUDA(cudaMemcpyAsync(state, h.data(), n * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
    SDC_CUDA(cudaStreamSynchronize(c->stream));
    if (step) *step = st;
    return SDC_OK;
}

int sdc_qdelta(int nodes, int rule, int sweep, double *qdelta) {
    if (nodes < 1 || nodes > kMaxNodes || sweep < 1 || !qdelta) return fail(SDC_EINVAL, "bad argument");
    if (rule < SDC_QDELTA_CLAMPED || rule > SDC_QDELTA_MIN_SR_S) return fail(SDC_EINVAL, "bad q-delta rule");
    std::vector<double> tau, Q, mss;
    radau_right(nodes, tau, Q);
    if (rule == SDC_QDELTA_MIN_SR_S && !min_sr_s_diagonal(nodes, tau, Q, mss))
        return fail(SDC_EUNSUPPORTED, "MIN-SR-S diagonal not reached for this node count");
    for (int m = 0; m < nodes; ++m) qdelta[m] = qdelta_value(rule, nodes, tau, mss, sweep, m);
    return SDC_OK;
}

int sdc_counters(const sdc_ctx *c, long long *evals, long long *solves, long long *launches) {
    if (!c) return fail(SDC_EINVAL, "ctx is NULL");
    if (evals) *evals = c->n_explicit;
    if (solves) *solves = c->n_solve;
    if (launches) *launches = c->n_launch;
    return SDC_OK;
}

int sdc_tendency_adjoint(sdc_ctx *c, const void *states, const void *abar, void *ubar, int batch) {
    if (!c || !states || !abar || !ubar) return fail(SDC_EINVAL, "NULL argument");
    if (batch < 1 || batch > c->M) return fail(SDC_EINVAL, "batch must be in [1, nodes]");
    const long long se = c->state_elems();
    int launches = 0;
    // forward evaluation records the base grid fields (its tendency output is scratch)
    cudaError_t e = tendency(c, batch, static_cast<const double2 *>(states), se, c->E, se, c->stream, &launches,
                             nullptr, grid_slot(c, 0));
    if (e != cudaSuccess) return cuda_fail(e, "tendency (record)");
    SDC_CUDA(cudaMemsetAsync(ubar, 0, sizeof(double2) * se * batch, c->stream));
    e = launch_tendency_adjoint(c->d, c->plan, c->precision != SDC_FP64, batch, grid_slot(c, 0),
                                static_cast<const double2 *>(abar), se, static_cast<double2 *>(ubar), se,
                                tables(c), Workspace{c->f1, c->f2, c->f3}, c->stream, &launches);
    if (e != cudaSuccess) return cuda_fail(e, "tendency adjoint");
    c->n_launch += launches;
    return SDC_OK;
}

int sdc_step_adjoint(sdc_ctx *c, const void *state_n, const void *ubar_next, void *ubar_n) {
    if (!c || !state_n || !ubar_next || !ubar_n) return fail(SDC_EINVAL, "NULL argument");
    if (c->method != SDC_METHOD_DSDC) return fail(SDC_EUNSUPPORTED, "the adjoint is built for the dSDC method");
    const size_t sbytes = 3ULL * c->d.ncoef * sizeof(double2);
    SDC_CUDA(cudaMemcpyAsync(c->un, state_n, sbytes, cudaMemcpyDeviceToDevice, c->stream));
    SDC_CUDA(cudaMemcpyAsync(c->ubnext, ubar_next, sbytes, cudaMemcpyDeviceToDevice, c->stream));
    int st = reverse_one(c, nullptr, false);
    if (st != SDC_OK) return st;
    SDC_CUDA(cudaMemcpyAsync(ubar_n, c->ubnext, sbytes, cudaMemcpyDeviceToDevice, c->stream));
    return SDC_OK;
}

static int adjoint_common(sdc_ctx *c, const void *state0, int nsteps, int nsnapshots, const void *ubar_final,
                          const double *h_target, double *loss_out, void *ubar_initial) {
    if (!c || !state0 || !ubar_initial) return fail(SDC_EINVAL, "NULL argument");
    if (c->method != SDC_METHOD_DSDC) return fail(SDC_EUNSUPPORTED, "the adjoint is built for the dSDC method");
    if (nsteps < 0 || nsteps > 4096) return fail(SDC_EINVAL, "nsteps must be in [0, 4096]");
    if (nsnapshots < 1 || nsnapshots > kMaxSnapshots) return fail(SDC_EINVAL, "nsnapshots must be in [1, 32]");
    const size_t sbytes = 3ULL * c->d.ncoef * sizeof(double2);
    SDC_CUDA(cudaMemcpyAsync(c->un, state0, sbytes, cudaMemcpyDeviceToDevice, c->stream));
    c->adj_forward_steps = 0;
    if (nsteps == 0) {
        if (h_target) {
            SDC_CUDA(cudaMemsetAsync(c->ubnext, 0, sbytes, c->stream));
            SDC_CUDA(launch_spec_to_grid(c->d, c->plan, c->un, c->phigrid, c->pbar, c->tw,
                                         static_cast<double2 *>(c->f1), c->stream));
            SDC_CUDA(launch_height_loss(c->d, c->plan, c->phigrid, h_target, 1.0 / c->phys.gravity,
                                        c->phys.mean_depth, c->rgrid, c->loss_part, c->loss_dev, c->ubnext,
                                        c->pbar, c->tw, static_cast<double2 *>(c->f2), c->stream));
        } else {
            SDC_CUDA(cudaMemcpyAsync(c->ubnext, ubar_final, sbytes, cudaMemcpyDeviceToDevice, c->stream));
        }
    } else {
        if (!h_target)
            SDC_CUDA(cudaMemcpyAsync(c->ubnext, ubar_final, sbytes, cudaMemcpyDeviceToDevice, c->stream));
        Reverser r;
        r.c = c;
        r.h_target = h_target;
        r.N = nsteps;
        r.sbytes = sbytes;
        const int sfree = nsnapshots - 1;
        r.sched.build(nsteps, sfree);
        for (int k = nsnapshots - 1; k >= 1; --k) r.free_slots.push_back(k);
        int st = r.store(0);
        if (st != SDC_OK) return st;
        st = r.rev(0, nsteps, sfree, 0);
        if (st != SDC_OK) return st;
    }
    SDC_CUDA(cudaMemcpyAsync(ubar_initial, c->ubnext, sbytes, cudaMemcpyDeviceToDevice, c->stream));
    if (loss_out) {
        SDC_CUDA(cudaMemcpyAsync(loss_out, c->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        SDC_CUDA(cudaStreamSynchronize(c->stream));
    }
    return SDC_OK;
}

int sdc_run_adjoint(sdc_ctx *c, const void *state0, int nsteps, int nsnapshots, const void *ubar_final,
                    void *ubar_initial, long long *forward_steps) {
    if (!ubar_final) return fail(SDC_EINVAL, "NULL argument");
    int st = adjoint_common(c, state0, nsteps, nsnapshots, ubar_final, nullptr, nullptr, ubar_initial);
    if (st == SDC_OK && forward_steps) {
        SDC_CUDA(cudaStreamSynchronize(c->stream));
        *forward_steps = c->adj_forward_steps;
    }
    return st;
}

int sdc_adjoint_run(sdc_ctx *c, const void *state0, int nsteps, int nsnapshots, const double *h_target,
                    double *loss_out, void *grad_out) {
    if (!h_target || !loss_out) return fail(SDC_EINVAL, "NULL argument");
    return adjoint_common(c, state0, nsteps, nsnapshots, nullptr, h_target, loss_out, grad_out);
}

int sdc_profile_step(sdc_ctx *c, void *state, double *ms, int *launches) {
    if (!c || !state || !ms || !launches) return fail(SDC_EINVAL, "NULL argument");
    StageTimer tm;
    tm.stream = c->stream;
    for (int i = 0; i <= StageTimer::kMax; ++i) {
        cudaError_t e = cudaEventCreate(&tm.ev[i]);
        if (e != cudaSuccess) {
            for (int k = 0; k < i; ++k) cudaEventDestroy(tm.ev[k]);
            return cuda_fail(e, "cudaEventCreate");
        }
    }
    const size_t sbytes = 3ULL * c->d.ncoef * sizeof(double2);
    int nl = 0;
    cudaError_t e = cudaMemcpyAsync(c->un, state, sbytes, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = enqueue_step(c, c->stream, false, &nl, &tm);
    tm.end();
    if (e == cudaSuccess) e = cudaMemcpyAsync(state, c->un, sbytes, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) {
        for (int k = 0; k < NSTAGES; ++k) { ms[k] = 0.0; launches[k] = 0; }
        for (int i = 0; i < tm.n; ++i) {
            float t = 0.f;
            cudaEventElapsedTime(&t, tm.ev[i], tm.ev[i + 1]);
            ms[tm.cls[i]] += t;
            launches[tm.cls[i]] += 1;
        }
        c->n_explicit += evals_per_step(c);
        c->n_solve += solves_per_step(c);
        c->n_launch += nl;
    }
    for (int i = 0; i <= StageTimer::kMax; ++i) cudaEventDestroy(tm.ev[i]);
    if (e != cudaSuccess) return cuda_fail(e, "profiled step");
    return SDC_OK;
}

int sdc_sync(sdc_ctx *c) {
    if (!c) return fail(SDC_EINVAL, "ctx is NULL");
    SDC_CUDA(cudaStreamSynchronize(c->stream));
    SDC_CUDA(cudaGetLastError());
    if (c->tc_err) {
        int flag = 0;
        SDC_CUDA(cudaMemcpy(&flag, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (flag) return fail(SDC_ECUDA, "a tensor-core kernel gave up a bounded wait (code " + std::to_string(flag) + ")");
    }
    return SDC_OK;
}

int sdc_launches_per_step(const sdc_ctx *c, int *launches) {
    if (!c || !launches) return fail(SDC_EINVAL, "NULL argument");
    sdc_ctx *cc = const_cast<sdc_ctx *>(c);
    int st = ensure_graph(cc, false);
    if (st != SDC_OK) return st;
    *launches = c->graph_launches[0];
    return SDC_OK;
}

}  // extern "C"
