/*
 * sdc.h -- C ABI of the GB300 node-parallel diagonal IMEX SDC sweep for the
 * rotating shallow-water equations in spherical-harmonic vorticity-divergence
 * form (Freese, Goetschel, Lunet, Ruprecht, Schreiber: "Parallel performance
 * of shared memory parallel spectral deferred corrections", arXiv 2403.20135,
 * the SWEET variant of Sec. 3.2 and Sec. 4.4).
 *
 * Conventions shared by every call
 * --------------------------------
 * State: three complex spectral fields in the order (Phi', zeta, div) -- the
 *   paper's U-hat of Sec. 3.2 (it writes rho for the divergence) -- stored as
 *   double2 (re, im) in DEVICE memory, layout state[3][ncoef].  Coefficient
 *   (n, m), 0 <= m <= n <= T, sits at m (2T + 3 - m) / 2 + (n - m)
 *   ("m-major triangular").  Basis: normalised associated Legendre functions
 *   (integral of Pbar^2 over [-1, 1] equal to 1, no Condon-Shortley phase)
 *   times e^{i m lambda}; a real field is f_0 + 2 Re sum_{m>0}.  Im of the
 *   m = 0 coefficients is 0 on input and stays 0.
 * Grid: nlat Gauss-Legendre latitudes ordered north to south, nlon equally
 *   spaced longitudes from 0; grid arrays are double [nlat][nlon].
 * Phi' = g (h - H) is the geopotential perturbation, Phibar = g H.
 * Streams: every call is asynchronous on the stream given to sdc_create,
 *   except where a HOST output (resid_out, loss_out, counters) is requested;
 *   those calls synchronise that stream before returning.
 * Ownership: the caller owns every state, grid and gradient buffer it passes;
 *   the library owns its tables, workspaces and CUDA graphs, all allocated in
 *   sdc_create and released in sdc_destroy.  No call other than sdc_create
 *   allocates device memory.
 * Errors: every call returns an sdc_status; no exception or abort crosses the
 *   ABI.  sdc_last_error() returns a thread-local description of the last
 *   failure on the calling thread.  After SDC_ECUDA the context must be
 *   destroyed.
 */
#ifndef SDC_H_
#define SDC_H_

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sdc_ctx sdc_ctx;

/* Physical constants: sphere radius a [m], rotation rate Omega [1/s],
 * gravity g [m/s^2], mean depth H [m] (Sec. 3.2, Eq. (4)). */
typedef struct {
    double radius;
    double omega;
    double gravity;
    double mean_depth;
} sdc_phys;

/* Arithmetic of the explicit tendency's spectral transforms.  The implicit
 * solves, the collocation (quadrature) accumulation and the residual norms
 * are FP64 in every mode. */
typedef enum {
    SDC_FP64 = 0,          /* transforms in FP64 */
    SDC_MIXED_FP32 = 1,    /* Legendre contractions and ring FFTs in FP32 */
    SDC_MIXED_BF16X3 = 2,  /* ring FFTs in FP32; Legendre contractions on the
                              tensor cores (tcgen05) with operands split into 2
                              BF16 pieces, 3 piece products, FP32 accumulation */
    SDC_MIXED_BF16X6 = 3   /* as SDC_MIXED_BF16X3 with 3 BF16 pieces and 6
                              piece products (about FP32 accuracy) */
} sdc_precision;

typedef enum {
    SDC_OK = 0,
    SDC_EINVAL = 1,        /* an argument is out of range (see each call) */
    SDC_ENOMEM = 2,        /* device or host allocation failed in sdc_create */
    SDC_ECUDA = 3,         /* a CUDA runtime call failed */
    SDC_EDIVERGED = 4,     /* a requested residual norm is not finite */
    SDC_ESTATE = 5,        /* call not valid in the context's current state */
    SDC_EUNSUPPORTED = 6   /* option/precision not available for these sizes */
} sdc_status;

/* Option keys for sdc_set_option. */
typedef enum {
    /* Diagonal coefficients q^Delta_{m,m} of the implicit part in Eq. (7)
     * (Sec. 4.2), at sweep k = 1..K:
     * SDC_QDELTA_CLAMPED (default): MIN-SR-FLEX tau_m / q(k) with
     *   q(k) = min(k, M) (the paper always runs K = M);
     * SDC_QDELTA_LITERAL: MIN-SR-FLEX with q(k) = k;
     * SDC_QDELTA_MIN_SR_NS: tau_m / M in every sweep (Q - diag(q^Delta) is
     *   nilpotent: the iteration's non-stiff limit);
     * SDC_QDELTA_IMPLICIT_EULER: tau_m in every sweep (one implicit Euler
     *   step from t_n to each node);
     * SDC_QDELTA_MIN_SR_S: in every sweep the positive diagonal, increasing
     *   in m, for which I - diag(q^Delta)^{-1} Q is nilpotent (the stiff limit
     *   of the sweep vanishes after M sweeps), found once per context by
     *   damped Newton; SDC_EUNSUPPORTED if it is not reached.
     * Any other value returns SDC_EINVAL.  Changing the rule re-uploads the
     * solve denominators and drops the captured graphs. */
    SDC_OPT_QDELTA_RULE = 1,
    /* The integrator sdc_step / sdc_run / sdc_profile_step advance with:
     * SDC_METHOD_DSDC (default): diagonal IMEX SDC, Algorithm 2, Eq. (7);
     * SDC_METHOD_SERIAL_SDC: serial IMEX SDC, Algorithm 1 with Eq. (6)
     *   (same nodes, collocation matrix and K; node updates sequential, each
     *   followed by one tendency evaluation: K M evaluations and K M solves
     *   per step);
     * SDC_METHOD_IMEX2: IMEX-o2 of Sec. 3.2, Strang splitting with
     *   Crank-Nicolson half steps on L_g around one Heun step on T_E
     *   (2 evaluations, 2 solves per step).
     * The reference integrators run in the context's precision for T_E and FP64
     * elsewhere; residual output and the adjoint calls (except
     * sdc_tendency_adjoint) need SDC_METHOD_DSDC and return SDC_EUNSUPPORTED
     * otherwise.  Selecting a reference integrator the first time allocates
     * max(2 nodes, 4) extra states (SDC_ECUDA / SDC_ENOMEM on failure). */
    SDC_OPT_METHOD = 2,
    /* Implicit node weights of serial IMEX SDC (SDC_METHOD_SERIAL_SDC), the
     * lower-triangular q^Delta of Eq. (6):
     * SDC_SERIAL_IMPLICIT_EULER (default): dtau_j, backward Euler across the
     *   node intervals as Eq. (6) writes it;
     * SDC_SERIAL_IMPLICIT_LU: the transpose of the upper factor of the
     *   Doolittle factorisation Q^T = L U (the lower-triangular choice of
     *   Sec. 4.2's first paragraph, which makes the stiff-limit sweep matrix
     *   I - q^Delta^{-1} Q = I - L^T nilpotent).
     * The explicit weights stay forward Euler (dtau_{j+1}). */
    SDC_OPT_SERIAL_IMPLICIT = 3,
    /* Source of the normalised Legendre functions in the FP32 synthesis
     * (SDC_MIXED_FP32 contexts only; SDC_EUNSUPPORTED in the other modes):
     * SDC_LEGENDRE_TABLE (default): rows of the precomputed FP32 table;
     * SDC_LEGENDRE_RECURRENCE: generated on the fly by the three-term
     *   recurrence in n of the normalised functions (the recurrence that also
     *   builds the table, SHTns-style regeneration, Sec. 6), in FP32-pair
     *   arithmetic from the FP64 values of Pbar_m^m and Pbar_{m+1}^m, so the
     *   synthesis streams no table.  Selecting it the first time builds and
     *   uploads its coefficient and seed tables (host work and a small device
     *   allocation; SDC_ECUDA on failure).  The analysis projection and the
     *   adjoint's transposed transforms keep the table.  Changing the source
     *   drops the captured graphs. */
    SDC_OPT_LEGENDRE = 4,
    /* Concurrent state chains of a tendency batch in the captured step and
     * retape graphs: 1 runs the transforms of the batch's states as one
     * launch per stage; 2 (default) to 4 split the states into that many
     * parts (at most one per state) whose transforms run on as many streams
     * inside the graph, so that one part's kernels fill the SMs the others'
     * leave idle.  The arithmetic and the results are the same.  The
     * tensor-core modes stay on one chain.  Any other value returns
     * SDC_EINVAL; changing it drops the captured graphs. */
    SDC_OPT_CHAINS = 5,
    /* Programmatic dependent launch inside the captured step and retape
     * graphs: 1 (default) launches the sweep and the FP32 synthesis, ring and
     * projection kernels as programmatic dependents of their predecessors, so
     * that their launch overlaps the predecessor's last blocks (the sweep lets
     * its successor start as soon as all its own blocks run); a kernel does
     * only the work that needs none of its predecessors' results (table and
     * twiddle prefetch, barrier set-up) before it waits for their completion,
     * so the results are the same.  0 launches every kernel after its
     * predecessor has completed.  Any other value returns SDC_EINVAL; changing
     * it drops the captured graphs. */
    SDC_OPT_PDL = 6
} sdc_option;
enum {
    SDC_LEGENDRE_TABLE = 0,
    SDC_LEGENDRE_RECURRENCE = 1
};
enum {
    SDC_QDELTA_CLAMPED = 0,
    SDC_QDELTA_LITERAL = 1,
    SDC_QDELTA_MIN_SR_NS = 2,
    SDC_QDELTA_IMPLICIT_EULER = 3,
    SDC_QDELTA_MIN_SR_S = 4
};
enum { SDC_METHOD_DSDC = 0, SDC_METHOD_SERIAL_SDC = 1, SDC_METHOD_IMEX2 = 2 };
enum { SDC_SERIAL_IMPLICIT_EULER = 0, SDC_SERIAL_IMPLICIT_LU = 1 };

/* Create a solver for truncation T on an nlat x nlon Gauss grid with M
 * Radau-right collocation nodes (tau_M = 1, Sec. 4.2), K sweeps per step
 * (Algorithm 2) and step size dt [s].
 * Requirements (else SDC_EINVAL): 1 <= T <= 1023; nlat even, nlat >= (3T+1)/2
 * (alias-free quadratic products), nlat <= 2048; nlon = 2^a 3^b with
 * nlon >= 3T + 1 and nlon <= 2304 (one latitude ring pair's FFTs live in
 * shared memory; SDC_FP64 contexts return SDC_EUNSUPPORTED above 2048
 * longitudes); 1 <= nodes <= 8; 1 <= sweeps <= 64;
 * dt > 0; phys non-NULL with radius, gravity, mean_depth > 0; precision one of
 * sdc_precision.  cuda_stream is a cudaStream_t (NULL = legacy default
 * stream) used by every later call.  On success *out owns all device memory
 * the solver needs; on failure *out is NULL and nothing is leaked. */
int sdc_create(sdc_ctx **out, int truncation, int nlat, int nlon, int nodes, int sweeps,
               double dt, const sdc_phys *phys, int precision, void *cuda_stream);

/* Release everything sdc_create allocated (waits for the stream).  NULL is a
 * no-op. */
int sdc_destroy(sdc_ctx *ctx);

/* Set an option (sdc_option); SDC_EINVAL for an unknown key or value,
 * SDC_EUNSUPPORTED if the MIN-SR-S diagonal is not reached, SDC_ECUDA /
 * SDC_ENOMEM if a reference integrator's first selection cannot allocate.
 * Synchronises the context's stream when the setting changes. */
int sdc_set_option(sdc_ctx *ctx, int key, int value);

/* Number of complex coefficients per field, (T+1)(T+2)/2; -1 for NULL. */
int sdc_ncoef(const sdc_ctx *ctx);

/* One dSDC step t_n -> t_n + dt: Algorithm 2 with the node update Eq. (7)
 * (f_I = L_g solved per spectral mode as in Eq. (8), f_E = T_E = L_c + N_a +
 * N_r of Eq. (4)).  state_in and state_out are device state[3][ncoef]; they
 * may be the same buffer.  resid_out (HOST, nullable) receives K x 3 doubles:
 * for each sweep k = 1..K and field (Phi', zeta, div), the maximum over the
 * nodes that sweep updates of the Parseval-weighted L2 norm of the
 * collocation residual u_n + dt sum_j q_mj F(u_j^{k-1}) - u_m^{k-1}; when
 * requested the call synchronises and returns SDC_EDIVERGED if any norm is
 * not finite. */
int sdc_step(sdc_ctx *ctx, const void *state_in, void *state_out, double *resid_out);

/* nsteps >= 0 steps in place on the device state[3][ncoef] (one CUDA graph
 * replay per step).  nsteps = 0 is a no-op. */
int sdc_run(sdc_ctx *ctx, void *state, int nsteps);

/* Explicit tendency T_E (Eq. (4): L_c + N_a + N_r through the spherical
 * harmonic transform) of `batch` states: states and tend are device arrays
 * [batch][3][ncoef]; 1 <= batch <= nodes. */
int sdc_tendency(sdc_ctx *ctx, const void *states, void *tend, int batch);

/* Discrete adjoint (reverse-mode derivative) of T_E: ubar = J_E(states)^T abar
 * for `batch` base states (1 <= batch <= nodes); states, abar and ubar are
 * device [batch][3][ncoef].  Adjoints use the real degrees of freedom of the
 * stored arrays: the real part of an adjoint coefficient is d/dRe, the
 * imaginary part d/dIm (the convention of torch's complex gradients). */
int sdc_tendency_adjoint(sdc_ctx *ctx, const void *states, const void *abar, void *ubar, int batch);

/* Adjoint of one dSDC step (Algorithm 2 with Eq. (7) transposed):
 * ubar_n = (d u_{n+1} / d u_n)^T ubar_next, where u_{n+1} is the step of
 * state_n.  The step is first re-run to record its node evaluations.  All
 * three are device state[3][ncoef]. */
int sdc_step_adjoint(sdc_ctx *ctx, const void *state_n, const void *ubar_next, void *ubar_n);

/* Adjoint of nsteps steps from state0: ubar_initial = (d u_N / d u_0)^T ubar_final.
 * Memory stays bounded by binomial checkpointing: at most nsnapshots states
 * (1..32, counting state0) are kept, the schedule minimising forward
 * recomputation for that budget; each reversed step is re-run once more to
 * record its evaluations.  forward_steps (HOST, nullable) receives the number
 * of recomputed forward steps (synchronises).  nsteps in [0, 4096]. */
int sdc_run_adjoint(sdc_ctx *ctx, const void *state0, int nsteps, int nsnapshots, const void *ubar_final,
                    void *ubar_initial, long long *forward_steps);

/* Height-misfit loss of the state after nsteps steps from state0,
 * L = 0.5 sum over the nlat x nlon grid of (h - h_target)^2 with
 * h = H + Phi'/g (h_target: device double[nlat][nlon]), written to *loss_out
 * (HOST; synchronises), and its gradient with respect to state0 in grad_out
 * (device state[3][ncoef]), with the checkpointing of sdc_run_adjoint. */
int sdc_adjoint_run(sdc_ctx *ctx, const void *state0, int nsteps, int nsnapshots, const double *h_target,
                    double *loss_out, void *grad_out);

/* Scalar transforms of one field (helpers for initial states and grid
 * diagnostics): spec is device double2[ncoef], grid is device
 * double[nlat][nlon].  grid_to_spec is the Gauss-quadrature analysis onto
 * degree <= T. */
int sdc_spec_to_grid(sdc_ctx *ctx, const void *spec, double *grid);
int sdc_grid_to_spec(sdc_ctx *ctx, const double *grid, void *spec);

/* Host copies of the grid and collocation data: mu[nlat] = sin(latitude),
 * w[nlat] Gauss weights, tau[nodes] Radau-right nodes, Q[nodes*nodes]
 * row-major collocation matrix q_{m,j} = int_0^{tau_m} l_j (Sec. 4.1).
 * Any pointer may be NULL. */
int sdc_grid_coords(const sdc_ctx *ctx, double *mu, double *w);
int sdc_collocation(const sdc_ctx *ctx, double *tau, double *Q);

/* Checkpoint and resume of a state (the paper keeps none between runs).
 * sdc_save writes to the file `path` (NUL-terminated) one JSON header line --
 * format tag "sdc-swe-state-1", the context's truncation, nlat, nlon, nodes,
 * sweeps, dt and physical constants, the caller's step index, ncoef, the field
 * order ["phi", "zeta", "div"] and the byte count -- followed by the raw FP64
 * state [3][ncoef] (16 bytes per complex coefficient, little-endian as in
 * memory).  sdc_load reads such a file into the device state of this context
 * and returns its step index through `step` (may be NULL).  state: device
 * memory of 3 * ncoef double2, owned by the caller.  Both synchronise the
 * context's stream.  SDC_EINVAL for NULL arguments, a file that cannot be
 * opened, written or read, a header of another format, truncation or size, a
 * header whose grid, nodes, sweeps, dt or physical constants differ from the
 * context's (compared exactly: the step index is a model time only under the
 * same configuration), or a data section of the wrong length; SDC_ECUDA if a
 * copy fails. */
int sdc_save(sdc_ctx *ctx, const void *state, long long step, const char *path);
int sdc_load(sdc_ctx *ctx, void *state, long long *step, const char *path);

/* The diagonal coefficients q^Delta_{m,m} (m = 0..nodes-1) that rule (an
 * SDC_QDELTA_* value) gives at sweep `sweep` (1-based) on Radau-right nodes
 * -- what a context with that rule uses (Sec. 4.2).  Host only (no GPU, no
 * context); qdelta is a HOST array of `nodes` doubles.  SDC_EINVAL for nodes
 * outside [1, 8], sweep < 1, an unknown rule or NULL; SDC_EUNSUPPORTED if the
 * MIN-SR-S iteration does not reach its root. */
int sdc_qdelta(int nodes, int rule, int sweep, double *qdelta);

/* Work counters since creation (HOST outputs, any may be NULL): explicit
 * tendency evaluations of single states, per-node implicit solves, and the
 * library's own kernel launches.  Algorithm 2 performs 1 + (K-1) M
 * evaluations and (K-1) M + 1 solves per step (Table 1). */
int sdc_counters(const sdc_ctx *ctx, long long *explicit_evals, long long *solves,
                 long long *kernel_launches);

/* One step like sdc_run(ctx, state, 1), but launched kernel by kernel (not
 * from the graph) with CUDA events between the launches; synchronises.
 * HOST outputs ms[6] and launches[6] receive the summed device time and the
 * number of launches of each kernel class: 0 Legendre synthesis, 1 ring
 * FFT/products, 2 Legendre analysis (projections), 3 analysis epilogue
 * (div/curl recombination per mode), 4 quadrature + implicit solve (sweep),
 * 5 residual reduction. */
int sdc_profile_step(sdc_ctx *ctx, void *state, double *ms, int *launches);

/* Wait for the context's stream; SDC_ECUDA if a CUDA error is pending or a
 * tensor-core kernel gave up a bounded wait (its results are then invalid). */
int sdc_sync(sdc_ctx *ctx);

/* Launches per step of the captured step graph (HOST output): 4 per tendency
 * batch (K per step) plus one sweep kernel per sweep. */
int sdc_launches_per_step(const sdc_ctx *ctx, int *launches);

/* FP64 fused multiply-add rate of the current device, measured: `repeats`
 * timed launches (after one warm-up launch) of blocks that fill every SM,
 * each thread running 8 independent FMA chains of `iters` steps; HOST output
 * *tflops in TFLOP/s, an FMA counting two flops.  The paper has no
 * counterpart: it is the peak the FP64 transform kernels are reported
 * against.  sink is a DEVICE double the kernel never writes for these
 * inputs (it keeps the chains from being optimised away).  Synchronises
 * cuda_stream (a cudaStream_t, NULL = legacy default); changes no GPU
 * setting.  SDC_EINVAL for NULL pointers or iters, repeats < 1, SDC_ECUDA if
 * a CUDA call fails; sdc_last_error() is not updated. */
int sdc_fp64_fma_rate(int iters, int repeats, void *cuda_stream, double *sink, double *tflops);

/* Spectral-to-grid transform of one field that allocates nothing and needs no
 * context.  The paper has no counterpart: this serves callers that cannot call
 * cudaMalloc -- host applications that own all device memory through their
 * own allocator and forbid other code from allocating, latency-critical loops
 * that cannot afford cudaMalloc/cudaFree (which may synchronise the device),
 * and processes under a fixed device-memory budget -- and therefore cannot
 * create an sdc_ctx.  It computes what sdc_spec_to_grid computes (same sizes
 * rules as sdc_create; spec is device double2[(T+1)(T+2)/2], grid is device
 * double[nlat][nlon], both owned by the caller) with the Gauss nodes, Legendre
 * functions and FFT twiddles generated on the fly.  Its only intermediate data
 * live in a static 2 MiB device array that every GPU loading the library holds
 * until exit: the call is rejected with SDC_EUNSUPPORTED unless
 * (nlat/2)*2*(T+1) + ceil(nlat/4) <= 131072 complex doubles (T255 on 384
 * latitudes fits; T511 on 768 does not).  SDC_EINVAL for NULL pointers or
 * invalid sizes, SDC_ECUDA if a CUDA call fails or if a CUDA error from
 * earlier work is already pending on the calling thread (it is then left
 * pending for its owner and nothing is launched); sdc_last_error() is not
 * updated.  The first call on each device does a one-time set-up on the
 * current device (looks up the array's device address, raises a kernel's
 * shared-memory limit); make that first call before any stream capture.  The
 * set-up is kept for the life of the process: after cudaDeviceReset() of a
 * device the kept address may be stale, so do not call this function on that
 * device again in the same process.
 * Every call shares the array: calls whose work overlaps on the GPU (several
 * streams or host threads) race and must be serialised by the caller.
 * Asynchronous on cuda_stream (a cudaStream_t, NULL = legacy default). */
int sdc_spec_to_grid_static(int truncation, int nlat, int nlon, const void *spec, double *grid,
                            void *cuda_stream);

const char *sdc_strerror(int status);
const char *sdc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SDC_H_ */
