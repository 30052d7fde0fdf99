/*
 * pbe.h - C ABI of the GB300 (sm_103a) solver for the crystallization
 * population balance equation (PBE) and its coupled solute balance.
 *
 * The model (Sec. 2.1, Eqs. 1-4):
 *   d n/dt + d(G1 n)/dL1 [+ d(G2 n)/dL2] = 0  on [0, lmax] (1-D) or
 *   [0, lmax1] x [0, lmax2] (2-D), growth-only transport with nucleation B
 *   entering the smallest-size cell; solute concentration C follows
 *   C^{k+1} = C^k - kappa (V(n^{k+1}) - V(n^k)) (Eq. 4) with the crystal
 *   volume V = sum x^3 n dL (1-D) or sum x1 x2^2 n dL1 dL2 (2-D).
 * The step (Eq. 3 in semi-discrete form; SI Sec. S1.1): van Leer
 * flux-limited upwind face fluxes, two-stage SSP Runge-Kutta, CFL time step
 * dt = cfl / (G1/dL1 + G2/dL2), clipped to land exactly on output times.
 *
 * Conventions for every call:
 *  - returns PBE_OK (0) or a PBE_E* code; pbe_last_error() gives the message
 *    of the last failure on the calling host thread;
 *  - a pbe_grid is owned by the library: create with pbe_create_grid, free
 *    with pbe_destroy_grid; its device buffers live on the CUDA device that
 *    was current at creation;
 *  - caller pointers stay owned by the caller; each one is host or device
 *    memory as the `mem` argument (PBE_MEM_HOST / PBE_MEM_DEVICE) says;
 *  - work is ordered on the stream given to pbe_set_stream (default: the
 *    legacy default stream).  Calls that return values to the host
 *    (pbe_step, pbe_solve, pbe_get_state, pbe_moments with host memory,
 *    pbe_vjp) synchronize that stream before returning;
 *  - arrays are float64; a 2-D distribution is row-major n[i * N2 + j],
 *    i along L1 (first size), j along L2 (second size); cell centres are
 *    x_i = (i + 1/2) dL.
 * No call falls back to the CPU: without a usable CUDA device every call
 * that needs one fails with PBE_ECUDA.
 */
#ifndef PBE_H
#define PBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int pbe_status;
#define PBE_OK 0
#define PBE_EINVAL 1     /* bad argument (size, pointer, order of times)      */
#define PBE_ENOMEM 2     /* device or pinned allocation failed                */
#define PBE_ECUDA 3      /* a CUDA runtime call or launch failed              */
#define PBE_ENONFINITE 4 /* NaN/Inf appeared in the state or kinetics         */
#define PBE_ETIMEOUT 5   /* step budget or a bounded device wait ran out      */
#define PBE_ESTATE 6     /* call out of order (e.g. solve before set_state)   */

#define PBE_MEM_HOST 0
#define PBE_MEM_DEVICE 1

/* kinetic models */
#define PBE_KINETICS_POWER_LAW 0 /* G_d = kg[d] s^g[d], B = kb s^b, s = max(C/c*(T) - 1, 0) */
#define PBE_KINETICS_FIXED 1     /* G_d = kg[d], B = kb, independent of S (tests)           */
#define PBE_KINETICS_MLP 2       /* learned closure set by pbe_set_closure                   */

/* time schemes */
#define PBE_SCHEME_SSPRK2 0 /* semi-discrete limited fluxes, two-stage SSP Runge-Kutta, both
                               directions at once, dt = cfl / (G1/dL1 + G2/dL2)           */
#define PBE_SCHEME_PAPER 1  /* Eq. 3 (one-step high resolution, van Leer limiter) with Godunov
                               dimensional splitting (L1 sweep then L2 sweep),
                               dt = cfl min(dL1/G1, dL2/G2) (SI Sec. S1.1); plain path only  */

/* execution paths of pbe_solve */
#define PBE_PATH_PLAIN 0 /* two stage kernels per step, device-resident scalars, CUDA graph loop */
#define PBE_PATH_FUSED 1 /* one persistent kernel for the whole solve                              */
#define PBE_PATH_AUTO 2  /* the faster path for the configuration: the fused path (faster than the
                            plain one at every measured size of the SSP-RK2 scheme, 1-D 200 to 2^20
                            cells, 2-D 128^2 to 2048^2), the plain path where the fused one does not
                            apply (the paper scheme of Eq. 3)                                      */

typedef struct pbe_grid pbe_grid;

/* Kinetics, solubility, cooling and scheme parameters (Sec. 2.1, Appendix A;
 * power-law forms with a polynomial solubility). */
typedef struct {
    int kind;          /* PBE_KINETICS_*                                        */
    double kg[2];      /* growth prefactor per direction, um/s                  */
    double g[2];       /* growth exponent per direction                         */
    double kb, b;      /* nucleation prefactor (#/(kg s)) and exponent          */
    double csat[3];    /* c*(T) = csat[0] + csat[1] T + csat[2] T^2, g/g        */
    double T0, T1;     /* linear cooling from T0 to T1 (deg C) ...              */
    double t_cool;     /* ... over t_cool seconds (> 0), constant afterwards    */
    double kappa;      /* rho_c k_v u: g/g of solute per um^3/kg of crystal     */
    double cfl;        /* Courant number nu of the CFL step (0 < cfl <= 1)      */
    int scheme;        /* PBE_SCHEME_SSPRK2 or PBE_SCHEME_PAPER                  */
    int growth_form;   /* 0: G = kg s^g; 1: Arrhenius G = kg exp(-ea/(T+273.15)) s^g (Appendix A);
                          2: polynomial G_m = sum_k a_mk s^k (Eq. 6, pbe_set_growth_poly)   */
    int solubility_form; /* 0: polynomial csat; 1: c* = csat[0] exp(csat[1] T) (Appendix A) */
    double ea[2];      /* activation temperatures of the Arrhenius form (K)      */
} pbe_kinetics;

/* Create a grid of ndim (1 or 2) dimensions with ncells[d] >= 1 cells on
 * [0, lmax[d]].  Allocates the state and work buffers on the current device.
 * Errors: PBE_EINVAL (ndim, sizes, lmax <= 0), PBE_ENOMEM, PBE_ECUDA. */
pbe_status pbe_create_grid(pbe_grid** out, int ndim, const int64_t* ncells, const double* lmax);

/* Free a grid and its device buffers (waits for its stream).  NULL is a no-op. */
pbe_status pbe_destroy_grid(pbe_grid* g);

/* Order all later work of this grid on `cuda_stream` (a cudaStream_t). */
pbe_status pbe_set_stream(pbe_grid* g, void* cuda_stream);

/* Select the execution path of pbe_solve and pbe_vjp (PBE_PATH_PLAIN,
 * PBE_PATH_FUSED or PBE_PATH_AUTO; AUTO behaves as FUSED, whose solves fall
 * back to the plain path for the paper scheme).  Both compute the same step;
 * results agree to rounding.  Errors: PBE_EINVAL for another value. */
pbe_status pbe_set_path(pbe_grid* g, int path);

/* Set the kinetic model (Sec. 2.1 S = c/c*; Appendix A growth law only for
 * S > 1).  Errors: PBE_EINVAL for kind, cfl not in (0, 1], t_cool <= 0. */
pbe_status pbe_set_kinetics(pbe_grid* g, const pbe_kinetics* k);

/* Weights of the learned kinetics closure (the empirical hybrid model of
 * Sec. 4.2: a network replaces the growth and nucleation expressions inside
 * the solver), used when the kinetics kind is PBE_KINETICS_MLP.  A 3 -> 64 ->
 * 64 -> 3 perceptron with SiLU hidden units: inputs x0 = 4 (S - 1),
 * x1 = (T - 25)/10, x2 = 1e-6 V/mu0 (V = mu3 in 1-D, mu12 in 2-D); outputs
 * ln G1 = o0 + ln 0.01, ln G2 = o1 + ln 0.005, ln B = o2 + ln 1e5; G = B = 0
 * for S <= 1.  w: HOST float array of 4611 values in the layout W1[64][3],
 * b1[64], W2[64][64], b2[64], W3[3][64], b3[3]; the weight matrices are stored
 * rounded to bf16 (round to nearest even), the biases in fp32; arithmetic is
 * fp32.  Rates that are not finite fall back to the power law
 * (pbe_set_closure_box).  On the fused path, solves with the closure (and
 * with the polynomial growth law) run in the persistent kernel of pbe_vjp,
 * without its reverse sweep. */
pbe_status pbe_set_closure(pbe_grid* g, const float* w, int count);

/* Coefficients of the polynomial growth law of Eq. 6 (the model of the
 * parameter estimation study of Sec. 4.1), used with growth_form 2:
 * G_m = sum_{k=1..K} a[m K + k - 1] s^k for s = S - 1 > 0 (0 otherwise),
 * m = 0 .. ndim-1 (one polynomial per growth direction); nucleation keeps
 * B = kb s^b.  a: HOST array of ndim * K doubles, 1 <= K <= 4096.  Call it
 * before pbe_set_kinetics selects growth_form 2; later calls replace the
 * coefficients in place.  Synchronizes the grid's stream.  Errors:
 * PBE_EINVAL (K, non-finite values), PBE_ENOMEM, PBE_ECUDA. */
pbe_status pbe_set_growth_poly(pbe_grid* g, const double* a, int K);

/* dL/da of the polynomial growth law from the last pbe_vjp of this grid
 * (fused path; growth_form 2): `count` = ndim * K HOST doubles in the layout
 * of pbe_set_growth_poly.  Synchronizes.  Errors: PBE_EINVAL (count),
 * PBE_ESTATE (no such gradient yet), PBE_ECUDA. */
pbe_status pbe_growth_poly_grad(pbe_grid* g, double* dL_da, int count);

/* Training box of the learned closure's inputs, and with it the plain-kinetics
 * fallback of the hybrid model (Sec. 4.2): at any kinetics evaluation whose
 * inputs (x0, x1, x2) of pbe_set_closure, in FP64, are not all inside
 * [lo[k], hi[k]], and at any evaluation where a network rate is not finite,
 * the rates are those of the power law of the pbe_kinetics parameters (kg,
 * g, kb, b) instead.  The non-finite test is always on; the box only after
 * this call.  pbe_vjp differentiates whichever rates each stage used.  lo,
 * hi: HOST arrays of 3 doubles, lo[k] <= hi[k]; both NULL removes the box.
 * Errors: PBE_EINVAL. */
pbe_status pbe_set_closure_box(pbe_grid* g, const double* lo, const double* hi);

/* Load the state: distribution n (ncell values, `mem` memory), solute
 * concentration C and time t.  Initial condition of Eqs. (5)-(9). */
pbe_status pbe_set_state(pbe_grid* g, const double* n, double C, double t, int mem);

/* Initial condition from a normal seed (SI Sec. S1.3, initial distribution
 * generation): n = exp(-q/2) at the cell centres, q the squared Mahalanobis
 * distance of the normal with means mean[ndim] (um), standard deviations
 * sd[ndim] > 0 (um) and, in 2-D, correlation corr in (-1, 1) (ignored in
 * 1-D), scaled so that the discrete zeroth moment sum(n) dA equals
 * total_number (# per kg of solvent).  Sets C = C0 and t = 0.  Host arrays;
 * synchronizes the grid's stream (the normalisation is read back).  Errors:
 * PBE_EINVAL (arguments, or a density that underflows at every cell
 * centre), PBE_ECUDA. */
pbe_status pbe_init_seed_gaussian(pbe_grid* g, const double* mean, const double* sd, double corr,
                                  double total_number, double C0);

/* The same normal seed scaled by the seed mass instead (the scale factor
 * beta of SI Sec. S1.3): rho_kv sum(x1 x2^2 n) dA = seed_mass in 2-D,
 * rho_kv sum(x^3 n) dL = seed_mass in 1-D, with rho_kv = rho_c k_v in the
 * mass units of seed_mass per um^3.  Arguments and errors as above. */
pbe_status pbe_init_seed_gaussian_mass(pbe_grid* g, const double* mean, const double* sd, double corr,
                                       double seed_mass, double rho_kv, double C0);

/* Read the state back (n may be NULL to read only C and t). */
pbe_status pbe_get_state(pbe_grid* g, double* n, double* C, double* t, int mem);

/* Advance by one SSP-RK2 step whose length is the CFL step, clipped so the
 * step ends no later than t_limit (> current t).  *dt_taken (may be NULL)
 * receives the step length.  Synchronizes the grid's stream. */
pbe_status pbe_step(pbe_grid* g, double t_limit, double* dt_taken);

/* March from the current state through the increasing output times
 * t_out[0..n_out) (t_out[0] >= current t; host memory), landing on each
 * exactly (Fig. 1 loop).  rows receives n_out rows of `ncol` doubles
 * (ncol = 6 in 1-D: t, mu0, mu1, mu2, mu3, C; ncol = 12 in 2-D: t, mu00,
 * mu10, mu01, mu20, mu11, mu02, mu30, mu21, mu12, mu03, C), in `mem`
 * memory.  *steps (may be NULL) receives the number of steps taken.
 * Moments follow the SI definition of mu_pq by the midpoint rule.
 * Synchronizes the grid's stream (the status and step count are read back).
 * Errors: PBE_EINVAL (times), PBE_ESTATE (no state/kinetics),
 * PBE_ENONFINITE, PBE_ETIMEOUT (more than the step budget), PBE_ECUDA. */
pbe_status pbe_solve(pbe_grid* g, const double* t_out, int n_out, double* rows, int mem,
                     int64_t* steps);

/* Moments of the current distribution: 4 values (mu0..mu3) in 1-D, 10 in
 * 2-D in the row order of pbe_solve (SI moment definition, midpoint rule). */
pbe_status pbe_moments(pbe_grid* g, double* mu, int mem);

/* Vector-Jacobian product of pbe_solve from the current state: the gradient
 * that parameter estimation by a gradient method needs (Sec. 4.1, Eq. 5),
 * computed by the hand-written discrete adjoint of the step (reverse mode
 * through every operation of the forward scheme, branches as the forward
 * pass took them: limiter derivative of the branch taken, zero for S <= 1,
 * the step length through its CFL or output-clip branch; the step count is
 * that of the forward pass).  Checkpointing: the forward pass keeps the state
 * every `checkpoint_every` steps; the reverse sweep recomputes each segment.
 *   t_out, n_out       output times as in pbe_solve (host memory)
 *   seeds              dL/d(rows): n_out x ncol doubles (`seeds_mem` memory);
 *                      the time column is ignored
 *   dL_dtheta          HOST, 6 doubles: d/d(kg[0], g[0], kg[1], g[1], kb, b)
 *                      (power-law kinetics; with fixed kinetics d/d(kg, kb);
 *                      with the polynomial growth law only kb and b, the
 *                      coefficients' gradient then comes from
 *                      pbe_growth_poly_grad)
 *   dL_dn0             optional, ncell doubles (`mem` memory): d/d(initial n)
 *   dL_dC0             optional HOST double: d/d(initial C)
 *   rows               optional, the forward rows (`mem` memory)
 *   dL_dweights        optional HOST, 4611 doubles: gradient with respect to the
 *                      learned closure's weights (PBE_KINETICS_MLP; the layout
 *                      of pbe_set_closure, taken at the stored bf16 values; on
 *                      the fused path from the recorded evaluations by the
 *                      kernel of pbe_closure_grad, on the plain path
 *                      accumulated per stage in fp64)
 * Paths: on PBE_PATH_FUSED one persistent cooperative launch runs the
 * forward pass (checkpoints, and the records of the current segment), the
 * recomputation of the earlier segments and the reverse sweep, with work
 * buffers kept by the grid between calls (grown when a call needs more); on
 * PBE_PATH_PLAIN per-stage kernels from the host, with buffers allocated per
 * call.  The polynomial growth law is differentiated on the fused path only
 * (PBE_EINVAL on the plain path).  Both agree to rounding.
 * On return the grid holds the state at the end of the solve; synchronizes
 * the stream.  With pbe_set_timing on, pbe_kernel_time gives the duration of
 * the fused path's persistent launch. */
pbe_status pbe_vjp(pbe_grid* g, const double* t_out, int n_out, const double* seeds, int seeds_mem,
                   int checkpoint_every, double* dL_dtheta, double* dL_dn0, double* dL_dC0, double* rows, int mem,
                   double* dL_dweights);

/* The learned closure's weight gradient summed over several trajectories (the
 * training step of the hybrid model of Sec. 4.2 on a minibatch): the sum of
 * dL/dweights of the last pbe_vjp of each of the `count` grids, computed by one
 * launch of the weight-gradient kernel over all their recorded closure
 * evaluations (the 64-wide layers on the tensor cores, bf16 operands with
 * fp32 accumulation, activations split into two bf16 parts).  Every grid must
 * use PBE_KINETICS_MLP with the same weights, be on one device, and have run
 * pbe_vjp on the fused path since its last closure change.  dL_dweights:
 * HOST, 4611 doubles (layout of pbe_set_closure).  Synchronizes every grid's
 * stream.  Errors: PBE_EINVAL (arguments, other weights or devices),
 * PBE_ESTATE (no gradient rows), PBE_ENOMEM, PBE_ECUDA. */
pbe_status pbe_closure_grad(pbe_grid* const* grids, int count, double* dL_dweights);

/* Upper bound on steps per pbe_solve call (default 1e6); exceeding it stops
 * the solve with PBE_ETIMEOUT. */
pbe_status pbe_set_max_steps(pbe_grid* g, int64_t max_steps);

/* Solve a 1-D problem without allocating any memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * once running (a fixed-budget real-time loop, a host framework whose
 * allocator owns all device memory, a process that already holds every byte
 * it may use).  It does the work of pbe_create_grid + pbe_set_kinetics +
 * pbe_set_state + pbe_solve on the plain path's arithmetic, with the caller's
 * buffers for inputs and outputs and a fixed working array built into the
 * library (about 0.56 MB of device memory per GPU that loads the library,
 * held until the process exits).
 *   k        kinetics (host memory)
 *   ncells   1 <= ncells <= 65536 cells on [0, lmax]; larger grids: PBE_EINVAL
 *   n        DEVICE memory, ncells doubles: initial distribution in, final out
 *   C0, t0   initial concentration and time
 *   t_out    HOST memory, 1 <= n_out <= 4096 increasing times, t_out[0] >= t0
 *   rows     DEVICE memory, n_out rows of 6 doubles (t, mu0..mu3, C)
 *   steps    optional (host) number of steps taken
 *   stream   cudaStream_t the work is ordered on; the call synchronizes it
 * The kinetics pass the same checks as in pbe_set_kinetics (PBE_EINVAL for a
 * non-finite parameter or a negative rate prefactor).  The whole solve runs
 * in ONE thread block with a fixed budget of 1e6 steps (PBE_ETIMEOUT beyond
 * it): on the largest grid one call can hold one SM for minutes.
 * The first call on each device looks up the working array's device address
 * and keeps it for the life of the process (make that first call before any
 * stream capture; a cudaDeviceReset after it is not supported, because the
 * kept address would then be stale).  All calls share the working array:
 * calls that overlap on a GPU race and must be serialized by the caller.  It
 * calls no cudaMalloc/cudaFree and no allocating library routine. */
pbe_status pbe_solve_1d_noalloc(const pbe_kinetics* k, int64_t ncells, double lmax, double* n, double C0,
                                double t0, const double* t_out, int n_out, double* rows, int64_t* steps,
                                void* stream);

/* ------------------------------------------------------------------------
 * Batched 1-D solves: many independent instances of the 1-D problem, each
 * with its own grid, kinetics, cooling profile, initial state and
 * CFL-limited step count, advanced by one persistent launch (replayed as a
 * CUDA graph) until every instance reaches the shared output times.  The
 * arithmetic per instance is the 1-D step above (fused-path quotient).
 * ------------------------------------------------------------------------ */
typedef struct pbe_batch pbe_batch;

typedef struct {
    int64_t ncells;     /* 1 <= ncells <= 6144 cells on [0, lmax]           */
    double lmax;
    pbe_kinetics kin;   /* per-instance kinetics and scheme (ndim = 1)      */
    double C0, t0;      /* initial concentration and time                   */
} pbe_instance;

/* Create a batch of `count` instances (host array).  Distributions are
 * packed back to back in instance order: instance i occupies cells
 * [offset[i], offset[i+1]) of the packed state (see pbe_batch_offsets).
 * Errors: PBE_EINVAL (sizes, parameters), PBE_ENOMEM, PBE_ECUDA. */
pbe_status pbe_batch_create(pbe_batch** out, const pbe_instance* inst, int count);
pbe_status pbe_batch_destroy(pbe_batch* b);
pbe_status pbe_batch_set_stream(pbe_batch* b, void* cuda_stream);

/* offsets[0..count] (host) of each instance in the packed state. */
pbe_status pbe_batch_offsets(pbe_batch* b, int64_t* offsets);

/* Load the packed distributions (offsets[count] doubles, `mem` memory) and
 * reset every instance's C and t to its C0 and t0.  Synchronizes. */
pbe_status pbe_batch_set_state(pbe_batch* b, const double* n_packed, int mem);

/* Read back the packed state, per-instance C and t (any may be NULL). */
pbe_status pbe_batch_get_state(pbe_batch* b, double* n_packed, double* C, double* t, int mem);

/* Advance every instance through the shared increasing output times
 * t_out[0..n_out) (host memory; t_out[0] >= every t0).  rows (`mem` memory)
 * receives count * n_out rows of 6 doubles (t, mu0..mu3, C), instance-major.
 * *total_steps (host, may be NULL) = steps summed over instances.
 * Synchronizes.  Errors as pbe_solve, naming the first failing instance. */
pbe_status pbe_batch_solve(pbe_batch* b, const double* t_out, int n_out, double* rows, int mem,
                           int64_t* total_steps);

/* Steps taken by each instance in the last pbe_batch_solve (host, count values). */
pbe_status pbe_batch_steps(pbe_batch* b, int64_t* steps);

/* Schedule of the batched launch: warps_per_block (1, 2, 3, 4, 6 or 8),
 * team_instances (0..count) and warp_cells (0..6144).  Team instances, each
 * solved by all warps of a block, are the team_instances instances of
 * largest estimated cost (cells x CFL steps at the peak supersaturation the
 * cooling alone gives) and every instance of more than warp_cells cells; the
 * others are solved by one warp each.  A warp's shared-memory slice holds
 * the largest warp instance, a block's whole allocation the largest team
 * instance, so a lower warp_cells leaves smaller slices and more blocks per
 * SM.  Results are bitwise identical under every schedule (moment sums are
 * formed over fixed 256-cell segments in a fixed order).  PBE_EINVAL when
 * the schedule does not fit in one block's shared memory.  pbe_batch_create
 * picks 4 warps, a cost-based team count and the largest warp_cells that
 * fits; pbe_batch_autotune times alternatives. */
pbe_status pbe_batch_set_schedule(pbe_batch* b, int warps_per_block, int team_instances, int warp_cells);
pbe_status pbe_batch_get_schedule(pbe_batch* b, int* warps_per_block, int* team_instances, int* warp_cells);

/* The learned closure of the batch's PBE_KINETICS_MLP instances (the
 * weights and box as pbe_set_closure / pbe_set_closure_box; one copy on the
 * device for the whole batch; such instances need growth_form 0, whose power
 * law is the closure's fallback).  The batch kernel then sums mu0 at every
 * stage for the closure's input ratio V / mu0.  pbe_batch_solve and
 * pbe_batch_autotune fail with PBE_ESTATE while a batch with closure
 * instances has no weights; the batched adjoint differentiates the power law
 * only (PBE_EINVAL for closure instances).  Synchronizes. */
pbe_status pbe_batch_set_closure(pbe_batch* b, const float* weights, int count);
pbe_status pbe_batch_set_closure_box(pbe_batch* b, const double* lo, const double* hi);

/* pbe_batch_set_schedule(b, warps_per_block, 0, 6144): one instance per warp. */
pbe_status pbe_batch_set_config(pbe_batch* b, int warps_per_block);

/* Gradients of a loss of every instance's output rows (the batched form of
 * pbe_vjp: the same hand-written discrete adjoint by a team of warps (one
 * block, pbe_batch_set_vjp_schedule) per instance, the forward with
 * checkpoints every `checkpoint_every` steps and the reverse sweep with
 * recomputation, up to 4096 steps per instance).  Starts from the
 * batch's current state; seeds: count * n_out rows of 6 doubles (dL/drows,
 * instance-major, `seeds_mem` memory); dL_dtheta HOST count x 6
 * (kg1, g1, kg2, g2, kb, b per instance); dL_dC0 optional HOST count;
 * dL_dn0 optional DEVICE packed state (mem must be PBE_MEM_DEVICE).  The
 * batch state is left unchanged.  Synchronizes. */
pbe_status pbe_batch_vjp(pbe_batch* b, const double* t_out, int n_out, const double* seeds, int seeds_mem,
                         int checkpoint_every, double* dL_dtheta, double* dL_dC0, double* dL_dn0, int mem);

/* Launch shape of pbe_batch_vjp: warps per instance (1, 2, 4 or 8; 0, the
 * default: 4 while there are at most 8 instances per SM, else 2) and
 * resident teams per SM (1..32, capped by what fits; 0, the default: 1
 * while there are at most 2 instances per SM, else 8 / warps).  Results
 * depend on the warps per instance (the order of the sums), not on
 * blocks_per_sm. */
pbe_status pbe_batch_set_vjp_schedule(pbe_batch* b, int warps, int blocks_per_sm);

/* Time schedules on this batch and these output times (every warps-per-block
 * setting with 0, 1/2, 1 and 2 times the cost-based team count; then, at the
 * fastest, the size cut of every higher occupancy level; then team counts
 * from 1/4 to 3 times the fastest one; the state is saved and restored
 * around every trial), keep the fastest and return its warps per block in
 * *chosen (may be NULL; pbe_batch_get_schedule gives the whole schedule). */
pbe_status pbe_batch_autotune(pbe_batch* b, const double* t_out, int n_out, int* chosen);

/* One Adam step (the optimizer of the paper's parameter estimation,
 * Appendix C) on DEVICE arrays of n doubles: moments m, v updated in place,
 * w -= lr * mhat / (sqrt(vhat) + eps) with bias corrections for step >= 1.
 * Ordered on `stream`; does not synchronize. */
pbe_status pbe_adam_update(double* w, const double* grad, double* m, double* v, int n, double lr, double beta1,
                           double beta2, double eps, int step, void* stream);

/* Kernel of the 2-D SSP-RK2 stages.  Plain path: -1 (default) the
 * register-window kernel when the grid gives it at least one block per SM,
 * else the tile kernel; 0 always the tile kernel; 1 always the window
 * kernel.  Fused path, grids too large for one tile per co-resident block:
 * -1 and 1 the persistent window kernel, 0 a loop over 16 x 32 tiles.  All
 * compute the same stage; results agree to rounding.  PBE_EINVAL for another
 * mode. */
pbe_status pbe_set_window(pbe_grid* g, int mode);

/* Limit of every device-wide wait of the fused path (seconds; < 0 restores
 * the default of about one second).  A wait that runs out ends the solve
 * with PBE_ETIMEOUT and leaves the context usable; a limit of 0 makes any
 * wait that does not complete at once run out (used to exercise that path). */
pbe_status pbe_set_wait_limit(pbe_grid* g, double seconds);

/* Most thread blocks the fused path's persistent launches of this grid may
 * use (the solve and the gradient; 0, the default: one per SM).  Grids
 * solved side by side on several streams (a minibatch of trajectories) can
 * then run at the same time: a cooperative launch starts only when all its
 * blocks fit.  The tiles are chosen again (several a block where needed);
 * results agree to rounding.  Synchronizes the grid's stream when the
 * limit changes.  PBE_EINVAL for a negative count. */
pbe_status pbe_set_block_limit(pbe_grid* g, int blocks);

/* Device timing of pbe_solve.  With `enable` != 0 every later pbe_solve
 * records two CUDA events on the grid's stream around the launch that
 * advances the state (the fused path's persistent kernel; the plain path's
 * graph or its chunked step launches) - the prologue, the output-row kernel
 * and the copies stay outside.  pbe_kernel_time writes that duration of the
 * last solve in milliseconds to the HOST double `ms` (-1 when timing was off
 * or the solve failed); pbe_solve has returned by then, so it does not wait.
 * Enabling creates the two events; it does not synchronize.  Errors:
 * PBE_EINVAL (null grid or `ms`), PBE_ECUDA (event creation). */
pbe_status pbe_set_timing(pbe_grid* g, int enable);
pbe_status pbe_kernel_time(pbe_grid* g, double* ms);

/* Message of the last failure on this host thread ("" if none). */
const char* pbe_last_error(void);

/* Library ABI version (major * 100 + minor). */
int pbe_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PBE_H */
