/*
 * slipspring.h -- C ABI of the GB300 (sm_103a) library for the single-chain
 * slip-spring model of T. Uneyama, arXiv:1106.2899.
 *
 * The library advances many independent chains.  Each chain has N beads R_i
 * (Sec. 2.1), Z slip-springs with bead index S_j and anchor A_j (Sec. 2.1,
 * Z <= z_max <= N, the paper's bound for one slot per bead, Sec. 3.2), and is
 * stepped by the three substeps of Sec. 3.1: Euler-Maruyama beads with
 * affinely advected anchors (Eqs. langevin_equation_bead_position,
 * dynamic_equation_anchoring_position), capped Glauber hops (Eqs.
 * transition_probability_s_plus/minus), creation and destruction at the chain
 * ends (Eqs. transition_probability_z_plus/minus).  After every step the
 * library samples the stress (Eq. stress_tensor_single_chain) and the virtual
 * stress (App. B) into a multiple-tau correlator for G(t) (Eq.
 * relaxation_modulus_tensor_green_kubo_form) and, every log_every steps, into
 * ensemble sums for <sigma>(t) and eta+(t) (Sec. 4.1).
 *
 * Conventions
 *  - Every function returns an int status: SS_OK (0) or a negative SS_E* code;
 *    ss_last_error() gives a message for the last failure on that context.
 *  - Units: b, kT and zeta as given in ss_params (the paper uses b = kT =
 *    zeta = 1, Sec. 3.1).  Stresses in kT per chain; G in rho0 kT (the
 *    per-chain correlation divided by N kT^2, c0 = rho0/N); time in units of
 *    the time step times dt.
 *  - Bead indices are 0-based (bead 0 = the paper's bead 1).
 *  - Host arrays are caller-owned, C-contiguous, and only read or written
 *    during the call.  The library owns every device allocation it makes.
 *  - Calls enqueue work on the context's CUDA stream and return; the calls
 *    that write host arrays synchronise that stream first.
 *  - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef SLIPSPRING_H
#define SLIPSPRING_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SS_OK 0
#define SS_EINVAL (-1)     /* invalid argument or parameter                        */
#define SS_ENOMEM (-2)     /* device or host allocation failed                     */
#define SS_ECUDA (-3)      /* a CUDA runtime call failed                           */
#define SS_EOVERFLOW (-4)  /* non-finite state, or the step counter would wrap 2^32 */
#define SS_ESTATE (-5)     /* call out of order (e.g. ss_run before ss_set_params)  */
#define SS_ETIMEOUT (-6)   /* reserved: a bounded device wait gave up              */
#define SS_ETOOBIG (-7)    /* request needs more than the no-allocation scratch    */

/* precisions */
#define SS_FP32 0 /* FP32 beads and anchors, FP64 ensemble sums */
#define SS_FP64 1 /* FP64 throughout                            */

/* correlator channels (Eq. relaxation_modulus_tensor_green_kubo_form) */
#define SS_CH_AUTO 0  /* (1/N) <sigma_ab(t) sigma_ab(0)>                 */
#define SS_CH_CROSS 1 /* (1/N) <sigma_ab(t) sigma^(v)_ab(0)>             */
#define SS_CH_TOTAL 2 /* AUTO + CROSS: the paper's G(t)                   */
/* with corr_tt = 1 (Sec. 4.1, Eq. relative_contribution_virtual_stress_to_
 * shear_relaxation_modulus: the virtual-stress share is VIRTUAL / TOTAL) */
#define SS_CH_TT 3      /* (1/N) <(sigma + sigma^(v))_ab(t) (sigma + sigma^(v))_ab(0)> */
#define SS_CH_VIRTUAL 4 /* TT - TOTAL = (1/N) <sigma^(v)_ab(t) (sigma + sigma^(v))_ab(0)> */

#define SS_CORR_POINTS 16 /* multiple-tau points per level */
#define SS_MAX_LEVELS 32
#define SS_MAX_BEADS 128  /* chain length limit of the library           */
#define SS_MAX_SLOTS 64   /* slip-springs per chain: z_max <= min(N, 64)  */

typedef struct ss_ctx ss_ctx;

/* One ensemble ("element") of independent chains of equal length. */
typedef struct {
    int32_t n_chains; /* >= 1                          */
    int32_t n_beads;  /* 2 .. SS_MAX_BEADS             */
} ss_element;

/* Parameters of the model (Sec. 2), the scheme (Sec. 3.1) and the observables.
 * Any field left 0 takes the default in brackets. */
typedef struct {
    double N0;      /* beads per slip-spring, <Z>_eq = N/N0 (Eq. average_slip_spring_number_and_
                       entanglement_bead_number); +inf switches slip-springs off [4]       */
    double Ns;      /* slip-spring strength (Eq. free_energy_single_chain) [0.5]          */
    double zeta_s;  /* slip-spring friction (Eqs. transition_probability_*) [0.1]         */
    double dt;      /* time step (Sec. 3.1) [0.01]                                       */
    double b;       /* bead size [1]                                                     */
    double kT;      /* thermal energy [1]                                                */
    double zeta;    /* bead friction [1]                                                 */
    double k_b;     /* bond stiffness; 0 -> 3 kT / b^2                                   */
    double k_s;     /* slip-spring stiffness; 0 -> 3 kT / (Ns b^2)                        */
    int32_t create_mode;    /* 0: K = z_max - Z creation attempts per end (GPU form of
                               Sec. 3.2); 1: K = 1 (CPU form) [0]                        */
    int32_t z_max;          /* slip-spring slots per chain, 1..min(N, SS_MAX_SLOTS)
                               [min(N, SS_MAX_SLOTS)]                                    */
    int32_t destroy_new;    /* 1: a spring created in a step may be destroyed in the same
                               step; 0: only springs that existed before [0]             */
    int32_t recenter_every; /* shift each chain and its anchors to the chain's centre of
                               mass every this many steps when the flow is non-zero; the
                               shift does not change any bond, spring length, rate or
                               stress [100]; < 0 never                                  */
    int32_t log_every;      /* ensemble stress sums every this many steps; 0: none        */
    int32_t max_logs;       /* capacity of the stress log per element [0]                */
    int32_t corr_levels;    /* multiple-tau levels, 1..SS_MAX_LEVELS [24]; < 0: none      */
    int32_t groups;         /* chain groups per element for standard errors [32]         */
    int32_t chunk_steps;    /* steps per kernel launch [1024]; 1 gives the plain
                               one-step-per-launch form.  With the correlator on, a
                               launch covers at most 1024 steps (larger values are
                               reduced to 1024): the launch's stress series, 24 B per
                               chain and step in FP32, is what the correlator reads.
                               The chain states and event counts do not depend on it
                               (random numbers are indexed by the absolute step); the
                               correlator folds its FP32 sums of each launch into FP64,
                               so its sums depend on it at the rounding level        */
    int32_t corr_tt;        /* 1: also correlate sigma + sigma^(v) with itself (channels
                               SS_CH_TT, SS_CH_VIRTUAL) [0]                             */
    int32_t integrator;     /* substep 1: SS_EULER, the Euler-Maruyama scheme of Sec. 3.1
                               [default], or SS_HEUN, the stochastic Heun scheme (the
                               second-order stochastic Runge-Kutta method for additive
                               noise that Sec. 3.1 names as the more accurate choice):
                               the Euler step predicts, the corrector averages the drift
                               (bead forces with this step's springs, flow terms) at the
                               start and at the predicted beads and anchors, with the
                               same noise; hops, creation and destruction unchanged.
                               Stationary bias O(dt^2) instead of O(dt).  The per-element
                               path only: batched mode, differentiation windows and
                               ss_run_noalloc refuse it with SS_EINVAL               */
} ss_params;

/* integrators (ss_params.integrator) */
#define SS_EULER 0
#define SS_HEUN 1

/* Create a context for n_elems elements.  precision: SS_FP32 or SS_FP64.
 * seed keys the counter-based random numbers (Philox4x32-10): chains with the
 * same seed and global chain id draw the same numbers in any run.  The global
 * chain id of chain m of element e is the sum of n_chains of elements < e plus
 * m.  cuda_stream: a cudaStream_t, or NULL for the default stream.
 * Errors: SS_EINVAL (bad element table), SS_ENOMEM, SS_ECUDA. */
int ss_create(ss_ctx** out, const ss_element* elems, int n_elems, int precision, uint64_t seed,
              void* cuda_stream);

/* Validate and apply parameters; allocates the device state.  Must precede the
 * first ss_run.  Validation: every physical parameter finite and > 0 (N0 may
 * be +inf), Euler stability dt (4 k_b + k_s)/zeta < 2, 1 <= z_max <= min(N, SS_MAX_SLOTS).
 * Calling it again resets the state, the observables and the step counter. */
int ss_set_params(ss_ctx* ctx, const ss_params* p);

/* Velocity gradient kappa (row-major, dR_a/dt contains kappa[3a+b] R_b) from
 * step from_step on, for element elem (-1: all).  Later entries of the
 * piecewise-constant schedule are replaced.  Applies to the bead update
 * (Eq. langevin_equation_bead_position) and the anchor advection (Eq.
 * dynamic_equation_anchoring_position). */
int ss_set_flow(ss_ctx* ctx, int elem, int64_t from_step, const double kappa[9]);

/* Many entries of the flow schedule at once (the batched multiscale use, one
 * velocity-gradient history per element): entry i sets kappa[9i..9i+8] for
 * element elem[i] from step from_step[i] on, as ss_set_flow does; within an
 * element the entries must be in increasing from_step order. */
int ss_set_flow_table(ss_ctx* ctx, int n, const int32_t* elem, const int64_t* from_step, const double* kappa);

/* Batched mode (support for many elements; not in the paper): when enabled,
 * ss_run advances all elements with one persistent launch per chunk of
 * chunk_steps steps, replayed from an explicitly built CUDA graph; CTAs take
 * (element, chain tile) work items from an atomic counter, longest chains
 * first.  Before the first batched launch an autotuner times the candidate lane
 * layouts of each chain length on a scratch ensemble and keeps the fastest (the
 * default layout unless another is at least 3% faster; results cached per
 * process).  Batched mode keeps the stress logs, not the
 * correlator: ss_run fails with SS_EINVAL unless corr_levels < 0.  The
 * numbers drawn and the results are those of the per-element path with the
 * same layout.  enable = 0 returns to the per-element path and its default
 * layouts. */
int ss_set_batched(ss_ctx* ctx, int enable);

/* Enqueue n_steps time steps for every element.  The first call on fresh state
 * samples the equilibrium initial state (Sec. 3.1: Gaussian chain, Poisson Z,
 * uniform S, Gaussian anchors).  Returns SS_EOVERFLOW if the step counter
 * would pass 2^32 (a Philox counter word); a non-finite state is reported by
 * ss_status(). */
int ss_run(ss_ctx* ctx, int64_t n_steps);

/* Ensemble stress log of element elem: for each log n, t[n] is the time
 * (steps * dt), mean[n][6] the chain average of sigma xx,yy,zz,xy,xz,yz and
 * sem[n][6] its standard error over the chain groups (either may be NULL).
 * Writes at most cap entries; *n_out receives the number available. */
int ss_stress(ss_ctx* ctx, int elem, double* t, double* mean, double* sem, int cap, int* n_out);

/* Relaxation modulus of element elem from the multiple-tau correlator, channel
 * SS_CH_*: t[n] the lag (steps * dt), G[n] in rho0 kT averaged over the xy, xz,
 * yz components, sem[n] its standard error over chain groups.  Lags are
 * ascending; lags without samples are left out.  *n_out = number available.
 * Writes at most cap entries (any of t, G, sem may be NULL); with cap = 0 or
 * all three NULL it only sets *n_out and reads nothing from the device.
 * Otherwise the group sums are reduced on the device and copied back once:
 * synchronises with the context's stream. */
int ss_correlator(ss_ctx* ctx, int elem, int channel, double* t, double* G, double* sem, int cap,
                  int* n_out);

/* Free every resource of the context (NULL is accepted). */
int ss_destroy(ss_ctx* ctx);

/* Message of the last failure on ctx ("" if none); static text for NULL. */
const char* ss_last_error(const ss_ctx* ctx);

/* ---- support calls -------------------------------------------------------- */

/* Copy element elem's state to host arrays (any may be NULL): R[M][N][3],
 * Z[M], S[M][z_max] (-1 for empty slots), A[M][z_max][3] (0 for empty),
 * in FP64 whatever the precision.  Synchronises. */
int ss_get_state(ss_ctx* ctx, int elem, double* R, int32_t* Z, int32_t* S, double* A);

/* Replace element elem's state from host arrays laid out as in ss_get_state.
 * Validation: 0 <= Z <= z_max, 0 <= S < N for j < Z, finite values.  Marks the
 * context initialised (no equilibrium sampling on the next ss_run). */
int ss_set_state(ss_ctx* ctx, int elem, const double* R, const int32_t* Z, const int32_t* S,
                 const double* A);

/* The same two calls on caller-owned DEVICE arrays in the same layout as
 * ss_get_state / ss_set_state (R [M][N][3] and A [M][z_max][3] double, S
 * [M][z_max] and Z [M] int32; the state converted to and from the library's
 * device layout by kernels, in FP64 whatever the precision), for callers whose
 * data already lives on the GPU (e.g. torch tensors).  cuda_stream: the
 * caller's cudaStream_t, or NULL for the context's stream.
 * ss_get_state_dev is asynchronous: the copy is ordered after the work already
 * enqueued on the context's stream, and work the caller enqueues on
 * cuda_stream afterwards sees the arrays written; any array may be NULL.
 * ss_set_state_dev waits on the context's stream for work already enqueued on
 * cuda_stream, validates the arrays as ss_set_state does (synchronising the
 * context's stream to read a 4-byte check flag) and replaces the state; the
 * caller's arrays may be reused when it returns.  Errors as ss_set_state. */
int ss_get_state_dev(ss_ctx* ctx, int elem, double* R, int32_t* Z, int32_t* S, double* A, void* cuda_stream);
int ss_set_state_dev(ss_ctx* ctx, int elem, const double* R, const int32_t* Z, const int32_t* S,
                     const double* A, void* cuda_stream);

/* Histogram of the slip-spring number Z over the chains of element elem (the
 * distribution of Eq. slip_spring_number_distribution_modified, Poisson(N/N0)
 * in equilibrium up to the z_max cap and the O(dt) bias of the scheme):
 * hist[z] = number of chains with Z = z, z = 0..z_max.  *n_out = z_max + 1;
 * with hist NULL or cap = 0 only *n_out is set.  Counted on the device, read
 * back once: synchronises.  SS_ESTATE before the state exists; SS_EOVERFLOW if
 * some chain's Z lies outside 0..z_max (a broken invariant, see ss_status;
 * those chains are in no bin). */
int ss_zhist(ss_ctx* ctx, int elem, int64_t* hist, int cap, int* n_out);

/* Global chain id of chain 0 of element 0 (default 0); the elements follow
 * contiguously.  A shard of a larger ensemble (one GPU or process of several)
 * passes the start of its contiguous chain range, so that every chain draws
 * the same Philox numbers whatever the number of shards.  Errors: SS_EINVAL if
 * offset + total chains passes 2^32. */
int ss_set_chain_offset(ss_ctx* ctx, uint32_t offset);

/* Steps taken so far. */
int ss_step_count(ss_ctx* ctx, int64_t* steps);
/* Set the step counter (resume from a saved state: the next step draws the
 * Philox numbers of step `step`, Sec. 3.1 with the counter mapping above).
 * The observables are reset, as by ss_reset_observables, so that correlator
 * and log windows start at the new step.  SS_EINVAL outside 0..2^32. */
int ss_set_step_count(ss_ctx* ctx, int64_t step);

/* Zero the correlator and the stress logs (e.g. after equilibration). */
int ss_reset_observables(ss_ctx* ctx);

/* Raw correlator sums of element elem: acc[g][level][16][2][3] (lag slot,
 * channel 0 = later sigma x origin sigma, 1 = later sigma x origin
 * sigma + sigma_v, component xy/xz/yz) summed over the chains of group g,
 * n_groups groups; *n_samples = samples per chain since the last reset.
 * Level l >= 1 only fills lag slots 8..15 (lag slot k means k 2^l steps). */
int ss_corr_sums(ss_ctx* ctx, int elem, double* acc, int* n_groups, int64_t* n_samples);
/* Group sums of channel TT, acc_tt[n_groups][levels][16][3] (lag-major as in
 * ss_corr_sums, one channel).  SS_ESTATE unless corr_tt = 1. */
int ss_corr_sums_tt(ss_ctx* ctx, int elem, double* acc_tt, int* n_groups, int64_t* n_samples);

/* Raw stress-log sums of element elem: sums[n][g][14] = sums over group g of
 * sigma xx,yy,zz,xy,xz,yz, their squares, Z and Z^2; log_step[n] = steps done
 * when log n was taken.  *n_out = logs available, *n_groups = groups. */
int ss_log_sums(ss_ctx* ctx, int elem, int64_t* log_step, double* sums, int cap, int* n_out,
                int* n_groups);

/* Event counters summed over all chains since ss_set_params: out[0] hops to
 * S+1, out[1] hops to S-1, out[2] springs created, out[3] springs destroyed,
 * out[4] creation attempts dropped at capacity (K = 1 form), out[5] kernel
 * launches, out[6] non-finite-state detections, out[7] broken-invariant
 * detections (see ss_status). */
int ss_counters(ss_ctx* ctx, int64_t out[8]);

/* Device status word, checked by every chain-kernel launch on the state it
 * leaves: 0 if all is well; bit 0 set if a bead position was not finite, bit 1
 * if a chain broke 0 <= Z <= z_max or 0 <= S_j < N (a defect of the step, not
 * of the model).  Synchronises. */
int ss_status(ss_ctx* ctx, int32_t* status);

/* Wait for the context's stream. */
int ss_synchronize(ss_ctx* ctx);

/* Kernel timing (support for benchmarks; not in the paper).  While enabled
 * (enable = 1), every launch of the chain kernel is bracketed by CUDA events on
 * the context's stream.  ss_kernel_time synchronises and returns the summed
 * event time of those launches and their number, then clears them.
 * enable = 0 stops recording. */
int ss_kernel_timing(ss_ctx* ctx, int enable);
int ss_kernel_time(ss_ctx* ctx, double* chain_kernel_ms, int64_t* chain_launches);

/* ---- differentiation windows (pathwise gradients; not in the paper) --------
 * A window of n_steps steps from the current state of a one-element context
 * with the correlator enabled and no flow.  The loss is a function L(G) of the
 * TOTAL channel of the relaxation modulus G measured over the window alone
 * (Eq. relaxation_modulus_tensor_green_kubo_form, App. B); the gradient is
 * the pathwise derivative of L with respect to (k_b, k_s, zeta) with every
 * discrete decision (hop, creation, destruction) frozen along the trajectory.
 *
 * ss_window_forward runs the window, resetting the observables at its start,
 * saving the state every checkpoint_every steps (checkpoint_every <=
 * chunk_steps; the last segment may be shorter) and the stress series of every
 * step.
 * replay = 0 records the decisions on a tape; replay = 1 re-runs a window of
 * the same length from the current state with the recorded decisions and the
 * recorded window's step indices, hence the same Gaussian noise (for finite
 * differences of the frozen-decision map at other parameters set with
 * ss_set_coefficients); the continuous update uses the current parameters
 * either way.  Device memory grows with n_steps x chains.
 *
 * ss_window_backward takes dL/dG for each multiple-tau slot of the TOTAL
 * channel, dL_dG[level][16] (G as returned by ss_correlator; unused slots 0),
 * and writes grad = dL/d(k_b, k_s, zeta).  It runs a hand-written adjoint of
 * the continuous update backwards through the window, recomputing each
 * checkpoint segment forward (with the recorded decisions) to obtain the
 * states it needs.  The live state is the window's final state afterwards. */
int ss_window_forward(ss_ctx* ctx, int64_t n_steps, int checkpoint_every, int replay);
/* Set the bond stiffness k_b, the slip-spring stiffness k_s and the bead
 * friction zeta (Sec. 3.1) without touching the state, the step counter, the
 * observables or a recorded window (ss_set_params would reset all of them).
 * SS_EINVAL for a non-positive value or an unstable Euler step
 * (dt (4 k_b + k_s) / zeta >= 2); SS_ESTATE before ss_set_params. */
int ss_set_coefficients(ss_ctx* ctx, double k_b, double k_s, double zeta);
int ss_window_backward(ss_ctx* ctx, const double* dL_dG, double grad[3]);

/* ---- allocation-free run ---------------------------------------------------
 * The paper has no counterpart to this call; it exists for callers that cannot
 * call cudaMalloc: a host application that owns all device memory through its
 * own pool and forbids allocations behind its back, a framework whose device
 * memory budget is fixed when it starts, and real-time loops in which an
 * allocation could block or synchronise the device.  It advances caller-owned
 * device state by n_steps with the same chain and correlator kernels as
 * ss_run, and keeps their working memory (correlator history and FP64 sums,
 * the stress series of a launch and the correlator's level samples, event
 * counters, the flow) in one file-scope device array of SS_NOALLOC_SCRATCH_BYTES
 * bytes that every GPU which loads the library holds until the process exits.
 * The series takes what the rest leaves, so the launch length shrinks as
 * n_chains grows.
 * It calls no cudaMalloc, cudaFree or allocating library routine.
 *
 * State (device pointers, read and written in place), with NP = n_beads
 * rounded up to a multiple of 16 for n_beads <= 64, and NP = 128 above:
 *   R [n_chains][3][NP], A [n_chains][3][NP] (float for SS_FP32, double for
 *   SS_FP64; entries beyond n_beads / beyond Z are ignored), S [n_chains][NP]
 *   int32 bead index of slot j (j < Z), Z [n_chains] int32.
 * params: as ss_set_params (log_every must be 0; chunk_steps splits the call
 *   into launches; channel TT is not accumulated); z_max <= min(n_beads, 64).
 * kappa: row-major constant velocity gradient for the whole call (host array,
 *   read during the call and handed to the GPU by value in a kernel's
 *   arguments), NULL for none.
 * seed, chain_base, t0: Philox key, global id of chain 0 and the index of the
 *   first step, so that consecutive calls with t0 advanced by n_steps draw the
 *   same numbers as one ss_run of the same chains.
 * corr_out (device, may be NULL): [corr_levels][16][2][3] double sums over all
 *   chains of the correlator products of this call alone (laid out as in
 *   ss_corr_sums for one group); the correlator history starts empty at every
 *   call.  status_out (device, may be NULL): set to 0, or 1 if a non-finite
 *   bead position was produced.
 * Errors: SS_EINVAL for invalid arguments, SS_ETOOBIG when the request needs
 *   more scratch than SS_NOALLOC_SCRATCH_BYTES (it grows with n_chains and
 *   corr_levels; with the correlator on, at least one step of series must fit),
 *   SS_EOVERFLOW if t0 + n_steps passes 2^32, SS_ECUDA.
 * The first call on a device looks up the device address of the array (with
 *   that device current) and caches it.  Every call, on any stream, uses the
 *   same array and leaves its contents behind; each call clears what must
 *   start at zero.  Calls that overlap on the GPU race on the array:
 *   serialise them (one stream, or events). */
#define SS_NOALLOC_SCRATCH_BYTES (32u << 20)
int ss_run_noalloc(const ss_params* params, int precision, uint64_t seed, int32_t n_chains,
                   int32_t n_beads, uint32_t chain_base, int64_t t0, int64_t n_steps,
                   const double* kappa, void* R, void* A, int32_t* S, int32_t* Z, double* corr_out,
                   int32_t* status_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
