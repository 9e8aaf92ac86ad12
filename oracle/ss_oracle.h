/*
 * ss_oracle.h -- plain FP64 CPU oracle of the single-chain slip-spring model
 * (T. Uneyama, "Single Chain Slip-Spring Model for Fast Rheology Simulations of
 * Entangled Polymers on GPU", arXiv:1106.2899).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists so that the CUDA library can be
 * checked against an independent, slow, obviously correct restatement of the
 * method.  Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it; the product path never does.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * Everything is double precision, one chain at a time, in the order the paper
 * gives the three substeps of one time step (Sec. 3.1).  Bead indices are
 * 0-based here (the paper counts 1..N): bead 0 is the paper's bead 1, bead N-1
 * the paper's bead N.
 *
 * Parity status of each function is stated beside it; "pinned" means a
 * `-m "not gpu"` test checks it against a closed form, an invariant of the
 * paper, brute-force enumeration, or published known-answer values.
 */
#ifndef SS_ORACLE_H
#define SS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_NMAX 128 /* largest chain length the oracle handles           */
#define OR_LMAX 32  /* largest number of multiple-tau levels              */
#define OR_P 16     /* points per multiple-tau level                      */

/* Philox counter word 2 ("purpose") values: which random draw a block feeds. */
enum {
    OR_PURPOSE_STEP = 1,      /* per step, per bead/slot index: noise + slot uniform  */
    OR_PURPOSE_CREATE = 2,    /* per step, per attempt index: anchor of a new spring */
    OR_PURPOSE_INIT_BOND = 3, /* init: bond vector i                                 */
    OR_PURPOSE_INIT_Z = 4,    /* init: number of slip-springs                        */
    OR_PURPOSE_INIT_S = 5,    /* init: bead index of spring j                        */
    OR_PURPOSE_INIT_A = 6     /* init: anchor of spring j                            */
};

/* Model and scheme parameters (Sec. 2, Sec. 3.1).  k_b and k_s are the bond and
 * slip-spring stiffnesses 3kT/b^2 and 3kT/(Ns b^2) of Eq. (free_energy); they
 * are filled from b, Ns, kT by or_params_derive() unless set > 0 beforehand. */
typedef struct {
    int N;           /* beads per chain, 2..OR_NMAX                              */
    int z_max;       /* slot capacity, 1..N (the paper's GPU bound Z <= N)       */
    int create_mode; /* 0: K = z_max - Z parallel attempts; 1: K = 1 (CPU form)  */
    int destroy_new; /* 1: a spring created this step may be destroyed this step */
    double N0;       /* mean beads per slip-spring, <Z>_eq = N/N0 (inf: none)    */
    double Ns;       /* slip-spring strength                                     */
    double zeta_s;   /* slip-spring friction                                     */
    double dt;       /* time step                                                */
    double b, kT, zeta;
    double k_b, k_s;
    int integrator; /* OR_EULER (the paper's scheme, Sec. 3.1) or OR_HEUN        */
} or_params;

/* Integrators of the bead/anchor substep (substep 1 of Sec. 3.1).  OR_HEUN is
 * the stochastic Heun scheme, the second-order stochastic Runge-Kutta method
 * for additive noise that Sec. 3.1 names as the more accurate alternative
 * (Honeycutt 1992): the Euler step is the predictor; the corrector adds half
 * the drift at the start and half the drift at the predicted state, with the
 * same noise.  Slip-spring indices and anchors of the step enter both drifts
 * (anchors at their predicted positions under a flow).  Hops, creation and
 * destruction are unchanged.  Pinned by the exact discrete Rouse closed form
 * of the scheme (per mode r = 1 - x + x^2/2 and variance scale (1 - x/2)^2,
 * x = dt k_b mu_p/zeta), whose stationary bias is second order in dt. */
enum { OR_EULER = 0, OR_HEUN = 1 };

/* Fill k_b, k_s from b, Ns, kT where they are <= 0. */
void or_params_derive(or_params* p);

/* One chain's state: positions R[i], Z springs with bead index S[j] (0-based)
 * and anchor A[j]; slots j >= Z are unused. */
typedef struct {
    double R[OR_NMAX][3];
    int Z;
    int S[OR_NMAX];
    double A[OR_NMAX][3];
} or_chain;

/* Philox4x32-10 of Salmon, Moraes, Dror and Shaw (SC'11).  Pinned by the
 * published known-answer vectors. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Decoding of one Philox block into the draws the scheme uses:
 * n[0..3] = two Box-Muller pairs from (w0,w1) and (w2,w3), radius from the
 * high 24 bits of the first word mapped to (0,1], angle pi*(2u-1) from the
 * high 24 bits of the second word; u = the low bytes of w0,w1,w2 as a 24-bit
 * uniform on [0,1).  Pinned by moment and KS tests. */
void or_decode_block(const uint32_t w[4], double n[4], double* u);

/* Equilibrium initial state (Sec. 3.1, sampling steps 1-3; Eqs.
 * bead_position_distribution, slip_spring_number_distribution_modified,
 * bead_index_distribution, anchoring_point_distribution).  Pinned by the
 * equilibrium-statistics tests. */
void or_init_chain(const or_params* p, const uint32_t key[2], uint32_t chain_id, or_chain* c);

/* Per-step decision record of one chain (test support). */
typedef struct {
    double min_margin; /* smallest |u - threshold| over all decisions of the step */
    int hops_up, hops_down, created, destroyed, dropped;
} or_step_info;

/* One time step t -> t+dt (Sec. 3.1, substeps 1-3).  kappa is row-major
 * (dR_a/dt contains kappa[a][b] R_b).  cd = Phi^{-1}(p_destroy) (the destroy
 * decision threshold on the block's fourth normal; +inf if p_destroy = 1).
 * Pinned by the Rouse closed form, the equilibrium invariants, hop detailed
 * balance and brute-force enumeration; its flow terms (kappa . R in the bead
 * update, affine anchor advection) by the frozen-bead linear map
 * (I + dt kappa)^n and the sheared-Rouse Lyapunov solution; the anchor spread
 * of new springs by the spring-vector variance kT/k_s in the dynamics.  Each of
 * these pins is shown to fail on a copy with a planted mistake. */
void or_step_chain(const or_params* p, const uint32_t key[2], uint32_t chain_id, uint32_t step,
                   const double kappa[9], double cd, or_chain* c, or_step_info* info);

/* The same step with a decision tape (test support for frozen-decision
 * finite differences): `record` (N bytes, may be NULL) receives the step's
 * decisions, `replay` (may be NULL) supplies them instead of the random draws.
 * Byte j: bit 0 spring j hopped to S+1, bit 1 to S-1, bit 2 attempt j created a
 * spring at bead 1, bit 3 at bead N, bit 4 old spring j destroyed, bit 5 the
 * spring of attempt j destroyed. */
void or_step_chain_tape(const or_params* p, const uint32_t key[2], uint32_t chain_id, uint32_t step,
                        const double kappa[9], double cd, or_chain* c, or_step_info* info, const uint8_t* replay,
                        uint8_t* record);

/* Stress of Eq. (stress_tensor_single_chain) and virtual stress of App. B
 * (sum over j = 1..z), both row-major 3x3, in units of kT.  Pinned. */
void or_stress(const or_params* p, const or_chain* c, double sigma[9], double sigma_v[9]);

/* Inverse standard normal CDF by bisection on erfc (host constant). */
double or_norm_ppf(double p);

/* Streaming multiple-tau correlator of one chain fed with the series
 * x[T][6] (signals sigma_xy, sigma_xz, sigma_yz and the same components of
 * sigma + sigma_v); adds into acc[levels][OR_P][2][3].  Pinned against the
 * batch definition (block means, lag products). */
void or_corr_series(const double* x, int64_t T, int levels, double* acc);
/* The same, also accumulating channel TT (later sigma + sigma_v times origin
 * sigma + sigma_v) into acc_tt[levels][OR_P][3] when acc_tt is not NULL. */
void or_corr_series_tt(const double* x, int64_t T, int levels, double* acc, double* acc_tt);

/* ---- operation counts (test infrastructure) -------------------------------
 * Built with -DOR_COUNT_OPS (single-threaded runs only), the oracle counts the
 * operations of the method it executes, by substep.  Rules: one operation per
 * arithmetic operator, comparison, integer shift/mask/logic operator and
 * int-to-float conversion; a library call (log, sqrt, sin, cos, exp) or a
 * reciprocal one; a product added in the same expression counts once with the
 * addition (a fused multiply-add); a 32x32 -> 64-bit product with both halves
 * once; a three-input xor once; constants of the parameters (dt kT/zeta_s,
 * k_s/(4 kT), ...) are formed once and not counted per use.  The velocity-
 * gradient terms count only when kappa is not zero.  The stress counts what
 * the outputs use (off-diagonal components every step, the diagonal at log
 * steps).  Loads, stores, index arithmetic, control flow and the test-support
 * bookkeeping (decision margins, traces, tapes) are not counted.  Without the
 * flag or_ops_get returns zeros and or_ops_enabled 0. */
enum {
    OR_OPC_PHILOX = 0, /* Philox4x32-10 blocks                             */
    OR_OPC_DECODE,     /* Box-Muller pairs and the 24-bit uniform          */
    OR_OPC_BOND,       /* bond forces                                      */
    OR_OPC_SPRING,     /* slip-spring forces                               */
    OR_OPC_EULER,      /* Euler-Maruyama update (with the flow term)       */
    OR_OPC_ADVECT,     /* affine anchor advection                          */
    OR_OPC_HOP,        /* hop probabilities and decisions                  */
    OR_OPC_CREATE,     /* creation attempts and new anchors                */
    OR_OPC_DESTROY,    /* destruction tests                                */
    OR_OPC_STRESS,     /* stress and virtual stress                        */
    OR_OPC_CORR,       /* multiple-tau correlator                          */
    OR_OPC_N
};
void or_ops_get(int64_t out[OR_OPC_N]);
void or_ops_reset(void);
int or_ops_enabled(void);

/* ---- ensemble runner (mirrors the library's calls) ----------------------- */
typedef struct or_ens or_ens;

/* M chains with global ids chain_offset .. chain_offset+M-1, split into G
 * contiguous groups for standard errors, multiple-tau correlator with `levels`
 * levels of OR_P points, logs every log_every steps (0: never). */
or_ens* or_ens_create(const or_params* p, uint64_t seed, int M, uint32_t chain_offset, int G,
                      int levels, int log_every, int max_logs);
void or_ens_destroy(or_ens* e);
void or_ens_init(or_ens* e);
/* piecewise-constant kappa from step `from_step` on (replaces later entries):
 * the step t -> t+1 uses the entry with the largest from_step <= t.  Pinned
 * by the schedule-switch closed form. */
int or_ens_set_flow(or_ens* e, int64_t from_step, const double kappa[9]);
/* Run n_steps.  Optional per-step traces (NULL to skip): Z_tr[n_steps][M],
 * S_tr[n_steps][M][z_max] (-1 for empty slots), margin_tr[n_steps][M]. */
int or_ens_run(or_ens* e, int64_t n_steps, int nthreads, int32_t* Z_tr, int32_t* S_tr,
               double* margin_tr);
/* or_ens_run with a decision tape [n_steps][M][N]: tape_mode 1 records, 2 replays. */
int or_ens_run_tape(or_ens* e, int64_t n_steps, int nthreads, int32_t* Z_tr, int32_t* S_tr,
                    double* margin_tr, uint8_t* tape, int tape_mode);
void or_ens_get_state(const or_ens* e, double* R, int32_t* Z, int32_t* S, double* A);
void or_ens_set_state(or_ens* e, const double* R, const int32_t* Z, const int32_t* S,
                      const double* A);
int64_t or_ens_step(const or_ens* e);
/* Position the step counter (the Philox counter of the next step); test
 * support for re-running a window from a saved state with the same noise. */
void or_ens_set_step(or_ens* e, int64_t step);
/* correlator group sums acc[G][levels][OR_P][2 channels][3 comps] and the
 * number of samples pushed so far (per chain) */
void or_ens_corr(const or_ens* e, double* acc, int64_t* n_samples);
/* group sums of channel TT, acc_tt[G][levels][OR_P][3 comps] */
void or_ens_corr_tt(const or_ens* e, double* acc_tt);
/* logs[n][G][14]: sums of sigma (xx,yy,zz,xy,xz,yz), sigma^2 (same order), Z, Z^2;
 * log_step[n] = step index after which log n was taken.  Returns n. */
int or_ens_logs(const or_ens* e, double* logs, int64_t* log_step, int cap);
void or_ens_reset_obs(or_ens* e);
/* counters: hops up, hops down, created, destroyed, dropped (summed) */
void or_ens_counters(const or_ens* e, int64_t out[5]);

#ifdef __cplusplus
}
#endif
#endif
