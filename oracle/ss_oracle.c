/*
 * ss_oracle.c -- plain FP64 CPU oracle of the single-chain slip-spring model.
 *
 * TEST INFRASTRUCTURE ONLY (see ss_oracle.h).  Built with -ffp-contract=off so
 * that every multiply and add rounds separately, in source order.
 *
 * The method (arXiv:1106.2899):
 *   state      beads R_i, springs (S_j, A_j), j < Z                  Sec. 2.1
 *   free energy F = sum_i k_b/2 |R_{i+1}-R_i|^2 + sum_j k_s/2 |R_Sj - A_j|^2
 *                                                      Eq. free_energy_single_chain
 *   step       1. Euler-Maruyama for R, affine advection for A       Sec. 3.1 item 1
 *              2. hops S_j -> S_j +- 1 with capped Glauber probabilities
 *                                                                    Sec. 3.1 item 2
 *              3. creation at the ends (K attempts), then destruction at the
 *                 ends, then re-indexing j = 1..Z                    Sec. 3.1 item 3
 *   stress     sigma = k_b sum QQ - N kT 1        Eq. stress_tensor_single_chain
 *   virtual    sigma_v = k_s sum_{j<Z} dd - Z kT 1, d = R_Sj - A_j   App. B
 *   G(t)       = (c0/kT)[<s(t)s(0)> + <s(t)s_v(0)>]   Eq. relaxation_modulus_..._green_kubo_form
 */
#include "ss_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------ operation counts --
 * With -DOR_COUNT_OPS (a separate, single-threaded build) every executed
 * operation of the method adds to a counter of its substep; the rules are in
 * ss_oracle.h.  Without it OR_OPS compiles to nothing. */
#ifdef OR_COUNT_OPS
static int64_t or_ops[OR_OPC_N];
#define OR_OPS(cat, n) (or_ops[(cat)] += (int64_t)(n))
void or_ops_get(int64_t out[OR_OPC_N]) { memcpy(out, or_ops, sizeof(or_ops)); }
void or_ops_reset(void) { memset(or_ops, 0, sizeof(or_ops)); }
int or_ops_enabled(void) { return 1; }
#else
#define OR_OPS(cat, n) ((void)0)
void or_ops_get(int64_t out[OR_OPC_N]) { memset(out, 0, sizeof(int64_t) * OR_OPC_N); }
void or_ops_reset(void) {}
int or_ops_enabled(void) { return 0; }
#endif

/* ---------------------------------------------------------------- Philox -- */
/* Philox4x32-10 as published by Salmon et al., SC'11: a 4x32-bit counter and a
 * 2x32-bit key; each round multiplies counter words 0 and 2 by two fixed odd
 * constants (full 64-bit products), swaps and xors the high halves with the
 * other counter words and the round key; the key is bumped by two Weyl
 * constants between rounds. */
#define OR_PHILOX_M0 0xD2511F53u
#define OR_PHILOX_M1 0xCD9E8D57u
#define OR_PHILOX_W0 0x9E3779B9u
#define OR_PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        OR_OPS(OR_OPC_PHILOX, round > 0 ? 6 : 4);
        if (round > 0) {
            k0 += OR_PHILOX_W0;
            k1 += OR_PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)OR_PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)OR_PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0;
        x1 = y1;
        x2 = y2;
        x3 = y3;
    }
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    out[3] = x3;
}

static void or_block(const uint32_t key[2], uint32_t index, uint32_t step, uint32_t purpose,
                     uint32_t chain, uint32_t w[4]) {
    uint32_t ctr[4] = {index, step, purpose, chain};
    or_philox4x32_10(ctr, key, w);
}

/* ------------------------------------------------------- random decoding -- */
static const double OR_TWO_M24 = 1.0 / 16777216.0; /* 2^-24 */
static const double OR_PI = 3.14159265358979323846;

/* Box-Muller: radius sqrt(-2 ln v), v in (0,1]; angle pi*(2u-1), u in [0,1). */
static void or_box_muller(uint32_t wa, uint32_t wb, double* n_cos, double* n_sin) {
    /* shift, +1, convert, scale, log, x(-2), sqrt; shift, convert, scale,
     * 2u - 1 (fused), x pi, cos, sin, two products */
    OR_OPS(OR_OPC_DECODE, 16);
    double v = ((double)(wa >> 8) + 1.0) * OR_TWO_M24;
    double u = (double)(wb >> 8) * OR_TWO_M24;
    double r = sqrt(-2.0 * log(v));
    double th = OR_PI * (2.0 * u - 1.0);
    *n_cos = r * cos(th);
    *n_sin = r * sin(th);
}

void or_decode_block(const uint32_t w[4], double n[4], double* u) {
    or_box_muller(w[0], w[1], &n[0], &n[1]);
    or_box_muller(w[2], w[3], &n[2], &n[3]);
    uint32_t lo = (w[0] & 0xFFu) | ((w[1] & 0xFFu) << 8) | ((w[2] & 0xFFu) << 16);
    *u = (double)lo * OR_TWO_M24;
    OR_OPS(OR_OPC_DECODE, 9); /* three masks, two shifts, two ors, convert, scale */
}

/* ------------------------------------------------------------ parameters -- */
void or_params_derive(or_params* p) {
    if (!(p->k_b > 0)) p->k_b = 3.0 * p->kT / (p->b * p->b);
    if (!(p->k_s > 0)) p->k_s = 3.0 * p->kT / (p->Ns * p->b * p->b);
}

/* Standard normal CDF via erfc; inverse by bisection (monotone, 200 halvings
 * reach the double spacing everywhere in [-40, 40]). */
static double or_norm_cdf(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

double or_norm_ppf(double p) {
    if (p >= 1.0) return INFINITY;
    if (p <= 0.0) return -INFINITY;
    double lo = -40.0, hi = 40.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        if (or_norm_cdf(mid) < p)
            lo = mid;
        else
            hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------ init -- */
/* Sec. 3.1 sampling: (1) ideal-chain bonds, variance kT/k_b = b^2/3 per
 * component (Eq. bead_position_distribution); (2) Z ~ Poisson(N/N0) by inverse
 * CDF on a 53-bit uniform (Eq. slip_spring_number_distribution_modified),
 * capped at z_max; (3) S_j uniform on the N beads (Eq. bead_index_distribution)
 * and A_j = R_Sj + sqrt(kT/k_s) n, variance Ns b^2/3 per component
 * (Eq. anchoring_point_distribution). */
void or_init_chain(const or_params* p, const uint32_t key[2], uint32_t chain_id, or_chain* c) {
    const int N = p->N;
    memset(c, 0, sizeof(*c));
    double sb = sqrt(p->kT / p->k_b);
    for (int i = 0; i + 1 < N; ++i) {
        uint32_t w[4];
        double n[4], u;
        or_block(key, (uint32_t)i, 0u, OR_PURPOSE_INIT_BOND, chain_id, w);
        or_decode_block(w, n, &u);
        for (int a = 0; a < 3; ++a) c->R[i + 1][a] = c->R[i][a] + sb * n[a];
    }
    /* Z */
    {
        uint32_t w[4];
        or_block(key, 0u, 0u, OR_PURPOSE_INIT_Z, chain_id, w);
        double u53 = ((double)(w[0] >> 5) * 67108864.0 + (double)(w[1] >> 6)) / 9007199254740992.0;
        double lam = (double)N / p->N0; /* 0 when N0 = inf */
        int Z = p->z_max;
        double pmf = exp(-lam), cdf = pmf;
        for (int k = 0; k < p->z_max; ++k) {
            if (u53 < cdf) {
                Z = k;
                break;
            }
            pmf *= lam / (double)(k + 1);
            cdf += pmf;
        }
        c->Z = Z;
    }
    double sa = sqrt(p->kT / p->k_s);
    for (int j = 0; j < c->Z; ++j) {
        uint32_t w[4];
        double n[4], u;
        or_block(key, (uint32_t)j, 0u, OR_PURPOSE_INIT_S, chain_id, w);
        c->S[j] = (int)(((uint64_t)w[0] * (uint64_t)N) >> 32);
        or_block(key, (uint32_t)j, 0u, OR_PURPOSE_INIT_A, chain_id, w);
        or_decode_block(w, n, &u);
        for (int a = 0; a < 3; ++a) c->A[j][a] = c->R[c->S[j]][a] + sa * n[a];
    }
}

/* ------------------------------------------------------------------ step -- */
void or_step_chain_tape(const or_params* p, const uint32_t key[2], uint32_t chain_id, uint32_t step,
                        const double kap[9], double cd, or_chain* c, or_step_info* info, const uint8_t* replay,
                        uint8_t* record);
static double or_dist2(const double x[3], const double y[3]) {
    double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
    return d0 * d0 + d1 * d1 + d2 * d2;
}

/* Capped hop probability of Sec. 3.1 item 2:
 * min{ dt kT/zeta_s [1 - tanh(y)], 1/2 },  y = k_s (|R'-A|^2 - |R-A|^2)/(4 kT)
 * (= 3/(4 Ns b^2) times the change of squared spring length).  1 - tanh(y) is
 * evaluated as 2/(1+exp(2y)), the same number without cancellation; y is
 * clamped to [-40, 40] where the expression is saturated anyway. */
static double or_hop_prob(const or_params* p, double d_new, double d_old) {
    /* difference, scale, 2 clamps, x2, exp, +1, reciprocal, x(2 pref), cap */
    OR_OPS(OR_OPC_HOP, 10);
    double y = p->k_s * (d_new - d_old) / (4.0 * p->kT);
    if (y > 40.0) y = 40.0;
    if (y < -40.0) y = -40.0;
    double w = (p->dt * p->kT / p->zeta_s) * (2.0 / (1.0 + exp(2.0 * y)));
    return w < 0.5 ? w : 0.5;
}

static void or_margin(double* m, double a, double b) {
    double d = fabs(a - b);
    if (d < *m) *m = d;
}

void or_step_chain(const or_params* p, const uint32_t key[2], uint32_t chain_id, uint32_t step,
                   const double kap[9], double cd, or_chain* c, or_step_info* info) {
    or_step_chain_tape(p, key, chain_id, step, kap, cd, c, info, NULL, NULL);
}

/* Decision tape (test support for frozen-decision finite differences): one
 * byte per slot/attempt index j and step; bit 0: spring j hopped to S+1, bit 1:
 * to S-1, bit 2: attempt j created a spring at bead 1, bit 3: at bead N, bit 4:
 * old spring j destroyed, bit 5: the spring created by attempt j destroyed.
 * With `replay` the decisions are read instead of drawn. */
void or_step_chain_tape(const or_params* p, const uint32_t key[2], uint32_t chain_id, uint32_t step,
                        const double kap[9], double cd, or_chain* c, or_step_info* info, const uint8_t* replay,
                        uint8_t* record) {
    uint8_t tape[OR_NMAX];
    memset(tape, 0, sizeof(tape));
    const int N = p->N;
    double nrm[OR_NMAX][4], uni[OR_NMAX];
    for (int i = 0; i < N; ++i) {
        uint32_t w[4];
        or_block(key, (uint32_t)i, step, OR_PURPOSE_STEP, chain_id, w);
        or_decode_block(w, nrm[i], &uni[i]);
    }
    or_step_info inf = {INFINITY, 0, 0, 0, 0, 0};

    /* ---- substep 1: forces on the state at time t, then the Euler update. */
    double F[OR_NMAX][3];
    for (int i = 0; i < N; ++i)
        for (int a = 0; a < 3; ++a) {
            double f = 0.0;
            if (i > 0) f += p->k_b * (c->R[i - 1][a] - c->R[i][a]);
            if (i + 1 < N) f += p->k_b * (c->R[i + 1][a] - c->R[i][a]);
            F[i][a] = f;
            OR_OPS(OR_OPC_BOND, 2 * ((i > 0) + (i + 1 < N))); /* difference, multiply-add */
        }
    for (int j = 0; j < c->Z; ++j) {
        int s = c->S[j];
        for (int a = 0; a < 3; ++a) F[s][a] += p->k_s * (c->A[j][a] - c->R[s][a]);
        OR_OPS(OR_OPC_SPRING, 6);
    }
    const double mob = p->dt / p->zeta;
    const double amp = sqrt(2.0 * p->kT * p->dt / p->zeta);
    double Rn[OR_NMAX][3];
    int kap_on = 0; /* the flow term of the method vanishes when kappa = 0 */
    for (int k = 0; k < 9; ++k) kap_on |= kap[k] != 0.0;
    OR_OPS(OR_OPC_EULER, (int64_t)N * (kap_on ? 6 + 9 : 6)); /* 2 multiply-adds (+3 flow, +1) per component */
    if (kap_on) OR_OPS(OR_OPC_ADVECT, (int64_t)c->Z * 12); /* kappa . A: 3, A + dt flow: 1 per component */
    double flowR[OR_NMAX][3], flowA[OR_NMAX][3];
    for (int i = 0; i < N; ++i)
        for (int a = 0; a < 3; ++a) {
            double flow = kap[3 * a + 0] * c->R[i][0] + kap[3 * a + 1] * c->R[i][1] +
                          kap[3 * a + 2] * c->R[i][2];
            flowR[i][a] = flow;
            Rn[i][a] = c->R[i][a] + mob * F[i][a] + p->dt * flow + amp * nrm[i][a];
        }
    double An[OR_NMAX][3];
    for (int j = 0; j < c->Z; ++j)
        for (int a = 0; a < 3; ++a) {
            double flow = kap[3 * a + 0] * c->A[j][0] + kap[3 * a + 1] * c->A[j][1] +
                          kap[3 * a + 2] * c->A[j][2];
            flowA[j][a] = flow;
            An[j][a] = c->A[j][a] + p->dt * flow;
        }
    if (p->integrator == OR_HEUN) {
        /* corrector: drifts at the predicted state (Rn, An) with the same
         * springs, then the average of both drifts and the same noise */
        double F2[OR_NMAX][3];
        for (int i = 0; i < N; ++i)
            for (int a = 0; a < 3; ++a) {
                double f = 0.0;
                if (i > 0) f += p->k_b * (Rn[i - 1][a] - Rn[i][a]);
                if (i + 1 < N) f += p->k_b * (Rn[i + 1][a] - Rn[i][a]);
                F2[i][a] = f;
                OR_OPS(OR_OPC_BOND, 2 * ((i > 0) + (i + 1 < N)));
            }
        for (int j = 0; j < c->Z; ++j) {
            int s = c->S[j];
            for (int a = 0; a < 3; ++a) F2[s][a] += p->k_s * (An[j][a] - Rn[s][a]);
            OR_OPS(OR_OPC_SPRING, 6);
        }
        const double hmob = 0.5 * mob, hdt = 0.5 * p->dt;
        OR_OPS(OR_OPC_EULER, (int64_t)N * (kap_on ? 9 + 9 : 9)); /* sum of forces, 2 multiply-adds, noise */
        if (kap_on) OR_OPS(OR_OPC_ADVECT, (int64_t)c->Z * 12);
        for (int i = 0; i < N; ++i) {
            double flow2[3];
            for (int a = 0; a < 3; ++a)
                flow2[a] = kap[3 * a + 0] * Rn[i][0] + kap[3 * a + 1] * Rn[i][1] + kap[3 * a + 2] * Rn[i][2];
            for (int a = 0; a < 3; ++a)
                Rn[i][a] = c->R[i][a] + hmob * (F[i][a] + F2[i][a]) + hdt * (flowR[i][a] + flow2[a]) +
                           amp * nrm[i][a];
        }
        for (int j = 0; j < c->Z; ++j) {
            double flow2[3];
            for (int a = 0; a < 3; ++a)
                flow2[a] = kap[3 * a + 0] * An[j][0] + kap[3 * a + 1] * An[j][1] + kap[3 * a + 2] * An[j][2];
            for (int a = 0; a < 3; ++a) An[j][a] = c->A[j][a] + hdt * (flowA[j][a] + flow2[a]);
        }
    }
    for (int j = 0; j < c->Z; ++j) memcpy(c->A[j], An[j], sizeof(double) * 3);
    memcpy(c->R, Rn, sizeof(double) * 3 * (size_t)N);

    /* ---- substep 2: hops on the post-substep-1 positions.  One uniform per
     * spring: [0, p+) -> S+1, [p+, p+ + p-) -> S-1, otherwise stay. */
    for (int j = 0; j < c->Z; ++j) {
        int s = c->S[j];
        /* three squared distances (3 differences, 3 products/multiply-adds
         * each), the decision: p+ + p-, two comparisons */
        OR_OPS(OR_OPC_HOP, 6 * (1 + (s < N - 1) + (s > 0)) + 3);
        double d0 = or_dist2(c->R[s], c->A[j]);
        double pp = (s < N - 1) ? or_hop_prob(p, or_dist2(c->R[s + 1], c->A[j]), d0) : 0.0;
        double pm = (s > 0) ? or_hop_prob(p, or_dist2(c->R[s - 1], c->A[j]), d0) : 0.0;
        double u = uni[j];
        or_margin(&inf.min_margin, u, pp);
        or_margin(&inf.min_margin, u, pp + pm);
        int up = u < pp, down = !up && u < pp + pm;
        if (replay) {
            up = (replay[j] & 1) != 0;
            down = (replay[j] & 2) != 0;
        }
        if (up) {
            c->S[j] = s + 1;
            inf.hops_up++;
            tape[j] |= 1;
        } else if (down) {
            c->S[j] = s - 1;
            inf.hops_down++;
            tape[j] |= 2;
        }
    }

    /* ---- substep 3a: creation.  K attempts, each choosing end 1 with
     * probability pc, end N with probability pc, nothing otherwise. */
    const int Zc = c->Z;
    int first = Zc, last = Zc; /* attempt indices [first, last) */
    if (Zc < p->z_max) last = (p->create_mode == 0) ? p->z_max : Zc + 1;
    if (Zc >= p->z_max && p->create_mode == 1) inf.dropped += 1; /* K = 1 form at capacity */
    int K = last - first;
    int new_end[OR_NMAX];
    double new_A[OR_NMAX][3];
    for (int j = 0; j < OR_NMAX; ++j) new_end[j] = -1;
    if (K > 0) {
        double pc = p->dt * p->kT / (p->zeta_s * p->N0 * (double)K);
        if (pc > 0.5) pc = 0.5;
        double sa = sqrt(p->kT / p->k_s);
        for (int j = first; j < last; ++j) {
            double u = uni[j];
            OR_OPS(OR_OPC_CREATE, 2); /* u < pc, u < 2 pc */
            or_margin(&inf.min_margin, u, pc);
            or_margin(&inf.min_margin, u, 2.0 * pc);
            int end = -1;
            if (u < pc)
                end = 0;
            else if (u < 2.0 * pc)
                end = N - 1;
            if (replay) end = (replay[j] & 4) ? 0 : ((replay[j] & 8) ? N - 1 : -1);
            if (end < 0) continue;
            tape[j] |= end == 0 ? 4 : 8;
            uint32_t w[4];
            double n[4], uu;
            or_block(key, (uint32_t)j, step, OR_PURPOSE_CREATE, chain_id, w);
            or_decode_block(w, n, &uu);
            new_end[j] = end;
            OR_OPS(OR_OPC_CREATE, 3); /* anchor: one multiply-add per component */
            for (int a = 0; a < 3; ++a) new_A[j][a] = c->R[end][a] + sa * n[a];
            inf.created++;
        }
    }

    /* ---- substep 3b: destruction of springs at either end with probability
     * pd = min(dt kT/zeta_s, 1).  The uniform is Phi(n3) of slot j's block, so
     * the test u < pd reads n3 < Phi^{-1}(pd) = cd. */
    int alive[OR_NMAX];
    for (int j = 0; j < Zc; ++j) {
        alive[j] = 1;
        int s = c->S[j];
        if (s == 0 || s == N - 1) {
            OR_OPS(OR_OPC_DESTROY, 1);
            or_margin(&inf.min_margin, nrm[j][3], cd);
            int kill = nrm[j][3] < cd;
            if (replay) kill = (replay[j] & 16) != 0;
            if (kill) {
                alive[j] = 0;
                inf.destroyed++;
                tape[j] |= 16;
            }
        }
    }
    for (int j = first; j < last; ++j) {
        if (new_end[j] < 0 || !p->destroy_new) continue;
        OR_OPS(OR_OPC_DESTROY, 1);
        or_margin(&inf.min_margin, nrm[j][3], cd);
        int kill = nrm[j][3] < cd;
        if (replay) kill = (replay[j] & 32) != 0;
        if (kill) {
            new_end[j] = -2; /* created and destroyed within the step */
            inf.destroyed++;
            tape[j] |= 32;
        }
    }

    /* ---- re-indexing: surviving springs keep their order, then the new ones
     * at bead 1 in attempt order, then the new ones at bead N. */
    or_chain out;
    int z = 0;
    for (int j = 0; j < Zc; ++j)
        if (alive[j]) {
            out.S[z] = c->S[j];
            memcpy(out.A[z], c->A[j], sizeof(double) * 3);
            ++z;
        }
    for (int pass = 0; pass < 2; ++pass) {
        int want = pass == 0 ? 0 : N - 1;
        for (int j = first; j < last; ++j)
            if (new_end[j] == want) {
                out.S[z] = want;
                memcpy(out.A[z], new_A[j], sizeof(double) * 3);
                ++z;
            }
    }
    c->Z = z;
    for (int j = 0; j < z; ++j) {
        c->S[j] = out.S[j];
        memcpy(c->A[j], out.A[j], sizeof(double) * 3);
    }
    for (int j = z; j < OR_NMAX; ++j) c->S[j] = 0;
    if (record) memcpy(record, tape, (size_t)N);
    if (info) *info = inf;
}

/* ---------------------------------------------------------------- stress -- */
void or_stress(const or_params* p, const or_chain* c, double sig[9], double sigv[9]) {
    for (int k = 0; k < 9; ++k) sig[k] = sigv[k] = 0.0;
    for (int i = 0; i + 1 < p->N; ++i) {
        double q[3];
        for (int a = 0; a < 3; ++a) q[a] = c->R[i + 1][a] - c->R[i][a];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) sig[3 * a + b] += p->k_b * q[a] * q[b];
    }
    for (int j = 0; j < c->Z; ++j) {
        double d[3];
        for (int a = 0; a < 3; ++a) d[a] = c->R[c->S[j]][a] - c->A[j][a];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) sigv[3 * a + b] += p->k_s * d[a] * d[b];
    }
    for (int a = 0; a < 3; ++a) {
        sig[4 * a] -= (double)p->N * p->kT;
        sigv[4 * a] -= (double)c->Z * p->kT;
    }
}

/* ----------------------------------------------------- multiple-tau ------ */
/* Level 0 holds the last OR_P raw samples and lags 0..OR_P-1.  Every two
 * samples of level l-1 give one sample of level l, their average, so a level-l
 * sample is the mean of 2^l consecutive raw samples; level l >= 1 contributes
 * lags k*2^l for k = OR_P/2 .. OR_P-1.  Each sample x holds six signals:
 * sigma_xy, sigma_xz, sigma_yz and the same components of sigma + sigma_v.
 * Channel 0 accumulates later sigma times origin sigma (AUTO); channel 1 later
 * sigma times origin sigma + sigma_v (TOTAL); the optional channel TT (acc_tt)
 * later sigma + sigma_v times origin sigma + sigma_v, whose difference with
 * TOTAL is the virtual-stress numerator of Sec. 4.1 (Eq.
 * relative_contribution_virtual_stress_to_shear_relaxation_modulus). */
typedef struct {
    double hist[OR_LMAX][OR_P][6];
    int64_t nfill[OR_LMAX];
    double pend[OR_LMAX][6];
    int npend[OR_LMAX];
} or_corr_chain;

static void or_corr_push(or_corr_chain* cc, double* acc /* [levels][P][2][3] */,
                         double* acc_tt /* [levels][P][3] or NULL */, int levels, int l, const double v[6]) {
    for (int k = OR_P - 1; k > 0; --k) memcpy(cc->hist[l][k], cc->hist[l][k - 1], sizeof(double) * 6);
    memcpy(cc->hist[l][0], v, sizeof(double) * 6);
    cc->nfill[l]++;
    int kmin = (l == 0) ? 0 : OR_P / 2;
    for (int k = kmin; k < OR_P; ++k) {
        if (cc->nfill[l] <= k) break;
        double* a = acc + ((size_t)l * OR_P + (size_t)k) * 6;
        OR_OPS(OR_OPC_CORR, 6); /* one multiply-add per product (the optional channel TT not counted) */
        for (int c = 0; c < 3; ++c) {
            a[c] += v[c] * cc->hist[l][k][c];
            a[3 + c] += v[c] * cc->hist[l][k][3 + c];
        }
        if (acc_tt) {
            double* b = acc_tt + ((size_t)l * OR_P + (size_t)k) * 3;
            for (int c = 0; c < 3; ++c) b[c] += v[3 + c] * cc->hist[l][k][3 + c];
        }
    }
    for (int s = 0; s < 6; ++s) cc->pend[l][s] += v[s];
    cc->npend[l]++;
    OR_OPS(OR_OPC_CORR, 6); /* block sums */
    if (cc->npend[l] == 2) {
        OR_OPS(OR_OPC_CORR, 6); /* block means */
        double up[6];
        for (int s = 0; s < 6; ++s) up[s] = 0.5 * cc->pend[l][s];
        memset(cc->pend[l], 0, sizeof(cc->pend[l]));
        cc->npend[l] = 0;
        if (l + 1 < levels) or_corr_push(cc, acc, acc_tt, levels, l + 1, up);
    }
}

void or_corr_series(const double* x, int64_t T, int levels, double* acc) {
    or_corr_series_tt(x, T, levels, acc, NULL);
}

void or_corr_series_tt(const double* x, int64_t T, int levels, double* acc, double* acc_tt) {
    or_corr_chain* cc = (or_corr_chain*)calloc(1, sizeof(or_corr_chain));
    for (int64_t t = 0; t < T; ++t) or_corr_push(cc, acc, acc_tt, levels, 0, x + 6 * t);
    free(cc);
}

/* ------------------------------------------------------------ ensemble --- */
typedef struct {
    int64_t from;
    double k[9];
} or_flow_entry;

struct or_ens {
    or_params p;
    uint32_t key[2];
    int M, G, levels, log_every, max_logs, nlogs;
    uint32_t chain_offset;
    int64_t step;
    double cd;
    or_chain* ch;
    or_corr_chain* cc;
    double* acc;  /* [G][levels][P][6] */
    double* acc_tt; /* [G][levels][P][3] */
    double* logs; /* [max_logs][G][14] */
    int64_t* log_step;
    int64_t n_samples;
    or_flow_entry* flow;
    int nflow, capflow;
    int64_t counters[5];
};

or_ens* or_ens_create(const or_params* p, uint64_t seed, int M, uint32_t chain_offset, int G,
                      int levels, int log_every, int max_logs) {
    if (M <= 0 || G <= 0 || G > M || levels < 1 || levels > OR_LMAX) return NULL;
    if (p->N < 2 || p->N > OR_NMAX || p->z_max < 1 || p->z_max > p->N) return NULL;
    if (p->integrator != OR_EULER && p->integrator != OR_HEUN) return NULL;
    or_ens* e = (or_ens*)calloc(1, sizeof(or_ens));
    e->p = *p;
    or_params_derive(&e->p);
    e->key[0] = (uint32_t)seed;
    e->key[1] = (uint32_t)(seed >> 32);
    e->M = M;
    e->G = G;
    e->levels = levels;
    e->log_every = log_every;
    e->max_logs = max_logs > 0 ? max_logs : 0;
    e->chain_offset = chain_offset;
    double pd = e->p.dt * e->p.kT / e->p.zeta_s;
    e->cd = or_norm_ppf(pd < 1.0 ? pd : 1.0);
    e->ch = (or_chain*)calloc((size_t)M, sizeof(or_chain));
    e->cc = (or_corr_chain*)calloc((size_t)M, sizeof(or_corr_chain));
    e->acc = (double*)calloc((size_t)G * levels * OR_P * 6, sizeof(double));
    e->acc_tt = (double*)calloc((size_t)G * levels * OR_P * 3, sizeof(double));
    e->logs = (double*)calloc((size_t)(e->max_logs ? e->max_logs : 1) * G * 14, sizeof(double));
    e->log_step = (int64_t*)calloc((size_t)(e->max_logs ? e->max_logs : 1), sizeof(int64_t));
    e->capflow = 16;
    e->flow = (or_flow_entry*)calloc((size_t)e->capflow, sizeof(or_flow_entry));
    e->nflow = 1; /* kappa = 0 from step 0 */
    return e;
}

void or_ens_destroy(or_ens* e) {
    if (!e) return;
    free(e->ch);
    free(e->cc);
    free(e->acc);
    free(e->acc_tt);
    free(e->logs);
    free(e->log_step);
    free(e->flow);
    free(e);
}

void or_ens_init(or_ens* e) {
    for (int m = 0; m < e->M; ++m) or_init_chain(&e->p, e->key, e->chain_offset + (uint32_t)m, &e->ch[m]);
    e->step = 0;
}

int or_ens_set_flow(or_ens* e, int64_t from_step, const double kappa[9]) {
    int n = 0;
    while (n < e->nflow && e->flow[n].from < from_step) ++n;
    if (n + 1 > e->capflow) {
        e->capflow = 2 * (n + 1);
        e->flow = (or_flow_entry*)realloc(e->flow, sizeof(or_flow_entry) * (size_t)e->capflow);
    }
    e->flow[n].from = from_step;
    memcpy(e->flow[n].k, kappa, sizeof(double) * 9);
    e->nflow = n + 1;
    return 0;
}

static const double* or_kappa_at(const or_ens* e, int64_t t) {
    const double* k = e->flow[0].k;
    for (int i = 0; i < e->nflow; ++i)
        if (e->flow[i].from <= t) k = e->flow[i].k;
    return k;
}

int or_ens_run(or_ens* e, int64_t n_steps, int nthreads, int32_t* Z_tr, int32_t* S_tr,
               double* margin_tr) {
    return or_ens_run_tape(e, n_steps, nthreads, Z_tr, S_tr, margin_tr, NULL, 0);
}

int or_ens_run_tape(or_ens* e, int64_t n_steps, int nthreads, int32_t* Z_tr, int32_t* S_tr,
                    double* margin_tr, uint8_t* tape, int tape_mode) {
    const int M = e->M, G = e->G, zmax = e->p.z_max;
    const int64_t t0 = e->step;
    const size_t per_acc = (size_t)e->levels * OR_P * 6;
    int nlog_new = 0;
    if (e->log_every > 0) {
        for (int64_t t = t0 + 1; t <= t0 + n_steps; ++t)
            if (t % e->log_every == 0) ++nlog_new;
        if (e->nlogs + nlog_new > e->max_logs) return -1;
        int n = e->nlogs;
        for (int64_t t = t0 + 1; t <= t0 + n_steps; ++t)
            if (t % e->log_every == 0) e->log_step[n++] = t;
    }
    int64_t cnt[5] = {0, 0, 0, 0, 0};
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : cnt[:5])
#else
    (void)nthreads;
#endif
    for (int g = 0; g < G; ++g) {
        int m0 = (int)(((int64_t)g * M) / G), m1 = (int)(((int64_t)(g + 1) * M) / G);
        double* acc = e->acc + (size_t)g * per_acc;
        for (int m = m0; m < m1; ++m) {
            or_chain* c = &e->ch[m];
            or_corr_chain* cc = &e->cc[m];
            int lg = e->nlogs;
            for (int64_t s = 0; s < n_steps; ++s) {
                int64_t t = t0 + s;
                or_step_info info;
                uint8_t* row = tape ? tape + ((size_t)s * M + m) * (size_t)e->p.N : NULL;
                or_step_chain_tape(&e->p, e->key, e->chain_offset + (uint32_t)m, (uint32_t)t, or_kappa_at(e, t),
                                   e->cd, c, &info, tape_mode == 2 ? row : NULL, tape_mode == 1 ? row : NULL);
                cnt[0] += info.hops_up;
                cnt[1] += info.hops_down;
                cnt[2] += info.created;
                cnt[3] += info.destroyed;
                cnt[4] += info.dropped;
                double sig[9], sigv[9];
                or_stress(&e->p, c, sig, sigv);
                /* the correlator needs the off-diagonal xy, xz, yz of sigma and
                 * sigma + sigma_v: per bond or spring 3 differences, 2 products,
                 * 3 multiply-adds; 3 additions per chain.  A log step adds the
                 * diagonal (3 multiply-adds per bond and spring, 3 subtractions). */
                OR_OPS(OR_OPC_STRESS, 8 * (int64_t)(e->p.N - 1 + c->Z) + 3);
                if (e->log_every > 0 && (t + 1) % e->log_every == 0)
                    OR_OPS(OR_OPC_STRESS, 3 * (int64_t)(e->p.N - 1 + c->Z) + 6);
                double v[6] = {sig[1], sig[2], sig[5], sig[1] + sigv[1], sig[2] + sigv[2], sig[5] + sigv[5]};
                or_corr_push(cc, acc, e->acc_tt + (size_t)g * e->levels * OR_P * 3, e->levels, 0, v);
                if (e->log_every > 0 && (t + 1) % e->log_every == 0) {
                    double* L = e->logs + ((size_t)lg * G + (size_t)g) * 14;
                    double comp[6] = {sig[0], sig[4], sig[8], sig[1], sig[2], sig[5]};
                    for (int k = 0; k < 6; ++k) {
                        L[k] += comp[k];
                        L[6 + k] += comp[k] * comp[k];
                    }
                    L[12] += (double)c->Z;
                    L[13] += (double)c->Z * (double)c->Z;
                    ++lg;
                }
                if (Z_tr) Z_tr[(size_t)s * M + m] = c->Z;
                if (S_tr)
                    for (int j = 0; j < zmax; ++j)
                        S_tr[((size_t)s * M + m) * zmax + j] = j < c->Z ? c->S[j] : -1;
                if (margin_tr) margin_tr[(size_t)s * M + m] = info.min_margin;
            }
        }
    }
    for (int k = 0; k < 5; ++k) e->counters[k] += cnt[k];
    e->nlogs += nlog_new;
    e->step += n_steps;
    e->n_samples += n_steps;
    return 0;
}

void or_ens_get_state(const or_ens* e, double* R, int32_t* Z, int32_t* S, double* A) {
    const int N = e->p.N, zm = e->p.z_max;
    for (int m = 0; m < e->M; ++m) {
        const or_chain* c = &e->ch[m];
        if (R) memcpy(R + (size_t)m * N * 3, c->R, sizeof(double) * 3 * (size_t)N);
        if (Z) Z[m] = c->Z;
        for (int j = 0; j < zm; ++j) {
            if (S) S[(size_t)m * zm + j] = j < c->Z ? c->S[j] : -1;
            for (int a = 0; a < 3; ++a)
                if (A) A[((size_t)m * zm + j) * 3 + a] = j < c->Z ? c->A[j][a] : 0.0;
        }
    }
}

void or_ens_set_state(or_ens* e, const double* R, const int32_t* Z, const int32_t* S, const double* A) {
    const int N = e->p.N, zm = e->p.z_max;
    for (int m = 0; m < e->M; ++m) {
        or_chain* c = &e->ch[m];
        memset(c, 0, sizeof(*c));
        memcpy(c->R, R + (size_t)m * N * 3, sizeof(double) * 3 * (size_t)N);
        c->Z = Z[m];
        for (int j = 0; j < c->Z; ++j) {
            c->S[j] = S[(size_t)m * zm + j];
            for (int a = 0; a < 3; ++a) c->A[j][a] = A[((size_t)m * zm + j) * 3 + a];
        }
    }
}

int64_t or_ens_step(const or_ens* e) { return e->step; }

void or_ens_set_step(or_ens* e, int64_t step) { e->step = step; }

void or_ens_corr(const or_ens* e, double* acc, int64_t* n_samples) {
    memcpy(acc, e->acc, sizeof(double) * (size_t)e->G * e->levels * OR_P * 6);
    if (n_samples) *n_samples = e->n_samples;
}

void or_ens_corr_tt(const or_ens* e, double* acc_tt) {
    memcpy(acc_tt, e->acc_tt, sizeof(double) * (size_t)e->G * e->levels * OR_P * 3);
}

int or_ens_logs(const or_ens* e, double* logs, int64_t* log_step, int cap) {
    int n = e->nlogs < cap ? e->nlogs : cap;
    if (logs) memcpy(logs, e->logs, sizeof(double) * (size_t)n * e->G * 14);
    if (log_step) memcpy(log_step, e->log_step, sizeof(int64_t) * (size_t)n);
    return e->nlogs;
}

void or_ens_reset_obs(or_ens* e) {
    memset(e->cc, 0, sizeof(or_corr_chain) * (size_t)e->M);
    memset(e->acc, 0, sizeof(double) * (size_t)e->G * e->levels * OR_P * 6);
    memset(e->acc_tt, 0, sizeof(double) * (size_t)e->G * e->levels * OR_P * 3);
    memset(e->logs, 0, sizeof(double) * (size_t)(e->max_logs ? e->max_logs : 1) * e->G * 14);
    e->nlogs = 0;
    e->n_samples = 0;
}

void or_ens_counters(const or_ens* e, int64_t out[5]) { memcpy(out, e->counters, sizeof(int64_t) * 5); }
