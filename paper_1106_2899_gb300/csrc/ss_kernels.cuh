// ss_kernels.cuh -- sm_103a kernels of the single-chain slip-spring time step
// (T. Uneyama, arXiv:1106.2899, Sec. 3.1), with a per-step stress series
// for the multiple-tau correlator (a separate kernel) and ensemble stress logs.
//
// Layout: one chain per W-lane segment of a warp (W = 32: one chain per warp,
// W = 16: two), B beads per lane: lane l of a segment owns beads and
// slip-spring slots l, l + W, ..., so N <= W*B and z_max <= N (the paper's
// one-slot-per-bead bound, Sec. 3.2); slots above 64 stay empty (z_max <= 64,
// so a 64-bit mask covers a bead's springs).  A launch advances each chain `nsteps`
// steps with its whole state in registers; neighbouring beads are read from a
// per-warp shared-memory position table, stresses are reduced with shuffles.
//
// Random numbers: Philox4x32-10 (Salmon et al., SC'11), counter = (index,
// step, purpose, chain id), key = seed.  Per step, slot/bead index l draws
// one block: two Box-Muller pairs give the bead noise (x, y, z) and a fourth
// normal n3; the low bytes of the first three words give a 24-bit uniform u.
// Slot l uses u for its hop (occupied) or its creation attempt (empty) and n3
// for its destruction test n3 < Phi^{-1}(p_destroy).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace ssk {

constexpr int kP = 16;      // multiple-tau points per level
constexpr int kCells = 32;  // (channel, lag) cells per level and component: channel*16 + lag
constexpr uint32_t kPurposeStep = 1, kPurposeCreate = 2, kPurposeInitBond = 3,
                   kPurposeInitZ = 4, kPurposeInitS = 5, kPurposeInitA = 6;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxBeads = 128;  // beads per chain
constexpr int kMaxSlots = 64;   // slip-spring slots per chain (z_max <= min(N, kMaxSlots))
constexpr int kSliceChains = 64;  // chains per FP64 correlator/log slice
constexpr int kMaxCorrLevels = 32;  // correlator levels the library accepts

// ---------------------------------------------------------------- Philox ----
// Ten rounds of the Philox4x32 bijection: words 0 and 2 are multiplied by
// the two round multipliers (high and low halves kept), the high halves are
// xored with words 1 and 3 and the round key, and the key advances by the
// two Weyl increments after every round.
__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c0;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c2;
        c0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        c2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

// The same bijection with the ten round keys precomputed (kernel parameters).
__device__ __forceinline__ uint4 philox4x32_10_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                  const uint32_t (&rk0)[10], const uint32_t (&rk1)[10]) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c0;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c2;
        c0 = (uint32_t)(p1 >> 32) ^ c1 ^ rk0[r];
        c2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk1[r];
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
    }
    return make_uint4(c0, c1, c2, c3);
}

// The same generator for the step draws of a fixed (index, purpose, chain):
// counter (idx, t, P, cid).  Round 0 and most of round 1 do not depend on the
// step t, so their results are computed once per slot (pre) and per step
// (shared by all slots of a lane); philox_step finishes rounds 1..9 and
// returns the same words as philox4x32_10_rk(idx, t, P, cid).
struct PhiloxPre {
    uint32_t c3_1;  // lo(M0 idx) after round 0
    uint32_t c0_2;  // hi(M1 c2_1) ^ lo(M1 P) ^ rk0[1]
    uint32_t c1_2;  // lo(M1 c2_1)
};
__device__ __forceinline__ PhiloxPre philox_pre(uint32_t idx, uint32_t P, uint32_t cid, const uint32_t (&rk0)[10],
                                                const uint32_t (&rk1)[10]) {
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * idx;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * P;
    const uint32_t c2_1 = (uint32_t)(p0 >> 32) ^ cid ^ rk1[0];
    const uint32_t c1_1 = (uint32_t)p1;
    const unsigned long long q1 = (unsigned long long)0xCD9E8D57u * c2_1;
    PhiloxPre r;
    r.c3_1 = (uint32_t)p0;
    r.c0_2 = (uint32_t)(q1 >> 32) ^ c1_1 ^ rk0[1];
    r.c1_2 = (uint32_t)q1;
    return r;
}
// step part shared by the slots: c0 after round 0 is hi(M1 P) ^ t ^ rk0[0]
__device__ __forceinline__ unsigned long long philox_step_shared(uint32_t t, uint32_t P, const uint32_t (&rk0)[10]) {
    const uint32_t c0_1 = (uint32_t)(((unsigned long long)0xCD9E8D57u * P) >> 32) ^ t ^ rk0[0];
    return (unsigned long long)0xD2511F53u * c0_1;
}
__device__ __forceinline__ uint4 philox_step(const PhiloxPre& pre, unsigned long long p0_1, const uint32_t (&rk0)[10],
                                             const uint32_t (&rk1)[10]) {
    uint32_t c0 = pre.c0_2, c1 = pre.c1_2;
    uint32_t c2 = (uint32_t)(p0_1 >> 32) ^ pre.c3_1 ^ rk1[1];
    uint32_t c3 = (uint32_t)p0_1;
#pragma unroll
    for (int r = 2; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c0;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c2;
        c0 = (uint32_t)(p1 >> 32) ^ c1 ^ rk0[r];
        c2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk1[r];
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
    }
    return make_uint4(c0, c1, c2, c3);
}

// ------------------------------------------------------------ math traits ---
template <typename T>
struct Mth;

template <>
struct Mth<float> {
    static __device__ __forceinline__ float neg2log(float x) { return __log2f(x) * -1.3862943611198906f; }
    // sqrt of x >= 0 by the hardware approximation (sqrt.approx); x = 0 gives 0
    static __device__ __forceinline__ float sqrt(float x) {
        float r;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    static __device__ __forceinline__ void sincos(float x, float* s, float* c) { __sincosf(x, s, c); }
    static __device__ __forceinline__ float exp(float x) { return __expf(x); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
    static __device__ __forceinline__ bool finite(float x) { return isfinite(x); }
};

template <>
struct Mth<double> {
    static __device__ __forceinline__ double neg2log(double x) { return -2.0 * ::log(x); }
    static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
    static __device__ __forceinline__ void sincos(double x, double* s, double* c) { ::sincos(x, s, c); }
    static __device__ __forceinline__ double exp(double x) { return ::exp(x); }
    static __device__ __forceinline__ double div(double a, double b) { return a / b; }
    static __device__ __forceinline__ bool finite(double x) { return isfinite(x); }
};

// pi / 2^23 in both precisions (a power-of-two scaling of pi)
template <typename T>
__device__ __forceinline__ T pi_over_2p23();
template <>
__device__ __forceinline__ float pi_over_2p23<float>() { return 3.14159265358979323846f / 8388608.0f; }
template <>
__device__ __forceinline__ double pi_over_2p23<double>() { return 3.14159265358979323846 / 8388608.0; }

// Box-Muller pair from two words: radius sqrt(-2 ln v), v = (hi24(wa)+1)/2^24
// in (0,1]; angle pi (2 hi24(wb)/2^24 - 1) in [-pi, pi).
template <typename T>
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, T& n_cos, T& n_sin) {
    const T v = T((wa >> 8) + 1u) * T(1.0 / 16777216.0);
    const T r = Mth<T>::sqrt(Mth<T>::neg2log(v));
    const T th = T(int(wb >> 8) - (1 << 23)) * pi_over_2p23<T>();
    T s, c;
    Mth<T>::sincos(th, &s, &c);
    n_cos = r * c;
    n_sin = r * s;
}

// 24-bit uniform in [0, 1) from the low bytes of words x, y, z
__device__ __forceinline__ uint32_t lo24_bits(uint4 w) {
    return (w.x & 0xFFu) | ((w.y & 0xFFu) << 8) | ((w.z & 0xFFu) << 16);
}
template <typename T>
__device__ __forceinline__ T uniform_lo24(uint4 w) {
    return T(lo24_bits(w)) * T(1.0 / 16777216.0);
}

// ---- packed FP32x2 arithmetic (sm_100 and later: one instruction per pair).
// Where a lane carries an even number of FP32 beads, the identical scalar
// operations of two beads (sub-slots 2p and 2p+1) are issued as one packed
// instruction; each half is rounded exactly as the scalar operation, so the
// results are bit-identical to the scalar forms.
__device__ __forceinline__ float2 pk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 pk(float a) { return make_float2(a, a); }

// Box-Muller pairs of two beads (words a_k, b_k of bead k), the operations of
// box_muller<float> on each.
__device__ __forceinline__ void box_muller_x2(uint32_t a0, uint32_t b0, uint32_t a1, uint32_t b1, float& c0,
                                              float& s0, float& c1, float& s1) {
    const float2 v = __fmul2_rn(pk(float((a0 >> 8) + 1u), float((a1 >> 8) + 1u)), pk(1.0f / 16777216.0f));
    const float2 m = __fmul2_rn(pk(__log2f(v.x), __log2f(v.y)), pk(-1.3862943611198906f));
    const float2 r = pk(Mth<float>::sqrt(m.x), Mth<float>::sqrt(m.y));
    const float2 th = __fmul2_rn(pk(float(int(b0 >> 8) - (1 << 23)), float(int(b1 >> 8) - (1 << 23))),
                                 pk(3.14159265358979323846f / 8388608.0f));
    float sa, ca, sb, cb;
    __sincosf(th.x, &sa, &ca);
    __sincosf(th.y, &sb, &cb);
    const float2 cc = __fmul2_rn(r, pk(ca, cb));
    const float2 ss = __fmul2_rn(r, pk(sa, sb));
    c0 = cc.x;
    c1 = cc.y;
    s0 = ss.x;
    s1 = ss.y;
}

template <typename T>
__device__ __forceinline__ T shfl(T v, int src, int width) {
    return __shfl_sync(kFull, v, src, width);
}

// ------------------------------------------------------------- arguments ----
template <typename T>
struct StepConst {
    T k_b, k_s;   // bond and slip-spring stiffness
    T mob;        // dt / zeta
    T amp;        // sqrt(2 kT dt / zeta)
    T dt;
    T pref;       // dt kT / zeta_s: hop and destruction prefactor
    T chop;       // k_s / (4 kT): Glauber exponent per change of squared length
    T sa;         // sqrt(kT / k_s): anchor spread of a new spring
    T cd;         // Phi^{-1}(min(dt kT/zeta_s, 1)) (+inf when that is 1)
    T NkT, kT;
    T pc[kMaxSlots + 1];  // creation probability per end and attempt, by K
    T two_pref;           // 2 dt kT / zeta_s
    T c2;                 // 2 chop log2(e): base-2 exponent per change of squared length
    T hmob, hdt;          // mob / 2, dt / 2: the stochastic Heun corrector
    uint32_t rk0[10], rk1[10];  // Philox round keys (key + r * Weyl increment)
};

struct ChunkArgs {
    void* R;            // [M][3][W] T
    void* A;            // [M][3][W] T
    int32_t* S;         // [M][W]
    int32_t* Z;         // [M]
    double* logs;       // [max_logs][groups][14]
    unsigned long long* counters;  // [8]: events 0..4, 6 non-finite states, 7 broken invariants
    int32_t* status;
    const double* kap;          // [n_kap][9]
    const long long* kap_from;  // [n_kap]
    int n_kap;
    int M, N, zmax, create_mode, destroy_new;
    int log_every, recenter_every;
    long long log_m0;           // logs are taken at steps m*log_every with m > log_m0
    int max_logs, groups, slices;  // slices of kSliceChains chains
    long long t0;               // first step index of this launch
    int nsteps;
    uint32_t key0, key1, chain_base;
    int nlog_chunk;             // log slots reserved in shared memory
    int W, B;                   // lane layout (read by the batched kernel)
    // differentiation windows (all optional, null when unused):
    uint8_t* tape;              // [steps][M][NP] decisions per slot and step
    int tape_mode;              // 0 off, 1 record, 2 replay (decisions frozen)
    long long tape_t0;          // step of tape row 0
    long long tape_rows;        // rows of the tape (steps outside are neither read nor written)
    void* snapR;                // [steps+1][M][3][NP] T: state before each step
    void* snapA;
    int32_t* snapS;             // [steps+1][M][NP]
    int32_t* snapZ;             // [steps+1][M]
    long long snap_t0;
    int snap_steps;
    // stress series for the correlator (null: not written): element
    // [((series_row0 + s) * M + m) * 6 + q] is, after step s of this launch,
    // sigma_off (q = 0..2: xy, xz, yz) or (sigma + sigma^(v))_off (q = 3..5)
    void* series;
    long long series_row0;
};

// decision byte of one slot in one step (tape): hop, creation, destruction
constexpr uint8_t kTapeUp = 1, kTapeDown = 2, kTapeNew0 = 4, kTapeNewN = 8, kTapeKillOld = 16, kTapeKillNew = 32;

// One slip-spring slot as the force loop reads it from shared memory:
// anchor and bead index (-1: empty slot), 16 bytes in FP32.
template <typename T>
struct __align__(16) SlotRec {
    T x, y, z;
    int s;
};

// One bead position in the per-warp shared position table.
template <typename T>
struct __align__(16) Pos {
    T x, y, z, w;
};

// threads per CTA of the chunk kernel, and resident CTAs per SM it is compiled for
constexpr int kChunkThreads = 128;
#ifndef SS_CTAS_PER_SM
#define SS_CTAS_PER_SM 6
#endif
#ifndef SS_CTAS_PER_SM_MULTI
#define SS_CTAS_PER_SM_MULTI 5  // for layouts with several beads per lane
#endif
#ifndef SS_CTAS_PER_SM_BATCHED_MULTI
#define SS_CTAS_PER_SM_BATCHED_MULTI 4  // the batched kernel with 3 or more beads per lane (it reads its
#endif                                  // arguments through a pointer; 2 beads per lane fit 5 CTAs/SM)

// shared memory carve-up (bytes), identical on host and device
struct SmemPlan {
    int off_tab, off_pos, off_bq, off_msk, off_log, total;
};

template <typename T>
__host__ __device__ inline SmemPlan smem_plan(int warps, int W, int B, int nlog_chunk) {
    SmemPlan p;
    p.off_tab = 0;
    // per chain NP slot records and one record of zeros that empty gathers read
    int sz = warps * (32 / W) * (W * B + 1) * (int)sizeof(SlotRec<T>);
    p.off_pos = (sz + 15) & ~15;
    sz = p.off_pos + warps * 32 * B * (int)sizeof(Pos<T>);
    p.off_bq = (sz + 15) & ~15;
    // per chain NP + 1 bond vectors: entry i + 1 holds bead i's, entry 0 zeros
    sz = p.off_bq + warps * (32 / W) * (W * B + 1) * (int)sizeof(Pos<T>);
    p.off_msk = (sz + 15) & ~15;
    sz = p.off_msk + warps * 32 * B * (int)sizeof(unsigned long long);
    p.off_log = (sz + 15) & ~15;
    sz = p.off_log + nlog_chunk * 14 * (int)sizeof(double);
    p.total = (sz + 15) & ~15;
    return p;
}

// -------------------------------------------------------------- helpers -----
// 1 + index of the lowest set bit (0 for none) of a 32- or 64-bit slot mask
__device__ __forceinline__ int mask_ffs(unsigned m) { return __ffs((int)m); }
__device__ __forceinline__ int mask_ffs(unsigned long long m) { return __ffsll((long long)m); }
// number of set bits of a slot mask
__device__ __forceinline__ int mask_popc(unsigned m) { return __popc(m); }
__device__ __forceinline__ int mask_popc(unsigned long long m) { return __popcll(m); }

// Sum over the W lanes of a segment; every lane of the segment gets the sum.
template <typename T, int W>
__device__ __forceinline__ T seg_sum(T v) {
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off, W);
    return v;
}

// Sums over the W lanes of a segment of six per-lane values v[0..5]
// (sigma_xy, sigma_xz, sigma_yz and the same components of sigma + sigma^(v))
// by a transpose reduction: the first round splits the two tensors between
// the lane halves, the second the xy/xz pair (yz summed on both sides), the
// third xy-or-xz against yz; butterflies finish.  On return lane ll holds
// the total of value seg6_value(ll).
template <int W>
__device__ __forceinline__ int seg6_value(int ll) {
    const int comp = (ll & (W / 8)) ? 2 : ((ll & (W / 4)) ? 1 : 0);
    return ((ll & (W / 2)) ? 3 : 0) + comp;
}
template <typename T, int W>
__device__ __forceinline__ T seg_reduce6(const T (&v)[8], int ll) {
    T w[3];
    {
        const bool hi = (ll & (W / 2)) != 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const T send = hi ? v[k] : v[k + 3];
            const T keep = hi ? v[k + 3] : v[k];
            w[k] = keep + __shfl_xor_sync(kFull, send, W / 2, W);
        }
    }
    T x, y;
    {
        const bool hi = (ll & (W / 4)) != 0;
        const T send = hi ? w[0] : w[1];
        const T keep = hi ? w[1] : w[0];
        x = keep + __shfl_xor_sync(kFull, send, W / 4, W);
        y = w[2] + __shfl_xor_sync(kFull, w[2], W / 4, W);
    }
    T r;
    {
        const bool hi = (ll & (W / 8)) != 0;
        const T send = hi ? x : y;
        const T keep = hi ? y : x;
        r = keep + __shfl_xor_sync(kFull, send, W / 8, W);
    }
#pragma unroll
    for (int off = W / 16; off > 0; off >>= 1) r += __shfl_xor_sync(kFull, r, off, W);
    return r;
}

// Glauber hop probability of Sec. 3.1 item 2, min{pref (1 - tanh y), 1/2},
// y = chop (d_new - d_old), with 1 - tanh y written 2 / (1 + e^{2y}) and y
// clamped to [-40, 40].
template <typename T>
__device__ __forceinline__ T hop_prob(const StepConst<T>& c, T d_new, T d_old) {
    T y = c.chop * (d_new - d_old);
    y = y > T(40) ? T(40) : (y < T(-40) ? T(-40) : y);
    const T w = c.pref * Mth<T>::div(T(2), T(1) + Mth<T>::exp(T(2) * y));
    return w < T(0.5) ? w : T(0.5);
}

// FP32 form of the same probability: e^{2y} = 2^t with t = c2 (d_new - d_old)
// (c2 = 2 chop log2 e) by ex2.approx, 2/(1+e^{2y}) by rcp.approx.  t is capped
// at 80 log2 e (y <= 40), where the probability is still a normal float; below
// y = -40 the expression already equals its limit 2 pref.
template <typename T>
__device__ __forceinline__ T hop_prob_fast(const StepConst<T>& c, T d_new, T d_old) {
    return hop_prob<T>(c, d_new, d_old);
}
template <>
__device__ __forceinline__ float hop_prob_fast<float>(const StepConst<float>& c, float d_new, float d_old) {
    const float t = fminf(c.c2 * (d_new - d_old), 115.41560327111707f);
    float e, r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(t));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(1.0f + e));
    return fminf(c.two_pref * r, 0.5f);
}
// The same for two moves from one slot (new squared lengths dnew.x, dnew.y),
// with the additions and multiplications packed; each half is rounded as in
// hop_prob_fast<float>.
__device__ __forceinline__ float2 hop_prob_x2(const StepConst<float>& c, float2 dnew, float d_old) {
    const float2 t = __fmul2_rn(pk(c.c2), __fadd2_rn(dnew, pk(-d_old)));
    float ea, eb, ra, rb;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(ea) : "f"(fminf(t.x, 115.41560327111707f)));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(eb) : "f"(fminf(t.y, 115.41560327111707f)));
    const float2 den = __fadd2_rn(pk(1.0f), pk(ea, eb));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(ra) : "f"(den.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rb) : "f"(den.y));
    const float2 w = __fmul2_rn(pk(c.two_pref), pk(ra, rb));
    return make_float2(fminf(w.x, 0.5f), fminf(w.y, 0.5f));
}

// ---------------------------------------------------------- chunk kernel ----
// W lanes per chain, B beads per lane: bead i and slot i of a chain live on
// lane i % W as its sub-slot i / W (NP = W*B >= N beads and slots).
// State of one chain before a step, for the recompute of a differentiation window.
template <typename T, int W, int B>
__device__ __forceinline__ void snapshot_store(const ChunkArgs& a, long long row, int mm, int ll, const T (&R)[B][3],
                                               const T (&A)[B][3], const int (&S)[B], int Z) {
    constexpr int NP = W * B;
    T* sR = static_cast<T*>(a.snapR) + ((size_t)row * a.M + mm) * 3 * NP;
    T* sA = static_cast<T*>(a.snapA) + ((size_t)row * a.M + mm) * 3 * NP;
    int32_t* sS = a.snapS + ((size_t)row * a.M + mm) * NP;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int i = ll + b * W;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            sR[d * NP + i] = R[b][d];
            sA[d * NP + i] = i < Z ? A[b][d] : T(0);
        }
        sS[i] = i < Z ? S[b] : -1;
    }
    if (ll == 0) a.snapZ[(size_t)row * a.M + mm] = Z;
}

// The chains of one CTA: chains cta_first .. cta_first + chains per CTA - 1 of
// the element described by `a` (all warps of the CTA call this together).
// FLOW: the velocity-gradient terms are compiled in (without them the launch
// must have kappa = 0 throughout; recentring is then never needed).
template <typename T, int W, int B, bool WIN, bool FLOW, bool HEUN = false>
__device__ __forceinline__ void run_chains(const ChunkArgs& a, const StepConst<T>& c, const int cta_first,
                                           const T NkT, const long long t0_, const int nsteps_,
                                           const long long log_m0_, const int nlog_) {
    constexpr int SEGS = 32 / W;
    constexpr int NP = W * B;
    constexpr int G8 = W / 8;        // lanes per value group after seg_reduce6
    constexpr bool PK = std::is_same<T, float>::value && (B % 2) == 0;  // packed FP32x2 bead pairs
    // per-bead slot masks: 32 bits cover every slot when NP <= 32
    using Mask = typename std::conditional<(NP <= 32), unsigned, unsigned long long>::type;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int seg = lane / W;
    const int ll = lane % W;
    const int cslot = warp * SEGS + seg;
    const int m = cta_first + cslot;
    const bool live = m < a.M;
    const int mm = live ? m : 0;
    const uint32_t chain_id = a.chain_base + (uint32_t)mm;
    const int N = a.N;
    const int tmode = WIN ? a.tape_mode : 0;  // differentiation windows only
    const unsigned segmask = (W == 32) ? kFull : (((1u << W) - 1u) << (seg * W));
    const unsigned lt = ((1u << lane) - 1u) & segmask;  // lanes of this segment below this one

    extern __shared__ __align__(16) unsigned char smem[];
    const SmemPlan plan = smem_plan<T>(nwarps, W, B, nlog_);
    SlotRec<T>* tab = reinterpret_cast<SlotRec<T>*>(smem + plan.off_tab) + (warp * SEGS + seg) * (NP + 1);
    Pos<T>* pos = reinterpret_cast<Pos<T>*>(smem + plan.off_pos) + (warp * SEGS + seg) * NP;
    // bond vectors Q_i = R_{i+1} - R_i of the current state, one entry up:
    // bq[i + 1] = Q_i, bq[0] = 0 (bead 0 has no left bond)
    Pos<T>* bq = reinterpret_cast<Pos<T>*>(smem + plan.off_bq) + (warp * SEGS + seg) * (NP + 1);
    Mask* msk = reinterpret_cast<Mask*>(smem + plan.off_msk) + (warp * SEGS + seg) * NP;
    double* slog = reinterpret_cast<double*>(smem + plan.off_log);

    for (int i = threadIdx.x; i < nlog_ * 14; i += blockDim.x) slog[i] = 0.0;

    // ---- load state
    const T* Rg = static_cast<const T*>(a.R);
    const T* Ag = static_cast<const T*>(a.A);
    T R[B][3], A[B][3];
    int S[B];
    int Z = live ? a.Z[mm] : 0;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int i = ll + b * W;
        S[b] = (live && i < Z) ? a.S[(size_t)mm * NP + i] : 0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            R[b][d] = (live && i < N) ? Rg[((size_t)mm * 3 + d) * NP + i] : T(0);
            A[b][d] = (live && i < Z) ? Ag[((size_t)mm * 3 + d) * NP + i] : T(0);
        }
        Pos<T> p0;
        p0.x = R[b][0];
        p0.y = R[b][1];
        p0.z = R[b][2];
        p0.w = T(0);
        pos[i] = p0;
    }

    // Values that change only with Z, kept from one change to the next: the
    // creation attempts of substep 3a (slots first = Z .. c_last - 1, each
    // creating with probability p_c(K = c_last - Z) at either end; c_drop: an
    // attempt dropped at the cap, counted on lane 0) and the largest Z of this
    // warp's chains (sub-slots at or above it hold no spring).
    int c_last = Z;
    T c_pc2 = T(0);  // 2 p_c
    int z_w = 0;
    bool c_drop = false;
    auto set_create = [&]() {
        c_drop = Z >= a.zmax && a.create_mode == 1 && ll == 0 && live;
        z_w = (int)__reduce_max_sync(kFull, (unsigned)Z);
        c_last = Z < a.zmax ? ((a.create_mode == 0) ? a.zmax : Z + 1) : Z;
        c_pc2 = T(2) * c.pc[c_last - Z];
    };
    set_create();

    // stress series of this launch (the correlator reads it afterwards)
    T* const ser = static_cast<T*>(a.series);
    const bool corr_on = ser != nullptr;
    const int gq = seg6_value<W>(ll);  // value this lane holds after seg_reduce6
    // one writer per value: the lowest lane of its group (yz is held twice over)
    T* const ser_m = (corr_on && live && (ll % G8) == 0 && !((gq % 3) == 2 && (ll & (W / 4))))
                         ? ser + ((size_t)a.series_row0 * a.M + mm) * 6 + gq
                         : nullptr;
    const size_t ser_step = (size_t)a.M * 6;
    if (nlog_ > 0)
        __syncthreads();  // the CTA's stress-log buffer is zeroed
    else
        __syncwarp();

    // ---- flow schedule and periodic events, as step offsets in this launch
    const int never = 0x7fffffff;
    auto rel = [&](long long t_abs) -> int {
        const long long r = t_abs - t0_;
        return r > (long long)never ? never : (int)r;
    };
    int ki = 0;
    T kap[9];
    bool kap_nz = false;
    int next_from = never;
    if constexpr (FLOW) {
        while (ki + 1 < a.n_kap && t0_ >= a.kap_from[ki + 1]) ++ki;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            kap[i] = T(a.kap[ki * 9 + i]);
            kap_nz |= (kap[i] != T(0));
        }
        next_from = (ki + 1 < a.n_kap) ? rel(a.kap_from[ki + 1]) : never;
    }
    int next_log = a.log_every > 0 ? rel((t0_ / a.log_every + 1) * a.log_every - 1) : never;
    int next_rc = a.recenter_every > 0 ? rel((t0_ / a.recenter_every + 1) * a.recenter_every - 1) : never;
    int log_slot = 0;
    const uint32_t t0lo = (uint32_t)t0_;

    unsigned cnt_up = 0, cnt_dn = 0, cnt_cr = 0, cnt_de = 0, cnt_drop = 0;

    // slot table: the spring vector d_j = R_{S_j} - A_j of every occupied slot
    // j, written at the end of each step for the next step's spring forces; a
    // recentring step rewrites it from the shifted coordinates, as a launch
    // computes it here at its start.  The re-indexing below also uses the
    // table as scratch.  Record NP is zero: an empty slot mask reads it.
    __syncwarp();  // positions of this warp's chains are in the table
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int i = ll + b * W;
        if (i < Z) {
            const Pos<T> ps = pos[S[b]];
            SlotRec<T> rec;
            rec.x = ps.x - A[b][0];
            rec.y = ps.y - A[b][1];
            rec.z = ps.z - A[b][2];
            rec.s = S[b];
            tab[i] = rec;
        }
    }
    PhiloxPre ppre[B];
#pragma unroll
    for (int b = 0; b < B; ++b) ppre[b] = philox_pre((uint32_t)(ll + b * W), kPurposeStep, chain_id, c.rk0, c.rk1);
    if (ll == 0) {
        SlotRec<T> zero;
        zero.x = zero.y = zero.z = T(0);
        zero.s = -1;
        tab[NP] = zero;
        Pos<T> z4;
        z4.x = z4.y = z4.z = z4.w = T(0);
        bq[0] = z4;
    }
    // Bond vectors of the current positions (the position table holds them):
    // the stress of a step and the bond forces of the next step both use
    // them.  The last bead and padding beads read themselves: Q = 0.
    T Q[B][3];
    auto bond_vectors = [&]() {
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int i = ll + b * W;
            const Pos<T> p1 = pos[i < N - 1 ? i + 1 : i];
            Q[b][0] = p1.x - R[b][0];
            Q[b][1] = p1.y - R[b][1];
            Q[b][2] = p1.z - R[b][2];
            Pos<T> qq;
            qq.x = Q[b][0];
            qq.y = Q[b][1];
            qq.z = Q[b][2];
            qq.w = T(0);
            bq[i + 1] = qq;
        }
    };
    bond_vectors();

    // Random numbers of step tt: block (i, tt, STEP, chain) per bead/slot i.
    // They do not depend on the state, so each step draws the next step's
    // at its end, where their integer work interleaves with the stress.
    auto draw = [&](const uint32_t tt, T (&nrm)[B][4], T (&u)[B]) {
        const unsigned long long p_shared = philox_step_shared(tt, kPurposeStep, c.rk0);
        if constexpr (PK) {
#pragma unroll
            for (int b = 0; b < B; b += 2) {
                const uint4 w0 = philox_step(ppre[b], p_shared, c.rk0, c.rk1);
                const uint4 w1 = philox_step(ppre[b + 1], p_shared, c.rk0, c.rk1);
                box_muller_x2(w0.x, w0.y, w1.x, w1.y, nrm[b][0], nrm[b][1], nrm[b + 1][0], nrm[b + 1][1]);
                box_muller_x2(w0.z, w0.w, w1.z, w1.w, nrm[b][2], nrm[b][3], nrm[b + 1][2], nrm[b + 1][3]);
                const float2 uu = __fmul2_rn(pk(float(lo24_bits(w0)), float(lo24_bits(w1))), pk(1.0f / 16777216.0f));
                u[b] = uu.x;
                u[b + 1] = uu.y;
            }
        } else if constexpr (std::is_same<T, float>::value) {
#pragma unroll
            for (int b = 0; b < B; ++b) {  // the bead's two Box-Muller pairs packed
                const uint4 w = philox_step(ppre[b], p_shared, c.rk0, c.rk1);
                box_muller_x2(w.x, w.y, w.z, w.w, nrm[b][0], nrm[b][1], nrm[b][2], nrm[b][3]);
                u[b] = uniform_lo24<T>(w);
            }
        } else {
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const uint4 w = philox_step(ppre[b], p_shared, c.rk0, c.rk1);
                box_muller<T>(w.x, w.y, nrm[b][0], nrm[b][1]);
                box_muller<T>(w.z, w.w, nrm[b][2], nrm[b][3]);
                u[b] = uniform_lo24<T>(w);
            }
        }
    };
    T nrm[B][4], u[B];
    draw(t0lo, nrm, u);
    for (int s = 0; s < nsteps_; ++s) {
        const uint32_t t = t0lo + (uint32_t)s;
        if (FLOW && s >= next_from) {
            while (ki + 1 < a.n_kap && t0_ + s >= a.kap_from[ki + 1]) ++ki;
            kap_nz = false;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                kap[i] = T(a.kap[ki * 9 + i]);
                kap_nz |= (kap[i] != T(0));
            }
            next_from = (ki + 1 < a.n_kap) ? rel(a.kap_from[ki + 1]) : never;
        }
        if (WIN && a.snapR != nullptr && live) {
            const long long sr = (long long)t0_ + s - a.snap_t0;
            if (sr >= 0 && sr <= a.snap_steps) snapshot_store<T, W, B>(a, sr, mm, ll, R, A, S, Z);
        }
        const long long trow = (long long)t0_ + s - a.tape_t0;
        const bool tape_row = WIN && tmode != 0 && live && trow >= 0 && trow < a.tape_rows;
        uint8_t tb[B];
#pragma unroll
        for (int b = 0; b < B; ++b)
            tb[b] = (tmode == 2 && tape_row) ? a.tape[((size_t)trow * a.M + mm) * NP + ll + b * W] : (uint8_t)0;
        // ---- per-bead slot masks for this step's spring forces
#pragma unroll
        for (int b = 0; b < B; ++b) msk[ll + b * W] = Mask(0);
        __syncwarp();
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int i = ll + b * W;
            if (i < Z) atomicOr(&msk[S[b]], Mask(1) << i);
        }

        // ---- substep 1: forces at time t, Euler-Maruyama, anchor advection.
        // Forces on positions Ro (this lane's beads; the other beads from the
        // position table) with the spring vectors of the slot table: bonds
        // k_b (R_{i-1} + R_{i+1} - 2 R_i), springs -k_s sum_{j: S_j = i} d_j.
        // With bonds_from_q the bond forces come from the bond vectors of the
        // state (this lane's Q and the left neighbour's from the table):
        // k_b (Q_i - Q_{i-1}), the same terms as from positions.
        auto forces = [&](T (&Fo)[B][3], const T (&Ro)[B][3], const bool bonds_from_q) {
            if (bonds_from_q) {
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    const Pos<T> qm = bq[ll + b * W];  // Q_{i-1} (0 for bead 0)
                    const T Qm[3] = {qm.x, qm.y, qm.z};
#pragma unroll
                    for (int d = 0; d < 3; ++d) Fo[b][d] = c.k_b * Q[b][d] - c.k_b * Qm[d];
                }
            } else {
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    const int i = ll + b * W;
                    const Pos<T> pl = pos[i > 0 ? i - 1 : 0];
                    const Pos<T> pr = pos[i < N - 1 ? i + 1 : i];
                    const T Rl[3] = {pl.x, pl.y, pl.z}, Rr[3] = {pr.x, pr.y, pr.z};
                    // an end bead reads itself for its missing neighbour: that term is 0
#pragma unroll
                    for (int d = 0; d < 3; ++d) Fo[b][d] = c.k_b * (Rl[d] - Ro[b][d]) + c.k_b * (Rr[d] - Ro[b][d]);
                }
            }
            __syncwarp();
            bool more = false;
            Mask mrest[B];
#pragma unroll
            for (int b = 0; b < B; ++b) {
                // springs on this bead: -k_s sum_j d_j, slots in ascending order
                // (an empty mask reads the zero record at NP)
                const Mask m0 = msk[ll + b * W];
                const Mask m1 = m0 & (m0 - Mask(1));
                const int j0 = m0 ? mask_ffs(m0) - 1 : NP;
                const int j1 = m1 ? mask_ffs(m1) - 1 : NP;
                const SlotRec<T> r0 = tab[j0], r1 = tab[j1];
                const Mask mb = m1 & (m1 - Mask(1));
                mrest[b] = mb;
                more |= mb != Mask(0);
                Fo[b][0] -= c.k_s * (r0.x + r1.x);
                Fo[b][1] -= c.k_s * (r0.y + r1.y);
                Fo[b][2] -= c.k_s * (r0.z + r1.z);
            }
            if (__any_sync(kFull, more)) {  // a third spring on one bead: rare
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    // the first two slots were added already; add the rest in order
                    Mask mb = mrest[b];
                    T sx = T(0), sy = T(0), sz = T(0);
                    while (mb) {
                        const SlotRec<T> r = tab[mask_ffs(mb) - 1];
                        mb &= mb - Mask(1);
                        sx += r.x;
                        sy += r.y;
                        sz += r.z;
                    }
                    Fo[b][0] -= c.k_s * sx;
                    Fo[b][1] -= c.k_s * sy;
                    Fo[b][2] -= c.k_s * sz;
                }
            }
        };
        T F[B][3];
        forces(F, R, true);
        // Padding beads (i >= N) are stepped like the others: their bond
        // vectors are zero, they exert no force, carry no spring, enter no
        // stress and are never stored.
        T Rn[B][3];
        [[maybe_unused]] T A0[B][3];
        if constexpr (HEUN) {
#pragma unroll
            for (int b = 0; b < B; ++b)
#pragma unroll
                for (int d = 0; d < 3; ++d) A0[b][d] = A[b][d];
        }
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int i = ll + b * W;
            if (kap_nz) {
                if constexpr (PK) {
                    // beads b and b + 1 together; the same operations as the FP32 form below
                    if ((b & 1) == 0) {
                        const float2 r0 = pk(R[b][0], R[b + 1][0]), r1 = pk(R[b][1], R[b + 1][1]),
                                     r2 = pk(R[b][2], R[b + 1][2]);
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            const float2 flow = __ffma2_rn(pk(kap[3 * d + 2]), r2,
                                                           __ffma2_rn(pk(kap[3 * d + 1]), r1,
                                                                      __fmul2_rn(pk(kap[3 * d]), r0)));
                            const float2 e = __ffma2_rn(
                                pk(c.amp), pk(nrm[b][d], nrm[b + 1][d]),
                                __ffma2_rn(pk(c.dt), flow,
                                           __ffma2_rn(pk(c.mob), pk(F[b][d], F[b + 1][d]), pk(R[b][d], R[b + 1][d]))));
                            Rn[b][d] = e.x;
                            Rn[b + 1][d] = e.y;
                        }
                    }
                } else if constexpr (std::is_same<T, float>::value) {
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const float flow = __fmaf_rn(kap[3 * d + 2], R[b][2],
                                                     __fmaf_rn(kap[3 * d + 1], R[b][1], __fmul_rn(kap[3 * d], R[b][0])));
                        Rn[b][d] = __fmaf_rn(c.amp, nrm[b][d], __fmaf_rn(c.dt, flow, __fmaf_rn(c.mob, F[b][d], R[b][d])));
                    }
                } else {
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const T flow = kap[3 * d] * R[b][0] + kap[3 * d + 1] * R[b][1] + kap[3 * d + 2] * R[b][2];
                        Rn[b][d] = R[b][d] + c.mob * F[b][d] + c.dt * flow + c.amp * nrm[b][d];
                    }
                }
            } else if constexpr (PK) {
                if ((b & 1) == 0) {  // beads b and b + 1 together
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const float2 e = __ffma2_rn(pk(c.amp), pk(nrm[b][d], nrm[b + 1][d]),
                                                    __ffma2_rn(pk(c.mob), pk(F[b][d], F[b + 1][d]),
                                                               pk(R[b][d], R[b + 1][d])));
                        Rn[b][d] = e.x;
                        Rn[b + 1][d] = e.y;
                    }
                }
            } else {
#pragma unroll
                for (int d = 0; d < 3; ++d) Rn[b][d] = R[b][d] + c.mob * F[b][d] + c.amp * nrm[b][d];
            }
            if (kap_nz && i < Z) {
                T An[3];
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    An[d] = A[b][d] + c.dt * (kap[3 * d] * A[b][0] + kap[3 * d + 1] * A[b][1] + kap[3 * d + 2] * A[b][2]);
#pragma unroll
                for (int d = 0; d < 3; ++d) A[b][d] = An[d];
            }
        }
        if constexpr (HEUN && !FLOW) {
            // Stochastic Heun corrector without a velocity gradient: the
            // anchors stay where they are, so the springs' force at the
            // predicted positions is the step's spring force less
            // k_s n_i (Rn_i - R_i), n_i the number of springs on bead i (the
            // same sum, reordered); only the bond forces are recomputed.
#pragma unroll
            for (int b = 0; b < B; ++b) {
                Pos<T> pn;
                pn.x = Rn[b][0];
                pn.y = Rn[b][1];
                pn.z = Rn[b][2];
                pn.w = T(0);
                pos[ll + b * W] = pn;
            }
            __syncwarp();
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int i = ll + b * W;
                const Pos<T> pl = pos[i > 0 ? i - 1 : 0];
                const Pos<T> pr = pos[i < N - 1 ? i + 1 : i];
                const Pos<T> qm = bq[i];  // Q_{i-1} of the step's start
                const T nsp = T(mask_popc(msk[i]));
                const T Rl[3] = {pl.x, pl.y, pl.z}, Rr[3] = {pr.x, pr.y, pr.z}, Qm[3] = {qm.x, qm.y, qm.z};
                T F2[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const T fb1 = c.k_b * Q[b][d] - c.k_b * Qm[d];  // the bond part of F
                    F2[d] = c.k_b * (Rl[d] - Rn[b][d]) + c.k_b * (Rr[d] - Rn[b][d]) + (F[b][d] - fb1) -
                            c.k_s * nsp * (Rn[b][d] - R[b][d]);
                }
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    Rn[b][d] = R[b][d] + c.hmob * (F[b][d] + F2[d]) + c.amp * nrm[b][d];
            }
        } else if constexpr (HEUN) {
            // Stochastic Heun corrector (the second-order stochastic Runge-Kutta
            // step for additive noise): the Euler state above is the predictor;
            // the drift is averaged between the start and the predicted state
            // (predicted anchors A under a flow), with the springs and the
            // noise of this step.
            __syncwarp();
#pragma unroll
            for (int b = 0; b < B; ++b) {
                Pos<T> pn;
                pn.x = Rn[b][0];
                pn.y = Rn[b][1];
                pn.z = Rn[b][2];
                pn.w = T(0);
                pos[ll + b * W] = pn;
            }
            __syncwarp();
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int i = ll + b * W;
                if (i < Z) {
                    const Pos<T> ps = pos[S[b]];
                    SlotRec<T> rec;
                    rec.x = ps.x - A[b][0];
                    rec.y = ps.y - A[b][1];
                    rec.z = ps.z - A[b][2];
                    rec.s = S[b];
                    tab[i] = rec;
                }
            }
            __syncwarp();
            T F2[B][3];
            forces(F2, Rn, false);
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int i = ll + b * W;
                T fl[3] = {T(0), T(0), T(0)};
                if (kap_nz) {
#pragma unroll
                    for (int d = 0; d < 3; ++d)
                        fl[d] = (kap[3 * d] * R[b][0] + kap[3 * d + 1] * R[b][1] + kap[3 * d + 2] * R[b][2]) +
                                (kap[3 * d] * Rn[b][0] + kap[3 * d + 1] * Rn[b][1] + kap[3 * d + 2] * Rn[b][2]);
                }
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    Rn[b][d] = R[b][d] + c.hmob * (F[b][d] + F2[b][d]) + c.hdt * fl[d] + c.amp * nrm[b][d];
                if (kap_nz && i < Z) {
                    T An[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d)
                        An[d] = A0[b][d] + c.hdt * ((kap[3 * d] * A0[b][0] + kap[3 * d + 1] * A0[b][1] +
                                                     kap[3 * d + 2] * A0[b][2]) +
                                                    (kap[3 * d] * A[b][0] + kap[3 * d + 1] * A[b][1] +
                                                     kap[3 * d + 2] * A[b][2]));
#pragma unroll
                    for (int d = 0; d < 3; ++d) A[b][d] = An[d];
                }
            }
        }
        // the Heun corrector above read other lanes' positions, so they are
        // overwritten only after a barrier; in the Euler step the last reads
        // of the position table lie behind the barriers of the slot masks and
        // of the forces already
        if constexpr (HEUN) __syncwarp();
#pragma unroll
        for (int b = 0; b < B; ++b) {
            Pos<T> pn;
            pn.x = Rn[b][0];
            pn.y = Rn[b][1];
            pn.z = Rn[b][2];
            pn.w = T(0);
            pos[ll + b * W] = pn;
        }
        __syncwarp();

        // ---- substep 2: hops on the new positions, one uniform per spring;
        // sub-slots above every chain's Z in this warp are skipped
        const int zw = z_w;
#pragma unroll
        for (int b = 0; b < B; ++b) {
            if (b * W >= zw) break;
            const int i = ll + b * W;
            const bool occ = i < Z;
            const int si = S[b];  // a valid bead index in every slot, occupied or not
            const int sm = si > 0 ? si - 1 : 0;
            const int sp = si < N - 1 ? si + 1 : N - 1;
            const Pos<T> q0 = pos[si], qp = pos[sp], qm = pos[sm];
            const T r0[3] = {q0.x - A[b][0], q0.y - A[b][1], q0.z - A[b][2]};
            const T rp[3] = {qp.x - A[b][0], qp.y - A[b][1], qp.z - A[b][2]};
            const T rm[3] = {qm.x - A[b][0], qm.y - A[b][1], qm.z - A[b][2]};
            const T d0 = r0[0] * r0[0] + r0[1] * r0[1] + r0[2] * r0[2];
            T pp, pm;
            if constexpr (std::is_same<T, float>::value) {
                // the moves up and down as one packed pair
                const float2 dpm = __ffma2_rn(pk(rp[2], rm[2]), pk(rp[2], rm[2]),
                                              __ffma2_rn(pk(rp[1], rm[1]), pk(rp[1], rm[1]),
                                                         __fmul2_rn(pk(rp[0], rm[0]), pk(rp[0], rm[0]))));
                const float2 ppm = hop_prob_x2(c, dpm, d0);
                pp = (si < N - 1) ? ppm.x : T(0);
                pm = (si > 0) ? ppm.y : T(0);
            } else {
                const T dp = rp[0] * rp[0] + rp[1] * rp[1] + rp[2] * rp[2];
                const T dm = rm[0] * rm[0] + rm[1] * rm[1] + rm[2] * rm[2];
                pp = (si < N - 1) ? hop_prob_fast<T>(c, dp, d0) : T(0);
                pm = (si > 0) ? hop_prob_fast<T>(c, dm, d0) : T(0);
            }
            bool up = occ && (u[b] < pp);
            bool dn = occ && !up && (u[b] < pp + pm);
            if (tmode == 2) {
                up = occ && (tb[b] & kTapeUp);
                dn = occ && (tb[b] & kTapeDown);
            }
            if (tmode == 1) tb[b] |= (up ? kTapeUp : 0) | (dn ? kTapeDown : 0);
            S[b] = up ? si + 1 : (dn ? si - 1 : S[b]);
            cnt_up += up ? 1u : 0u;
            cnt_dn += dn ? 1u : 0u;
        }

        // ---- substep 3a: creation, K attempts at both ends
        const int Zc = Z;
        const int first = Zc, last = c_last;
        if (c_drop) ++cnt_drop;
        const T pc = T(0.5) * c_pc2;
        // a slot can change only if it may create (u < 2 p_c on an attempt) or
        // sits at an end with a destruction hit: the detailed work below runs
        // only when some slot of the warp can
        bool cand = WIN;
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int i = ll + b * W;
            cand |= ((i >= first) && (i < last) && (u[b] < c_pc2)) ||
                    ((i < Zc) && (S[b] == 0 || S[b] == N - 1) && (nrm[b][3] < c.cd));
        }
        if (__any_sync(kFull, cand)) {
        int end_new[B];
        bool any_new = false;
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int i = ll + b * W;
            const bool att = (i >= first) && (i < last);
            end_new[b] = !att ? -1 : (u[b] < pc ? 0 : (u[b] < c_pc2 ? N - 1 : -1));
            if (tmode == 2) end_new[b] = !att ? -1 : ((tb[b] & kTapeNew0) ? 0 : ((tb[b] & kTapeNewN) ? N - 1 : -1));
            if (tmode == 1) tb[b] |= end_new[b] == 0 ? kTapeNew0 : (end_new[b] > 0 ? kTapeNewN : 0);
            any_new |= end_new[b] >= 0;
        }
        T Anew[B][3];
#pragma unroll
        for (int b = 0; b < B; ++b) Anew[b][0] = Anew[b][1] = Anew[b][2] = T(0);
        const bool some_new = __any_sync(kFull, any_new);
        if (some_new) {
#pragma unroll
            for (int b = 0; b < B; ++b) {
                if (end_new[b] >= 0) {
                    const Pos<T> pe = pos[end_new[b]];
                    const uint4 wc = philox4x32_10_rk((uint32_t)(ll + b * W), t, kPurposeCreate, chain_id, c.rk0,
                                                      c.rk1);
                    T n3[4];
                    box_muller<T>(wc.x, wc.y, n3[0], n3[1]);
                    box_muller<T>(wc.z, wc.w, n3[2], n3[3]);
                    Anew[b][0] = pe.x + c.sa * n3[0];
                    Anew[b][1] = pe.y + c.sa * n3[1];
                    Anew[b][2] = pe.z + c.sa * n3[2];
                    ++cnt_cr;
                }
            }
        }

        // ---- substep 3b: destruction at the ends, then re-indexing
        bool alive_old[B], alive_new[B];
        bool any_change = false;
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int i = ll + b * W;
            const bool hit = nrm[b][3] < c.cd;
            bool kill_old = (i < Zc) && (S[b] == 0 || S[b] == N - 1) && hit;
            bool kill_new = (end_new[b] >= 0) && a.destroy_new && hit;
            if (tmode == 2) {
                kill_old = (i < Zc) && (tb[b] & kTapeKillOld);
                kill_new = (end_new[b] >= 0) && (tb[b] & kTapeKillNew);
            }
            if (tmode == 1) {
                tb[b] |= (kill_old ? kTapeKillOld : 0) | (kill_new ? kTapeKillNew : 0);
                if (tape_row) a.tape[((size_t)trow * a.M + mm) * NP + ll + b * W] = tb[b];
            }
            alive_old[b] = (i < Zc) && !kill_old;
            alive_new[b] = (end_new[b] >= 0) && !kill_new;
            cnt_de += (kill_old ? 1u : 0u) + (kill_new ? 1u : 0u);
            any_change |= kill_old || (end_new[b] >= 0);
        }
        if (__any_sync(kFull, any_change)) {
            // slot order: sub-slot major, then lane; survivors, then new springs at
            // bead 1 in attempt order, then new springs at bead N
            int dest[B];
            int base = 0;
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const unsigned kb = __ballot_sync(kFull, alive_old[b]) & segmask;
                dest[b] = alive_old[b] ? base + __popc(kb & lt) : -1;
                base += __popc(kb);
            }
            if (some_new) {  // new springs in this warp: at bead 1, then at bead N
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const bool e0 = alive_new[b] && end_new[b] == 0;
                const unsigned nb = __ballot_sync(kFull, e0) & segmask;
                if (e0) dest[b] = base + __popc(nb & lt);
                base += __popc(nb);
            }
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const bool eN = alive_new[b] && end_new[b] == N - 1;
                const unsigned nb = __ballot_sync(kFull, eN) & segmask;
                if (eN) dest[b] = base + __popc(nb & lt);
                base += __popc(nb);
            }
            }
            const int Znew = base;
            __syncwarp();
#pragma unroll
            for (int b = 0; b < B; ++b) {
                if (dest[b] >= 0) {
                    SlotRec<T> rec;
                    rec.x = alive_old[b] ? A[b][0] : Anew[b][0];
                    rec.y = alive_old[b] ? A[b][1] : Anew[b][1];
                    rec.z = alive_old[b] ? A[b][2] : Anew[b][2];
                    rec.s = alive_old[b] ? S[b] : end_new[b];
                    tab[dest[b]] = rec;
                }
            }
            __syncwarp();
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int i = ll + b * W;
                if (i < Znew) {
                    const SlotRec<T> rec = tab[i];
                    S[b] = rec.s;
                    A[b][0] = rec.x;
                    A[b][1] = rec.y;
                    A[b][2] = rec.z;
                }
            }
            __syncwarp();
            Z = Znew;
            set_create();
        }
        }  // candidates
        draw(t + 1u, nrm, u);  // the next step's random numbers
#pragma unroll
        for (int b = 0; b < B; ++b)
#pragma unroll
            for (int d = 0; d < 3; ++d) R[b][d] = Rn[b][d];

        // ---- spring vectors of the new state, d_j = R_{S_j} - A_j (0 for an
        // empty slot): next step's spring forces and this step's stress;
        // sub-slots above every chain's Z in this warp hold none
        const int zn = z_w;
        T dd[B][3];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            dd[b][0] = dd[b][1] = dd[b][2] = T(0);
            if (b * W < zn) {
                const int i = ll + b * W;
                const Pos<T> ps = pos[i < Z ? S[b] : 0];
                if (i < Z) {
                    dd[b][0] = ps.x - A[b][0];
                    dd[b][1] = ps.y - A[b][1];
                    dd[b][2] = ps.z - A[b][2];
                    SlotRec<T> rec;
                    rec.x = dd[b][0];
                    rec.y = dd[b][1];
                    rec.z = dd[b][2];
                    rec.s = S[b];
                    tab[i] = rec;
                }
            }
        }

        // ---- bond vectors of the new state: this step's stress, the next
        // step's bond forces
        bond_vectors();

        // ---- stress of the new state (Eq. stress_tensor_single_chain, App. B)
        const bool do_log = (s == next_log);
        if (do_log) next_log += a.log_every;
        const bool do_rc = (s == next_rc) && kap_nz;
        if (s == next_rc) next_rc += a.recenter_every;
        // per-lane parts of the off-diagonal sigma_ab (bonds) and sigma_ab +
        // sigma^(v)_ab (v[0..5]), and with `diag` the bond part of sigma_aa
        auto stress_parts = [&](T (&v)[8], T (&dgp)[3], const bool diag) {
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = T(0);
            dgp[0] = dgp[1] = dgp[2] = T(0);
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const T (&q)[3] = Q[b];  // the last bead's is 0
                T kq0, kq1;
                if constexpr (std::is_same<T, float>::value) {  // (xy, xz) as a packed pair
                    const float2 kq = __fmul2_rn(pk(c.k_b), pk(q[0], q[1]));
                    kq0 = kq.x;
                    kq1 = kq.y;
                    const float2 v01 = __ffma2_rn(pk(kq0), pk(q[1], q[2]), pk(v[0], v[1]));
                    v[0] = v01.x;
                    v[1] = v01.y;
                    v[2] += kq1 * q[2];
                    if (b * W < zn) {  // springs (an empty slot's d is 0)
                        const float2 kd = __fmul2_rn(pk(c.k_s), pk(dd[b][0], dd[b][1]));
                        const float2 v34 = __ffma2_rn(pk(kd.x), pk(dd[b][1], dd[b][2]), pk(v[3], v[4]));
                        v[3] = v34.x;
                        v[4] = v34.y;
                        v[5] += kd.y * dd[b][2];
                    }
                } else {
                    kq0 = c.k_b * q[0];
                    kq1 = c.k_b * q[1];
                    v[0] += kq0 * q[1];
                    v[1] += kq0 * q[2];
                    v[2] += kq1 * q[2];
                    if (b * W < zn) {  // springs (an empty slot's d is 0)
                        const T kd0 = c.k_s * dd[b][0], kd1 = c.k_s * dd[b][1];
                        v[3] += kd0 * dd[b][1];
                        v[4] += kd0 * dd[b][2];
                        v[5] += kd1 * dd[b][2];
                    }
                }
                if (diag) {
                    dgp[0] += kq0 * q[0];
                    dgp[1] += kq1 * q[1];
                    dgp[2] += c.k_b * q[2] * q[2];
                }
            }
            v[3] += v[0];
            v[4] += v[1];
            v[5] += v[2];
        };
        if (corr_on) {  // every step: the correlator's input
            T v[8], dgp[3];
            stress_parts(v, dgp, false);
            const T red = seg_reduce6<T, W>(v, ll);
            if (ser_m != nullptr) ser_m[(size_t)s * ser_step] = red;
        }
        if (do_log) {
            // a log step (warp-uniform, every log_every steps): the stress
            // again with its diagonal, kept out of the every-step path
            T v[8], dgp[3];
            stress_parts(v, dgp, true);
            const T red = seg_reduce6<T, W>(v, ll);
            T sig[3], dg[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                sig[d] = shfl(red, d == 0 ? 0 : (d == 1 ? W / 4 : W / 8), W);
                dg[d] = seg_sum<T, W>(dgp[d]) - NkT;
            }
            const int slot = log_slot++;
            if (live && ll == 0 && slot < nlog_) {
                double* L = slog + slot * 14;
                const double v6[6] = {(double)dg[0], (double)dg[1], (double)dg[2],
                                      (double)sig[0], (double)sig[1], (double)sig[2]};
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    atomicAdd(L + k, v6[k]);
                    atomicAdd(L + 6 + k, v6[k] * v6[k]);
                }
                atomicAdd(L + 12, (double)Z);
                atomicAdd(L + 13, (double)Z * (double)Z);
            }
        }
        if (do_rc) {
            T csum[3] = {T(0), T(0), T(0)};
#pragma unroll
            for (int b = 0; b < B; ++b)
#pragma unroll
                for (int d = 0; d < 3; ++d) csum[d] += (ll + b * W < N) ? R[b][d] : T(0);
            T com[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) com[d] = seg_sum<T, W>(csum[d]) / T(N);
            __syncwarp();
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int i = ll + b * W;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    if (i < N) R[b][d] -= com[d];
                    if (i < Z) A[b][d] -= com[d];
                }
                Pos<T> pn;
                pn.x = R[b][0];
                pn.y = R[b][1];
                pn.z = R[b][2];
                pn.w = T(0);
                pos[i] = pn;
            }
            // the spring and bond vectors from the shifted coordinates, as a
            // launch starting here computes them: results do not depend on
            // where the launches end
            __syncwarp();
            bond_vectors();
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int i = ll + b * W;
                if (i < Z) {
                    const Pos<T> ps = pos[S[b]];
                    SlotRec<T> rec;
                    rec.x = ps.x - A[b][0];
                    rec.y = ps.y - A[b][1];
                    rec.z = ps.z - A[b][2];
                    rec.s = S[b];
                    tab[i] = rec;
                }
            }
        }
        __syncwarp();
    }

    if (WIN && a.snapR != nullptr && live) {
        const long long sr = (long long)t0_ + nsteps_ - a.snap_t0;
        if (sr >= 0 && sr <= a.snap_steps) snapshot_store<T, W, B>(a, sr, mm, ll, R, A, S, Z);
    }

    // ---- store state
    T* Rw = static_cast<T*>(a.R);
    T* Aw = static_cast<T*>(a.A);
    bool bad = false, broken = false;  // non-finite position; broken invariant 0 <= Z <= z_max, 0 <= S < N
    if (live) {
        if (ll == 0) a.Z[mm] = Z;
        broken = Z < 0 || Z > a.zmax;
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int i = ll + b * W;
            a.S[(size_t)mm * NP + i] = (i < Z) ? S[b] : -1;
            broken |= (i < Z) && (S[b] < 0 || S[b] >= N);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (i < N) {
                    Rw[((size_t)mm * 3 + d) * NP + i] = R[b][d];
                    bad |= !Mth<T>::finite(R[b][d]);
                }
                Aw[((size_t)mm * 3 + d) * NP + i] = (i < Z) ? A[b][d] : T(0);
            }
        }
    }
    if (__any_sync(kFull, bad) && lane == 0) {
        atomicOr(a.status, 1);
        atomicAdd(a.counters + 6, 1ull);
    }
    if (__any_sync(kFull, broken) && lane == 0) {
        atomicOr(a.status, 2);
        atomicAdd(a.counters + 7, 1ull);
    }

    // ---- event counters (padding segments beyond the element's chains count nothing)
    {
        unsigned v[5] = {cnt_up, cnt_dn, cnt_cr, cnt_de, cnt_drop};
        if (!live) v[0] = v[1] = v[2] = v[3] = v[4] = 0u;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            unsigned x = v[k];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(kFull, x, off);
            if (lane == 0 && x) atomicAdd(a.counters + k, (unsigned long long)x);
        }
    }

    // ---- stress logs: add this CTA's sums to its group
    if (a.log_every > 0 && nlog_ > 0) {
        __syncthreads();
        const long long first_m = t0_ / a.log_every + 1;  // first log multiple in or after t0+1
        const int slice = cta_first / kSliceChains;
        const int grp = (int)(((long long)slice * a.groups) / a.slices);
        for (int i = threadIdx.x; i < nlog_ * 14; i += blockDim.x) {
            const int slot = i / 14, k = i % 14;
            const long long idx = first_m + slot - log_m0_ - 1;
            const long long step = (first_m + slot) * a.log_every;
            if (step <= t0_ + nsteps_ && idx >= 0 && idx < a.max_logs && slog[i] != 0.0)
                atomicAdd(a.logs + ((size_t)idx * a.groups + grp) * 14 + k, slog[i]);
        }
    }
}

// WIN: the differentiation-window hooks (decision tape, snapshots, stress
// series) are compiled in; the plain kernel carries none of them.  FLOW: the
// velocity-gradient terms are compiled in (launches with kappa = 0 throughout
// may use the instantiation without them).  HEUN: the stochastic Heun
// integrator instead of Euler-Maruyama for substep 1.
template <typename T, int W, int B, bool WIN, bool FLOW, bool HEUN = false>
__global__ void __launch_bounds__(kChunkThreads, B == 1 ? SS_CTAS_PER_SM : (B >= 4 ? 4 : SS_CTAS_PER_SM_MULTI))
    chunk_kernel(const ChunkArgs a, const StepConst<T> c) {
    run_chains<T, W, B, WIN, FLOW, HEUN>(a, c, blockIdx.x * (kChunkThreads / W), c.NkT, a.t0, a.nsteps, a.log_m0,
                                         a.nlog_chunk);
}

// ------------------------------------------------------ batched kernel ------
// Many elements in one persistent launch per lane layout: each CTA takes work
// items (element, first chain of a CTA tile) of its layout class from an
// atomic counter until the list is exhausted, and runs the tile for all steps
// of the launch.  The counter is only ever incremented: no CTA waits for
// another.  Each element's arguments (state pointers, sizes, flow schedule,
// log buffers) live in a device array and are read in place.
struct RunInfo {
    long long t0;     // first step of this launch
    int nsteps;
    long long log_m0;
};

template <typename T, int W, int B>
__global__ void __launch_bounds__(kChunkThreads, B == 1 ? SS_CTAS_PER_SM : (B == 2 ? SS_CTAS_PER_SM_MULTI : SS_CTAS_PER_SM_BATCHED_MULTI))
    batched_kernel(const ChunkArgs* __restrict__ elems, const int2* __restrict__ items, int n_items,
                   unsigned* __restrict__ next_item, const RunInfo info, const StepConst<T> c) {
    __shared__ int item_s;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) item_s = (int)atomicAdd(next_item, 1u);
        __syncthreads();
        const int it = item_s;
        if (it >= n_items) break;
        const int2 wi = items[it];
        const ChunkArgs& a = elems[wi.x];
        const int nlog = a.log_every > 0 ? (int)((info.t0 + info.nsteps) / a.log_every - info.t0 / a.log_every) : 0;
        run_chains<T, W, B, false, true>(a, c, wi.y, T((double)a.N) * c.kT, info.t0, info.nsteps, info.log_m0, nlog);
    }
}

// ----------------------------------------------------- correlator kernels ----
// Multiple-tau lag products of one launch's stress series (Eq.
// relaxation_modulus_tensor_green_kubo_form, App. B).  Level 0 holds the raw
// samples; level l >= 1 the means of two consecutive level-(l-1) samples, i.e.
// of blocks of 2^l raw samples aligned to the absolute sample index.  At level
// l, lag k (0..15 at level 0, 8..15 above) adds x_l(j) y_l(j - k) for every
// sample j completed in this launch, with x = sigma_off (the later value) and
// y = sigma_off (AUTO channel) or (sigma + sigma^(v))_off (TOTAL channel).
//
// One thread per (chain, series row q): q = 0..2 are sigma_off (xy, xz, yz),
// q = 3..5 (sigma + sigma^(v))_off; a warp holds 5 chains x 6 rows, and the
// later value x of row q is row q % 3 of the same chain, taken by a shuffle.
// Samples of a level are [j][M][6] arrays (the chain kernel's series for
// level 0).  hist [M][L][6][16] keeps the newest 16 samples of every level
// and row (oldest first, zero after a reset): the lags reach back into
// earlier launches through a 16-entry register ring; each level's pass
// writes its own history when it ends.  A CTA covers one slice of
// kSliceChains chains and adds its chains' sums of this launch, in chain
// order, to the slice's FP64 sums acc64 [slices][L][3][32] (component,
// channel * 16 + lag).  With TT the rows of sigma + sigma^(v) also take their
// own samples as the later value (channel TT, acc64tt [slices][L][3][16]).
constexpr int kCorrChainsPerWarp = 5;
constexpr int kCorrWarps = (kSliceChains + kCorrChainsPerWarp - 1) / kCorrChainsPerWarp;  // 13
constexpr int kCorrThreads = kCorrWarps * 32;
constexpr int kCorrMaxSteps = 1024;  // samples per launch (the level-sample buffers hold half)

// This slice's FP32 sums of one level (each thread's lags k0..15 of its row),
// folded in chain order into FP64.
// Channel TT of the rows q >= 3, folded the same way into out [3][16].
// Sum of column i over the kSliceChains rows of red (row stride `stride`), in
// chain order, in FP64.  FP32 rows go in blocks of eight: a block is summed in
// FP32 while the rounding error of every addition is kept exactly (TwoSum,
// Knuth) and summed beside it, then the block's sum and error are added in
// FP64.  The result has FP64 accuracy with a quarter of the FP64 conversions
// and additions (the FP64 pipe runs at a small fraction of the FP32 rate).
template <typename T>
__device__ __forceinline__ double slice_column_sum(const T* red, int stride, int i) {
    static_assert(kSliceChains % 8 == 0, "blocks of eight chains");
    double sum = 0.0;
    if constexpr (sizeof(T) == 4) {
        for (int c0 = 0; c0 < kSliceChains; c0 += 8) {
            float s = red[(size_t)c0 * stride + i], e = 0.0f;
#pragma unroll
            for (int c = 1; c < 8; ++c) {
                const float x = red[(size_t)(c0 + c) * stride + i];
                const float t = s + x;
                const float bp = t - s;
                e += (s - (t - bp)) + (x - bp);
                s = t;
            }
            sum += (double)s;
            sum += (double)e;
        }
    } else {
        for (int c = 0; c < kSliceChains; ++c) sum += (double)red[(size_t)c * stride + i];
    }
    return sum;
}

template <typename T>
__device__ __forceinline__ void corr_fold_slice_tt(const T (&acc2)[16], int k0, bool live, int slot, int q,
                                                   double* __restrict__ out, T* red) {
    __syncthreads();  // the first fold has read red
    if (slot < kSliceChains && q >= 3) {
        T* row = red + (size_t)slot * 48 + (q - 3) * kP;
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (k >= k0) row[k] = live ? acc2[k] : T(0);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 48; i += blockDim.x) {
        if (i % kP < k0) continue;
        out[i] += slice_column_sum(red, 48, i);
    }
}

template <typename T>
__device__ __forceinline__ void corr_fold_slice(const T (&acc)[16], int k0, bool live, int slot, int q,
                                                double* __restrict__ out, T* red) {
    // red: [kSliceChains][96] T in shared memory, free once every thread is here
    __syncthreads();
    if (slot < kSliceChains) {
        T* row = red + (size_t)slot * 96 + (q % 3) * kCells + (q / 3) * kP;
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (k >= k0) row[k] = live ? acc[k] : T(0);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 96; i += blockDim.x) {
        const int lag = i % kP;
        if (lag < k0) continue;
        out[i] += slice_column_sum(red, 96, i);
    }
}

// Ring of the newest 16 samples of one row: r[i] holds sample base + i - 16
// when the next sample to enter is sample base (i.e. after a whole number of
// 16-sample blocks).  Products of n new samples, sample j given by get(j) (a
// load), each later value x taken from lane src_lane; emit(j, y) sees every
// sample in order (the pair means of the level above are formed there).  nr
// returns the ring position of the next sample (the number of samples in the
// last partial block).  With TT, acc2 also takes the row's own sample as the
// later value (for the rows of sigma + sigma^(v): channel TT).
template <typename T, int K0, bool TT, typename Get, typename Emit>
__device__ __forceinline__ void corr_ring_products(T (&r)[16], T (&acc)[16], T (&acc2)[16], Get get, Emit emit,
                                                   int n, int src_lane, int& nr) {
    int j = 0;
    for (; j + 16 <= n; j += 16) {
        T yv[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) yv[u] = get(j + u);  // independent loads first
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            emit(j + u, yv[u]);
            const T xv = __shfl_sync(kFull, yv[u], src_lane);
            r[u] = yv[u];
#pragma unroll
            for (int k = K0; k < 16; ++k) acc[k] += xv * r[(u - k) & 15];
            if constexpr (TT) {
#pragma unroll
                for (int k = K0; k < 16; ++k) acc2[k] += yv[u] * r[(u - k) & 15];
            }
        }
    }
    const int rem = n - j;
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        if (u < rem) {
            const T yv = get(j + u);
            emit(j + u, yv);
            const T xv = __shfl_sync(kFull, yv, src_lane);
            r[u] = yv;
#pragma unroll
            for (int k = K0; k < 16; ++k) acc[k] += xv * r[(u - k) & 15];
            if constexpr (TT) {
#pragma unroll
                for (int k = K0; k < 16; ++k) acc2[k] += yv * r[(u - k) & 15];
            }
        }
    }
    nr = rem;
}

// The newest 16 samples in ring order after `nr` samples of a partial block:
// out[i] = r[(nr + i) & 15].
template <typename T>
__device__ __forceinline__ void corr_ring_newest(const T (&r)[16], int nr, T* out) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        T v = r[0];
#pragma unroll
        for (int s2 = 1; s2 < 16; ++s2)
            if (((nr + i) & 15) == s2) v = r[s2];
        out[i] = v;
    }
}

// All levels of one launch in one kernel.  Level l's pass reads the level-l
// samples of this launch (the series rows for level 0, else the samples the
// pass below stored), adds their products, and, as the samples stream by,
// stores the pairwise means that are the level-(l+1) samples into one of the
// ping-pong buffers lev (lev_half elements each).  A mean may pair the newest
// level-l sample of the previous launch (the last entry of the level's
// history) with the first new one.  Every thread reads only rows it wrote
// itself (its chain and series row); the block synchronises only for the
// slice folds.
template <typename T, bool TT>
__global__ void __launch_bounds__(kCorrThreads, (sizeof(T) == 4 && !TT) ? 2 : 1)
    corr_kernel(const T* __restrict__ ser, int ns, long long n0, int M, int L, T* __restrict__ hist,
                T* __restrict__ lev, size_t lev_half, double* __restrict__ acc64, double* __restrict__ acc64tt) {
    __shared__ T red[kSliceChains * 96];
    const int lane = threadIdx.x & 31;
    const int cc = lane / 6, q = lane % 6;
    const int slot = (threadIdx.x >> 5) * kCorrChainsPerWarp + cc;  // chain within the slice
    const int fslot = lane < 30 ? slot : kSliceChains;
    const int m = blockIdx.x * kSliceChains + slot;
    const bool live = lane < 30 && slot < kSliceChains && m < M;
    const int mm = live ? m : 0;
    const int src_lane = min(cc * 6 + q % 3, 31);
    const size_t stride = (size_t)M * 6;
    auto cl_of = [&](int l) { return (int)(((n0 + ns) >> l) - (n0 >> l)); };

    const T* yin = ser;  // level-l samples of this launch
    int cl = ns;
    for (int l = 0; l < L && cl > 0; ++l) {
        const int k0 = l == 0 ? 0 : kP / 2;
        T* h = hist + (((size_t)mm * L + l) * 6 + q) * 16;
        T r[16], acc[16], acc2[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            r[i] = live ? h[i] : T(0);
            acc[i] = T(0);
            acc2[i] = T(0);
        }
        // level-(l+1) sample J is the mean of level-l samples off + 2J and
        // off + 2J + 1 of this launch; sample -1 is the newest before it
        const int cn = l + 1 < L ? cl_of(l + 1) : 0;
        const int off = (int)(2 * (n0 >> (l + 1)) - (n0 >> l));  // -1 or 0
        T* const yout = lev + (size_t)(l & 1) * lev_half;
        T* const orow = yout + (size_t)mm * 6 + q;
        T prev = r[15];
        auto emit = [&](int a, T y) {
            const int J = (a - off - 1) >> 1;
            if (((a - off - 1) & 1) == 0 && J < cn && live) orow[(size_t)J * stride] = T(0.5) * (prev + y);
            prev = y;
        };
        const T* yrow = yin + (size_t)mm * 6 + q;
        int nr = 0;
        if (l == 0)
            corr_ring_products<T, 0, TT>(r, acc, acc2, [&](int j) { return yrow[(size_t)j * stride]; }, emit, cl,
                                         src_lane, nr);
        else
            corr_ring_products<T, kP / 2, TT>(r, acc, acc2, [&](int j) { return yrow[(size_t)j * stride]; }, emit,
                                              cl, src_lane, nr);
        corr_fold_slice(acc, k0, live, fslot, q, acc64 + ((size_t)blockIdx.x * L + l) * 96, red);
        if constexpr (TT) corr_fold_slice_tt(acc2, k0, live, fslot, q, acc64tt + ((size_t)blockIdx.x * L + l) * 48, red);
        if (live) {
            T nh[16];
            corr_ring_newest(r, nr, nh);
#pragma unroll
            for (int i = 0; i < 16; ++i) h[i] = nh[i];
        }
        yin = yout;
        cl = cn;
    }
}

// ------------------------------------------------------- state upload ------
// A caller's state in the host layout (R [M][N][3], A [M][zm][3] double;
// S [M][zm], Z [M] int32), staged on the device as it is, checked and then
// converted to the device layout.  One thread per (chain, bead or slot i).
// bad: bit 1 Z out of 0..zm, 2 S out of 0..N-1, 4 A not finite, 8 R not finite.
__global__ void state_check_kernel(const double* __restrict__ R, const double* __restrict__ A,
                                   const int32_t* __restrict__ S, const int32_t* __restrict__ Z, int M, int N,
                                   int zm, int width, int* __restrict__ bad) {
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long long)M * width) return;
    const int m = (int)(id / width), i = (int)(id % width);
    const int z = Z[m];
    int f = 0;
    if (i == 0 && (z < 0 || z > zm)) f |= 1;
    if (i < N)
        for (int d = 0; d < 3; ++d)
            if (!isfinite(R[((size_t)m * N + i) * 3 + d])) f |= 8;
    if (i < zm && i < z) {
        const int sj = S[(size_t)m * zm + i];
        if (sj < 0 || sj >= N) f |= 2;
        for (int d = 0; d < 3; ++d)
            if (!isfinite(A[((size_t)m * zm + i) * 3 + d])) f |= 4;
    }
    if (f) atomicOr(bad, f);
}

template <typename T>
__global__ void state_convert_kernel(const double* __restrict__ Rh, const double* __restrict__ Ah,
                                     const int32_t* __restrict__ Sh, const int32_t* __restrict__ Zh, int M, int N,
                                     int zm, int NP, T* __restrict__ R, T* __restrict__ A, int32_t* __restrict__ S,
                                     int32_t* __restrict__ Z) {
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long long)M * NP) return;
    const int m = (int)(id / NP), i = (int)(id % NP);
    const int z = Zh[m];
    if (i == 0) Z[m] = z;
    for (int d = 0; d < 3; ++d) {
        R[((size_t)m * 3 + d) * NP + i] = i < N ? T(Rh[((size_t)m * N + i) * 3 + d]) : T(0);
        A[((size_t)m * 3 + d) * NP + i] = i < z ? T(Ah[((size_t)m * zm + i) * 3 + d]) : T(0);
    }
    S[(size_t)m * NP + i] = i < z ? Sh[(size_t)m * zm + i] : -1;
}

// The state in the caller's layout (R [M][N][3], A [M][zm][3] double; S
// [M][zm] int32 with -1 for empty slots, Z [M]) from the device layout, into
// caller-owned device arrays (any may be null).  One thread per (chain, i).
template <typename T>
__global__ void state_export_kernel(const T* __restrict__ R, const T* __restrict__ A, const int32_t* __restrict__ S,
                                    const int32_t* __restrict__ Z, int M, int N, int zm, int NP, double* __restrict__ Ro,
                                    double* __restrict__ Ao, int32_t* __restrict__ So, int32_t* __restrict__ Zo) {
    const int width = N > zm ? N : zm;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long long)M * width) return;
    const int m = (int)(id / width), i = (int)(id % width);
    const int z = Z[m];
    if (i == 0 && Zo) Zo[m] = z;
    if (i < N && Ro)
        for (int d = 0; d < 3; ++d) Ro[((size_t)m * N + i) * 3 + d] = (double)R[((size_t)m * 3 + d) * NP + i];
    if (i < zm) {
        const bool occ = i < z;
        if (So) So[(size_t)m * zm + i] = occ ? S[(size_t)m * NP + i] : -1;
        if (Ao)
            for (int d = 0; d < 3; ++d)
                Ao[((size_t)m * zm + i) * 3 + d] = occ ? (double)A[((size_t)m * 3 + d) * NP + i] : 0.0;
    }
}

// Histogram of the slip-spring numbers Z of M chains: hist[z] += number of
// chains with Z = z, z = 0..nb-1 (nb <= kMaxSlots + 1), bins per CTA in shared
// memory.  A Z outside 0..nb-1 (never produced by the step) is counted in bin
// nb, the overflow bin.
__global__ void zhist_kernel(const int32_t* __restrict__ Z, int M, int nb, unsigned long long* __restrict__ hist) {
    __shared__ unsigned int h[kMaxSlots + 2];
    for (int i = threadIdx.x; i <= nb; i += blockDim.x) h[i] = 0u;
    __syncthreads();
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        const int z = Z[m];
        atomicAdd(&h[(z >= 0 && z < nb) ? z : nb], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= nb; i += blockDim.x)
        if (h[i]) atomicAdd(hist + i, (unsigned long long)h[i]);
}

// Correlator group sums from the slice sums: out[g][l][lag][ch][d] (the layout
// of ss_corr_sums) = sum over the slices of group g, in slice order, of
// acc64[s][l][d * 32 + ch * 16 + lag].  One thread per (g, l, cell).
__global__ void corr_group_kernel(const double* __restrict__ acc64, int slices, int groups, int L,
                                  double* __restrict__ out) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= groups * L * 96) return;
    const int g = id / (L * 96), l = (id / 96) % L, i = id % 96;
    const int d = i / 32, ch = (i % 32) / 16, lag = i % 16;
    // slices of group g: s with floor(s * groups / slices) == g
    const int s0 = (int)(((long long)g * slices + groups - 1) / groups);
    const int s1 = (int)(((long long)(g + 1) * slices + groups - 1) / groups);
    double sum = 0.0;
    for (int sl = s0; sl < s1; ++sl) sum += acc64[((size_t)sl * L + l) * 96 + i];
    out[((((size_t)g * L + l) * 16 + lag) * 2 + ch) * 3 + d] = sum;
}

// ------------------------------------------------------------ init kernel ----
// Equilibrium initial state (Sec. 3.1 sampling): ideal-chain bonds with
// variance kT/k_b per component, Z ~ Poisson(N/N0) by inverse CDF on a 53-bit
// uniform (capped at z_max), S uniform on the beads, anchors Gaussian around
// their bead with variance kT/k_s.  One thread per chain, FP64 arithmetic.
template <typename T, int NP>
__global__ void init_kernel(T* R, T* A, int32_t* S, int32_t* Z, int M, int N, int zmax, double sb,
                            double sa, double lam, uint32_t key0, uint32_t key1, uint32_t chain_base) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const uint32_t cid = chain_base + (uint32_t)m;
    double r[kMaxBeads][3];
    r[0][0] = r[0][1] = r[0][2] = 0.0;
    for (int i = 0; i + 1 < N; ++i) {
        const uint4 w = philox4x32_10((uint32_t)i, 0u, kPurposeInitBond, cid, key0, key1);
        double n[4];
        box_muller<double>(w.x, w.y, n[0], n[1]);
        box_muller<double>(w.z, w.w, n[2], n[3]);
        for (int d = 0; d < 3; ++d) r[i + 1][d] = r[i][d] + sb * n[d];
    }
    for (int i = 0; i < NP; ++i)
        for (int d = 0; d < 3; ++d) R[((size_t)m * 3 + d) * NP + i] = i < N ? T(r[i][d]) : T(0);
    int z = zmax;
    {
        const uint4 w = philox4x32_10(0u, 0u, kPurposeInitZ, cid, key0, key1);
        const double u53 = ((double)(w.x >> 5) * 67108864.0 + (double)(w.y >> 6)) / 9007199254740992.0;
        double pmf = exp(-lam), cdf = pmf;
        for (int k = 0; k < zmax; ++k) {
            if (u53 < cdf) {
                z = k;
                break;
            }
            pmf *= lam / (double)(k + 1);
            cdf += pmf;
        }
    }
    Z[m] = z;
    for (int j = 0; j < NP; ++j) {
        int sj = -1;
        double an[3] = {0.0, 0.0, 0.0};
        if (j < z) {
            const uint4 ws = philox4x32_10((uint32_t)j, 0u, kPurposeInitS, cid, key0, key1);
            sj = (int)(((unsigned long long)ws.x * (unsigned long long)N) >> 32);
            const uint4 wa = philox4x32_10((uint32_t)j, 0u, kPurposeInitA, cid, key0, key1);
            double n[4];
            box_muller<double>(wa.x, wa.y, n[0], n[1]);
            box_muller<double>(wa.z, wa.w, n[2], n[3]);
            for (int d = 0; d < 3; ++d) an[d] = r[sj][d] + sa * n[d];
        }
        S[(size_t)m * NP + j] = sj;
        for (int d = 0; d < 3; ++d) A[((size_t)m * 3 + d) * NP + j] = T(an[d]);
    }
}

}  // namespace ssk
