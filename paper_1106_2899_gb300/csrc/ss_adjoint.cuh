// ss_adjoint.cuh -- reverse-mode (adjoint) kernels for pathwise gradients of a
// G(t)-fit loss with respect to the bond stiffness k_b, the slip-spring
// stiffness k_s and the bead friction zeta, with every discrete decision (hop,
// creation, destruction) frozen along the trajectory.
//
// The differentiated map is the continuous part of Sec. 3.1 item 1,
//   R' = R + (dt/zeta) F(R, A; k_b, k_s) + sqrt(2 kT dt / zeta) w,
// F = -k_b L R (path Laplacian L) + k_s sum_{j: S_j = i} (A_j - R_i),
// the anchor of a new spring A = R'_end + sqrt(kT/k_s) n (Sec. 3.1 item 3),
// the re-indexing of the springs (a permutation of their adjoints), and the
// stress samples x = sigma_off, y = (sigma + sigma^(v))_off of every step
// (Eq. stress_tensor_single_chain, App. B) that feed the multiple-tau sums of
// the TOTAL channel of G (Eq. relaxation_modulus_tensor_green_kubo_form).
// Flow is zero in differentiation windows (anchors then move only when
// created).
#pragma once
#include "ss_kernels.cuh"

namespace ssk {

// ------------------------------------------------- correlator adjoint ------
// dL/dx(t) and dL/dy(t) for every chain and component p = 3 m + c from the
// per-(level, lag) weights wgt[l][k] = dL/d(sum of later x origin products).
// Level l pairs block means X_l(j) Y_l(j - k) of 2^l raw samples over complete
// blocks j < n_l = floor(n / 2^l); a block mean depends on each of its samples
// with weight 2^-l, so every sample t of block j = t >> l gets
//   dL/dx += sum_k w_lk Y_l(j - k) / 2^l,   dL/dy += sum_k w_lk X_l(j + k) / 2^l.
// Three passes, each one thread per (block or sample, p) with p fastest:
// block means of every level (pairwise, as the forward correlator forms them),
// the per-block sums cx_l(j), cy_l(j), and the sum over levels per sample.
// Level arrays are [off_l + j][P] with off_l = sum_{l' < l} n_l'.

// level 0 from the series ([t][M][6]: sigma_off, then (sigma + sigma^(v))_off)
template <typename T>
__global__ void adj_level0_kernel(const T* __restrict__ series, long long n, int M, T* __restrict__ X,
                                  T* __restrict__ Y) {
    const long long P = 3ll * M;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * P) return;
    const long long t = i / P;
    const int p = (int)(i % P), m = p / 3, c = p % 3;
    X[i] = series[((size_t)t * M + m) * 6 + c];
    Y[i] = series[((size_t)t * M + m) * 6 + 3 + c];
}

// level l from level l - 1: pairwise means
template <typename T>
__global__ void adj_level_mean_kernel(T* __restrict__ X, T* __restrict__ Y, long long off_prev, long long off,
                                      long long nl, long long P) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nl * P) return;
    const long long j = i / P, p = i % P;
    const long long a = (off_prev + 2 * j) * P + p;
    X[off * P + i] = T(0.5) * (X[a] + X[a + P]);
    Y[off * P + i] = T(0.5) * (Y[a] + Y[a + P]);
}

// cx_l(j), cy_l(j) for one level
template <typename T>
__global__ void adj_block_sums_kernel(const T* __restrict__ X, const T* __restrict__ Y, T* __restrict__ CX,
                                      T* __restrict__ CY, long long off, long long nl, long long P, int l,
                                      const double* __restrict__ wgt) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nl * P) return;
    const long long j = i / P, p = i % P;
    const T inv = T(1.0 / (double)(1ll << l));
    T ax = T(0), ay = T(0);
    for (int k = (l == 0 ? 0 : kP / 2); k < kP; ++k) {
        const T w = T(wgt[l * kP + k]);
        if (w == T(0)) continue;
        if (j - k >= 0) ax += w * Y[(off + j - k) * P + p];
        if (j + k < nl) ay += w * X[(off + j + k) * P + p];
    }
    CX[off * P + i] = ax * inv;
    CY[off * P + i] = ay * inv;
}

// dL/dx(t), dL/dy(t): sum over the levels whose block of t is complete
template <typename T>
__global__ void adj_sample_sums_kernel(const T* __restrict__ CX, const T* __restrict__ CY, long long n, long long P,
                                       int L, T* __restrict__ xbar, T* __restrict__ ybar) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * P) return;
    const long long t = i / P, p = i % P;
    T xb = T(0), yb = T(0);
    long long off = 0;
    for (int l = 0; l < L; ++l) {
        const long long nl = n >> l, j = t >> l;
        if (j >= nl) break;
        xb += CX[(off + j) * P + p];
        yb += CY[(off + j) * P + p];
        off += nl;
    }
    xbar[i] = xb;  // [t][M][3]
    ybar[i] = yb;
}

// ------------------------------------------------------- reverse sweep -----
struct AdjArgs {
    const void* snapR;    // [ns+1][M][3][NP] state before each step of the segment (and after the last)
    const void* snapA;
    const int32_t* snapS;
    const int32_t* snapZ;
    const uint8_t* tape;  // [ns][M][NP] decisions of the segment
    const void* xbar;     // [ns][M][3] dL/dx at the sample taken after each step
    const void* ybar;
    void* Rb;             // [M][3][NP] adjoint of the bead positions (in/out)
    void* Ab;             // [M][3][NP] adjoint of the anchors (in/out)
    double* grad;         // [M][3] accumulated dL/d(k_b, k_s, zeta) per chain
    int M, N, ns;
    long long t0;         // absolute step of the segment's first step
    uint32_t key0, key1, chain_base;
    int destroy_new, create_mode, zmax;
};

template <typename T, int W, int B>
__global__ void __launch_bounds__(kChunkThreads, B == 1 ? SS_CTAS_PER_SM : SS_CTAS_PER_SM_MULTI)
    adjoint_kernel(const AdjArgs a, const StepConst<T> c) {
    constexpr int SEGS = 32 / W;
    constexpr int NP = W * B;
    using Mask = unsigned long long;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int seg = lane / W, ll = lane % W;
    const int cpc = (blockDim.x >> 5) * SEGS;
    const int m = blockIdx.x * cpc + warp * SEGS + seg;
    const bool live = m < a.M;
    const int mm = live ? m : 0;
    const uint32_t chain_id = a.chain_base + (uint32_t)mm;
    const int N = a.N;
    const unsigned segmask = (W == 32) ? kFull : (((1u << W) - 1u) << (seg * W));
    const unsigned lt = ((1u << lane) - 1u) & segmask;

    extern __shared__ __align__(16) unsigned char smem[];
    // per chain: a position table (Pos), a vector table (Pos), a slot table (SlotRec), slot masks
    Pos<T>* pos = reinterpret_cast<Pos<T>*>(smem) + (warp * SEGS + seg) * NP;
    Pos<T>* vec = reinterpret_cast<Pos<T>*>(smem) + (blockDim.x / 32) * 32 * B + (warp * SEGS + seg) * NP;
    SlotRec<T>* tab = reinterpret_cast<SlotRec<T>*>(reinterpret_cast<Pos<T>*>(smem) + 2 * (blockDim.x / 32) * 32 * B) +
                      (warp * SEGS + seg) * NP;
    Mask* msk = reinterpret_cast<Mask*>(reinterpret_cast<SlotRec<T>*>(reinterpret_cast<Pos<T>*>(smem) +
                                                                      2 * (blockDim.x / 32) * 32 * B) +
                                        (blockDim.x / 32) * 32 * B) +
                (warp * SEGS + seg) * NP;

    const T* sR = static_cast<const T*>(a.snapR);
    const T* sA = static_cast<const T*>(a.snapA);
    T Rb[B][3], Ab[B][3];
    T* gRb = static_cast<T*>(a.Rb);
    T* gAb = static_cast<T*>(a.Ab);
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            Rb[b][d] = live ? gRb[((size_t)mm * 3 + d) * NP + ll + b * W] : T(0);
            Ab[b][d] = live ? gAb[((size_t)mm * 3 + d) * NP + ll + b * W] : T(0);
        }
    // gradient sums: per-step parts in T, folded into FP64 every 32 steps
    double gkb = 0.0, gks = 0.0, gz = 0.0;
    T tkb = T(0), tks = T(0), tz = T(0);
    const T mu = c.mob, kb = c.k_b, ks = c.k_s;
    const double zeta = (double)c.dt / (double)c.mob;
    const double inv_zeta = 1.0 / zeta;
    const T half_amp = T(0.5) * c.amp;

    // per-bead slot masks of a state (springs grouped by bead, in slot order)
    auto build_masks = [&](const int (&Sx)[B], int Zx) {
#pragma unroll
        for (int b = 0; b < B; ++b) msk[ll + b * W] = 0ull;
        __syncwarp();
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int i = ll + b * W;
            if (i < Zx) atomicOr(&msk[Sx[b]], 1ull << i);
        }
        __syncwarp();
    };

    PhiloxPre ppre[B];
#pragma unroll
    for (int b = 0; b < B; ++b) ppre[b] = philox_pre((uint32_t)(ll + b * W), kPurposeStep, chain_id, c.rk0, c.rk1);
    for (int t = a.ns - 1; t >= 0; --t) {
        // ------------------------------------------ state after the step
        T Ra[B][3], Aa[B][3];
        int Sa[B];
        const int Za = a.snapZ[(size_t)(t + 1) * a.M + mm];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int i = ll + b * W;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                Ra[b][d] = sR[(((size_t)(t + 1) * a.M + mm) * 3 + d) * NP + i];
                Aa[b][d] = sA[(((size_t)(t + 1) * a.M + mm) * 3 + d) * NP + i];
            }
            Sa[b] = a.snapS[((size_t)(t + 1) * a.M + mm) * NP + i];
        }
        // ---- (1) the stress sample after the step: dL/dx, dL/dy
        {
            const T* xb = static_cast<const T*>(a.xbar) + ((size_t)t * a.M + mm) * 3;
            const T* yb = static_cast<const T*>(a.ybar) + ((size_t)t * a.M + mm) * 3;
            T g[3], h[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                h[d] = live ? yb[d] : T(0);
                g[d] = (live ? xb[d] : T(0)) + h[d];  // sigma enters x and y
            }
            __syncwarp();
#pragma unroll
            for (int b = 0; b < B; ++b) {
                Pos<T> p;
                p.x = Ra[b][0];
                p.y = Ra[b][1];
                p.z = Ra[b][2];
                p.w = T(0);
                pos[ll + b * W] = p;
            }
            __syncwarp();
            // bonds: sigma_ab += k_b q_a q_b, q = R_{i+1} - R_i
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int i = ll + b * W;
                const Pos<T> p1 = pos[i < N - 1 ? i + 1 : i];
                T q[3] = {p1.x - Ra[b][0], p1.y - Ra[b][1], p1.z - Ra[b][2]};
                if (!(i < N - 1)) q[0] = q[1] = q[2] = T(0);
                Pos<T> v;  // d(g . sigma_bond)/dq
                v.x = kb * (g[0] * q[1] + g[1] * q[2]);
                v.y = kb * (g[0] * q[0] + g[2] * q[2]);
                v.z = kb * (g[1] * q[0] + g[2] * q[1]);
                v.w = T(0);
                vec[i] = v;
                tkb += g[0] * q[0] * q[1] + g[1] * q[0] * q[2] + g[2] * q[1] * q[2];
            }
            __syncwarp();
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int i = ll + b * W;
                const Pos<T> vi = vec[i];
                const Pos<T> vm = vec[i > 0 ? i - 1 : 0];
                if (i < N - 1) {
                    Rb[b][0] -= vi.x;
                    Rb[b][1] -= vi.y;
                    Rb[b][2] -= vi.z;
                }
                if (i > 0 && i < N) {
                    Rb[b][0] += vm.x;
                    Rb[b][1] += vm.y;
                    Rb[b][2] += vm.z;
                }
            }
            // springs: sigma^(v)_ab += k_s d_a d_b, d = R_S - A
            build_masks(Sa, Za);
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int i = ll + b * W;
                const Pos<T> ps = pos[i < Za ? Sa[b] : 0];
                T dd[3] = {ps.x - Aa[b][0], ps.y - Aa[b][1], ps.z - Aa[b][2]};
                if (!(i < Za)) dd[0] = dd[1] = dd[2] = T(0);
                const T wx = ks * (h[0] * dd[1] + h[1] * dd[2]);
                const T wy = ks * (h[0] * dd[0] + h[2] * dd[2]);
                const T wz = ks * (h[1] * dd[0] + h[2] * dd[1]);
                Ab[b][0] -= wx;
                Ab[b][1] -= wy;
                Ab[b][2] -= wz;
                SlotRec<T> r;
                r.x = wx;
                r.y = wy;
                r.z = wz;
                r.s = 0;
                tab[i] = r;
                tks += h[0] * dd[0] * dd[1] + h[1] * dd[0] * dd[2] + h[2] * dd[1] * dd[2];
            }
            __syncwarp();
#pragma unroll
            for (int b = 0; b < B; ++b) {
                Mask mb = msk[ll + b * W];
                while (mb) {
                    const SlotRec<T> r = tab[__ffsll((long long)mb) - 1];
                    mb &= mb - 1ull;
                    Rb[b][0] += r.x;
                    Rb[b][1] += r.y;
                    Rb[b][2] += r.z;
                }
            }
            __syncwarp();
        }

        // ------------------------------------------ state before the step
        T R0[B][3], A0[B][3];
        int S0[B];
        const int Z0 = a.snapZ[(size_t)t * a.M + mm];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int i = ll + b * W;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                R0[b][d] = sR[(((size_t)t * a.M + mm) * 3 + d) * NP + i];
                A0[b][d] = sA[(((size_t)t * a.M + mm) * 3 + d) * NP + i];
            }
            S0[b] = a.snapS[((size_t)t * a.M + mm) * NP + i];
        }
        uint8_t tb[B];
#pragma unroll
        for (int b = 0; b < B; ++b) tb[b] = live ? a.tape[((size_t)t * a.M + mm) * NP + ll + b * W] : (uint8_t)0;
        const uint32_t tt = (uint32_t)(a.t0 + t);

        // ---- (2) re-indexing and creation: adjoints of the springs after the
        // step back to the springs present after the hops (slot order of time t)
        {
            const int Zc = Z0;
            int first = Zc, last = Zc;
            if (Zc < a.zmax) last = (a.create_mode == 0) ? a.zmax : Zc + 1;
            bool alive_old[B], alive_new[B];
            int end_new[B];
            bool any = false;
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int i = ll + b * W;
                const bool att = (i >= first) && (i < last);
                end_new[b] = !att ? -1 : ((tb[b] & kTapeNew0) ? 0 : ((tb[b] & kTapeNewN) ? N - 1 : -1));
                alive_old[b] = (i < Zc) && !(tb[b] & kTapeKillOld);
                alive_new[b] = (end_new[b] >= 0) && !(tb[b] & kTapeKillNew);
                any |= (i < Zc && !alive_old[b]) || end_new[b] >= 0;
            }
            if (__any_sync(kFull, any)) {
                int dest[B];
                int base = 0;
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    const unsigned kbm = __ballot_sync(kFull, alive_old[b]) & segmask;
                    dest[b] = alive_old[b] ? base + __popc(kbm & lt) : -1;
                    base += __popc(kbm);
                }
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
                // adjoints of the springs after the step, by slot
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    SlotRec<T> r;
                    r.x = Ab[b][0];
                    r.y = Ab[b][1];
                    r.z = Ab[b][2];
                    r.s = 0;
                    tab[ll + b * W] = r;
                }
                __syncwarp();
                T anew[B][3];
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    const SlotRec<T> r = tab[dest[b] >= 0 ? dest[b] : 0];
                    const bool has = dest[b] >= 0;
                    const T x = has ? r.x : T(0), y = has ? r.y : T(0), z = has ? r.z : T(0);
                    anew[b][0] = alive_new[b] ? x : T(0);
                    anew[b][1] = alive_new[b] ? y : T(0);
                    anew[b][2] = alive_new[b] ? z : T(0);
                    Ab[b][0] = alive_old[b] ? x : T(0);
                    Ab[b][1] = alive_old[b] ? y : T(0);
                    Ab[b][2] = alive_old[b] ? z : T(0);
                }
                __syncwarp();
                // a new spring's anchor R'_end + sqrt(kT/k_s) n: adjoint to the
                // end bead (summed in attempt order) and to k_s
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    SlotRec<T> r;
                    r.x = anew[b][0];
                    r.y = anew[b][1];
                    r.z = anew[b][2];
                    r.s = alive_new[b] ? end_new[b] : -1;
                    tab[ll + b * W] = r;
                    if (alive_new[b]) {
                        const uint4 wc = philox4x32_10_rk((uint32_t)(ll + b * W), tt, kPurposeCreate, chain_id,
                                                          c.rk0, c.rk1);
                        T n3[4];
                        box_muller<T>(wc.x, wc.y, n3[0], n3[1]);
                        box_muller<T>(wc.z, wc.w, n3[2], n3[3]);
                        // d sqrt(kT/k_s) / d k_s = -sqrt(kT/k_s) / (2 k_s)
                        gks += -(double)c.sa / (2.0 * (double)ks) *
                               (double)(anew[b][0] * n3[0] + anew[b][1] * n3[1] + anew[b][2] * n3[2]);
                    }
                }
                __syncwarp();
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    const int i = ll + b * W;
                    if (i == 0 || i == N - 1) {
                        for (int j = 0; j < NP; ++j) {
                            const SlotRec<T> r = tab[j];
                            if (r.s == i) {
                                Rb[b][0] += r.x;
                                Rb[b][1] += r.y;
                                Rb[b][2] += r.z;
                            }
                        }
                    }
                }
                __syncwarp();
            }
        }

        // ---- (3) the Euler step on the state before it (hops do not move beads)
        {
            // R-bar' of all beads, for the Laplacian and the spring terms
#pragma unroll
            for (int b = 0; b < B; ++b) {
                Pos<T> p;
                p.x = Rb[b][0];
                p.y = Rb[b][1];
                p.z = Rb[b][2];
                p.w = T(0);
                vec[ll + b * W] = p;
                Pos<T> q;
                q.x = R0[b][0];
                q.y = R0[b][1];
                q.z = R0[b][2];
                q.w = T(0);
                pos[ll + b * W] = q;
                SlotRec<T> r;
                r.x = A0[b][0];
                r.y = A0[b][1];
                r.z = A0[b][2];
                r.s = 0;
                tab[ll + b * W] = r;
            }
            build_masks(S0, Z0);  // also orders the table writes above
            T Rn[B][3];
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int i = ll + b * W;
                const bool bead = i < N;
                const Pos<T> vl = vec[i > 0 ? i - 1 : 0], vr = vec[i < N - 1 ? i + 1 : i];
                const Pos<T> pl = pos[i > 0 ? i - 1 : 0], pr = pos[i < N - 1 ? i + 1 : i];
                const T rb[3] = {Rb[b][0], Rb[b][1], Rb[b][2]};
                const T bl[3] = {vl.x, vl.y, vl.z}, br[3] = {vr.x, vr.y, vr.z};
                const T xl[3] = {pl.x, pl.y, pl.z}, xr[3] = {pr.x, pr.y, pr.z};
                // springs on this bead
                Mask mb = msk[i];
                const T nsp = T(__popcll(mb));
                T asum[3] = {T(0), T(0), T(0)};
                while (mb) {
                    const SlotRec<T> r = tab[__ffsll((long long)mb) - 1];
                    mb &= mb - 1ull;
                    asum[0] += r.x;
                    asum[1] += r.y;
                    asum[2] += r.z;
                }
                // noise of this bead in this step
                const uint4 w = philox_step(ppre[b], philox_step_shared(tt, kPurposeStep, c.rk0), c.rk0, c.rk1);
                T nrm[4];
                box_muller<T>(w.x, w.y, nrm[0], nrm[1]);
                box_muller<T>(w.z, w.w, nrm[2], nrm[3]);
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    T fbk = T(0), lap = T(0);  // bond force / k_b, Laplacian of the adjoint
                    if (i > 0) {
                        fbk += xl[d] - R0[b][d];
                        lap += bl[d] - rb[d];
                    }
                    if (i < N - 1) {
                        fbk += xr[d] - R0[b][d];
                        lap += br[d] - rb[d];
                    }
                    const T fb = kb * fbk;
                    const T fs = ks * (asum[d] - nsp * R0[b][d]);
                    Rn[b][d] = bead ? rb[d] + mu * (kb * lap - ks * nsp * rb[d]) : T(0);
                    if (bead) {
                        // d/dk_b of mu F_b is mu F_b / k_b; d/dzeta of the update is
                        // -(mu F + amp w / 2) / zeta
                        tkb += mu * rb[d] * fbk;
                        tz += rb[d] * (mu * (fb + fs) + half_amp * nrm[d]);
                    }
                }
            }
            // anchors: A_j enters the force on bead S_j
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int i = ll + b * W;
                if (i < Z0) {
                    const Pos<T> vs = vec[S0[b]];
                    const Pos<T> ps = pos[S0[b]];
                    Ab[b][0] += mu * ks * vs.x;
                    Ab[b][1] += mu * ks * vs.y;
                    Ab[b][2] += mu * ks * vs.z;
                    tks += mu * (vs.x * (A0[b][0] - ps.x) + vs.y * (A0[b][1] - ps.y) + vs.z * (A0[b][2] - ps.z));
                } else {
                    Ab[b][0] = Ab[b][1] = Ab[b][2] = T(0);
                }
            }
#pragma unroll
            for (int b = 0; b < B; ++b)
#pragma unroll
                for (int d = 0; d < 3; ++d) Rb[b][d] = Rn[b][d];
            __syncwarp();
        }
        if ((t & 31) == 0) {
            gkb += (double)tkb;
            gks += (double)tks;
            gz -= (double)tz * inv_zeta;
            tkb = tks = tz = T(0);
        }
    }
    // ---- carry the adjoints to the previous segment, add this chain's gradient
    if (live) {
#pragma unroll
        for (int b = 0; b < B; ++b)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                gRb[((size_t)mm * 3 + d) * NP + ll + b * W] = Rb[b][d];
                gAb[((size_t)mm * 3 + d) * NP + ll + b * W] = Ab[b][d];
            }
    }
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) {
        gkb += __shfl_xor_sync(kFull, gkb, off, W);
        gks += __shfl_xor_sync(kFull, gks, off, W);
        gz += __shfl_xor_sync(kFull, gz, off, W);
    }
    if (live && ll == 0) {
        a.grad[(size_t)mm * 3 + 0] += gkb;
        a.grad[(size_t)mm * 3 + 1] += gks;
        a.grad[(size_t)mm * 3 + 2] += gz;
    }
}

}  // namespace ssk
