"""Exact transition matrix of the slip-spring occupation on a flat-energy chain
(test helper, no library or oracle code).

With all beads coincident and frozen, every hop changes no spring length, so
each hop probability is min(dt kT/zeta_s, 1/2) (Eqs. transition_probability_
s_plus/minus) and the occupation vector (n_0 .. n_{N-1}) is a finite Markov
chain under the substeps of Sec. 3.1: hops, K creation attempts (Eq.
transition_probability_z_plus), destruction at the ends (Eq.
transition_probability_z_minus).  Its stationary law is the finite-dt
counterpart of the Poisson slip-spring number (Eq.
slip_spring_number_distribution_modified).
"""
import itertools
import math

import numpy as np
from scipy import stats


def stationary_law(states, T, zm, N):
    """(pi_Z [zm + 1], mean occupation per site [N]) of the stationary law of T."""
    w, V = np.linalg.eig(T.T)
    pi = np.real(V[:, np.argmin(np.abs(w - 1))])
    pi /= pi.sum()
    piZ = np.zeros(zm + 1)
    occ = np.zeros(N)
    for n, q in zip(states, pi):
        piZ[sum(n)] += q
        occ += q * np.array(n)
    return piZ, occ


def flat_chain_matrix(N, zm, pdt, pc_fn, pdes, create_mode, destroy_new):
    """Exact transition matrix of the occupation vector (n_0..n_{N-1}) when every
    hop has probability pdt (coincident beads): hops, then K creation
    attempts, then destruction at the ends."""
    states = [n for n in itertools.product(range(zm + 1), repeat=N) if sum(n) <= zm]
    index = {n: i for i, n in enumerate(states)}
    T = np.zeros((len(states), len(states)))

    def site_moves(s, cnt):
        # distribution over (up, down, stay) counts of cnt springs at site s
        pu = pdt if s < N - 1 else 0.0
        pd_ = pdt if s > 0 else 0.0
        out = []
        for u in range(cnt + 1):
            for d in range(cnt - u + 1):
                st_ = cnt - u - d
                pr = math.factorial(cnt) / (math.factorial(u) * math.factorial(d) * math.factorial(st_))
                pr *= pu ** u * pd_ ** d * (1 - pu - pd_) ** st_
                if pr > 0:
                    out.append((u, d, pr))
        return out

    for n in states:
        Z = sum(n)
        # hops
        after = {}
        for combo in itertools.product(*[site_moves(s, n[s]) for s in range(N)]):
            occ = [0] * N
            pr = 1.0
            for s, (u, d, q) in enumerate(combo):
                pr *= q
                occ[s] += n[s] - u - d
                if u:
                    occ[s + 1] += u
                if d:
                    occ[s - 1] += d
            after[tuple(occ)] = after.get(tuple(occ), 0.0) + pr
        K = (zm - Z) if create_mode == 0 else (1 if Z < zm else 0)
        pc = pc_fn(K) if K > 0 else 0.0
        for occ, ph in after.items():
            for c0 in range(K + 1):
                for cN in range(K - c0 + 1):
                    pcr = (math.factorial(K) / (math.factorial(c0) * math.factorial(cN)
                                                * math.factorial(K - c0 - cN))
                           * pc ** c0 * pc ** cN * (1 - 2 * pc) ** (K - c0 - cN))
                    if pcr == 0:
                        continue
                    old0, oldN = occ[0], occ[N - 1]
                    el0 = old0 + (c0 if destroy_new else 0)
                    elN = oldN + (cN if destroy_new else 0)
                    for k0 in range(el0 + 1):
                        p0 = stats.binom.pmf(k0, el0, pdes)
                        for kN in range(elN + 1):
                            pN = stats.binom.pmf(kN, elN, pdes)
                            fin = list(occ)
                            fin[0] += c0 - k0
                            fin[N - 1] += cN - kN
                            T[index[n], index[tuple(fin)]] += ph * pcr * p0 * pN
    return states, T
