"""Pins of the oracle's model layer against what the paper fixes (CPU only).

* Equilibrium initial state (Sec. 3.1 sampling; Eqs. bead_position_distribution,
  slip_spring_number_distribution_modified, bead_index_distribution,
  anchoring_point_distribution): bond variance b^2/3, Z ~ Poisson(N/N0) (chi^2),
  S uniform (chi^2), R_S - A variance Ns b^2/3, <sigma_aa> = -kT
  (Eq. stress_tensor_single_chain_equilibrium_average), <sigma_v> = 0.
* Hop detailed balance (Eqs. transition_probability_s_plus/minus): with beads
  frozen, P(s -> s+1) / P(s+1 -> s) = exp(-dF/kT) exactly at finite dt while
  the 1/2 caps are inactive.
* Brute-force enumeration of one step's discrete moves on a tiny chain
  (hop, K creation attempts, destruction, re-indexing) against frequencies.
* Flat-energy Markov chain: coincident frozen beads make every hop
  probability dt kT/zeta_s, so the slip-spring occupation is a finite Markov
  chain; its exact stationary law is compared with long oracle runs.
* Stress of a hand-built state against the definition's invariants.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from flat_chain import flat_chain_matrix as _flat_chain_matrix
from oracle import Params

FROZEN = 1e30  # bead friction that freezes the beads: drift dt/zeta and noise ~ 1e-16


# --------------------------------------------------------------------- init --
def test_init_equilibrium_statistics():
    p = Params(N=16, N0=4.0)
    M = 6000
    ens = oracle.Ensemble(p, seed=11, M=M)
    ens.init()
    st = ens.get_state()
    R, Z, S, A = st["R"], st["Z"], st["S"], st["A"]
    assert np.all(R[:, 0, :] == 0.0)
    Q = np.diff(R, axis=1).reshape(-1, 3)
    v = Q.var(axis=0)
    assert np.allclose(v, 1 / 3, rtol=4 * np.sqrt(2 / len(Q)) * 1.5)
    # Z ~ Poisson(N/N0) capped at z_max = N
    lam = p.N / p.N0
    kmax = 12
    obs = np.bincount(np.minimum(Z, kmax), minlength=kmax + 1)
    pk = stats.poisson.pmf(np.arange(kmax), lam)
    pk = np.append(pk, 1 - pk.sum())
    chi = stats.chisquare(obs, pk * M)
    assert chi.pvalue > 1e-3
    assert abs(Z.mean() - lam) < 4 * np.sqrt(lam / M)
    # S uniform on the N beads, R_S - A Gaussian with variance Ns/3
    mask = S >= 0
    s = S[mask]
    obs = np.bincount(s, minlength=p.N)
    assert stats.chisquare(obs).pvalue > 1e-3
    m_idx, j_idx = np.nonzero(mask)
    d = R[m_idx, S[mask], :] - A[m_idx, j_idx, :]
    assert np.allclose(d.var(axis=0), p.Ns / 3, rtol=0.05)
    assert np.allclose(d.mean(axis=0), 0, atol=4 * np.sqrt(p.Ns / 3 / len(d)))
    # <sigma_aa> = -kT, <sigma_v> = 0 in equilibrium
    sig = np.zeros((M, 3, 3))
    sigv = np.zeros((M, 3, 3))
    for m in range(0, M, 10):
        sig[m], sigv[m] = oracle.stress(p, {"R": R[m], "Z": Z[m], "S": S[m], "A": A[m]})
    sel = np.arange(0, M, 10)
    diag = sig[sel][:, [0, 1, 2], [0, 1, 2]]
    assert abs(diag.mean() + 1.0) < 4 * diag.std() / np.sqrt(diag.size)
    assert abs(sigv[sel].mean()) < 4 * sigv[sel].std() / np.sqrt(sigv[sel].size)


def test_stress_definition_on_handmade_state():
    p = Params(N=3, N0=4.0, Ns=0.5)
    R = np.array([[0, 0, 0], [1.0, 2.0, 0.0], [1.0, 2.0, 3.0]])
    st = {"R": R, "Z": 1, "S": [2], "A": [[0.0, 0.0, 0.0]]}
    s, sv = oracle.stress(p, st)
    assert np.allclose(s, s.T) and np.allclose(sv, sv.T)
    # trace identity: tr sigma = k_b sum |Q|^2 - 3 N kT, tr sigma_v = k_s sum |d|^2 - 3 Z kT
    assert np.trace(s) == pytest.approx(3.0 * (5.0 + 9.0) - 9.0)
    assert np.trace(sv) == pytest.approx(6.0 * 14.0 - 3.0)
    # a bond along z only contributes to sigma_zz
    assert s[0, 2] == pytest.approx(0.0) and s[1, 2] == pytest.approx(0.0)
    assert s[0, 1] == pytest.approx(3.0 * 2.0)


# -------------------------------------------------------------- detailed balance
def _one_step_batch(p, seed, state, M, chain_offset=0):
    ens = oracle.Ensemble(p, seed=seed, M=M, chain_offset=chain_offset)
    st = {
        "R": np.repeat(state["R"][None], M, axis=0),
        "Z": np.full(M, state["Z"], dtype=np.int32),
        "S": np.repeat(np.asarray(state["S"], dtype=np.int32)[None], M, axis=0),
        "A": np.repeat(np.asarray(state["A"], dtype=np.float64)[None], M, axis=0),
    }
    ens.set_state(st)
    ens.run(1)
    return ens.get_state()


def test_hop_detailed_balance_frozen_beads():
    """P(s->s+1)/P(s+1->s) = exp(-(F(s+1)-F(s))/kT) with F = k_s/2 |R_s - A|^2."""
    N = 8
    p = Params(N=N, N0=np.inf, zeta=FROZEN, zeta_s=0.1, dt=0.01)
    rng = np.random.default_rng(5)
    R = np.cumsum(rng.normal(0, np.sqrt(1 / 3), size=(N, 3)), axis=0)
    A = R[3] + np.array([0.15, -0.1, 0.2])
    k_s = 3.0 / p.Ns
    M = 300000
    out = {}
    for s in (3, 4):
        st = {"R": R, "Z": 1, "S": np.array([s] + [-1] * (N - 1)),
              "A": np.vstack([A, np.zeros((N - 1, 3))])}
        res = _one_step_batch(p, seed=77 + s, state=st, M=M)
        assert np.all(res["Z"] == 1)
        s_new = res["S"][:, 0]
        out[s] = (np.mean(s_new == s + 1), np.mean(s_new == s - 1))
    p_up = out[3][0]
    p_dn = out[4][1]
    F = lambda i: 0.5 * k_s * np.sum((R[i] - A) ** 2)
    ratio_exact = math.exp(-(F(4) - F(3)))
    ratio = p_up / p_dn
    se = ratio * np.sqrt((1 - p_up) / (p_up * M) + (1 - p_dn) / (p_dn * M))
    assert p_up < 0.5 and p_dn < 0.5
    assert abs(ratio - ratio_exact) < 4 * se, (ratio, ratio_exact, se)


# ----------------------------------------------------------- enumeration ----
def _hop_p(p, R, A, s, t, dtks):
    """(1 - tanh y) rate of Eqs. transition_probability_s_plus/minus, capped at 1/2."""
    k_s = 3.0 * p.kT / (p.Ns * p.b ** 2)
    dF = k_s * (np.sum((R[t] - A) ** 2) - np.sum((R[s] - A) ** 2)) / (4 * p.kT)
    return min(dtks * (1 - math.tanh(dF)), 0.5)


def _enumerate_one_step(p, R, S, A):
    """Exact distribution of the re-indexed bead-index tuple after one step from
    (S, A) with frozen beads, following Sec. 3.1 items 2 and 3."""
    N, zm = p.N, p.zm
    dtks = p.dt * p.kT / p.zeta_s
    Z = len(S)
    hop_opts = []
    for j, s in enumerate(S):
        pu = _hop_p(p, R, A[j], s, s + 1, dtks) if s < N - 1 else 0.0
        pdn = _hop_p(p, R, A[j], s, s - 1, dtks) if s > 0 else 0.0
        hop_opts.append([(s + 1, pu), (s - 1, pdn), (s, 1 - pu - pdn)])
    if p.create_mode == 0:
        attempts = list(range(Z, zm)) if Z < zm else []
    else:
        attempts = [Z] if Z < zm else []
    K = len(attempts)
    pc = min(dtks / (p.N0 * K), 0.5) if K > 0 else 0.0
    pdes = min(dtks, 1.0)
    dist = {}
    for hops in itertools.product(*hop_opts):
        ph = np.prod([h[1] for h in hops])
        if ph == 0:
            continue
        s_after = [h[0] for h in hops]
        for cre in itertools.product([0, N - 1, None], repeat=K):
            pcr = np.prod([pc if c is not None else 1 - 2 * pc for c in cre])
            if pcr == 0:
                continue
            elig_old = [j for j in range(Z) if s_after[j] in (0, N - 1)]
            new = [c for c in cre if c is not None]
            elig_new = list(range(len(new))) if p.destroy_new else []
            n_el = len(elig_old) + len(elig_new)
            for kill in itertools.product([False, True], repeat=n_el):
                pk = np.prod([pdes if k else 1 - pdes for k in kill])
                if pk == 0:
                    continue
                kill_old = dict(zip(elig_old, kill[:len(elig_old)]))
                kill_new = dict(zip(elig_new, kill[len(elig_old):]))
                surv = [s_after[j] for j in range(Z) if not kill_old.get(j, False)]
                new_alive = [new[i] for i in range(len(new)) if not kill_new.get(i, False)]
                final = tuple(surv + [c for c in new_alive if c == 0]
                              + [c for c in new_alive if c == N - 1])
                dist[final] = dist.get(final, 0.0) + ph * pcr * pk
    return dist


@pytest.mark.parametrize("create_mode,destroy_new", [(0, 0), (0, 1), (1, 0)])
def test_one_step_enumeration(create_mode, destroy_new):
    N = 4
    p = Params(N=N, z_max=4, N0=0.5, zeta=FROZEN, create_mode=create_mode, destroy_new=destroy_new,
               dt=0.01, zeta_s=0.05)
    rng = np.random.default_rng(3)
    R = np.cumsum(rng.normal(0, 0.25, size=(N, 3)), axis=0)
    S = [1, 3]
    A = np.array([R[1] + [0.1, 0.0, -0.1], R[3] + [-0.2, 0.1, 0.0]])
    exact = _enumerate_one_step(p, R, S, A)
    assert abs(sum(exact.values()) - 1) < 1e-12
    M = 200000
    st = {"R": R, "Z": 2, "S": np.array(S + [-1, -1]), "A": np.vstack([A, np.zeros((2, 3))])}
    res = _one_step_batch(p, seed=1000 + 10 * create_mode + destroy_new, state=st, M=M)
    emp = {}
    for m in range(M):
        key = tuple(int(x) for x in res["S"][m, :res["Z"][m]])
        emp[key] = emp.get(key, 0) + 1
    assert set(emp) <= set(exact), set(emp) - set(exact)
    keys = sorted(exact, key=lambda k: -exact[k])
    big = [k for k in keys if exact[k] * M >= 20]
    small = [k for k in keys if exact[k] * M < 20]
    obs = [emp.get(k, 0) for k in big] + [sum(emp.get(k, 0) for k in small)]
    expct = [exact[k] * M for k in big] + [sum(exact[k] for k in small) * M]
    if expct[-1] == 0:
        obs, expct = obs[:-1], expct[:-1]
    chi = stats.chisquare(obs, np.array(expct) * sum(obs) / sum(expct))
    assert chi.pvalue > 1e-4, (chi, list(zip(big, obs, expct)))


# ------------------------------------------------------- flat-energy chain --
@pytest.mark.parametrize("create_mode,destroy_new", [(0, 0), (1, 1)])
def test_flat_energy_stationary_law(create_mode, destroy_new):
    N, zm = 4, 4
    p = Params(N=N, z_max=zm, N0=2.0, zeta=FROZEN, dt=0.02, zeta_s=0.1,
               create_mode=create_mode, destroy_new=destroy_new)
    dtks = p.dt * p.kT / p.zeta_s
    states, T = _flat_chain_matrix(N, zm, min(dtks, 0.5), lambda K: min(dtks / (p.N0 * K), 0.5),
                                   min(dtks, 1.0), create_mode, destroy_new)
    assert np.allclose(T.sum(axis=1), 1.0)
    w, V = np.linalg.eig(T.T)
    pi = np.real(V[:, np.argmin(np.abs(w - 1))])
    pi /= pi.sum()
    piZ = np.zeros(zm + 1)
    occ = np.zeros(N)
    for n, q in zip(states, pi):
        piZ[sum(n)] += q
        occ += q * np.array(n)
    M = 4000
    ens = oracle.Ensemble(p, seed=42 + create_mode, M=M)
    st = {"R": np.zeros((M, N, 3)), "Z": np.zeros(M, dtype=np.int32),
          "S": -np.ones((M, zm), dtype=np.int32), "A": np.zeros((M, zm, 3))}
    ens.set_state(st)
    ens.run(400)
    hist = np.zeros(zm + 1)
    socc = np.zeros(N)
    snaps = 8
    for _ in range(snaps):
        ens.run(150)
        s = ens.get_state()
        hist += np.bincount(s["Z"], minlength=zm + 1)
        Sv = s["S"][s["S"] >= 0]
        socc += np.bincount(Sv, minlength=N)
    chi = stats.chisquare(hist, piZ * hist.sum())
    assert chi.pvalue > 1e-4, (hist / hist.sum(), piZ)
    assert np.allclose(socc / (M * snaps), occ, atol=4 * np.sqrt(occ.max() / (M * snaps)))
