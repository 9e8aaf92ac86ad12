"""The support calls ss_zhist, ss_get_state_dev and ss_set_state_dev (GPU).

* ss_zhist on the parity workload (256 chains, N = 16, FP64, 1e4 steps, seed 0):
  the histogram counted on the device equals the oracle's Z histogram at the
  same steps (Z is bit-exact in FP64), and the pooled histogram of snapshots
  1000 steps apart agrees with Poisson(N/N0) (Eq.
  slip_spring_number_distribution_modified) by chi^2.
* ss_zhist on the flat-energy chain (coincident frozen beads): the slip-spring
  number follows the exact stationary law of the occupation Markov chain at
  finite dt (tests/flat_chain.py), in FP64 and FP32.
* ss_get_state_dev / ss_set_state_dev: the same arrays as the host calls,
  through torch CUDA tensors and a caller stream; a run restarted from a state
  set through device memory continues exactly as one restarted from host
  memory; invalid states are refused.
"""
import numpy as np
import pytest
from scipy import stats

import oracle
import synth
from flat_chain import flat_chain_matrix, stationary_law
from paper_1106_2899_gb300 import SlipSpring
from paper_1106_2899_gb300._native import SlipSpringError

pytestmark = pytest.mark.gpu


def _poisson_chi2(hist, lam, zm):
    k = np.arange(zm + 1)
    pm = stats.poisson.pmf(k, lam)
    pm[zm] += stats.poisson.sf(zm, lam)  # the z_max cap collects the tail
    exp = pm * hist.sum()
    big = exp >= 5
    obs, ex = hist[big], exp[big]
    if (~big).any():  # lump the sparse bins into one
        obs, ex = np.append(obs, hist[~big].sum()), np.append(ex, exp[~big].sum())
    return stats.chisquare(obs, ex * obs.sum() / ex.sum())


def test_zhist_parity_workload_matches_oracle_and_poisson(cuda_ok):
    w = synth.WORKLOADS["parity"]
    M, N = w["M"], w["N"]
    g = SlipSpring([(M, N)], precision="fp64", seed=w["seed"])
    g.set_params(corr_levels=-1, **synth.PAPER)
    o = oracle.Ensemble(oracle.Params(N=N, **synth.PAPER), seed=w["seed"], M=M)
    g.run(0)
    o.init()
    zm = N
    pooled = np.zeros(zm + 1, dtype=np.int64)
    for k in range(11):
        if k:
            g.run(1000)
            o.run(1000)
        h = g.zhist()
        assert h.shape == (zm + 1,) and h.sum() == M
        want = np.bincount(o.get_state()["Z"], minlength=zm + 1)
        assert np.array_equal(h, want), (k, h, want)
        if k:
            pooled += h
    assert abs((pooled * np.arange(zm + 1)).sum() / pooled.sum() - N / synth.PAPER["N0"]) < 0.2
    chi = _poisson_chi2(pooled, N / synth.PAPER["N0"], zm)
    assert chi.pvalue > 1e-3, (chi, pooled)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_zhist_flat_energy_stationary_law(cuda_ok, precision):
    N, zm, N0, dt, zeta_s = 4, 4, 2.0, 0.02, 0.1
    dtks = dt / zeta_s
    states, T = flat_chain_matrix(N, zm, min(dtks, 0.5), lambda K: min(dtks / (N0 * K), 0.5), min(dtks, 1.0), 0, 0)
    piZ, _ = stationary_law(states, T, zm, N)
    M = 16384
    g = SlipSpring([(M, N)], precision=precision, seed=77)
    g.set_params(N0=N0, dt=dt, zeta_s=zeta_s, zeta=1e30, z_max=zm, corr_levels=-1)
    g.set_state({"R": np.zeros((M, N, 3)), "Z": np.zeros(M, dtype=np.int32),
                 "S": -np.ones((M, zm), dtype=np.int32), "A": np.zeros((M, zm, 3))})
    g.run(400)
    hist = np.zeros(zm + 1, dtype=np.int64)
    for _ in range(8):
        g.run(150)
        hist += g.zhist()
    chi = stats.chisquare(hist, piZ * hist.sum())
    assert chi.pvalue > 1e-4, (hist / hist.sum(), piZ)
    # the finite-dt law is resolved away from Poisson(N/N0) capped at z_max
    pois = _poisson_chi2(hist, N / N0, zm)
    assert pois.pvalue < 1e-6


@pytest.mark.parametrize("precision,N", [("fp64", 16), ("fp32", 32), ("fp32", 80)])
def test_state_dev_calls_match_host_calls(cuda_ok, precision, N):
    import torch

    M, seed = 300, 21
    zm = min(N, 64)
    g = SlipSpring([(M, N)], precision=precision, seed=seed)
    g.set_params(corr_levels=-1)
    g.run(0)
    g.run(57)
    host = g.get_state()
    side = torch.cuda.Stream()
    dev = {"R": torch.full((M, N, 3), np.nan, dtype=torch.float64, device="cuda"),
           "Z": torch.full((M,), -9, dtype=torch.int32, device="cuda"),
           "S": torch.full((M, zm), -9, dtype=torch.int32, device="cuda"),
           "A": torch.full((M, zm, 3), np.nan, dtype=torch.float64, device="cuda")}
    g.get_state_dev(dev["R"], dev["Z"], dev["S"], dev["A"], stream=side.cuda_stream)
    with torch.cuda.stream(side):
        got = {k: v.clone() for k, v in dev.items()}  # ordered after the export on the side stream
    side.synchronize()
    for k in ("R", "Z", "S", "A"):
        assert np.array_equal(got[k].cpu().numpy(), host[k]), k

    # a new state through device memory and through host memory: the same
    # arrays, and the same continuation from the same step
    st = synth.random_state(M, N, zm, seed=4, z_mean=N / 4)
    t = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in st.items()}
    t["Z"] = t["Z"].to(torch.int32)
    t["S"] = t["S"].to(torch.int32)
    torch.cuda.synchronize()
    runs = []
    for via_dev in (True, False):
        if via_dev:
            g.set_state_dev(t["R"], t["Z"], t["S"], t["A"], stream=torch.cuda.current_stream().cuda_stream)
        else:
            g.set_state(st)
        g.step = 57
        a = g.get_state()
        g.run(200)
        runs.append((a, g.get_state()))
    for k in ("R", "Z", "S", "A"):
        assert np.array_equal(runs[0][0][k], runs[1][0][k]), k
        assert np.array_equal(runs[0][1][k], runs[1][1][k]), k

    # invalid states are refused and leave the state untouched
    bad = t["S"].clone()
    bad[0, 0] = N
    t["Z"][0] = max(int(t["Z"][0]), 1)
    before = g.get_state()
    with pytest.raises(SlipSpringError, match="SS_EINVAL"):
        g.set_state_dev(t["R"], t["Z"], bad, t["A"])
    badR = t["R"].clone()
    badR[1, 2, 0] = float("inf")
    with pytest.raises(SlipSpringError, match="SS_EINVAL"):
        g.set_state_dev(badR, t["Z"], t["S"], t["A"])
    after = g.get_state()
    for k in ("R", "Z", "S", "A"):
        assert np.array_equal(before[k], after[k]), k
    g.close()
