"""Linear viscoelasticity and its N dependence (Sec. 4.1; GPU, FP32 beads /
FP64 sums).  One equilibrium run per chain length N (the paper's parameters,
G(t) from the TOTAL channel of the multiple-tau correlator), long enough for
G(t) to decay by about three decades, shared by the tests below.

* Plateau modulus: the paper reads G_N ~ 0.1 rho0 kT (so N_e = rho0 kT / G_N
  ~ 10, Eq. entanglement_bead_number_rubber_elasticity_definition) from the
  plateau of G at N = 80; checked as a +-30% band (the paper's printed
  numbers are qualitative).
* Entangled scaling: tau_d ~ (N - 1)^3.48 (1/tau_d = -lim ln G(t)/t) and
  eta0 ~ (N - 1)^3.40 (eta0 = int G); exponents between N = 40 and 80
  within +-0.3.
* Unentangled side: for small N the paper finds tau_d ~ (N - 1)^2 (Rouse)
  and eta0 ~ N - 1; the exponents between N = 4 and 8 within +-0.3 of 2 and
  1, and the crossover of the two eta0 power laws at N_c ~ 14.2 ~ 1.4 N_e,
  checked as a band 10..21 (+-45%).
* G'(w), G''(w) for N = 10, 20, 40, 80 (Eqs. storage_modulus_definition,
  loss_modulus_definition; the paper's Figure of the storage and loss
  moduli): the terminal regime G' ~ w^2, G'' ~ w at w tau_d << 1 and G''/w ->
  eta0 for every N; above the terminal peak of G'' its log-slope flattens
  more the longer the chain (the entanglement plateau): the flattest slope
  in w tau_d = 3 .. 300 decreases from N = 10 to N = 80; it turns negative (a
  G'' minimum) for N = 40 and 80 and stays positive for N = 10 (Rouse-like).
"""
import functools

import numpy as np
import pytest

import synth
from paper_1106_2899_gb300 import SlipSpring, rheology

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

# chains and steps (after 20000 steps of equilibration) per chain length
RUNS = {4: (16384, 20000), 6: (16384, 30000), 8: (16384, 50000), 10: (16384, 100000), 20: (16384, 300000),
        40: (16384, 1500000), 80: (4096, 5000000)}


@functools.lru_cache(maxsize=None)
def equilibrium_G(N):
    M, steps = RUNS[N]
    g = SlipSpring([(M, N)], precision="fp32", seed=N + 1)
    g.set_params(**synth.PAPER, corr_levels=24, groups=32)
    g.run(20000)
    g.reset_observables()
    g.run(steps)
    assert g.status() == 0
    t, G, se = g.correlator("total")
    g.close()
    o = np.argsort(t)
    return t[o], G[o], se[o]


def _resolved(N):
    t, G, se = equilibrium_G(N)
    ok = (se < 0.3 * np.abs(G)) | (t < 1)  # lags resolved to 30%
    return t[ok], G[ok]


def eta0_tau_d(N):
    t, G = _resolved(N)
    eta0 = rheology.zero_shear_viscosity(t, G)
    tr = t[G > 0]
    tau_d = rheology.longest_relaxation_time(t, G, t_min=tr.max() / 10)  # the last resolved decade
    return eta0, tau_d


@pytest.fixture(scope="module", autouse=True)
def _gpu(cuda_ok):
    from paper_1106_2899_gb300 import build
    build.build()
    yield


def test_plateau_modulus_at_N80():
    t, G, se = equilibrium_G(80)
    # the plateau: G where ln G(t) is flattest over a factor 4 in time, 1 <= t <= 1000
    sel = (t >= 1) & (t <= 1000) & (G > 0) & (se < 0.05 * G)
    lt, lg = np.log(t[sel]), np.log(G[sel])
    slopes, vals = [], []
    for j in range(len(lt)):
        k = np.searchsorted(lt, lt[j] + np.log(4.0))
        if k >= len(lt):
            break
        slopes.append(abs((lg[k] - lg[j]) / (lt[k] - lt[j])))
        vals.append(np.exp(0.5 * (lg[j] + lg[k])))
    i = int(np.argmin(slopes))
    GN = vals[i]
    print("\nN=80: plateau G = %.4f rho0 kT (log-slope %.3f); N_e = %.1f" % (GN, slopes[i], 1.0 / GN))
    assert slopes[i] < 0.2  # a plateau region exists
    assert 0.07 <= GN <= 0.13, GN


def test_entangled_scaling_exponents_between_N40_and_N80():
    e40, t40 = eta0_tau_d(40)
    e80, t80 = eta0_tau_d(80)
    r = np.log(79.0 / 39.0)
    a_eta, a_tau = np.log(e80 / e40) / r, np.log(t80 / t40) / r
    print("\neta0 %.4g -> %.4g, tau_d %.4g -> %.4g: exponents eta0 %.2f (paper 3.40), tau_d %.2f (paper 3.48)"
          % (e40, e80, t40, t80, a_eta, a_tau))
    assert abs(a_eta - 3.40) <= 0.3, a_eta
    assert abs(a_tau - 3.48) <= 0.3, a_tau


def test_unentangled_scaling_and_crossover_chain_length():
    Ns = [4, 6, 8, 10, 20, 40, 80]
    e = {N: eta0_tau_d(N) for N in Ns}
    for N in Ns:
        print("N=%d: eta0 %.4g, tau_d %.4g" % (N, e[N][0], e[N][1]))
    # small N: Rouse-like (paper: tau_d ~ (N-1)^2, eta0 ~ N-1 for N <~ 10)
    x = np.log([N - 1.0 for N in (4, 6, 8)])
    a_eta = np.polyfit(x, np.log([e[N][0] for N in (4, 6, 8)]), 1)[0]
    a_tau = np.polyfit(x, np.log([e[N][1] for N in (4, 6, 8)]), 1)[0]
    # crossover: the small-N line eta0 = c (N-1) meets the large-N power law
    # through N = 40 and 80
    c = np.exp(np.mean(np.log([e[N][0] / (N - 1.0) for N in (4, 6, 8)])))
    big = np.polyfit(np.log([39.0, 79.0]), np.log([e[40][0], e[80][0]]), 1)
    Nc = 1.0 + np.exp((big[1] - np.log(c)) / (1.0 - big[0]))
    print("\nsmall-N exponents: eta0 %.2f (paper 1), tau_d %.2f (paper 2); crossover N_c = %.1f (paper 14.2)"
          % (a_eta, a_tau, Nc))
    assert abs(a_eta - 1.0) <= 0.3, a_eta
    assert abs(a_tau - 2.0) <= 0.4, a_tau
    assert 10.0 <= Nc <= 21.0, Nc


def test_storage_and_loss_moduli_N10_to_N80():
    flat = {}
    for N in (10, 20, 40, 80):
        t, G = _resolved(N)
        eta0, tau_d = eta0_tau_d(N)
        w = np.geomspace(1e-3 / tau_d, 10.0, 120)
        Gp, Gpp = rheology.storage_loss_moduli(t, G, w)
        # terminal regime, w tau_d in [0.01, 0.05]
        term = (w * tau_d >= 0.01) & (w * tau_d <= 0.05)
        sp = np.polyfit(np.log(w[term]), np.log(Gp[term]), 1)[0]
        spp = np.polyfit(np.log(w[term]), np.log(Gpp[term]), 1)[0]
        assert abs(sp - 2.0) < 0.25 and abs(spp - 1.0) < 0.15, (N, sp, spp)
        # G''/w -> eta0 at low frequency
        assert abs(Gpp[0] / w[0] / eta0 - 1) < 0.05, (N, Gpp[0] / w[0], eta0)
        # the flattest log-slope of G'' above its terminal peak
        lw, lg = np.log(w), np.log(Gpp)
        slope = np.gradient(lg, lw)
        band = (w * tau_d >= 3) & (w * tau_d <= 300) & (w <= 1.0)
        flat[N] = float(slope[band].min())
        j = int(np.argmin(np.where(band, slope, np.inf)))
        print("N=%d: tau_d %.3g, terminal slopes %.2f %.2f, flattest G'' slope %.3f at w tau_d = %.3g (G' %.3f)"
              % (N, tau_d, sp, spp, flat[N], w[j] * tau_d, Gp[j]))
    assert flat[10] > flat[20] > flat[40] > flat[80], flat
    # entangled chains: G'' has a minimum (its slope turns negative); N = 10 none
    assert flat[80] < 0 and flat[40] < 0 and flat[10] > 0.15, flat
