"""Pins of the oracle's stochastic Heun integrator (CPU only).

Sec. 3.1 names the stochastic Runge-Kutta method (Honeycutt) as the more
accurate alternative to its Euler-Maruyama bead update.  For the additive
noise of the bead equation the second-order scheme is the stochastic Heun
step: predictor R* = R + dt f(R) + a w, corrector R' = R + dt/2 (f(R) + f(R*))
+ a w with the same noise, anchors by the Heun step of their linear flow
equation.  What fixes it:

* Rouse chain (no slip-springs): the scheme is linear, each bond mode is
  mapped by r = 1 - x + x^2/2 with its noise scaled by (1 - x/2), x = k_b dt
  mu_p/zeta, so the stress autocorrelation is exact in closed form at finite
  dt (same algebra as the Euler pin); at dt = 0.03 it differs from the Euler
  closed form by many standard errors.
* The closed form's stationary bias against the continuous Rouse modulus is
  second order in dt (first order for Euler).
* Frozen beads and slip-spring moves under a velocity gradient: beads and
  anchors follow (I + dt kappa + (dt kappa)^2/2)^n exactly.
* Sheared Rouse chain: <sigma_xy> and sigma_xx - sigma_yy from the discrete
  Lyapunov equation of the Heun map.
"""
import numpy as np
import pytest

import oracle
from oracle import CORR_P, Params, corr_lags
from test_oracle_flow import FROZEN, KAPPA, sheared_rouse_stress
from test_oracle_observables import _group_G, _rouse_exact


@pytest.mark.slow
def test_heun_rouse_closed_form_autocorrelation():
    N, M, G, levels, dt = 8, 1024, 32, 9, 0.03
    p = Params(N=N, N0=np.inf, dt=dt, integrator=1)
    ens = oracle.Ensemble(p, seed=2025, M=M, groups=G, levels=levels)
    ens.init()
    ens.run(1000)
    ens.reset_observables()
    ens.run(12000)
    acc, n = ens.corr_sums()
    est = _group_G(acc, n, M, G, levels)
    heun = _rouse_exact(N, 3.0, dt, 1.0, 1.0, levels, scheme="heun")
    euler = _rouse_exact(N, 3.0, dt, 1.0, 1.0, levels, scheme="euler")
    lags = corr_lags(levels)
    checked, far = 0, 0
    for l in range(levels):
        for k in range(CORR_P):
            if lags[l, k] < 0 or lags[l, k] > 150:
                continue
            g = est[:, l, k, 0]
            m, se = g.mean(), g.std(ddof=1) / np.sqrt(G)
            assert abs(m - heun[l, k]) < 4.5 * se + 1e-12, (l, k, m, heun[l, k], se)
            far += abs(m - euler[l, k]) > 6 * se
            checked += 1
    assert checked > 30 and far >= 5


def test_heun_closed_form_bias_is_second_order():
    N = 8
    L = np.diag([1] + [2] * (N - 2) + [1]) - np.eye(N, k=1) - np.eye(N, k=-1)
    mu = np.linalg.eigvalsh(L)[1:]
    cont = np.sum(mu ** 2 * (1.0 / (3.0 * mu)) ** 2) * 9.0  # k_b^2 sum mu^2 V^2, V = kT/(k_b mu)
    ratios = {}
    for scheme in ("euler", "heun"):
        b = [abs(_rouse_exact(N, 3.0, h, 1.0, 1.0, 1, scheme=scheme)[0, 0] / cont - 1) for h in (0.02, 0.01, 0.005)]
        ratios[scheme] = (b[0] / b[1], b[1] / b[2])
    assert all(1.8 < r < 2.2 for r in ratios["euler"]), ratios
    assert all(3.6 < r < 4.4 for r in ratios["heun"]), ratios


def test_heun_frozen_beads_and_anchors_follow_second_order_flow_map():
    p = Params(N=10, zeta=FROZEN, zeta_s=FROZEN, dt=0.01, integrator=1)
    e = oracle.Ensemble(p, seed=8, M=16, levels=4)
    e.init()
    s0 = e.get_state()
    e.set_flow(0, KAPPA)
    n = 120
    e.run(n)
    s1 = e.get_state()
    hk = p.dt * KAPPA
    F = np.linalg.matrix_power(np.eye(3) + hk + 0.5 * hk @ hk, n)
    occ = np.arange(p.zm)[None, :] < s0["Z"][:, None]
    wantR, wantA = s0["R"] @ F.T, s0["A"] @ F.T
    assert np.allclose(s1["R"], wantR, rtol=1e-12, atol=1e-12 * np.abs(wantR).max())
    assert np.allclose(s1["A"][occ], wantA[occ], rtol=1e-12, atol=1e-12 * np.abs(wantA).max())
    # the Euler map is distinguishable at this size
    FE = np.linalg.matrix_power(np.eye(3) + hk, n)
    assert np.abs(s0["R"] @ FE.T - wantR).max() > 1e-3 * np.abs(wantR).max()


@pytest.mark.slow
def test_heun_sheared_rouse_matches_lyapunov():
    N, M, G, gdot, dt = 8, 1024, 32, 0.5, 0.02
    p = Params(N=N, N0=np.inf, dt=dt, integrator=1)
    kap = np.zeros((3, 3))
    kap[0, 1] = gdot
    every, burn, steps = 10, 1000, 10000
    e = oracle.Ensemble(p, seed=32, M=M, groups=G, levels=4, log_every=every, max_logs=steps // every + 1)
    e.init()
    e.set_flow(0, kap)
    e.run(burn)
    e.reset_observables()
    e.run(steps)
    _, L = e.logs()
    per = np.array([(g + 1) * M // G - g * M // G for g in range(G)], dtype=float)
    grp = L[:, :, :6].mean(axis=0) / per[:, None]
    want = sheared_rouse_stress(N, 3.0, dt, 1.0, 1.0, kap, scheme="heun")
    euler = sheared_rouse_stress(N, 3.0, dt, 1.0, 1.0, kap)
    for name, v, w in [("xy", grp[:, 3], want[0, 1]), ("N1", grp[:, 0] - grp[:, 1], want[0, 0] - want[1, 1]),
                       ("xx", grp[:, 0], want[0, 0])]:
        se = v.std(ddof=1) / np.sqrt(G)
        assert abs(v.mean() - w) < 4.0 * se, (name, v.mean(), w, se)
    # the diagonal stress separates the schemes (their O(dt) bias differs)
    v = grp[:, 0]
    assert abs(euler[0, 0] - want[0, 0]) > 6 * v.std(ddof=1) / np.sqrt(G)
