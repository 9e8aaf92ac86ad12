"""Pins of the oracle's flow terms and of the spring-vector distribution in the
dynamics (CPU only).

The velocity gradient enters the bead update (Eq. langevin_equation_bead_position,
the kappa . R term) and the affine anchor advection (Eq.
dynamic_equation_anchoring_position); the library applies it as a piecewise-
constant schedule.  What the mathematics fixes:

* Frozen beads (zeta -> infinity: the drift dt/zeta and the noise
  sqrt(2 kT dt/zeta) vanish below rounding).  Every bead then follows the
  linear map R <- (I + dt kappa) R, so R_n = (I + dt kappa)^n R_0, for any
  kappa; a transposed kappa or a missing dt gives a different matrix power.
  With slip-springs on and their moves frozen as well (zeta_s -> infinity:
  hop, creation and destruction probabilities all vanish), the anchors follow
  the same map.
* A schedule kappa_1 from step 0, kappa_2 from step s: the state after n steps
  is (I + dt kappa_2)^(n-s) (I + dt kappa_1)^s R_0 for n >= s, and
  (I + dt kappa_1)^n R_0 before -- the switch happens exactly at step s.
* Sheared Rouse chain (slip-springs off, N0 = inf).  The Euler scheme maps the
  bond vectors linearly, Q' = (I - dt k_b/zeta D D^T) Q + dt Q kappa^T + noise,
  so their stationary covariance solves a discrete Lyapunov equation (the
  algebra of the Rouse pin with the shear coupling); <sigma_xy> and
  <sigma_xx - sigma_yy> follow from it exactly at finite dt.
* Spring vectors d = R_S - A in the dynamics (Sec. 2.1, Eq.
  anchoring_point_distribution: d_a has variance N_s b^2/3 = kT/k_s).  With the
  beads frozen, a spring is born at an end with A Gaussian around that bead,
  hops by moves that are exactly reversible with respect to exp(-k_s d^2/2kT)
  at any dt (the capped Glauber ratio, uncapped at these parameters), and dies
  at an end with the same probability whatever A is.  The stationary density
  of springs over (S, A) is then proportional to exp(-k_s |R_S - A|^2/2kT), so
  the spring-averaged d_a^2 equals kT/k_s exactly, for any frozen chain.  The
  anchor spread of new springs (substep 3a) sets it.
"""
import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import Params

FROZEN = 1e60  # friction that freezes beads (zeta) or slip-spring moves (zeta_s)

# a non-symmetric traceless velocity gradient (a transposed kappa differs)
KAPPA = np.array([[0.1, 0.7, -0.2], [0.05, -0.3, 0.4], [0.3, -0.1, 0.2]])
KAPPA2 = np.array([[-0.4, 0.1, 0.3], [-0.6, 0.1, 0.0], [0.2, 0.5, 0.3]])


def _mat_power_apply(F, n, X):
    """X [..][3] row vectors mapped n times by x <- F x."""
    return X @ np.linalg.matrix_power(F, n).T


def test_frozen_beads_follow_linear_flow_map():
    p = Params(N=12, N0=np.inf, zeta=FROZEN, dt=0.01)
    M = 16
    e = oracle.Ensemble(p, seed=5, M=M, levels=4)
    e.init()
    R0 = e.get_state()["R"]
    assert np.all(e.get_state()["Z"] == 0)
    e.set_flow(0, KAPPA)
    F = np.eye(3) + p.dt * KAPPA
    for n in (1, 2, 50, 200):
        e.run(n - (e.step))
        R = e.get_state()["R"]
        want = _mat_power_apply(F, n, R0)
        assert np.allclose(R, want, rtol=1e-12, atol=1e-12 * np.abs(want).max()), n
    # the deformation is large enough that kappa^T or a missing dt cannot pass
    wrong = _mat_power_apply(np.eye(3) + p.dt * KAPPA.T, 200, R0)
    assert np.abs(wrong - want).max() > 1e-2 * np.abs(want).max()


def test_frozen_anchors_follow_linear_flow_map():
    # springs on, all slip-spring moves frozen: Z and S stay, anchors advect
    p = Params(N=12, zeta=FROZEN, zeta_s=FROZEN, dt=0.01)
    M = 32
    e = oracle.Ensemble(p, seed=6, M=M, levels=4)
    e.init()
    s0 = e.get_state()
    assert s0["Z"].sum() > 50
    e.set_flow(0, KAPPA)
    F = np.eye(3) + p.dt * KAPPA
    n = 150
    e.run(n)
    s1 = e.get_state()
    assert np.array_equal(s1["Z"], s0["Z"]) and np.array_equal(s1["S"], s0["S"])
    c = e.counters()
    assert c["hops_up"] + c["hops_down"] + c["created"] + c["destroyed"] == 0
    occ = np.arange(p.zm)[None, :] < s0["Z"][:, None]
    wantA = _mat_power_apply(F, n, s0["A"])
    scale = np.abs(wantA[occ]).max()
    assert np.allclose(s1["A"][occ], wantA[occ], rtol=1e-12, atol=1e-12 * scale)
    wantR = _mat_power_apply(F, n, s0["R"])
    assert np.allclose(s1["R"], wantR, rtol=1e-12, atol=1e-12 * np.abs(wantR).max())


def test_flow_schedule_switches_exactly_at_from_step():
    p = Params(N=10, zeta=FROZEN, zeta_s=FROZEN, dt=0.01)
    M, s1, s2 = 8, 7, 12
    e = oracle.Ensemble(p, seed=7, M=M, levels=4)
    e.init()
    st0 = e.get_state()
    e.set_flow(0, KAPPA)
    e.set_flow(s1, KAPPA2)
    e.set_flow(s2, np.zeros((3, 3)))
    F1, F2 = np.eye(3) + p.dt * KAPPA, np.eye(3) + p.dt * KAPPA2
    occ = np.arange(p.zm)[None, :] < st0["Z"][:, None]
    for n in range(1, 18):
        e.run(1)
        st = e.get_state()
        n1 = min(n, s1)
        n2 = min(max(n - s1, 0), s2 - s1)
        Fn = np.linalg.matrix_power(F2, n2) @ np.linalg.matrix_power(F1, n1)
        wantR = st0["R"] @ Fn.T
        wantA = st0["A"] @ Fn.T
        assert np.allclose(st["R"], wantR, rtol=1e-13, atol=1e-13 * np.abs(wantR).max()), n
        assert np.allclose(st["A"][occ], wantA[occ], rtol=1e-13, atol=1e-13 * np.abs(wantA).max()), n


def sheared_rouse_stress(N, k_b, dt, zeta, kT, kappa, scheme="euler"):
    """Stationary <sigma> (3x3, per chain, kT units) of the Euler scheme for a
    Rouse chain (no slip-springs) under a constant velocity gradient: the bond
    vectors Q [N-1][3] obey Q' = Mq Q + dt Q kappa^T + D W sqrt(2 kT dt/zeta),
    Mq = I - (dt k_b/zeta) D D^T, so vec(Q) (columns x, y, z) has the transition
    matrix I_3 (x) Mq + dt kappa (x) I and noise covariance (2 kT dt/zeta)
    I_3 (x) D D^T; its stationary covariance C solves C = T C T^T + Sigma."""
    n = N - 1
    D = np.zeros((n, N))
    for i in range(n):
        D[i, i], D[i, i + 1] = -1.0, 1.0
    DDt = D @ D.T
    Mq = np.eye(n) - (dt * k_b / zeta) * DDt
    T = np.kron(np.eye(3), Mq) + dt * np.kron(kappa, np.eye(n))
    Sig = (2.0 * kT * dt / zeta) * np.kron(np.eye(3), DDt)
    if scheme == "heun":
        # stochastic Heun: q' = (I + h Dr + h^2 Dr^2/2) q + (I + h Dr/2) xi with
        # the drift operator Dr = (T - I)/h
        hD = T - np.eye(3 * n)
        B = np.eye(3 * n) + 0.5 * hD
        T = np.eye(3 * n) + hD + 0.5 * hD @ hD
        Sig = B @ Sig @ B.T
    C = scipy.linalg.solve_discrete_lyapunov(T, Sig)
    sig = np.zeros((3, 3))
    for a in range(3):
        for b in range(3):
            sig[a, b] = k_b * np.trace(C[a * n:(a + 1) * n, b * n:(b + 1) * n])
    return sig - N * kT * np.eye(3)


def test_sheared_rouse_lyapunov_helper_reduces_to_equilibrium():
    # kappa = 0: <Q_a^2> per bond is the discrete Rouse variance; the stress
    # is isotropic and equals the sum of (1/3)/(1 - 1.5 mu_p dt) - N kT
    N, dt = 8, 0.01
    sig = sheared_rouse_stress(N, 3.0, dt, 1.0, 1.0, np.zeros((3, 3)))
    L = np.diag([1.0] + [2.0] * (N - 2) + [1.0]) - np.eye(N, k=1) - np.eye(N, k=-1)
    mu = np.linalg.eigvalsh(L)[1:]
    want = 3.0 * np.sum((1.0 / 3.0) / (1.0 - 1.5 * mu * dt)) - N
    assert np.allclose(np.diag(sig), want, rtol=1e-10)
    assert np.allclose(sig - np.diag(np.diag(sig)), 0.0, atol=1e-10)


@pytest.mark.slow
def test_sheared_rouse_steady_stress_matches_lyapunov():
    N, M, G, gdot = 8, 1024, 32, 0.5
    p = Params(N=N, N0=np.inf, dt=0.01)
    kap = np.zeros((3, 3))
    kap[0, 1] = gdot
    every, burn, steps = 10, 2000, 20000
    e = oracle.Ensemble(p, seed=31, M=M, groups=G, levels=4, log_every=every, max_logs=steps // every + 1)
    e.init()
    e.set_flow(0, kap)
    e.run(burn)
    e.reset_observables()
    e.run(steps)
    _, L = e.logs()  # [n][G][14]: sums of xx, yy, zz, xy, xz, yz over each group's chains
    per = np.array([(g + 1) * M // G - g * M // G for g in range(G)], dtype=float)
    grp = L[:, :, :6].mean(axis=0) / per[:, None]  # time-averaged chain means per group
    want = sheared_rouse_stress(N, 3.0, p.dt, 1.0, 1.0, kap)
    for name, v, w in [("xy", grp[:, 3], want[0, 1]), ("N1", grp[:, 0] - grp[:, 1], want[0, 0] - want[1, 1]),
                       ("yz", grp[:, 5], want[1, 2])]:
        se = v.std(ddof=1) / np.sqrt(G)
        assert abs(v.mean() - w) < 4.0 * se + 1e-12, (name, v.mean(), w, se)
    # the shear response is resolved: many standard errors from zero
    assert abs(want[0, 1]) > 20 * grp[:, 3].std(ddof=1) / np.sqrt(G)
    assert abs(want[0, 0] - want[1, 1]) > 10 * (grp[:, 0] - grp[:, 1]).std(ddof=1) / np.sqrt(G)


def _spring_vector_sums(st):
    """Per chain: sums over its springs of d_a^2 (a = x, y, z), of d_x d_y and
    the number of springs, d = R_S - A."""
    occ = np.arange(st["S"].shape[1])[None, :] < st["Z"][:, None]
    S = np.where(occ, st["S"], 0)
    RS = np.take_along_axis(st["R"], S[:, :, None].repeat(3, axis=2), axis=1)
    d = np.where(occ[:, :, None], RS - st["A"], 0.0)
    return np.concatenate([(d ** 2).sum(axis=1), (d[:, :, 0] * d[:, :, 1]).sum(axis=1)[:, None],
                           occ.sum(axis=1)[:, None]], axis=1)


@pytest.mark.slow
def test_spring_vector_variance_in_dynamics_with_frozen_beads():
    # short chains: every spring is at most one hop from an end, so springs
    # live tens of steps and the run replaces every one of them many times
    N, M, G = 4, 2048, 32
    p = Params(N=N, N0=2.0, zeta=FROZEN, dt=0.01)  # default Ns = 0.5: kT/k_s = 1/6
    e = oracle.Ensemble(p, seed=41, M=M, levels=4)
    e.init()
    e.run(500)
    acc = np.zeros((M, 5))
    for _ in range(100):
        e.run(20)
        acc += _spring_vector_sums(e.get_state())
    c = e.counters()
    assert c["created"] > 100 * M and c["destroyed"] > 100 * M and c["hops_up"] > 50 * M
    # chains are independent: ratio estimates per group of chains, SE across groups
    grp = acc.reshape(G, M // G, 5).sum(axis=1)
    est = grp[:, :4] / grp[:, 4:5]
    want = p.Ns * p.b ** 2 / 3.0
    mean, se = est.mean(axis=0), est.std(axis=0, ddof=1) / np.sqrt(G)
    for a in range(3):
        assert abs(mean[a] - want) < 4 * se[a], (a, mean[a], want, se[a])
        assert se[a] < 0.015 * want  # resolved to 1.5%
    assert abs(mean[3]) < 4 * se[3]
