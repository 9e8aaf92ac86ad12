"""Pathwise adjoint of a differentiation window (GPU, through the C ABI).

The gradient of L = sum (ln G - ln G_target)^2 over fitted multiple-tau slots
with respect to (k_b, k_s, zeta) (Sec. 3.1; G of Eq.
relaxation_modulus_tensor_green_kubo_form, App. B) is taken with every discrete
decision frozen.  It is checked

* against central finite differences of the same frozen-decision map on the
  GPU (relative step 1e-3, the recorded decisions replayed and the same noise),
* against an oracle gradient: central finite differences in FP64 of the
  oracle's own window, replaying the oracle's own decision tape (no value of
  the CUDA path enters it),
* and through torch.autograd.

A replay at the base parameters must reproduce the recorded window bit for bit.
"""
import time

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import Params
from paper_1106_2899_gb300 import SlipSpring
from paper_1106_2899_gb300.adjoint import GFit, fit_mask, log_loss, window_G

pytestmark = pytest.mark.gpu

THETA0 = np.array([3.0, 6.0, 1.0])  # k_b = 3kT/b^2, k_s = 3kT/(Ns b^2), zeta at the paper's defaults
EPS = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _gpu(cuda_ok):
    from paper_1106_2899_gb300 import build
    build.build()
    yield


def _ctx(M, N, precision, levels, seed, burn, chunk=256):
    g = SlipSpring([(M, N)], precision=precision, seed=seed)
    g.set_params(**synth.PAPER, corr_levels=levels, groups=16, chunk_steps=chunk)
    g.run(burn)
    return g


def _wiggle_target(G):
    """A smooth positive target that differs from G slot by slot."""
    idx = np.arange(G.size).reshape(G.shape)
    return G * np.exp(0.3 * np.sin(0.7 * idx))


def _fd(fit, theta0, eps=EPS):
    out = np.zeros(3)
    for p in range(3):
        h = eps * theta0[p]
        tp, tm = theta0.copy(), theta0.copy()
        tp[p] += h
        tm[p] -= h
        lp, _ = fit.evaluate(tp, replay=True)
        lm, _ = fit.evaluate(tm, replay=True)
        out[p] = (lp - lm) / (2 * h)
    return out


def _oracle_G(acc, n, M, N, levels, kT=1.0):
    """TOTAL-channel G per slot from oracle sums (one group), written out from
    the Green-Kubo estimator: sum of products / (3 components x products x M x N kT^2)."""
    cnt = oracle.corr_counts(n, levels)
    G = np.full((levels, 16), np.nan)
    ok = cnt > 0
    G[ok] = acc[0, :, :, 1, :].sum(axis=-1)[ok] / (3.0 * cnt[ok] * M * N * kT * kT)
    return G


def test_replay_at_base_parameters_is_bit_identical():
    M, N = 256, 24
    g = _ctx(M, N, "fp32", 8, seed=3, burn=200)
    start = g.get_state()
    t0 = g.step
    g.window_forward(600, 256)
    G0, _, _ = window_G(g)
    s0 = g.get_state()
    g.set_state(start)
    g.step = t0
    g.window_forward(600, 256, replay=True)
    G1, _, _ = window_G(g)
    s1 = g.get_state()
    for k in ("R", "A", "Z", "S"):
        assert np.array_equal(s0[k], s1[k]), k
    assert np.array_equal(G0[np.isfinite(G0)], G1[np.isfinite(G1)])
    # a plain (recording) window from the same start draws the same numbers too
    g.set_state(start)
    g.step = t0
    g.window_forward(600, 256)
    s2 = g.get_state()
    assert np.array_equal(s0["R"], s2["R"]) and np.array_equal(s0["S"], s2["S"])
    assert g.status() == 0


def test_backward_restores_final_state_and_zero_loss_gives_zero_gradient():
    M, N = 128, 16
    g = _ctx(M, N, "fp64", 6, seed=5, burn=100)
    g.window_forward(300, 128)
    s0 = g.get_state()
    grad = g.window_backward(np.zeros((6, 16)))
    assert np.array_equal(grad, np.zeros(3))
    s1 = g.get_state()
    for k in ("R", "A", "Z", "S"):
        assert np.array_equal(s0[k], s1[k]), k


@pytest.mark.parametrize("N,ce", [(24, 256), (16, 100), (40, 128), (80, 128)])
def test_fp64_adjoint_matches_replayed_finite_differences(N, ce):
    M, levels = 256, 8
    g = _ctx(M, N, "fp64", levels, seed=7, burn=300)
    start = g.get_state()
    # base window: records the decisions; the target wiggles around its G
    fit = GFit(g, start, n_steps=600, checkpoint_every=ce, target=np.ones((levels, 16)))
    fit.evaluate(THETA0)
    fit.target = _wiggle_target(fit.G)
    fit.mask = fit_mask(fit.G, fit.sem, fit.target)
    assert fit.mask.sum() >= 10
    L0, dL = log_loss(fit.G, fit.target, fit.mask)
    adj = fit.gradient(dL)
    fd = _fd(fit, THETA0)
    assert np.all(np.isfinite(adj)) and np.all(np.abs(fd) > 0)
    scale = np.abs(fd).max()
    # central differences carry an O(h^2) truncation error (a few 1e-5 relative
    # at h = 1e-3 here); Richardson extrapolation with h/2 removes it
    assert np.all(np.abs(adj - fd) <= 1e-3 * np.abs(fd) + 1e-6 * scale), (adj, fd)
    fd2 = _fd(fit, THETA0, EPS / 2)
    rich = (4 * fd2 - fd) / 3
    assert np.all(np.abs(adj - rich) <= 1e-6 * np.abs(rich) + 1e-8 * scale), (adj, rich)
    assert g.status() == 0


def test_fp64_adjoint_matches_oracle_gradient():
    """Oracle: same chains and numbers, its own decision tape, FD in FP64."""
    M, N, levels, burn, n = 128, 24, 8, 300, 600
    seed = 11
    g = _ctx(M, N, "fp64", levels, seed=seed, burn=burn)
    start = g.get_state()
    fit = GFit(g, start, n_steps=n, checkpoint_every=256, target=np.ones((levels, 16)))
    fit.evaluate(THETA0)
    target = _wiggle_target(fit.G)
    fit.target = target
    fit.mask = fit_mask(fit.G, fit.sem, target)
    assert fit.mask.sum() >= 10
    _, dL = log_loss(fit.G, target, fit.mask)
    adj = fit.gradient(dL)
    G_gpu = fit.G.copy()
    s_gpu = g.get_state()

    p0 = Params(N=N, **synth.PAPER)
    o = oracle.Ensemble(p0, seed=seed, M=M, levels=levels)
    o.init()
    o.run(burn)
    ost = o.get_state()
    assert np.array_equal(ost["Z"], start["Z"]) and np.array_equal(ost["S"], start["S"])
    tape = np.zeros((n, M, N), dtype=np.uint8)
    o.reset_observables()
    o.run_tape(n, tape, 1)
    acc, ns = o.corr_sums()
    G_or = _oracle_G(acc, ns, M, N, levels)
    fin = o.get_state()
    # the windows agree: same decisions (integers) and the same G to rounding
    assert np.array_equal(fin["Z"], s_gpu["Z"]) and np.array_equal(fin["S"], s_gpu["S"])
    ok = np.isfinite(G_gpu)
    assert np.allclose(G_or[ok], G_gpu[ok], rtol=1e-9, atol=1e-12 * np.nanmax(np.abs(G_gpu)))

    def oracle_loss(theta):
        p = Params(N=N, **{**synth.PAPER, "zeta": theta[2]}, k_b=theta[0], k_s=theta[1])
        e = oracle.Ensemble(p, seed=seed, M=M, levels=levels)
        e.set_state(ost)
        e.step = burn
        e.run_tape(n, tape, 2)
        a, k = e.corr_sums()
        Gx = _oracle_G(a, k, M, N, levels)
        r = np.log(Gx[fit.mask]) - np.log(target[fit.mask])
        return float(np.sum(r * r))

    def fd_at(eps):
        fd = np.zeros(3)
        for p in range(3):
            h = eps * THETA0[p]
            tp, tm = THETA0.copy(), THETA0.copy()
            tp[p] += h
            tm[p] -= h
            fd[p] = (oracle_loss(tp) - oracle_loss(tm)) / (2 * h)
        return fd

    fd = fd_at(EPS)
    scale = np.abs(fd).max()
    assert np.all(np.abs(adj - fd) <= 1e-3 * np.abs(fd) + 1e-6 * scale), (adj, fd)
    rich = (4 * fd_at(EPS / 2) - fd) / 3
    assert np.all(np.abs(adj - rich) <= 1e-6 * np.abs(rich) + 1e-8 * scale), (adj, rich)


def test_torch_autograd_function():
    M, N, levels = 256, 24, 8
    g = _ctx(M, N, "fp64", levels, seed=9, burn=200)
    start = g.get_state()
    fit = GFit(g, start, n_steps=512, checkpoint_every=256, target=np.ones((levels, 16)))
    fit.evaluate(THETA0)
    fit.target = _wiggle_target(fit.G)
    fit.mask = fit_mask(fit.G, fit.sem, fit.target)
    theta = torch.tensor(THETA0, dtype=torch.float64, requires_grad=True)
    loss = fit(theta)
    loss.backward()
    L, dL = log_loss(fit.G, fit.target, fit.mask)
    assert abs(loss.item() - L) <= 1e-12 * abs(L)
    direct = fit.gradient(dL)
    assert np.allclose(theta.grad.numpy(), direct, rtol=1e-12, atol=0)


@pytest.mark.slow
def test_fp32_full_window_against_finite_differences_and_oracle_target():
    """8192 chains of N=24, FP32 forward, FP64 loss; a 1e4-step window with a
    checkpoint every 256 steps; the target G from the oracle at (k_b, k_s, zeta)
    x 1.10; fitted lags where both moduli are positive and resolved to 20%."""
    w = synth.WORKLOADS["adjoint"]
    M, N, n, ce = w["M"], w["N"], w["steps"], w["checkpoint"]
    levels, burn = 14, 2000
    # target: oracle ensemble at perturbed parameters
    th_t = THETA0 * 1.10
    pt = Params(N=N, **{**synth.PAPER, "zeta": th_t[2]}, k_b=th_t[0], k_s=th_t[1])
    Mo = 512
    o = oracle.Ensemble(pt, seed=w["seed"] + 1, M=Mo, groups=16, levels=levels)
    o.init()
    o.run(burn)
    o.reset_observables()
    o.run(n)
    acc, ns = o.corr_sums()
    cnt = oracle.corr_counts(ns, levels)
    per = acc[:, :, :, 1, :].sum(axis=-1) / (3.0 * np.maximum(cnt, 1)[None] * (Mo / 16) * N)
    Gt = np.where(cnt > 0, per.mean(axis=0), np.nan)
    set_ = per.std(axis=0, ddof=1) / 4.0
    target = np.where(set_ < 0.2 * np.abs(Gt), Gt, np.nan)

    g = SlipSpring([(M, N)], precision="fp32", seed=w["seed"])
    g.set_params(**synth.PAPER, corr_levels=levels, groups=32, chunk_steps=1024)
    g.run(burn)
    start = g.get_state()
    fit = GFit(g, start, n_steps=n, checkpoint_every=ce, target=target)
    theta = torch.tensor(THETA0, dtype=torch.float64, requires_grad=True)
    g.synchronize()
    t_a = time.perf_counter()
    loss = fit(theta)
    g.synchronize()
    t_b = time.perf_counter()
    loss.backward()
    g.synchronize()
    t_c = time.perf_counter()
    adj = theta.grad.numpy().copy()
    print("\nwindow of %d chains x N=%d x %d steps: forward %.3g bead-steps/s, backward %.3g bead-steps/s"
          % (M, N, n, M * N * n / (t_b - t_a), M * N * n / (t_c - t_b)))
    assert fit.mask.sum() >= 20
    fd = _fd(fit, THETA0)
    print("\nadjoint %s\nFD      %s\nloss %.6g over %d slots" % (adj, fd, loss.item(), fit.mask.sum()))
    scale = np.abs(fd).max()
    # FP32 forward: the difference quotient carries rounding noise of ~1e-7 / h
    assert np.all(np.abs(adj - fd) <= 2e-3 * np.abs(fd) + 2e-4 * scale), (adj, fd)
    assert g.status() == 0
