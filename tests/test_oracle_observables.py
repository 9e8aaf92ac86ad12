"""Pins of the oracle's observables (CPU only).

* Multiple-tau correlator: the streaming implementation against the batch
  definition written with numpy (block means of 2^l raw samples, lag products
  summed over all origins).
* Rouse closed form (slip-springs off, N0 = inf): the Euler-Maruyama scheme of
  Sec. 3.1 item 1 is linear, so its stationary stress autocorrelation is
  exact: <s_xy(n) s_xy(0)> = k_b^2 sum_p mu_p^2 V_p^2 r_p^(2n) with mu_p the
  path-Laplacian eigenvalues, r_p = 1 - k_b dt mu_p / zeta and
  V_p = (2 kT dt/zeta) / (1 - r_p^2); block-averaged levels take the exact
  triangular average of that sum.  The continuous-time limit is the Rouse
  relaxation modulus the paper invokes for small N (Sec. 4.1).
* Equilibrium with slip-springs (Sec. 2.1): <Q_a^2> = b^2/3, <sigma_aa> = -kT,
  G_TOTAL(0) = G_AUTO(0) = (N-1)/N, G_CROSS(0) = 0, <Z> = N/N0 -- each up to
  the O(dt) bias of the scheme, checked to shrink with dt.
"""
import numpy as np
import pytest

import oracle
from oracle import CORR_P, Params, corr_counts, corr_lags


# ---------------------------------------------------- correlator definition --
def _batch_multitau(x, levels, P=CORR_P):
    T = x.shape[0]
    acc = np.zeros((levels, P, 2, 3))
    for l in range(levels):
        B = 1 << l
        nb = T // B
        if nb == 0:
            break
        X = x[: nb * B].reshape(nb, B, 6).mean(axis=1)
        for k in range(P):
            if l > 0 and k < P // 2:
                continue
            if k >= nb:
                continue
            later = X[k:, 0:3]
            acc[l, k, 0] = np.sum(later * X[: nb - k, 0:3], axis=0)
            acc[l, k, 1] = np.sum(later * X[: nb - k, 3:6], axis=0)
    return acc


@pytest.mark.parametrize("T", [1, 15, 16, 33, 1000, 4097])
def test_multitau_streaming_equals_batch_definition(T):
    rng = np.random.default_rng(T)
    x = rng.normal(size=(T, 6)) + 0.3
    levels = 10
    got = oracle.corr_series(x, levels)
    want = _batch_multitau(x, levels)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-9)
    # the pair counts used for normalisation match the definition
    cnt = corr_counts(T, levels)
    ones = oracle.corr_series(np.ones((T, 6)), levels)
    assert np.allclose(ones[:, :, 0, 0], cnt)


@pytest.mark.parametrize("T", [33, 1000])
def test_multitau_tt_channel_equals_batch_definition(T):
    """Channel TT (later and origin both sigma + sigma_v, the numerator of the
    virtual-stress share of Sec. 4.1 minus TOTAL): the batch definition applied
    to the series whose sigma columns are the sigma + sigma_v columns."""
    rng = np.random.default_rng(T + 7)
    x = rng.normal(size=(T, 6)) + 0.2
    levels = 9
    acc, acc_tt = oracle.corr_series(x, levels, tt=True)
    assert np.allclose(acc, oracle.corr_series(x, levels), rtol=0, atol=0)
    swapped = np.concatenate([x[:, 3:6], x[:, 3:6]], axis=1)
    want = _batch_multitau(swapped, levels)[:, :, 0, :]
    assert np.allclose(acc_tt, want, rtol=1e-12, atol=1e-9)


# -------------------------------------------------------------- Rouse -------
def _rouse_exact(N, k_b, dt, zeta, kT, levels, scheme="euler"):
    """Exact stress autocorrelation of the discrete scheme (see the module
    docstring); scheme "heun": the stochastic Heun step maps each bond mode by
    r = 1 - x + x^2/2 and scales its noise by (1 - x/2), x = k_b dt mu/zeta."""
    L = np.zeros((N, N))
    for i in range(N - 1):
        L[i, i] += 1
        L[i + 1, i + 1] += 1
        L[i, i + 1] -= 1
        L[i + 1, i] -= 1
    mu = np.linalg.eigvalsh(L)[1:]
    x = k_b * dt * mu / zeta
    if scheme == "heun":
        r = 1 - x + x * x / 2
        V = (2 * kT * dt / zeta) * (1 - x / 2) ** 2 / (1 - r ** 2)
    else:
        r = 1 - x
        V = (2 * kT * dt / zeta) / (1 - r ** 2)
    amp = k_b ** 2 * mu ** 2 * V ** 2

    def C(n):
        n = np.abs(np.asarray(n))
        return np.sum(amp[None, :] * r[None, :] ** (2 * n[:, None]), axis=1)

    lags = corr_lags(levels)
    G = np.full((levels, CORR_P), np.nan)
    for l in range(levels):
        B = 1 << l
        d = np.arange(-(B - 1), B)
        w = (B - np.abs(d)) / B ** 2
        for k in range(CORR_P):
            if lags[l, k] < 0:
                continue
            G[l, k] = np.sum(w * C(k * B + d))
    return G  # <s_xy(t) s_xy(0)> (kT^2 units), block-averaged


def _group_G(acc, n, M, G_groups, levels):
    """Per-group estimate of <later*origin> [G][levels][P][2] averaged over comps."""
    cnt = corr_counts(n, levels)
    per = M // G_groups
    with np.errstate(invalid="ignore", divide="ignore"):
        est = acc.mean(axis=4) / (cnt[None, :, :, None] * per)
    return est


@pytest.mark.slow
def test_rouse_closed_form_autocorrelation():
    N, M, G, levels = 8, 1024, 32, 9
    p = Params(N=N, N0=np.inf, dt=0.01)
    ens = oracle.Ensemble(p, seed=2024, M=M, groups=G, levels=levels)
    ens.init()
    ens.run(2000)
    ens.reset_observables()
    ens.run(24000)
    acc, n = ens.corr_sums()
    est = _group_G(acc, n, M, G, levels)
    exact = _rouse_exact(N, 3.0, p.dt, 1.0, 1.0, levels)
    lags = corr_lags(levels)
    checked = 0
    for l in range(levels):
        for k in range(CORR_P):
            if lags[l, k] < 0 or lags[l, k] > 400:
                continue
            g = est[:, l, k, 0]
            m, se = g.mean(), g.std(ddof=1) / np.sqrt(G)
            assert abs(m - exact[l, k]) < 4.5 * se + 1e-12, (l, k, m, exact[l, k], se)
            # no slip-springs: sigma_v = 0, TOTAL = AUTO exactly
            assert np.allclose(est[:, l, k, 1], est[:, l, k, 0])
            checked += 1
    assert checked > 40
    # G(0) per bead is (1/N) sum_p 1/(1 - a mu_p/2)^2 -- near (N-1)/N, above it
    assert exact[0, 0] / N > (N - 1) / N


@pytest.mark.slow
def test_rouse_discrete_form_is_distinguishable_from_continuous():
    """The exact discrete G differs from the continuous Rouse G by more than the
    test resolution at short lags, so the closed-form pin is sharp."""
    N = 8
    exact = _rouse_exact(N, 3.0, 0.01, 1.0, 1.0, 1)[0, :4]
    L = np.diag([1] + [2] * (N - 2) + [1]) - np.eye(N, k=1) - np.eye(N, k=-1)
    mu = np.linalg.eigvalsh(L)[1:]
    cont = np.array([np.sum(np.exp(-2 * 3.0 * mu * 0.01 * n)) for n in range(4)])
    assert np.all(np.abs(exact / cont - 1) > 0.01)


# -------------------------------------------------- equilibrium w/ springs --
def _equilibrium_run(dt, steps):
    N, M, G, levels = 12, 768, 32, 2
    p = Params(N=N, N0=3.0, dt=dt)
    ens = oracle.Ensemble(p, seed=99, M=M, groups=G, levels=levels, log_every=25,
                          max_logs=steps // 25 + 2)
    ens.init()
    ens.run(steps)
    acc, n = ens.corr_sums()
    est = _group_G(acc, n, M, G, levels)
    t, L = ens.logs()
    st = ens.get_state()
    Q = np.diff(st["R"], axis=1)
    return p, est, L, st, Q


@pytest.mark.slow
def test_equilibrium_invariants_with_slip_springs():
    res = {}
    for dt, steps in [(0.01, 6000), (0.0025, 12000)]:
        p, est, L, st, Q = _equilibrium_run(dt, steps)
        N = p.N
        g0_auto = est[:, 0, 0, 0] / N
        g0_tot = est[:, 0, 0, 1] / N
        cross = g0_tot - g0_auto
        Msum = L.sum(axis=1)  # [n][14] sums over groups
        nchain = 768
        sig_diag = Msum[:, 0:3].mean() / nchain
        Zmean = Msum[:, 12].mean() / nchain
        res[dt] = dict(g0_auto=g0_auto.mean(), g0_se=g0_auto.std(ddof=1) / np.sqrt(len(g0_auto)),
                       cross=cross.mean(), cross_se=cross.std(ddof=1) / np.sqrt(len(cross)),
                       sig=sig_diag, Z=Zmean, Q2=(Q ** 2).mean() * 3)
    exact_g0 = (12 - 1) / 12
    for dt, r in res.items():
        # CROSS(0) = <s_xy s_v,xy> = 0: d = R_S - A is independent of the bonds
        assert abs(r["cross"]) < 4 * r["cross_se"] + 0.01
        assert abs(r["Z"] / 4.0 - 1) < 0.05
        assert abs(r["Q2"] - 1) < 0.08
        # <sigma_aa> = k_b sum <Q_a^2> - N kT = -kT up to the scheme's O(dt)
        # inflation of the bond variance (k_b (N-1) times a few percent)
        assert abs(r["sig"] + 1.0) < 5.0 * dt * 11
    # the bias of <sigma_aa> is first order in dt: quartering dt quarters it
    b1, b2 = res[0.01]["sig"] + 1.0, res[0.0025]["sig"] + 1.0
    assert 0.15 < b2 / b1 < 0.4
    # O(dt) bias shrinks: the small-dt run is closer to (N-1)/N than the large one,
    # and within a few percent
    err_big = abs(res[0.01]["g0_auto"] - exact_g0)
    err_small = abs(res[0.0025]["g0_auto"] - exact_g0)
    assert err_small < 0.04 + 4 * res[0.0025]["g0_se"]
    assert err_small < err_big + 4 * res[0.0025]["g0_se"]
