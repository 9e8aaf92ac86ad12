"""Parity of the CUDA library (through its C ABI) with the FP64 CPU oracle.

Criteria (FP32 beads, FP64 sums):
  * integers (Z, S) bit-exact per chain per step, up to that chain's first
    decision whose oracle margin |u - threshold| is below 1e-5 (a near-tie,
    where FP32 rounding may legitimately decide the other way); FP64 runs
    must match without that exception;
  * positions within 1e-4 relative (|dR| <= 1e-4 max(1, |R|)) in the chain's
    centre-of-mass frame while the integers agree; FP64 within 1e-10;
  * correlator and log sums: FP64 runs within 1e-9 relative of the oracle's
    group totals; long FP32 runs within 3 standard errors and 2% where the
    oracle's relative standard error is below 0.5%.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import Params
from paper_1106_2899_gb300 import SlipSpring

pytestmark = pytest.mark.gpu
TIE = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu(cuda_ok):
    from paper_1106_2899_gb300 import build
    build.build()
    yield


def _gpu_ctx(p: Params, M, seed, precision, levels=24, log_every=0, max_logs=0, groups=8, chunk=1024,
             recenter=100):
    g = SlipSpring([(M, p.N)], precision=precision, seed=seed)
    g.set_params(N0=p.N0, Ns=p.Ns, zeta_s=p.zeta_s, dt=p.dt, b=p.b, kT=p.kT, zeta=p.zeta, k_b=p.k_b,
                 k_s=p.k_s, create_mode=p.create_mode, z_max=p.zm, destroy_new=p.destroy_new,
                 recenter_every=recenter, log_every=log_every, max_logs=max_logs,
                 corr_levels=levels if levels > 0 else -1, groups=groups, chunk_steps=chunk)
    return g


def _com_frame(st):
    c = st["R"].mean(axis=1, keepdims=True)
    R = st["R"] - c
    A = st["A"] - c
    A[st["S"] < 0] = 0.0
    return R, A


def _compare_states(go, oo, ok, rtol, what):
    """Compare GPU and oracle states on chains `ok` (bool [M])."""
    assert np.array_equal(go["Z"][ok], oo["Z"][ok]), what + ": Z differs"
    assert np.array_equal(go["S"][ok], oo["S"][ok]), what + ": S differs"
    Rg, Ag = _com_frame(go)
    Ro, Ao = _com_frame(oo)
    scale = np.maximum(1.0, np.abs(Ro[ok]))
    assert np.all(np.abs(Rg[ok] - Ro[ok]) <= rtol * scale), what + ": R differs %g" % np.max(
        np.abs(Rg[ok] - Ro[ok]) / scale)
    occ = (go["S"][ok] >= 0)[..., None]
    scaleA = np.maximum(1.0, np.abs(Ao[ok]))
    dA = np.where(occ, np.abs(Ag[ok] - Ao[ok]), 0.0)
    assert np.all(dA <= rtol * scaleA), what + ": A differs %g" % np.max(dA / scaleA)


# --------------------------------------------------------------- init -----
@pytest.mark.parametrize("precision,N", [("fp64", 16), ("fp32", 32), ("fp32", 11), ("fp64", 100)])
def test_equilibrium_init_matches_oracle(precision, N):
    p = Params(N=N, z_max=min(N, 64))
    M = 300
    g = _gpu_ctx(p, M, seed=5, precision=precision)
    g.run(0)
    go = g.get_state()
    o = oracle.Ensemble(p, seed=5, M=M)
    o.init()
    oo = o.get_state()
    assert np.array_equal(go["Z"], oo["Z"])
    assert np.array_equal(go["S"], oo["S"])
    tol = 1e-12 if precision == "fp64" else 1e-6
    assert np.allclose(go["R"], oo["R"], rtol=tol, atol=tol)
    assert np.allclose(go["A"], oo["A"], rtol=tol, atol=tol)


# ---------------------------------------------------- FP64 step parity ----
def _fp64_stepwise(p, M, seed, steps_each, blocks, kappa=None, start=None, levels=24, log_every=0,
                   total_steps=None):
    total = total_steps if total_steps else steps_each * blocks
    max_logs = total // log_every + 1 if log_every else 0
    G = min(4, M)
    g = _gpu_ctx(p, M, seed, "fp64", levels=levels, log_every=log_every, max_logs=max_logs, groups=G)
    o = oracle.Ensemble(p, seed=seed, M=M, groups=G, levels=max(levels, 1), log_every=log_every,
                        max_logs=max_logs)
    if kappa is not None:
        g.set_flow(kappa, 0)
        o.set_flow(0, kappa)
    if start is None:
        o.init()
        g.run(0)
    else:
        o.set_state(start)
        g.set_state(start)
    for b in range(blocks):
        g.run(steps_each)
        o.run(steps_each)
        _compare_states(g.get_state(), o.get_state(), np.ones(M, bool), 1e-10, "block %d" % b)
    # event counters are integers: equal, whatever the padding of the last CTA
    gc, oc = g.counters(), o.counters()
    for k in ("hops_up", "hops_down", "created", "destroyed", "dropped"):
        assert gc[k] == oc[k], k
    return g, o


def test_fp64_parity_workload_bit_exact_integers():
    """Parity workload: 256 chains of N = 16, FP64, seed 0 -- integers bit-exact
    at every one of the first 300 steps and every 500 steps to 10^4; positions
    within 1e-10; correlator, stress-log and counter sums equal."""
    w = synth.WORKLOADS["parity"]
    p = Params(N=w["N"], **{k: v for k, v in synth.PAPER.items()})
    M = w["M"]
    g, o = _fp64_stepwise(p, M, w["seed"], 1, 300, log_every=100, total_steps=w["steps"])
    for b in range(19):
        g.run(500)
        o.run(500)
        _compare_states(g.get_state(), o.get_state(), np.ones(M, bool), 1e-10, "step %d" % g.step)
    assert g.step == 9800
    g.run(200)
    o.run(200)
    _compare_states(g.get_state(), o.get_state(), np.ones(M, bool), 1e-10, "final")
    # correlator group sums (totals over groups)
    ga, gn = g.corr_sums()
    oa, on = o.corr_sums()
    assert gn == on == 10000
    gt, ot = ga.sum(axis=0), oa.sum(axis=0)
    lags = oracle.corr_lags(24)
    used = lags >= 0
    scale = np.abs(ot[used]).max()
    assert np.allclose(gt[used], ot[used], rtol=1e-9, atol=1e-12 * scale)
    # stress logs
    gts, gl = g.log_sums()
    ots, ol = o.logs()
    assert np.array_equal(gts, ots)
    assert np.allclose(gl.sum(axis=1), ol.sum(axis=1), rtol=1e-9, atol=1e-9)
    # event counters are integers: exactly equal
    gc, oc = g.counters(), o.counters()
    for k in ("hops_up", "hops_down", "created", "destroyed", "dropped"):
        assert gc[k] == oc[k], k
    assert g.status() == 0


@pytest.mark.parametrize("case", ["N2", "zmax1", "no_springs", "cpu_mode", "destroy_new", "M1",
                                  "ragged", "fast_create", "N48", "N64", "N33_crowded", "N80", "N128_zcap"])
def test_fp64_edge_cases(case):
    kw = dict(N=16)
    M = 37
    if case == "N2":
        kw = dict(N=2, N0=0.5)
    elif case == "zmax1":
        kw = dict(N=8, z_max=1, N0=2.0)
    elif case == "no_springs":
        kw = dict(N=12, N0=np.inf)
    elif case == "cpu_mode":
        kw = dict(N=16, create_mode=1, z_max=6, N0=1.0)
    elif case == "destroy_new":
        kw = dict(N=16, destroy_new=1, N0=1.0)
    elif case == "M1":
        M = 1
    elif case == "ragged":
        kw = dict(N=20)
        M = 8 * 3 + 5  # 8 chains per CTA at N > 16: a partial last CTA
    elif case == "fast_create":
        kw = dict(N=6, N0=0.05, zeta_s=0.02)  # creation capped at 1/2 per attempt
    elif case == "N48":
        kw = dict(N=48)  # three beads per lane
    elif case == "N64":
        kw = dict(N=64, N0=2.0)  # four beads per lane, up to 64 springs
    elif case == "N33_crowded":
        kw = dict(N=33, N0=0.6)  # sub-slots beyond the first 16 are occupied
    elif case == "N80":
        kw = dict(N=80, z_max=64)  # 32 lanes x 4 beads (the paper's longest chains)
    elif case == "N128_zcap":
        kw = dict(N=128, z_max=64, N0=2.0)  # <Z> pressed against the 64-slot cap
    p = Params(**kw)
    _fp64_stepwise(p, M, seed=17, steps_each=1, blocks=150)


def test_fp64_shear_flow_com_frame():
    """Startup shear kappa_xy = 0.3 with recentring every 100 steps on the GPU:
    the centre-of-mass frame state equals the oracle's absolute-frame state."""
    p = Params(N=16)
    _fp64_stepwise(p, 48, seed=3, steps_each=250, blocks=12, kappa=synth.shear_kappa(0.3))


def test_fp64_general_flow_schedule_and_set_state():
    p = Params(N=12, N0=2.0)
    M = 40
    st = synth.random_state(M, p.N, p.zm, seed=9, z_mean=5.0)
    g = _gpu_ctx(p, M, 21, "fp64", groups=4)
    o = oracle.Ensemble(p, seed=21, M=M, groups=4, levels=24)
    g.set_state(st)
    o.set_state(st)
    rng = np.random.default_rng(1)
    for k in range(4):
        kap = rng.normal(0, 0.2, size=(3, 3))
        kap -= np.trace(kap) / 3 * np.eye(3)
        g.set_flow(kap, 100 * k)
        o.set_flow(100 * k, kap)
    for b in range(8):
        g.run(60)
        o.run(60)
        _compare_states(g.get_state(), o.get_state(), np.ones(M, bool), 1e-10, "block %d" % b)


# ---------------------------------------------------- FP32 step parity ----
def _first_tie(margins):
    """Index of each chain's first step with a near-tie (n_steps if none)."""
    tie = margins < TIE
    first = np.where(tie.any(axis=0), tie.argmax(axis=0), margins.shape[0])
    return first


@pytest.mark.parametrize("N,kappa", [(32, None), (16, None), (24, 0.05), (48, None), (80, 0.02), (128, None),
                                     (11, 0.03), (2, None)])
def test_fp32_stepwise_parity_until_near_tie(N, kappa):
    p = Params(N=N, z_max=min(N, 64))
    M = 512 if N > 16 else 1024
    steps = 600
    g = _gpu_ctx(p, M, 1, "fp32")
    o = oracle.Ensemble(p, seed=1, M=M)
    if kappa is not None:
        g.set_flow(synth.shear_kappa(kappa), 0)
        o.set_flow(0, synth.shear_kappa(kappa))
    o.init()
    g.run(0)
    compared = 0
    for s in range(steps):
        g.run(1)
        Zt, St, mg = o.run(1, trace=True)
        if s == 0:
            first_tie = np.full(M, steps)
        tie_now = mg[0] < TIE
        first_tie = np.where((first_tie == steps) & tie_now, s, first_tie)
        ok = first_tie > s  # no near-tie at or before this step
        go, oo = g.get_state(), o.get_state()
        _compare_states(go, oo, ok, 1e-4, "step %d" % s)
        compared += ok.sum()
    assert compared > 0.5 * M * steps


def test_fp32_full_size_sampled_chains():
    """LVE workload size (65536 chains, N = 32) in the benchmark's launch shape
    (1024 steps per launch): sampled chains match the oracle run on those
    chains alone unless a near-tie occurred; sizes, counters and finiteness
    hold for every chain."""
    w = synth.WORKLOADS["lve"]
    M, N = w["M"], w["N"]
    p = Params(N=N)
    g = _gpu_ctx(p, M, w["seed"], "fp32", chunk=1024)
    g.run(0)
    st0 = g.get_state()
    g.run(1024)
    go = g.get_state()
    assert g.status() == 0
    assert np.all((go["Z"] >= 0) & (go["Z"] <= N))
    occ = np.arange(N)[None, :] < go["Z"][:, None]
    assert np.all((go["S"] >= 0) == occ) and np.all(go["S"][occ] < N)
    assert np.all(np.isfinite(go["R"]))
    c = g.counters()
    assert int(go["Z"].sum()) - int(st0["Z"].sum()) == c["created"] - c["destroyed"]
    rng = np.random.default_rng(0)
    ids = np.sort(rng.choice(M, size=48, replace=False))
    agree = 0
    for m in ids:
        o = oracle.Ensemble(p, seed=w["seed"], M=1, chain_offset=int(m), levels=1)
        o.init()
        _, _, mg = o.run(1024, trace=True)
        if np.any(mg[:, 0] < TIE):
            continue
        oo = o.get_state()
        one = {k: v[m:m + 1] for k, v in go.items()}
        _compare_states(one, oo, np.ones(1, bool), 1e-4, "chain %d" % m)
        agree += 1
    assert agree >= 8


# ------------------------------------------------ statistical parity -------
@pytest.mark.slow
def test_fp32_relaxation_modulus_statistics():
    """G(t) (AUTO and TOTAL) of a long FP32 GPU run against an independent
    oracle ensemble: within 3 combined standard errors at every lag up to
    1000 steps, and within 2% where the oracle's relative error is < 0.5%."""
    p = Params(N=16)
    Mg, Mo, burn, steps, G = 32768, 2048, 1000, 12000, 32
    g = _gpu_ctx(p, Mg, 7, "fp32", levels=10, groups=G)
    g.run(burn)
    g.reset_observables()
    g.run(steps)
    o = oracle.Ensemble(p, seed=1234567, M=Mo, groups=G, levels=10)
    o.init()
    o.run(burn)
    o.reset_observables()
    o.run(steps)
    oacc, on = o.corr_sums()
    cnt = oracle.corr_counts(on, 10)
    lags = oracle.corr_lags(10)
    per = Mo // G
    for ch_name, ch in (("auto", 0), ("total", 1)):
        t, Gg, sg = g.correlator(ch_name)
        # lag slots without samples (count 0) are never compared below
        est = oacc[:, :, :, ch, :].mean(axis=3) / (np.maximum(cnt, 1)[None] * per * p.N)
        checked = 0
        for i, tt in enumerate(t):
            lag = int(round(tt / p.dt))
            if lag > 1000:
                continue
            l, k = np.argwhere(lags == lag)[0]
            ov = est[:, l, k]
            om, ose = ov.mean(), ov.std(ddof=1) / np.sqrt(G)
            comb = np.sqrt(sg[i] ** 2 + ose ** 2)
            assert abs(Gg[i] - om) <= 3 * comb, (ch_name, lag, Gg[i], om, comb)
            if ose < 0.005 * abs(om):
                assert abs(Gg[i] - om) <= 0.02 * abs(om)
            checked += 1
        assert checked > 30


# ------------------------------------------------------------ errors -------
def test_error_paths():
    from paper_1106_2899_gb300._native import SlipSpringError
    g = SlipSpring([(10, 8)], precision="fp32", seed=0)
    with pytest.raises(SlipSpringError, match="SS_ESTATE"):
        g.run(1)
    with pytest.raises(SlipSpringError, match="SS_EINVAL"):
        g.set_params(dt=1.0)  # unstable Euler step
    with pytest.raises(SlipSpringError, match="SS_EINVAL"):
        g.set_params(z_max=9)
    g.set_params(log_every=10, max_logs=2)
    with pytest.raises(SlipSpringError, match="SS_EINVAL"):
        g.run(100)  # log capacity
    st = synth.random_state(10, 8, 8, seed=1)
    st["S"][0, 0] = 8
    st["Z"][0] = max(st["Z"][0], 1)
    with pytest.raises(SlipSpringError, match="SS_EINVAL"):
        g.set_state(st)
    with pytest.raises(SlipSpringError, match="SS_EINVAL"):
        g.set_flow(np.full(9, np.nan))
    g.run(20)
    assert g.status() == 0


# ------------------------------------------------- resume, failure detection --
def test_resume_from_saved_state_is_bit_exact():
    """Checkpoint/resume: the state after 300 steps, loaded into a new context
    with the step counter set to 300, continues bit for bit like one 600-step
    run (counter-based random numbers), with and without flow (recentring
    happens at absolute steps)."""
    for kappa in (None, synth.shear_kappa(0.05)):
        p = Params(N=24)
        ref = _gpu_ctx(p, 100, 7, "fp32", levels=-1)
        if kappa is not None:
            ref.set_flow(kappa, 0)
        ref.run(600)
        a = _gpu_ctx(p, 100, 7, "fp32", levels=-1)
        if kappa is not None:
            a.set_flow(kappa, 0)
        a.run(300)
        saved = a.get_state()
        b = _gpu_ctx(p, 100, 7, "fp32", levels=-1)
        if kappa is not None:
            b.set_flow(kappa, 0)
        b.set_state(saved)
        b.step = 300
        b.run(300)
        s_ref, s_b = ref.get_state(), b.get_state()
        for k in ("R", "A", "Z", "S"):
            assert np.array_equal(s_ref[k], s_b[k]), (k, kappa is not None)


def test_nonfinite_state_is_reported_not_faulted():
    """Failure detection on the device: a chain driven to overflow (bond forces
    beyond FP32 range) sets status bit 0 and the non-finite counter; the other
    chains, the integer state and the invariant bit are unaffected."""
    g = SlipSpring([(40, 16)], precision="fp32", seed=3)
    g.set_params(**synth.PAPER, corr_levels=8, groups=4)
    g.run(10)
    st = g.get_state()
    st["R"][5, ::2] += 3.0e38  # finite in FP32, but the next bond forces overflow
    g.set_state(st)
    g.run(5)
    s = g.status()
    c = g.counters()
    assert s & 1 and c["nonfinite"] >= 1
    assert not (s & 2) and c["broken"] == 0
    out = g.get_state()
    ok = np.ones(40, bool)
    ok[5] = False
    assert np.all(np.isfinite(out["R"][ok]))
    assert np.all((out["Z"] >= 0) & (out["Z"] <= 16))
