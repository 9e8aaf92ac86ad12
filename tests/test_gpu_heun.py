"""The stochastic Heun integrator (SS_HEUN) of the library against the
oracle's (GPU).

* FP64: integers bit-exact and positions within 1e-10 (centre-of-mass frame)
  at every compared step, with and without a velocity gradient, through
  launch boundaries; event counters equal.
* FP32 (N = 32): integers equal up to each chain's first near-tie, positions
  within 1e-4 relative until then.
* The Heun step is not the Euler step: the same seed gives different states.
* Paths that run only the Euler-Maruyama step refuse the integrator.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth
from oracle import Params
from paper_1106_2899_gb300 import SlipSpring
from paper_1106_2899_gb300 import _native as nat
from paper_1106_2899_gb300._native import SlipSpringError
from test_gpu_parity import TIE, _compare_states

pytestmark = pytest.mark.gpu


def _ctx(p, M, seed, precision, integrator=1, levels=8, chunk=64):
    g = SlipSpring([(M, p.N)], precision=precision, seed=seed)
    g.set_params(N0=p.N0, Ns=p.Ns, zeta_s=p.zeta_s, dt=p.dt, b=p.b, kT=p.kT, zeta=p.zeta, z_max=p.zm,
                 corr_levels=levels, groups=4, chunk_steps=chunk, integrator=integrator)
    return g


@pytest.mark.parametrize("N,gdot", [(16, 0.0), (24, 0.05), (48, 0.0), (80, 0.02)])
def test_heun_fp64_matches_oracle(cuda_ok, N, gdot):
    p = Params(N=N, z_max=min(N, 64), integrator=1, **synth.PAPER)
    M, seed = 160, 31
    g = _ctx(p, M, seed, "fp64")
    o = oracle.Ensemble(p, seed=seed, M=M, groups=4, levels=8)
    if gdot:
        g.set_flow(synth.shear_kappa(gdot), 0)
        o.set_flow(0, synth.shear_kappa(gdot))
    g.run(0)
    o.init()
    for blk, n in enumerate([1, 1, 3, 50, 150, 300]):
        g.run(n)
        o.run(n)
        _compare_states(g.get_state(), o.get_state(), np.ones(M, bool), 1e-10, "N=%d block %d" % (N, blk))
    gc, oc = g.counters(), o.counters()
    for k in ("hops_up", "hops_down", "created", "destroyed"):
        assert gc[k] == oc[k], k
    ga, _ = g.corr_sums()
    oa, _ = o.corr_sums()
    assert np.allclose(ga.sum(0), oa.sum(0), rtol=1e-9, atol=1e-9 * np.abs(oa).max())


def test_heun_fp32_matches_oracle_until_near_ties(cuda_ok):
    p = Params(N=32, integrator=1, **synth.PAPER)
    M, seed, steps = 256, 7, 120
    g = _ctx(p, M, seed, "fp32")
    o = oracle.Ensemble(p, seed=seed, M=M, levels=8)
    g.run(0)
    o.init()
    g.run(steps)
    _, _, mg = o.run(steps, trace=True)
    ok = ~(mg < TIE).any(axis=0)
    assert ok.sum() > 0.7 * M
    _compare_states(g.get_state(), o.get_state(), ok, 1e-4, "fp32 heun")


def test_heun_differs_from_euler_and_is_refused_elsewhere(cuda_ok):
    p = Params(N=16, **synth.PAPER)
    st = []
    for integ in (0, 1):
        g = _ctx(p, 64, 3, "fp64", integrator=integ)
        g.run(0)
        g.run(20)
        st.append(g.get_state())
        g.close()
    assert not np.allclose(st[0]["R"], st[1]["R"], atol=1e-8)
    # batched mode and differentiation windows run the Euler-Maruyama step only
    g = SlipSpring([(64, 16), (32, 24)], precision="fp32", seed=1)
    g.set_params(corr_levels=-1, integrator=1)
    g.set_batched(True)
    with pytest.raises(SlipSpringError, match="SS_EINVAL"):
        g.run(10)
    g = SlipSpring([(64, 16)], precision="fp32", seed=1)
    g.set_params(integrator=1)
    with pytest.raises(SlipSpringError, match="SS_EINVAL"):
        g.window_forward(100, 50)
    with pytest.raises(SlipSpringError, match="SS_EINVAL"):
        g.set_params(integrator=2)
    params = nat.ss_params()
    params.integrator = 1
    lib = nat.load()
    rc = lib.ss_run_noalloc(C.byref(params), nat.SS_FP32, 0, 8, 16, 0, 0, 1, None, C.c_void_p(1), C.c_void_p(1),
                            C.c_void_p(1), C.c_void_p(1), None, None, None)
    assert rc == -1
