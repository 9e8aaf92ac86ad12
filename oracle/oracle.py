"""ctypes binding of the FP64 C oracle (ss_oracle.c).  TEST INFRASTRUCTURE ONLY.

Array layouts (all C-contiguous):
  R  [M][N][3] float64     bead positions, bead 0 = the paper's bead 1
  Z  [M]       int32       number of slip-springs
  S  [M][z_max] int32      0-based bead index of spring j, -1 for empty slots
  A  [M][z_max][3] float64 anchor of spring j
"""
import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import build as _build

CORR_P = 16
_lib = None


class _CParams(C.Structure):
    _fields_ = [("N", C.c_int), ("z_max", C.c_int), ("create_mode", C.c_int),
                ("destroy_new", C.c_int), ("N0", C.c_double), ("Ns", C.c_double),
                ("zeta_s", C.c_double), ("dt", C.c_double), ("b", C.c_double),
                ("kT", C.c_double), ("zeta", C.c_double), ("k_b", C.c_double),
                ("k_s", C.c_double), ("integrator", C.c_int)]


class _CChain(C.Structure):
    _fields_ = [("R", C.c_double * 3 * 128), ("Z", C.c_int), ("S", C.c_int * 128),
                ("A", C.c_double * 3 * 128)]


class _CInfo(C.Structure):
    _fields_ = [("min_margin", C.c_double), ("hops_up", C.c_int), ("hops_down", C.c_int),
                ("created", C.c_int), ("destroyed", C.c_int), ("dropped", C.c_int)]


OPS_CATEGORIES = ["philox", "decode", "bond", "spring", "euler", "advect", "hop", "create", "destroy", "stress",
                  "correlator"]
_count_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    _lib = _configure(C.CDLL(_build.build()))
    return _lib


def _load_counting():
    global _count_lib
    if _count_lib is None:
        _count_lib = _configure(C.CDLL(_build.build_counting()))
    return _count_lib


def _configure(lib):
    P = C.POINTER
    dp, ip, lp = P(C.c_double), P(C.c_int32), P(C.c_int64)
    u32p = P(C.c_uint32)
    lib.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
    lib.or_decode_block.argtypes = [u32p, dp, dp]
    lib.or_norm_ppf.argtypes = [C.c_double]
    lib.or_norm_ppf.restype = C.c_double
    lib.or_params_derive.argtypes = [P(_CParams)]
    lib.or_init_chain.argtypes = [P(_CParams), u32p, C.c_uint32, P(_CChain)]
    lib.or_step_chain.argtypes = [P(_CParams), u32p, C.c_uint32, C.c_uint32, dp, C.c_double,
                                  P(_CChain), P(_CInfo)]
    lib.or_stress.argtypes = [P(_CParams), P(_CChain), dp, dp]
    lib.or_ens_create.argtypes = [P(_CParams), C.c_uint64, C.c_int, C.c_uint32, C.c_int, C.c_int,
                                  C.c_int, C.c_int]
    lib.or_ens_create.restype = C.c_void_p
    lib.or_ens_destroy.argtypes = [C.c_void_p]
    lib.or_ens_init.argtypes = [C.c_void_p]
    lib.or_ens_set_flow.argtypes = [C.c_void_p, C.c_int64, dp]
    lib.or_ens_run.argtypes = [C.c_void_p, C.c_int64, C.c_int, ip, ip, dp]
    lib.or_ens_run.restype = C.c_int
    lib.or_ens_get_state.argtypes = [C.c_void_p, dp, ip, ip, dp]
    lib.or_ens_set_state.argtypes = [C.c_void_p, dp, ip, ip, dp]
    lib.or_ens_step.argtypes = [C.c_void_p]
    lib.or_ens_step.restype = C.c_int64
    lib.or_ens_corr.argtypes = [C.c_void_p, dp, lp]
    lib.or_ens_logs.argtypes = [C.c_void_p, dp, lp, C.c_int]
    lib.or_ens_logs.restype = C.c_int
    lib.or_ens_reset_obs.argtypes = [C.c_void_p]
    lib.or_ens_counters.argtypes = [C.c_void_p, lp]
    lib.or_corr_series.argtypes = [dp, C.c_int64, C.c_int, dp]
    lib.or_ens_run_tape.argtypes = [C.c_void_p, C.c_int64, C.c_int, ip, ip, dp, P(C.c_uint8), C.c_int]
    lib.or_ens_run_tape.restype = C.c_int
    lib.or_ens_set_step.argtypes = [C.c_void_p, C.c_int64]
    lib.or_ens_set_step.restype = None
    lib.or_corr_series_tt.argtypes = [dp, C.c_int64, C.c_int, dp, dp]
    lib.or_corr_series_tt.restype = None
    lib.or_ens_corr_tt.argtypes = [C.c_void_p, dp]
    lib.or_ens_corr_tt.restype = None
    lib.or_ops_get.argtypes = [lp]
    lib.or_ops_get.restype = None
    lib.or_ops_reset.argtypes = []
    lib.or_ops_reset.restype = None
    lib.or_ops_enabled.argtypes = []
    lib.or_ops_enabled.restype = C.c_int
    return lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


@dataclass
class Params:
    """Model parameters; the defaults are the paper's (Sec. 4.1: N0 = 4, Ns = 0.5,
    zeta_s = 0.1, dt = 0.01; units b = kT = zeta = 1, Sec. 3.1)."""
    N: int = 32
    z_max: int = 0            # 0 -> N
    create_mode: int = 0      # 0: K = z_max - Z; 1: K = 1
    destroy_new: int = 0
    N0: float = 4.0
    Ns: float = 0.5
    zeta_s: float = 0.1
    dt: float = 0.01
    b: float = 1.0
    kT: float = 1.0
    zeta: float = 1.0
    k_b: float = 0.0          # 0 -> 3 kT / b^2
    k_s: float = 0.0          # 0 -> 3 kT / (Ns b^2)
    integrator: int = 0       # 0: Euler-Maruyama (Sec. 3.1); 1: stochastic Heun (second-order SRK)

    def c(self):
        zm = self.z_max if self.z_max > 0 else self.N
        p = _CParams(self.N, zm, self.create_mode, self.destroy_new, self.N0, self.Ns,
                     self.zeta_s, self.dt, self.b, self.kT, self.zeta, self.k_b, self.k_s, self.integrator)
        _load().or_params_derive(C.byref(p))
        return p

    @property
    def zm(self):
        return self.z_max if self.z_max > 0 else self.N


def _key(seed):
    return np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)


def philox(ctr, key):
    """Philox4x32-10 of one 4-word counter under a 2-word key."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.or_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def decode_block(w):
    """Four normals and one 24-bit uniform from a Philox block."""
    lib = _load()
    ww = np.ascontiguousarray(w, dtype=np.uint32)
    n = np.zeros(4)
    u = C.c_double()
    lib.or_decode_block(_ptr(ww, C.c_uint32), _ptr(n, C.c_double), C.byref(u))
    return n, u.value


def norm_ppf(p):
    return _load().or_norm_ppf(float(p))


def _chain_from(state, N, zm):
    c = _CChain()
    R = np.asarray(state["R"], dtype=np.float64)
    for i in range(N):
        for a in range(3):
            c.R[i][a] = R[i, a]
    c.Z = int(state["Z"])
    for j in range(c.Z):
        c.S[j] = int(state["S"][j])
        for a in range(3):
            c.A[j][a] = float(state["A"][j][a])
    return c


def _chain_to(c, N, zm):
    R = np.array([[c.R[i][a] for a in range(3)] for i in range(N)])
    S = np.full(zm, -1, dtype=np.int32)
    A = np.zeros((zm, 3))
    for j in range(c.Z):
        S[j] = c.S[j]
        A[j] = [c.A[j][a] for a in range(3)]
    return {"R": R, "Z": c.Z, "S": S, "A": A}


def init_chain(p: Params, seed: int, chain_id: int):
    """Equilibrium initial state of one chain (Sec. 3.1 sampling procedure)."""
    lib = _load()
    cp = p.c()
    c = _CChain()
    lib.or_init_chain(C.byref(cp), _ptr(_key(seed), C.c_uint32), chain_id, C.byref(c))
    return _chain_to(c, p.N, p.zm)


def step_chain(p: Params, seed: int, chain_id: int, step: int, state, kappa=None):
    """One time step of one chain (Sec. 3.1 substeps 1-3); returns (state, info)."""
    lib = _load()
    cp = p.c()
    c = _chain_from(state, p.N, p.zm)
    kap = np.zeros(9) if kappa is None else np.ascontiguousarray(kappa, dtype=np.float64).ravel()
    pd = min(cp.dt * cp.kT / cp.zeta_s, 1.0)
    cd = norm_ppf(pd)
    info = _CInfo()
    lib.or_step_chain(C.byref(cp), _ptr(_key(seed), C.c_uint32), chain_id, step,
                      _ptr(kap, C.c_double), cd, C.byref(c), C.byref(info))
    return _chain_to(c, p.N, p.zm), {
        "min_margin": info.min_margin, "hops_up": info.hops_up, "hops_down": info.hops_down,
        "created": info.created, "destroyed": info.destroyed, "dropped": info.dropped}


def stress(p: Params, state):
    """(sigma, sigma_v) as 3x3 arrays (Eq. stress_tensor_single_chain, App. B)."""
    lib = _load()
    cp = p.c()
    c = _chain_from(state, p.N, p.zm)
    s = np.zeros(9)
    sv = np.zeros(9)
    lib.or_stress(C.byref(cp), C.byref(c), _ptr(s, C.c_double), _ptr(sv, C.c_double))
    return s.reshape(3, 3), sv.reshape(3, 3)


class Ensemble:
    """M independent chains run by the oracle, with the same calls as the library:
    init, set_flow, run, get/set_state, correlator sums, stress logs.
    counting=True uses the operation-counting build (single-threaded)."""

    def __init__(self, p: Params, seed: int, M: int, chain_offset: int = 0, groups: int = 1,
                 levels: int = 24, log_every: int = 0, max_logs: int = 0, counting: bool = False):
        self.lib = _load_counting() if counting else _load()
        self.p = p
        self.M, self.G, self.levels = M, groups, levels
        self.N, self.zm = p.N, p.zm
        self.log_every = log_every
        self._cp = p.c()
        self.k_b, self.k_s = self._cp.k_b, self._cp.k_s
        self.h = self.lib.or_ens_create(C.byref(self._cp), seed, M, chain_offset, groups, levels,
                                        log_every, max_logs)
        if not self.h:
            raise ValueError("oracle: invalid ensemble parameters")

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.or_ens_destroy(self.h)
            self.h = None

    def init(self):
        self.lib.or_ens_init(self.h)

    def set_flow(self, from_step, kappa):
        k = np.ascontiguousarray(kappa, dtype=np.float64).ravel()
        self.lib.or_ens_set_flow(self.h, int(from_step), _ptr(k, C.c_double))

    def run(self, n_steps, nthreads=0, trace=False):
        """Advance n_steps; with trace=True return per-step Z [n][M], S [n][M][z_max]
        and the smallest decision margin [n][M]."""
        Z = S = mg = None
        if trace:
            Z = np.zeros((n_steps, self.M), dtype=np.int32)
            S = np.zeros((n_steps, self.M, self.zm), dtype=np.int32)
            mg = np.zeros((n_steps, self.M))
        rc = self.lib.or_ens_run(self.h, int(n_steps), int(nthreads), _ptr(Z, C.c_int32),
                                 _ptr(S, C.c_int32), _ptr(mg, C.c_double))
        if rc != 0:
            raise RuntimeError("oracle: log capacity exceeded")
        return (Z, S, mg) if trace else None

    def run_tape(self, n_steps, tape, mode, nthreads=0):
        """Advance n_steps recording (mode 1) or replaying (mode 2) the decision
        tape, a uint8 array [n_steps][M][N]."""
        assert tape.dtype == np.uint8 and tape.shape == (n_steps, self.M, self.N) and tape.flags.c_contiguous
        rc = self.lib.or_ens_run_tape(self.h, int(n_steps), int(nthreads), None, None, None,
                                      _ptr(tape, C.c_uint8), int(mode))
        if rc != 0:
            raise RuntimeError("oracle: log capacity exceeded")

    @property
    def step(self):
        return self.lib.or_ens_step(self.h)

    @step.setter
    def step(self, value):
        self.lib.or_ens_set_step(self.h, int(value))

    def get_state(self):
        R = np.zeros((self.M, self.N, 3))
        Z = np.zeros(self.M, dtype=np.int32)
        S = np.zeros((self.M, self.zm), dtype=np.int32)
        A = np.zeros((self.M, self.zm, 3))
        self.lib.or_ens_get_state(self.h, _ptr(R, C.c_double), _ptr(Z, C.c_int32),
                                  _ptr(S, C.c_int32), _ptr(A, C.c_double))
        return {"R": R, "Z": Z, "S": S, "A": A}

    def set_state(self, st):
        R = np.ascontiguousarray(st["R"], dtype=np.float64)
        Z = np.ascontiguousarray(st["Z"], dtype=np.int32)
        S = np.ascontiguousarray(st["S"], dtype=np.int32)
        A = np.ascontiguousarray(st["A"], dtype=np.float64)
        self.lib.or_ens_set_state(self.h, _ptr(R, C.c_double), _ptr(Z, C.c_int32),
                                  _ptr(S, C.c_int32), _ptr(A, C.c_double))

    def corr_sums(self):
        """Group sums [G][levels][P][2][3] of later*origin products and the
        number of samples pushed per chain."""
        acc = np.zeros((self.G, self.levels, CORR_P, 2, 3))
        n = C.c_int64()
        self.lib.or_ens_corr(self.h, _ptr(acc, C.c_double), C.byref(n))
        return acc, n.value

    def corr_sums_tt(self):
        """Group sums [G][levels][P][3] of channel TT (later sigma + sigma_v times
        origin sigma + sigma_v)."""
        acc = np.zeros((self.G, self.levels, CORR_P, 3))
        self.lib.or_ens_corr_tt(self.h, _ptr(acc, C.c_double))
        return acc

    def logs(self):
        """(log_step [n], sums [n][G][14]) — sums of sigma xx,yy,zz,xy,xz,yz,
        their squares, Z and Z^2 over each group's chains."""
        n = self.lib.or_ens_logs(self.h, None, None, 0)
        L = np.zeros((max(n, 1), self.G, 14))
        t = np.zeros(max(n, 1), dtype=np.int64)
        self.lib.or_ens_logs(self.h, _ptr(L, C.c_double), _ptr(t, C.c_int64), n)
        return t[:n], L[:n]

    def reset_observables(self):
        self.lib.or_ens_reset_obs(self.h)

    def counters(self):
        out = np.zeros(5, dtype=np.int64)
        self.lib.or_ens_counters(self.h, _ptr(out, C.c_int64))
        return dict(zip(["hops_up", "hops_down", "created", "destroyed", "dropped"], out.tolist()))


def op_counts(p: Params, seed: int, M: int, steps: int, levels: int = 24, warm: int = 200, kappa=None,
              log_every: int = 0):
    """Operations of the method per bead-step, by substep (ss_oracle.h states the
    counting rules), from the counting build of the oracle run single-threaded
    on M chains for `steps` steps after `warm` steps of warm-up."""
    e = Ensemble(p, seed=seed, M=M, levels=levels, log_every=log_every,
                 max_logs=(warm + steps) // log_every + 1 if log_every else 0, counting=True)
    lib = e.lib
    assert lib.or_ops_enabled() == 1
    e.init()
    if kappa is not None:
        e.set_flow(0, kappa)
    e.run(warm, nthreads=1)
    lib.or_ops_reset()
    e.run(steps, nthreads=1)
    out = np.zeros(len(OPS_CATEGORIES), dtype=np.int64)
    lib.or_ops_get(_ptr(out, C.c_int64))
    per = out / float(M * p.N * steps)
    return dict(zip(OPS_CATEGORIES, per.tolist()))


def corr_series(x, levels: int, tt: bool = False):
    """Streaming multiple-tau sums [levels][P][2][3] of one series x[T][6]; with
    tt also the channel-TT sums [levels][P][3]."""
    xx = np.ascontiguousarray(x, dtype=np.float64)
    acc = np.zeros((levels, CORR_P, 2, 3))
    if not tt:
        _load().or_corr_series(_ptr(xx, C.c_double), xx.shape[0], levels, _ptr(acc, C.c_double))
        return acc
    acc_tt = np.zeros((levels, CORR_P, 3))
    _load().or_corr_series_tt(_ptr(xx, C.c_double), xx.shape[0], levels, _ptr(acc, C.c_double),
                              _ptr(acc_tt, C.c_double))
    return acc, acc_tt


def corr_counts(n_samples: int, levels: int, P: int = CORR_P):
    """Number of later/origin pairs behind each (level, lag) of the multiple-tau
    correlator after n_samples pushes of one chain: level l has n_l =
    floor(n/2^l) samples and lag k gets max(0, n_l - k) pairs."""
    cnt = np.zeros((levels, P))
    for l in range(levels):
        nl = n_samples >> l
        for k in range(P):
            if l > 0 and k < P // 2:
                continue
            cnt[l, k] = max(0, nl - k)
    return cnt


def corr_lags(levels: int, P: int = CORR_P):
    """Lag in steps of each (level, lag-slot); -1 where the slot is unused."""
    lag = -np.ones((levels, P), dtype=np.int64)
    for l in range(levels):
        for k in range(P):
            if l > 0 and k < P // 2:
                continue
            lag[l, k] = k << l
    return lag

