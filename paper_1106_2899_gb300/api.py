"""Python binding of the slip-spring library: argument marshalling only.

Every step of the model runs in the library's CUDA kernels; this module turns
NumPy arrays and keyword arguments into the C ABI's pointers and structs.

    ens = SlipSpring([(65536, 32)], precision="fp32", seed=1)
    ens.set_params(N0=4, Ns=0.5, zeta_s=0.1, dt=0.01)
    ens.run(10000)
    t, G, sem = ens.correlator(channel="total")
"""
import ctypes as C

import numpy as np

from . import _native as nat

CHANNELS = {"auto": nat.SS_CH_AUTO, "cross": nat.SS_CH_CROSS, "total": nat.SS_CH_TOTAL, "tt": nat.SS_CH_TT,
            "virtual": nat.SS_CH_VIRTUAL}


def _p(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


class SlipSpring:
    """A context of one or more elements (ensembles of equal-length chains)."""

    def __init__(self, elements, precision="fp32", seed=0, stream=None, chain_offset=0):
        self.lib = nat.load()
        els = [(int(m), int(n)) for m, n in elements]
        arr = (nat.ss_element * len(els))(*[nat.ss_element(m, n) for m, n in els])
        self.elements = els
        self.precision = precision
        h = C.c_void_p()
        prec = {"fp32": nat.SS_FP32, "fp64": nat.SS_FP64}[precision]
        st = C.c_void_p(int(stream)) if stream is not None else None
        nat.check(self.lib.ss_create(C.byref(h), arr, len(els), prec, int(seed), st), None, "ss_create")
        self.h = h
        self.params = None
        if chain_offset:
            self._chk(self.lib.ss_set_chain_offset(self.h, int(chain_offset)), "ss_set_chain_offset")

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.ss_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, rc, what):
        nat.check(rc, self.h, what)

    # ------------------------------------------------------------ setup ---
    def set_params(self, **kw):
        p = nat.ss_params()
        for k, v in kw.items():
            if not hasattr(p, k):
                raise TypeError("unknown parameter %r" % k)
            setattr(p, k, v)
        self._chk(self.lib.ss_set_params(self.h, C.byref(p)), "ss_set_params")
        self.params = dict(kw)

    def set_flow(self, kappa, from_step=0, elem=-1):
        k = np.ascontiguousarray(np.asarray(kappa, dtype=np.float64).reshape(9))
        self._chk(self.lib.ss_set_flow(self.h, int(elem), int(from_step), _p(k, C.c_double)), "ss_set_flow")

    def set_flow_table(self, elem, from_step, kappa):
        """Many flow-schedule entries at once: element indices, first steps and
        kappa matrices [n][3][3] (in increasing step order within an element)."""
        e = np.ascontiguousarray(elem, dtype=np.int32)
        f = np.ascontiguousarray(from_step, dtype=np.int64)
        k = np.ascontiguousarray(np.asarray(kappa, dtype=np.float64).reshape(len(e), 9))
        self._chk(self.lib.ss_set_flow_table(self.h, len(e), _p(e, C.c_int32), _p(f, C.c_int64),
                                             _p(k, C.c_double)), "ss_set_flow_table")

    def set_batched(self, enable=True):
        """One persistent, graph-replayed launch per chunk over all elements."""
        self._chk(self.lib.ss_set_batched(self.h, 1 if enable else 0), "ss_set_batched")

    def set_coefficients(self, k_b, k_s, zeta):
        """New (k_b, k_s, zeta) keeping the state, step counter and a recorded window."""
        self._chk(self.lib.ss_set_coefficients(self.h, float(k_b), float(k_s), float(zeta)), "ss_set_coefficients")

    def run(self, n_steps):
        self._chk(self.lib.ss_run(self.h, int(n_steps)), "ss_run")

    # ------------------------------------------------ differentiation ---
    def window_forward(self, n_steps, checkpoint_every=256, replay=False):
        """Run a differentiation window (observables reset at its start); with
        replay the recorded decisions and noise are reused."""
        self._chk(self.lib.ss_window_forward(self.h, int(n_steps), int(checkpoint_every), 1 if replay else 0),
                  "ss_window_forward")

    def window_backward(self, dL_dG):
        """dL/d(k_b, k_s, zeta) from dL/dG [levels][16] of the window's TOTAL channel."""
        levels = (self.params or {}).get("corr_levels", 0) or 24
        g = np.ascontiguousarray(dL_dG, dtype=np.float64)
        if g.shape != (levels, 16):
            raise ValueError("dL_dG must have shape (%d, 16)" % levels)
        out = np.zeros(3)
        self._chk(self.lib.ss_window_backward(self.h, _p(g, C.c_double), _p(out, C.c_double)),
                  "ss_window_backward")
        return out

    def synchronize(self):
        self._chk(self.lib.ss_synchronize(self.h), "ss_synchronize")

    def reset_observables(self):
        self._chk(self.lib.ss_reset_observables(self.h), "ss_reset_observables")

    @property
    def step(self):
        s = C.c_int64()
        self._chk(self.lib.ss_step_count(self.h, C.byref(s)), "ss_step_count")
        return s.value

    @step.setter
    def step(self, value):
        """Position the step counter (resets the observables)."""
        self._chk(self.lib.ss_set_step_count(self.h, int(value)), "ss_set_step_count")

    # ------------------------------------------------------------ state ---
    def _zm(self, elem):
        zm = (self.params or {}).get("z_max", 0)
        return zm if zm > 0 else min(self.elements[elem][1], nat.SS_MAX_SLOTS)

    def get_state(self, elem=0):
        M, N = self.elements[elem]
        zm = self._zm(elem)
        R = np.zeros((M, N, 3))
        Z = np.zeros(M, dtype=np.int32)
        S = np.zeros((M, zm), dtype=np.int32)
        A = np.zeros((M, zm, 3))
        self._chk(self.lib.ss_get_state(self.h, elem, _p(R, C.c_double), _p(Z, C.c_int32), _p(S, C.c_int32),
                                        _p(A, C.c_double)), "ss_get_state")
        return {"R": R, "Z": Z, "S": S, "A": A}

    def set_state(self, st, elem=0):
        R = np.ascontiguousarray(st["R"], dtype=np.float64)
        Z = np.ascontiguousarray(st["Z"], dtype=np.int32)
        S = np.ascontiguousarray(st["S"], dtype=np.int32)
        A = np.ascontiguousarray(st["A"], dtype=np.float64)
        self._chk(self.lib.ss_set_state(self.h, elem, _p(R, C.c_double), _p(Z, C.c_int32), _p(S, C.c_int32),
                                        _p(A, C.c_double)), "ss_set_state")

    def get_state_dev(self, R, Z, S, A, elem=0, stream=None):
        """Copy the state into caller-owned CUDA tensors (R [M][N][3], A [M][z_max][3]
        float64; S [M][z_max], Z [M] int32), ordered before later work on `stream`."""
        st = C.c_void_p(int(stream)) if stream is not None else None
        ptr = [C.c_void_p(t.data_ptr()) if t is not None else None for t in (R, Z, S, A)]
        self._chk(self.lib.ss_get_state_dev(self.h, elem, *ptr, st), "ss_get_state_dev")

    def set_state_dev(self, R, Z, S, A, elem=0, stream=None):
        """Replace the state from CUDA tensors laid out as in get_state_dev."""
        st = C.c_void_p(int(stream)) if stream is not None else None
        ptr = [C.c_void_p(t.data_ptr()) for t in (R, Z, S, A)]
        self._chk(self.lib.ss_set_state_dev(self.h, elem, *ptr, st), "ss_set_state_dev")

    # ------------------------------------------------------ observables ---
    def zhist(self, elem=0):
        """Histogram of the slip-spring number Z over the element's chains, z = 0..z_max."""
        n = C.c_int()
        self._chk(self.lib.ss_zhist(self.h, elem, None, 0, C.byref(n)), "ss_zhist")
        h = np.zeros(n.value, dtype=np.int64)
        self._chk(self.lib.ss_zhist(self.h, elem, _p(h, C.c_int64), n.value, C.byref(n)), "ss_zhist")
        return h

    def stress(self, elem=0):
        """(t, mean[n][6], sem[n][6]) of sigma xx,yy,zz,xy,xz,yz at the log times."""
        n = C.c_int()
        self._chk(self.lib.ss_stress(self.h, elem, None, None, None, 0, C.byref(n)), "ss_stress")
        k = n.value
        t = np.zeros(k)
        mean = np.zeros((k, 6))
        sem = np.zeros((k, 6))
        if k:
            self._chk(self.lib.ss_stress(self.h, elem, _p(t, C.c_double), _p(mean, C.c_double),
                                         _p(sem, C.c_double), k, C.byref(n)), "ss_stress")
        return t, mean, sem

    def correlator(self, channel="total", elem=0):
        """(t, G, sem) of the relaxation modulus in rho0 kT (Green-Kubo, App. B)."""
        ch = CHANNELS[channel] if isinstance(channel, str) else int(channel)
        n = C.c_int()
        self._chk(self.lib.ss_correlator(self.h, elem, ch, None, None, None, 0, C.byref(n)), "ss_correlator")
        k = n.value
        t, G, sem = np.zeros(k), np.zeros(k), np.zeros(k)
        if k:
            self._chk(self.lib.ss_correlator(self.h, elem, ch, _p(t, C.c_double), _p(G, C.c_double),
                                             _p(sem, C.c_double), k, C.byref(n)), "ss_correlator")
        return t, G, sem

    def corr_sums(self, elem=0):
        """(acc [G][levels][16][2][3], n_samples) raw correlator group sums."""
        levels = (self.params or {}).get("corr_levels", 0) or 24
        g = C.c_int()
        n = C.c_int64()
        self._chk(self.lib.ss_corr_sums(self.h, elem, None, C.byref(g), C.byref(n)), "ss_corr_sums")
        acc = np.zeros((g.value, levels, 16, 2, 3))
        self._chk(self.lib.ss_corr_sums(self.h, elem, _p(acc, C.c_double), C.byref(g), C.byref(n)),
                  "ss_corr_sums")
        return acc, n.value

    def corr_sums_tt(self, elem=0):
        """(acc [G][levels][16][3], n_samples) group sums of channel TT (corr_tt=1)."""
        levels = (self.params or {}).get("corr_levels", 0) or 24
        g = C.c_int()
        n = C.c_int64()
        self._chk(self.lib.ss_corr_sums_tt(self.h, elem, None, C.byref(g), C.byref(n)), "ss_corr_sums_tt")
        acc = np.zeros((g.value, levels, 16, 3))
        self._chk(self.lib.ss_corr_sums_tt(self.h, elem, _p(acc, C.c_double), C.byref(g), C.byref(n)),
                  "ss_corr_sums_tt")
        return acc, n.value

    def log_sums(self, elem=0):
        """(log_step [n], sums [n][G][14]) raw stress-log group sums."""
        n = C.c_int()
        g = C.c_int()
        self._chk(self.lib.ss_log_sums(self.h, elem, None, None, 0, C.byref(n), C.byref(g)), "ss_log_sums")
        k = n.value
        t = np.zeros(k, dtype=np.int64)
        L = np.zeros((k, g.value, 14))
        if k:
            self._chk(self.lib.ss_log_sums(self.h, elem, _p(t, C.c_int64), _p(L, C.c_double), k, C.byref(n),
                                           C.byref(g)), "ss_log_sums")
        return t, L

    def counters(self):
        out = np.zeros(8, dtype=np.int64)
        self._chk(self.lib.ss_counters(self.h, _p(out, C.c_int64)), "ss_counters")
        return dict(zip(["hops_up", "hops_down", "created", "destroyed", "dropped", "launches",
                         "nonfinite", "broken"], out.tolist()))

    def kernel_timing(self, enable=True):
        """Bracket each chain-kernel launch with CUDA events (benchmark support)."""
        self._chk(self.lib.ss_kernel_timing(self.h, 1 if enable else 0), "ss_kernel_timing")

    def kernel_time(self):
        """(summed chain-kernel milliseconds, launches) since timing was enabled."""
        ms = C.c_double()
        n = C.c_int64()
        self._chk(self.lib.ss_kernel_time(self.h, C.byref(ms), C.byref(n)), "ss_kernel_time")
        return ms.value, n.value

    def status(self):
        s = C.c_int32()
        self._chk(self.lib.ss_status(self.h, C.byref(s)), "ss_status")
        return s.value
