"""ctypes declarations of the C ABI in include/slipspring.h.

Loading fails loudly when the compiled library is missing: there is no CPU
fallback.  Build it with `python -m paper_1106_2899_gb300.build`.
"""
import ctypes as C
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libslipspring.so")

SS_OK = 0
ERRORS = {-1: "SS_EINVAL", -2: "SS_ENOMEM", -3: "SS_ECUDA", -4: "SS_EOVERFLOW", -5: "SS_ESTATE",
          -6: "SS_ETIMEOUT", -7: "SS_ETOOBIG"}
SS_NOALLOC_SCRATCH_BYTES = 32 << 20
SS_FP32, SS_FP64 = 0, 1
SS_EULER, SS_HEUN = 0, 1
SS_MAX_BEADS, SS_MAX_SLOTS = 128, 64
SS_CH_AUTO, SS_CH_CROSS, SS_CH_TOTAL, SS_CH_TT, SS_CH_VIRTUAL = 0, 1, 2, 3, 4

# every symbol include/slipspring.h declares
EXPORTS = ["ss_create", "ss_set_params", "ss_set_flow", "ss_run", "ss_stress", "ss_correlator",
           "ss_destroy", "ss_last_error", "ss_get_state", "ss_set_state", "ss_step_count",
           "ss_reset_observables", "ss_corr_sums", "ss_log_sums", "ss_counters", "ss_status",
           "ss_synchronize", "ss_run_noalloc", "ss_kernel_timing", "ss_kernel_time",
           "ss_set_chain_offset", "ss_set_flow_table", "ss_set_batched", "ss_window_forward",
           "ss_window_backward", "ss_set_coefficients", "ss_set_step_count", "ss_corr_sums_tt",
           "ss_get_state_dev", "ss_set_state_dev", "ss_zhist"]


class ss_element(C.Structure):
    _fields_ = [("n_chains", C.c_int32), ("n_beads", C.c_int32)]


class ss_params(C.Structure):
    _fields_ = [("N0", C.c_double), ("Ns", C.c_double), ("zeta_s", C.c_double), ("dt", C.c_double),
                ("b", C.c_double), ("kT", C.c_double), ("zeta", C.c_double), ("k_b", C.c_double),
                ("k_s", C.c_double), ("create_mode", C.c_int32), ("z_max", C.c_int32),
                ("destroy_new", C.c_int32), ("recenter_every", C.c_int32), ("log_every", C.c_int32),
                ("max_logs", C.c_int32), ("corr_levels", C.c_int32), ("groups", C.c_int32),
                ("chunk_steps", C.c_int32), ("corr_tt", C.c_int32), ("integrator", C.c_int32)]


class SlipSpringError(RuntimeError):
    pass


_lib = None


def load(path: str = LIB_PATH):
    """Load the library and declare its signatures (once)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise SlipSpringError(
            "libslipspring.so not found at %s: build it with `python -m paper_1106_2899_gb300.build` "
            "(there is no CPU fallback)" % path)
    lib = C.CDLL(path)
    P = C.POINTER
    vp, dp, i32p, i64p = C.c_void_p, P(C.c_double), P(C.c_int32), P(C.c_int64)
    sig = {
        "ss_create": [P(vp), P(ss_element), C.c_int, C.c_int, C.c_uint64, vp],
        "ss_set_params": [vp, P(ss_params)],
        "ss_set_flow": [vp, C.c_int, C.c_int64, dp],
        "ss_run": [vp, C.c_int64],
        "ss_stress": [vp, C.c_int, dp, dp, dp, C.c_int, P(C.c_int)],
        "ss_correlator": [vp, C.c_int, C.c_int, dp, dp, dp, C.c_int, P(C.c_int)],
        "ss_destroy": [vp],
        "ss_get_state": [vp, C.c_int, dp, i32p, i32p, dp],
        "ss_set_state": [vp, C.c_int, dp, i32p, i32p, dp],
        "ss_step_count": [vp, i64p],
        "ss_reset_observables": [vp],
        "ss_corr_sums": [vp, C.c_int, dp, P(C.c_int), i64p],
        "ss_log_sums": [vp, C.c_int, i64p, dp, C.c_int, P(C.c_int), P(C.c_int)],
        "ss_counters": [vp, i64p],
        "ss_status": [vp, i32p],
        "ss_synchronize": [vp],
        "ss_kernel_timing": [vp, C.c_int],
        "ss_set_chain_offset": [vp, C.c_uint32],
        "ss_set_flow_table": [vp, C.c_int, i32p, i64p, dp],
        "ss_set_batched": [vp, C.c_int],
        "ss_window_forward": [vp, C.c_int64, C.c_int, C.c_int],
        "ss_window_backward": [vp, dp, dp],
        "ss_set_coefficients": [vp, C.c_double, C.c_double, C.c_double],
        "ss_set_step_count": [vp, C.c_int64],
        "ss_corr_sums_tt": [vp, C.c_int, dp, P(C.c_int), i64p],
        "ss_kernel_time": [vp, dp, i64p],
        "ss_get_state_dev": [vp, C.c_int, vp, vp, vp, vp, vp],
        "ss_set_state_dev": [vp, C.c_int, vp, vp, vp, vp, vp],
        "ss_zhist": [vp, C.c_int, i64p, C.c_int, P(C.c_int)],
        "ss_run_noalloc": [P(ss_params), C.c_int, C.c_uint64, C.c_int32, C.c_int32, C.c_uint32, C.c_int64,
                           C.c_int64, dp, vp, vp, vp, vp, vp, vp, vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.ss_last_error.argtypes = [vp]
    lib.ss_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def check(rc: int, ctx=None, what: str = ""):
    if rc != SS_OK:
        msg = ""
        if ctx is not None and _lib is not None:
            msg = (_lib.ss_last_error(ctx) or b"").decode()
        raise SlipSpringError("%s failed: %s %s" % (what, ERRORS.get(rc, rc), msg))
