"""CPU-side checks of the C-ABI library: it builds, loads without a GPU and
exports every function include/slipspring.h declares; host-side validation
paths that need no device run here too."""
import ctypes as C
import os
import re

import pytest

from paper_1106_2899_gb300 import _native as nat
from paper_1106_2899_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    hdr = open(os.path.join(ROOT, "include", "slipspring.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(ss_[a-z_]+)\s*\(", hdr, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return nat.load()


def test_header_declarations_match_binding():
    assert _declared() == sorted(nat.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_argument_validation_without_device(lib):
    # argument checks that happen before any CUDA call
    h = C.c_void_p()
    el = (nat.ss_element * 1)(nat.ss_element(4, 1))  # N = 1 is not a chain
    assert lib.ss_create(C.byref(h), el, 1, nat.SS_FP32, 0, None) == -1
    el = (nat.ss_element * 1)(nat.ss_element(4, 129))  # longer than this build supports
    assert lib.ss_create(C.byref(h), el, 1, nat.SS_FP32, 0, None) == -1
    el = (nat.ss_element * 1)(nat.ss_element(4, 16))
    assert lib.ss_create(C.byref(h), el, 1, 7, 0, None) == -1  # bad precision
    assert lib.ss_create(None, el, 1, nat.SS_FP32, 0, None) == -1
    assert lib.ss_run(None, 10) == -1
    assert lib.ss_destroy(None) == 0
    assert lib.ss_last_error(None) == b"no context"



def test_empty_and_oversized_ensembles_are_refused(lib):
    h = C.c_void_p()
    assert lib.ss_create(C.byref(h), None, 1, nat.SS_FP32, 0, None) == -1  # no element array
    el = (nat.ss_element * 1)(nat.ss_element(4, 16))
    assert lib.ss_create(C.byref(h), el, 0, nat.SS_FP32, 0, None) == -1  # no elements
    el = (nat.ss_element * 2)(nat.ss_element(4, 16), nat.ss_element(0, 16))  # an element without chains
    assert lib.ss_create(C.byref(h), el, 2, nat.SS_FP32, 0, None) == -1
    el = (nat.ss_element * 1)(nat.ss_element(-3, 16))
    assert lib.ss_create(C.byref(h), el, 1, nat.SS_FP64, 0, None) == -1
    # global chain ids are 32-bit Philox counter words: more than 2^32 chains in all is refused
    el = (nat.ss_element * 3)(*[nat.ss_element(2 ** 31 - 1, 16) for _ in range(3)])
    assert lib.ss_create(C.byref(h), el, 3, nat.SS_FP32, 0, None) == -1
    assert not h.value


def test_noalloc_argument_checks_before_any_device_call(lib):
    p = nat.ss_params()
    one = C.c_void_p(16)  # never dereferenced: every case is refused first

    def call(prec=nat.SS_FP32, M=8, N=16, base=0, t0=0, n=10, kap=None, R=one, params=p):
        return lib.ss_run_noalloc(C.byref(params) if params is not None else None, prec, 0, M, N, base, t0, n,
                                  kap, R, one, one, one, None, None, None)

    assert call(params=None) == -1
    assert call(R=None) == -1
    assert call(prec=5) == -1
    assert call(M=0) == -1 and call(M=-1) == -1  # no chains
    assert call(N=1) == -1 and call(N=129) == -1  # not a chain / longer than supported
    assert call(t0=-1) == -1 and call(n=-1) == -1
    assert call(base=2 ** 32 - 4) == -1  # chain ids past 2^32
    assert call(t0=2 ** 32 - 5, n=10) == -4  # the step counter would wrap
    kap = (C.c_double * 9)(*([0.0] * 8 + [float("nan")]))
    assert call(kap=kap) == -1  # non-finite velocity gradient
    q = nat.ss_params()
    q.log_every = 10
    assert call(params=q) == -1  # stress logs need a context
    q = nat.ss_params()
    q.integrator = nat.SS_HEUN
    assert call(params=q) == -1  # the allocation-free call steps Euler-Maruyama only
