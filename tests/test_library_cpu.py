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

