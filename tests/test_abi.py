"""The C ABI library: it loads, exports every entry point include/hweno.h declares, and validates
arguments on the host (no device work is issued by these calls)."""
import ctypes
import os
import re

import pytest

from paper_2411_11229_gb300 import _capi as C

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "hweno.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hweno_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    lib = C.load()
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
        assert n in C.SIGNATURES, n


def _create(*args):
    h = ctypes.c_void_p()
    rc = C.load().hweno_create(*args, ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("args", [
    (3, 2, 64, 64, 0.1, 0.1, 1.4, 0),     # dim
    (1, 7, 64, 1, 0.1, 0.1, 1.4, 0),      # system
    (1, 2, 4, 1, 0.1, 0.1, 1.4, 0),       # nx < 5
    (2, 2, 64, 3, 0.1, 0.1, 1.4, 0),      # ny < 5
    (1, 2, 64, 1, -0.1, 0.1, 1.4, 0),     # dx <= 0
    (1, 2, 64, 1, 0.1, 0.1, 1.0, 0),      # gamma <= 1
    (1, 2, 64, 1, 0.1, 0.1, 1.4, 9),      # bc
])
def test_create_rejects_invalid(args):
    rc, h = _create(*args)
    assert rc == C.HWENO_EINVAL and not h.value


def test_sizes_and_params():
    lib = C.load()
    rc, h = _create(2, C.HWENO_EULER, 40, 30, 0.05, 0.05, 1.4, C.HWENO_BC_PERIODIC)
    assert rc == 0
    try:
        assert lib.hweno_state_doubles(h) == 3 * 4 * 40 * 30
        ws = lib.hweno_workspace_bytes(h)
        assert ws >= 8 * (3 * 4 + 2 * 4 + 2 * 3 * 4 + 4) * 40 * 30
        assert lib.hweno_set_params(h, 1.5, 0.9, 1e-10, 0.6, 1, 1) == C.HWENO_EINVAL
        assert lib.hweno_set_params(h, 0.9, 0.9, 0.0, 0.6, 1, 1) == C.HWENO_EINVAL
        assert lib.hweno_set_params(h, 0.9, 0.9, 1e-10, 0.6, 1, 1) == C.HWENO_OK
        # no state bound yet: calls that need one report ESTATE without touching the device
        assert lib.hweno_step(h, 0.1) == C.HWENO_ESTATE
        assert lib.hweno_rhs(h, 8, 16, 24) == C.HWENO_ESTATE
        assert lib.hweno_bind(h, None, None) == C.HWENO_EINVAL
        assert lib.hweno_launch_count(h) == 0
    finally:
        lib.hweno_destroy(h)
    assert lib.hweno_strerror(C.HWENO_ENONPHYS).startswith(b"non-physical")
