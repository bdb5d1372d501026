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
    (1, 2, (1 << 28) + 1, 1, 0.1, 0.1, 1.4, 0),    # nx beyond the largest axis
    (2, 2, 1 << 16, (1 << 15) + 1, 0.1, 0.1, 1.4, 0),  # nx * ny beyond 2^31 cells
    (2, 2, 64, 64, float("inf"), 0.1, 1.4, 0),     # non-finite spacing
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


def _ext(flags=0, sides=(0, 0, 0, 0), grav=0.0, fixed=None):
    e = C.HwenoExt()
    e.flags = flags
    for k, t in enumerate(sides):
        e.side[k] = t
    e.grav = grav
    for k, U in (fixed or {}).items():
        for j, u in enumerate(U):
            e.fixed[k][j] = u
    return e


def _create_ex(dim, system, e, nx=40, ny=30):
    h = ctypes.c_void_p()
    rc = C.load().hweno_create_ex(dim, system, nx, ny, 0.05, 0.05, 1.4, ctypes.byref(e), ctypes.byref(h))
    return rc, h


P, T, R, F = C.HWENO_BC_PERIODIC, C.HWENO_BC_TRANSMISSIVE, C.HWENO_BC_REFLECTIVE, C.HWENO_BC_FIXED


@pytest.mark.parametrize("dim,system,e", [
    (2, C.HWENO_EULER, _ext(flags=32)),                                       # unknown flag
    (2, C.HWENO_EULER, _ext(sides=(P, T, P, P))),                             # periodic on one end
    (2, C.HWENO_EULER, _ext(sides=(P, P, T, P))),
    (2, C.HWENO_EULER, _ext(sides=(P, P, 4, 4))),                             # unknown type
    (2, C.HWENO_BURGERS, _ext(sides=(R, R, P, P))),                           # reflective scalar
    (1, C.HWENO_EULER, _ext(grav=1.0)),                                       # gravity in 1D
    (2, C.HWENO_BURGERS, _ext(grav=1.0)),                                     # gravity, scalar
    (2, C.HWENO_EULER, _ext(sides=(F, T, P, P), fixed={0: [-1.0, 0, 0, 2.5]})),  # rho <= 0
    (2, C.HWENO_EULER, _ext(sides=(F, T, P, P), fixed={0: [1.0, 3.0, 0, 1.0]})),  # P <= 0
])
def test_create_ex_rejects_invalid(dim, system, e):
    rc, h = _create_ex(dim, system, e)
    assert rc == C.HWENO_EINVAL and not h.value


def test_create_ex_sizes_and_adjoint_refusal():
    """R2 keeps four face states per cell and direction (and those of the line-end ghosts); the
    plain configuration keeps the plain workspace; the adjoint refuses extended handles."""
    lib = C.load()
    rc0, h0 = _create(2, C.HWENO_EULER, 40, 30, 0.05, 0.05, 1.4, C.HWENO_BC_PERIODIC)
    rc1, h1 = _create_ex(2, C.HWENO_EULER, _ext())                     # plain, through the ex entry
    rc2, h2 = _create_ex(2, C.HWENO_EULER, _ext(flags=C.HWENO_FLAG_R2))
    rc3, h3 = _create_ex(2, C.HWENO_EULER, _ext(flags=C.HWENO_FLAG_CD2, grav=1.0))
    try:
        assert rc0 == rc1 == rc2 == rc3 == 0
        w0, w1, w2, w3 = (lib.hweno_workspace_bytes(h) for h in (h0, h1, h2, h3))
        assert w0 == w1 == w3
        assert w2 >= w0 + 8 * 2 * 4 * 4 * 40 * 30
        for h in (h2, h3):
            assert lib.hweno_adjoint_step(h, 8, 0.1, 16, 24, 32, 256) == C.HWENO_EINVAL
            assert lib.hweno_stage_vjp(h, 8, 16, 24, 32, 40, 256) == C.HWENO_EINVAL
    finally:
        for h in (h0, h1, h2, h3):
            lib.hweno_destroy(h)


def test_pipeline_and_stage_copy_refuse_invalid_arguments_on_the_host():
    """hweno_pipeline and hweno_step_stages check their arguments before any device work; the
    bounds-check entry points report -1 in the normal build."""
    lib = C.load()
    rc, h = _create(2, C.HWENO_EULER, 40, 30, 0.05, 0.05, 1.4, C.HWENO_BC_PERIODIC)
    assert rc == 0
    try:
        state = lib.hweno_state_doubles(h) * 8
        assert lib.hweno_pipeline_slot_bytes(h) == ((state + 255) // 256) * 256 + lib.hweno_workspace_bytes(h)
        assert lib.hweno_pipeline_slot_bytes(None) == 0
        fake = ctypes.c_void_p(1 << 20)  # never dereferenced: every call below fails validation
        one = (ctypes.c_void_p * 1)(1 << 21)
        nul = (ctypes.c_void_p * 1)(None)
        P = lib.hweno_pipeline
        assert P(None, 1, one, one, 1, 2, fake) == C.HWENO_EINVAL
        assert P(h, -1, one, one, 1, 2, fake) == C.HWENO_EINVAL
        assert P(h, 1, one, one, -1, 2, fake) == C.HWENO_EINVAL
        assert P(h, 1, one, one, 1, 0, fake) == C.HWENO_EINVAL
        assert P(h, 1, one, one, 1, 9, fake) == C.HWENO_EINVAL
        assert P(h, 1, one, one, 1, 2, None) == C.HWENO_EINVAL
        assert P(h, 1, one, one, 1, 2, ctypes.c_void_p((1 << 20) + 8)) == C.HWENO_EINVAL
        assert P(h, 1, None, one, 1, 2, fake) == C.HWENO_EINVAL
        assert P(h, 1, one, nul, 1, 2, fake) == C.HWENO_EINVAL
        S = lib.hweno_step_stages
        assert S(h, 0.0, None, fake) == C.HWENO_EINVAL
        assert S(h, float("nan"), fake, fake) == C.HWENO_EINVAL
        assert S(h, 0.0, fake, fake) == C.HWENO_ESTATE  # nothing bound
        where = ctypes.c_int(7)
        assert lib.hweno_bounds_status(ctypes.byref(where)) == -1 and where.value == 0
        assert lib.hweno_bounds_selftest() == -1
    finally:
        lib.hweno_destroy(h)
