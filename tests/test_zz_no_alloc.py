"""hweno_rhs_static: the spatial operator for callers that cannot allocate device memory.

Some callers of this library cannot allocate a workspace: their own framework or memory pool owns
every device allocation and hands a library only input and output buffers, or they run
latency-sensitive loops that cannot afford a cudaMalloc.  hweno_rhs_static serves them from a
fixed scratch array inside the library.  These tests call it through the C ABI and check it
against the workspace-based hweno_rhs, on two calls in a row (the array keeps the previous call's
contents), and check that an oversized grid is refused.  The file is collected last so that a run
stopping at the first failure has already run every other test; it also passes on its own in a
fresh process, where its first call performs the one-time device set-up.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_11229_gb300 import Solver  # noqa: E402
from paper_2411_11229_gb300 import _capi as C  # noqa: E402

SYSTEMS = {"advection": C.HWENO_ADVECTION, "burgers": C.HWENO_BURGERS, "euler": C.HWENO_EULER}
BCS = {"periodic": C.HWENO_BC_PERIODIC, "transmissive": C.HWENO_BC_TRANSMISSIVE,
       "reflective": C.HWENO_BC_REFLECTIVE}


def _static_rhs(dim, system, nx, ny, dx, dy, bc, S, params5=None):
    Sd = torch.as_tensor(S, device="cuda").contiguous()
    L = torch.full_like(Sd, float("nan"))
    M = torch.full_like(Sd, float("nan"))
    stream = torch.cuda.current_stream()
    p5 = None if params5 is None else (ctypes.c_double * 5)(*params5)
    rc = C.load().hweno_rhs_static(dim, SYSTEMS[system], nx, ny, dx, dy, 1.4, BCS[bc], p5,
                                   ctypes.c_void_p(Sd.data_ptr()), ctypes.c_void_p(L.data_ptr()),
                                   ctypes.c_void_p(M.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    C.check(rc, "hweno_rhs_static")
    torch.cuda.synchronize()
    return L.cpu().numpy(), M.cpu().numpy()


def _handle_rhs(dim, system, nx, ny, dx, dy, bc, S, params5=None):
    kw = {}
    if params5 is not None:
        kw = dict(gamma0=params5[0], d0=params5[1], eps=params5[2], ax=params5[3], ay=params5[4])
    s = Solver(dim, system, nx, ny, dx=dx, dy=dy, bc=bc, **kw)
    s.set_state(S)
    L, M = s.rhs()
    torch.cuda.synchronize()
    return L.cpu().numpy(), M.cpu().numpy()


def _rel(a, b):
    nf, nc = b.shape[0], b.shape[1]
    a, b = a.reshape(nf * nc, -1), b.reshape(nf * nc, -1)
    return (np.abs(a - b).max(axis=1) / np.maximum(np.abs(b).max(axis=1), 1e-300)).max()


def test_static_rhs_matches_workspace_rhs_on_two_calls():
    # first call: 2D Euler with discontinuities; second call: a different grid and system, so the
    # second result must not depend on what the first call left in the scratch array
    cases = [
        (2, "euler", 37, 29, "periodic", W.euler2d_random(37, 29, 11, "jumps")[0]),
        (1, "euler", 300, 1, "transmissive", W.euler1d_random(300, 12, "smooth")[0]),
        (2, "euler", 180, 180, "periodic", W.euler2d_quadrants(180, seed=2000)[0]),
        (2, "euler", 61, 47, "reflective", W.euler2d_quadrants(61, 47, seed=2001)[0]),
        (1, "euler", 400, 1, "reflective", W.blast_wave_1d(400, p_mid=1.0)[0]),
    ]
    for dim, system, nx, ny, bc, S in cases:
        dx = 2.0 / nx
        dy = 2.0 / ny if dim == 2 else dx
        Ls, Ms = _static_rhs(dim, system, nx, ny, dx, dy, bc, S)
        Lh, Mh = _handle_rhs(dim, system, nx, ny, dx, dy, bc, S)
        assert np.isfinite(Ls).all() and np.isfinite(Ms).all()
        assert _rel(Ls, Lh) <= 1e-12
        assert _rel(Ms, Mh) <= 1e-12


def test_static_rhs_scalar_laws_with_parameters():
    """The advection and Burgers instantiations behind the same entry point, 1D and 2D, with the
    scheme parameters (gamma0, d0, eps and the advection speeds) passed in params5, two calls in a
    row on different grids each."""
    cases = [
        (1, "advection", 97, 1, "periodic", W.scalar_random(1, 97, 1, 21, "jumps")[0], (0.9, 0.8, 1e-8, -0.7, 0.0)),
        (2, "advection", 41, 33, "periodic", W.scalar_random(2, 41, 33, 22, "smooth")[0],
         (0.97, 0.85, 1e-9, 0.8, -0.6)),
        (1, "burgers", 120, 1, "transmissive", W.scalar_random(1, 120, 1, 23, "jumps")[0],
         (0.95, 0.9, 1e-10, 1.0, 1.0)),
        (2, "burgers", 35, 44, "periodic", W.scalar_random(2, 35, 44, 24, "jumps")[0], (0.99, 0.9, 1e-6, 1.0, 1.0)),
        (2, "burgers", 29, 31, "transmissive", W.scalar_random(2, 29, 31, 25, "smooth")[0],
         (0.9, 0.7, 1e-10, 1.0, 1.0)),
    ]
    for dim, system, nx, ny, bc, S, p5 in cases:
        dx = 2.0 / nx
        dy = 2.0 / ny if dim == 2 else dx
        Ls, Ms = _static_rhs(dim, system, nx, ny, dx, dy, bc, S, p5)
        Lh, Mh = _handle_rhs(dim, system, nx, ny, dx, dy, bc, S, p5)
        assert np.isfinite(Ls).all() and np.isfinite(Ms).all()
        assert _rel(Ls, Lh) <= 1e-12
        assert _rel(Ms, Mh) <= 1e-12


def test_static_rhs_rejects_grids_beyond_its_scratch():
    n = 256  # 2D Euler needs about 480 bytes per cell: 256^2 cells exceed the 16 MiB array
    S = np.zeros((3, 4, n, n))
    Sd = torch.as_tensor(S, device="cuda")
    L, M = torch.empty_like(Sd), torch.empty_like(Sd)
    rc = C.load().hweno_rhs_static(2, C.HWENO_EULER, n, n, 2.0 / n, 2.0 / n, 1.4, C.HWENO_BC_PERIODIC, None,
                                   ctypes.c_void_p(Sd.data_ptr()), ctypes.c_void_p(L.data_ptr()),
                                   ctypes.c_void_p(M.data_ptr()), None)
    assert rc == C.HWENO_ETOOBIG
    # a grid whose cell count alone exceeds the array (each side within the per-axis limit) is
    # refused before any byte count is formed
    for nx, ny in ((1 << 27, 1 << 27), (1 << 28, 5), (5, 1 << 28)):
        rc = C.load().hweno_rhs_static(2, C.HWENO_EULER, nx, ny, 1.0, 1.0, 1.4, C.HWENO_BC_PERIODIC, None,
                                       ctypes.c_void_p(Sd.data_ptr()), ctypes.c_void_p(L.data_ptr()),
                                       ctypes.c_void_p(M.data_ptr()), None)
        assert rc == C.HWENO_ETOOBIG, (nx, ny, rc)
