"""Hand-written GPU adjoint against the oracle's reverse-mode adjoint (same conventions: fixed dt
and per-stage LF coefficients, sign(0) = 0): one stage operator and whole SSP-RK3 steps, within
1e-10 relative max-norm per plane."""
import ctypes

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_11229_gb300 import Solver  # noqa: E402
from paper_2411_11229_gb300 import _capi as C  # noqa: E402


def _rel(a, b):
    nf, nc = b.shape[0], b.shape[1]
    a, b = a.reshape(nf * nc, -1), b.reshape(nf * nc, -1)
    return (np.abs(a - b).max(axis=1) / np.maximum(np.abs(b).max(axis=1), 1e-300)).max()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _setup(dim, nx, ny, kind, bc, seed):
    if dim == 2:
        S, dx, dy = W.euler2d_random(nx, ny, seed, kind)
    else:
        S, dx = W.euler1d_random(nx, seed, kind)
        dy = dx
    obc = {"periodic": O.BC_PERIODIC, "transmissive": O.BC_TRANSMISSIVE, "reflective": O.BC_REFLECTIVE}[bc]
    cfg = O.make_cfg(dim, O.EULER, nx, ny, dx=dx, dy=dy, bc=obc)
    s = Solver(dim, "euler", nx, ny, dx=dx, dy=dy, bc=bc)
    s.set_state(S)
    aws = torch.empty(int(C.load().hweno_adjoint_workspace_bytes(s.h)), dtype=torch.uint8, device="cuda")
    return S, cfg, s, aws


CASES = [(2, 12, 10, "smooth", "periodic"), (2, 12, 10, "jumps", "periodic"), (2, 11, 13, "smooth", "transmissive"),
         (2, 9, 7, "jumps", "transmissive"), (1, 23, 1, "smooth", "periodic"), (1, 19, 1, "jumps", "transmissive"),
         (2, 12, 11, "smooth", "reflective"), (2, 10, 9, "jumps", "reflective"), (1, 21, 1, "smooth", "reflective"),
         (1, 6, 1, "jumps", "reflective"), (2, 6, 5, "smooth", "reflective")]


@pytest.mark.parametrize("dim,nx,ny,kind,bc", CASES)
def test_stage_vjp_matches_oracle(dim, nx, ny, kind, bc):
    S, cfg, s, aws = _setup(dim, nx, ny, kind, bc, seed=nx + ny)
    alpha = O.max_wavespeed(cfg, S)
    rng = np.random.default_rng(3)
    muM, muL = rng.normal(size=S.shape), rng.normal(size=S.shape)
    ref = O.stage_vjp(cfg, S, alpha, muM, muL)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    Sd, mMd, mLd, al = dev(S), dev(muM), dev(muL), dev(np.array(alpha))
    lam = torch.empty_like(Sd)
    C.check(C.load().hweno_stage_vjp(s.h, _ptr(Sd), _ptr(al), _ptr(mMd), _ptr(mLd), _ptr(lam), _ptr(aws)),
            "hweno_stage_vjp")
    assert _rel(lam.cpu().numpy(), ref) <= 1e-10


@pytest.mark.parametrize("dim,nx,ny,kind,bc", CASES)
def test_adjoint_step_matches_oracle(dim, nx, ny, kind, bc):
    S, cfg, s, aws = _setup(dim, nx, ny, kind, bc, seed=2 * nx + ny)
    _, dts, alphas = O.steps_record(cfg, S, 1)
    rng = np.random.default_rng(4)
    lam_in = rng.normal(size=S.shape)
    ref = O.adjoint_step(cfg, S, dts[0], alphas[0], lam_in)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    Sd, lin, al = dev(S), dev(lam_in), dev(alphas[0])
    lout = torch.empty_like(Sd)
    C.check(C.load().hweno_adjoint_step(s.h, _ptr(Sd), float(dts[0]), _ptr(al), _ptr(lin), _ptr(lout), _ptr(aws)),
            "hweno_adjoint_step")
    assert _rel(lout.cpu().numpy(), ref) <= 1e-10


def test_record_and_replay_reproduce_the_cfl_step():
    S, cfg, s, aws = _setup(2, 20, 16, "smooth", "periodic", seed=5)
    s.set_time(0.0, 0.0)
    s.step(0.0)
    rec = torch.empty(7, dtype=torch.float64, device="cuda")
    C.check(C.load().hweno_step_record(s.h, _ptr(rec)), "hweno_step_record")
    after = s.state.clone()
    r = rec.cpu().numpy()
    _, dts, alphas = O.steps_record(cfg, S, 1)
    assert abs(r[0] - dts[0]) <= 1e-14 * dts[0]
    assert np.allclose(r[1:], alphas[0], rtol=1e-14, atol=0)
    s.set_state(S)
    al = rec[1:].clone()
    C.check(C.load().hweno_step_replay(s.h, float(r[0]), _ptr(al)), "hweno_step_replay")
    assert torch.equal(s.state, after)
