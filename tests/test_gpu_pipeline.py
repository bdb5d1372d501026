"""hweno_pipeline: independent problems host memory to host memory on several device slots in turn.
Each problem's result equals, bit for bit, the same problem stepped on its own (upload, CFL steps,
download on one handle); a non-physical problem is reported; invalid arguments are refused on the
host before any device work."""
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


def _problems(count, nx, ny):
    out = []
    for k in range(count):
        S, dx, dy = W.euler2d_random(nx, ny, 700 + k, "jumps" if k % 2 else "smooth")
        out.append(torch.from_numpy(np.ascontiguousarray(S)).pin_memory())
    return out, dx, dy


@pytest.mark.parametrize("depth", [1, 2, 3])
@pytest.mark.parametrize("flags", [0, C.HWENO_FLAG_R2])
def test_pipeline_matches_single_problems(depth, flags):
    nx, ny, nsteps = 37, 29, 2
    ins, dx, dy = _problems(7, nx, ny)
    outs = [torch.empty_like(t).pin_memory() for t in ins]
    s = Solver(2, "euler", nx, ny, dx=dx, dy=dy, bc="transmissive", flags=flags)
    s.pipeline(ins, outs, nsteps, depth)
    for k, S in enumerate(ins):
        r = Solver(2, "euler", nx, ny, dx=dx, dy=dy, bc="transmissive", flags=flags)
        r.set_state(S)
        r.set_time(0.0, 0.0)
        r.step(0.0, nsteps)
        assert torch.equal(outs[k], r.state.cpu()), k


def test_pipeline_in_place_and_reuse():
    """host_out[i] = host_in[i], and a second call on the same slots."""
    nx = 200
    S, dx = W.euler1d_random(nx, 5, "jumps")
    a = torch.from_numpy(np.ascontiguousarray(S)).pin_memory()
    b = a.clone().pin_memory()
    s = Solver(1, "euler", nx, dx=dx, bc="transmissive")
    s.pipeline([a], [a], 3, 2)
    s.pipeline([b], [b], 1, 2)
    s.pipeline([b], [b], 2, 2)
    assert torch.equal(a, b)


def test_pipeline_reports_a_non_physical_problem():
    nx, ny = 12, 10
    ins, dx, dy = _problems(3, nx, ny)
    ins[1][0, 0, 4, 5] = -1.0  # negative density planted on the host
    outs = [torch.empty_like(t).pin_memory() for t in ins]
    s = Solver(2, "euler", nx, ny, dx=dx, dy=dy)
    with pytest.raises(C.HwenoError) as e:
        s.pipeline(ins, outs, 1, 2)
    assert e.value.code == C.HWENO_ENONPHYS


def test_pipeline_refuses_invalid_arguments():
    nx, ny = 12, 10
    ins, dx, dy = _problems(1, nx, ny)
    outs = [torch.empty_like(ins[0]).pin_memory()]
    s = Solver(2, "euler", nx, ny, dx=dx, dy=dy)
    lib = C.load()
    mem = torch.empty(2 * int(lib.hweno_pipeline_slot_bytes(s.h)) + 512, dtype=torch.uint8, device="cuda")
    pin = (ctypes.c_void_p * 1)(ins[0].data_ptr())
    pout = (ctypes.c_void_p * 1)(outs[0].data_ptr())
    base = mem.data_ptr()
    assert lib.hweno_pipeline(s.h, 1, pin, pout, 1, 0, ctypes.c_void_p(base)) == C.HWENO_EINVAL
    assert lib.hweno_pipeline(s.h, 1, pin, pout, 1, 9, ctypes.c_void_p(base)) == C.HWENO_EINVAL
    assert lib.hweno_pipeline(s.h, 1, pin, pout, -1, 2, ctypes.c_void_p(base)) == C.HWENO_EINVAL
    assert lib.hweno_pipeline(s.h, 1, pin, pout, 1, 2, ctypes.c_void_p(base + 8)) == C.HWENO_EINVAL
    assert lib.hweno_pipeline(s.h, 1, pin, pout, 1, 2, None) == C.HWENO_EINVAL
    nul = (ctypes.c_void_p * 1)(None)
    assert lib.hweno_pipeline(s.h, 1, nul, pout, 1, 2, ctypes.c_void_p(base)) == C.HWENO_EINVAL
    assert lib.hweno_pipeline(s.h, 0, None, None, 1, 2, ctypes.c_void_p(base)) == C.HWENO_OK
