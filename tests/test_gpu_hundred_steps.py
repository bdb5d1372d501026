"""100 SSP-RK3 steps of the 2D Euler workload at 1024^2 (periodic [0, 2]^2, CFL 0.6, gamma 1.4) on
the GPU against the oracle, element by element: the scheme of Eq. (2Dfully-hweno) with the dt of
every step computed on each side from its own state.

Smooth wave (rho = 1 + 0.2 sin(pi (x + y)), velocity (0.7, 0.3), P = 1): within 1e-10 relative
max-norm per (field, component) plane.  Seeded four-quadrant Riemann data (seed 2000): the waves
from the quadrant corners steepen into shocks, which rounding moves by a fraction of a cell, so the
state is compared per plane in the relative L1 norm against ten times the largest drift of that
plane among four oracle runs from inputs moved by one ulp (or 1e-10), and the conserved totals to
round-off; the step count is exact, and the end time (the step sizes follow the largest
wavespeed, found at a shock) within ten times the end-time drift of the same four runs.  The
oracle runs on all host cores (its results do not depend on the thread count).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_11229_gb300 import Solver  # noqa: E402

N = 1024
STEPS = 100


def _gpu_run(S, dx, dy):
    s = Solver(2, "euler", N, N, dx=dx, dy=dy)
    s.set_state(S)
    s.set_time(0.0, 0.0)
    s.step(0.0, STEPS)
    _, t = s.last_dt()
    return s.state.cpu().numpy(), t


def _oracle_run(S, dx, dy):
    O.set_threads(0)
    cfg = O.make_cfg(2, O.EULER, N, N, dx=dx, dy=dy)
    out, n, t = O.run(cfg, S, 0.0, 0.6, 1.0, max_steps=STEPS)
    assert n == STEPS
    return out, t


def _rel_max(a, b):
    a, b = a.reshape(12, -1), b.reshape(12, -1)
    return np.abs(a - b).max(axis=1) / np.maximum(np.abs(b).max(axis=1), 1e-300)


def _rel_l1(a, b):
    a, b = a.reshape(12, -1), b.reshape(12, -1)
    return np.abs(a - b).sum(axis=1) / np.maximum(np.abs(b).sum(axis=1), 1e-300)


def test_smooth_1024_hundred_steps():
    S, dx, dy = W.euler2d_smooth(N)
    gpu, tg = _gpu_run(S, dx, dy)
    ref, t = _oracle_run(S, dx, dy)
    err = _rel_max(gpu, ref)
    print("smooth 1024^2, 100 steps: per-plane relative max-norm", err.max(), "time", tg, t)
    assert abs(tg - t) <= 1e-13 * t, (tg, t)
    assert err.max() <= 1e-10, err


def test_quadrants_1024_hundred_steps():
    S, dx, dy = W.euler2d_quadrants(N, seed=2000)
    gpu, tg = _gpu_run(S, dx, dy)
    ref, t = _oracle_run(S, dx, dy)
    env, env_t = np.zeros(12), 0.0
    for seed in (11, 12, 13, 14):
        sign = np.random.default_rng(seed).choice([-1.0, 1.0], S.shape)
        pert, tp = _oracle_run(S * (1.0 + sign * 2.0 ** -52), dx, dy)
        env = np.maximum(env, _rel_l1(pert, ref))
        env_t = max(env_t, abs(tp - t))
    err = _rel_l1(gpu, ref)
    print("quadrants 1024^2, 100 steps: per-plane relative L1", err, "envelope", env,
          "max-norm", _rel_max(gpu, ref).max(), "time", tg, t, "time envelope", env_t)
    # the step sizes come from the largest wavespeed, which sits at a shock: the end time drifts
    # with the shocks' positions, and is held to the same envelope
    assert abs(tg - t) <= max(1e-12 * t, 10.0 * env_t), (tg, t, env_t)
    assert np.all(err <= np.maximum(1e-10, 10.0 * env)), (err, env)
    for k in range(4):  # periodic: every conserved total agrees to round-off
        tot = np.abs(ref[0, k]).sum()
        assert abs(gpu[0, k].sum() - ref[0, k].sum()) <= 1e-12 * tot
