"""The adjoint workload: 2D Euler gamma = 1.4 on periodic [0, 2]^2 at 1024^2, the smooth wave plus
8 seeded Fourier modes (amplitude 0.05 in rho and P), J = 1/2 sum rho(T)^2 dx dy after 200 SSP-RK3
steps, gradient with respect to the initial state (conserved variables and their derivatives)
through the checkpointed autograd rollout (checkpoints every 20 steps).  Checked against central
differences of J along 16 seeded directions (same recorded dt and alphas), against the oracle's
adjoint at 128^2, and for independence of the checkpoint interval and of keeping every step's stage
inputs instead of checkpoints."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_11229_gb300 import Solver  # noqa: E402
from paper_2411_11229_gb300.adjoint import Rollout, replay  # noqa: E402


def _gradient(n, nsteps, every, keep_stages=False):
    S0n, dx, dy = W.euler2d_adjoint_init(n, seed=4000)
    s = Solver(2, "euler", n, n, dx=dx, dy=dy)
    S0 = torch.as_tensor(S0n, device="cuda").requires_grad_(True)
    ST = Rollout.apply(S0, s, nsteps, every, keep_stages)
    J = 0.5 * (ST[0, 0] ** 2).sum() * dx * dy
    J.backward()
    # the recorded steps, for the replays
    s.set_state(S0n)
    s.set_time(0.0, 0.0)
    rec = torch.empty((nsteps, 7), dtype=torch.float64, device="cuda")
    for k in range(nsteps):
        s.step(0.0)
        s.record(rec[k])
    return S0n, dx, dy, s, S0.grad.detach(), rec


def test_config5_gradient_against_central_differences():
    n, nsteps = 1024, 200
    S0n, dx, dy, s, g, rec = _gradient(n, nsteps, 20)
    dts = rec[:, 0].cpu().numpy()
    S0 = torch.as_tensor(S0n, device="cuda")
    scale = torch.as_tensor(np.abs(S0n).max(axis=(2, 3), keepdims=True), device="cuda")
    J = lambda S: (0.5 * (S[0, 0] ** 2).sum() * dx * dy).item()
    eps = 1e-5
    for k in range(16):
        d = torch.as_tensor(np.random.default_rng(5000 + k).normal(size=S0n.shape), device="cuda") * scale
        fd = (J(replay(S0 + eps * d, s, dts, rec)) - J(replay(S0 - eps * d, s, dts, rec))) / (2 * eps)
        ad = (g * d).sum().item()
        assert abs(ad - fd) <= 1e-6 * abs(ad), (k, ad, fd)


def test_config5_gradient_against_oracle_at_128():
    n, nsteps = 128, 3
    S0n, dx, dy, s, g, rec = _gradient(n, nsteps, 2)
    cfg = O.make_cfg(2, O.EULER, n, n, dx=dx, dy=dy)
    r = rec.cpu().numpy()
    states = [S0n]
    for k in range(nsteps):
        states.append(O.steps_replay(cfg, states[-1], r[k:k + 1, 0], r[k:k + 1, 1:]))
    lam = np.zeros_like(S0n)
    lam[0, 0] = states[-1][0, 0] * dx * dy
    for k in range(nsteps - 1, -1, -1):
        lam = O.adjoint_step(cfg, states[k], r[k, 0], r[k, 1:], lam)
    got = g.cpu().numpy()
    # J depends on the initial derivative fields six orders of magnitude more weakly than on U
    # (max |dJ/dV| ~ 4e-10 against max |dJ/dU| ~ 3e-4 here), so the bar is relative to the max-norm
    # of the whole gradient; each field (U, V, W) must also agree to 1e-8 of its own max-norm.
    assert np.abs(got - lam).max() <= 1e-10 * np.abs(lam).max()
    for f in range(3):
        assert np.abs(got[f] - lam[f]).max() <= 1e-8 * np.abs(lam[f]).max(), f


def test_checkpoint_interval_does_not_change_the_gradient():
    grads = [_gradient(64, 12, every)[4] for every in (1, 5, 12)]
    assert torch.equal(grads[0], grads[1]) and torch.equal(grads[0], grads[2])


def test_kept_stages_give_the_checkpointed_gradient():
    """Keeping every step's input and stage inputs in the forward pass (no replay) gives the
    gradient of the checkpointed rollout bit for bit: the CFL step and its replay with the recorded
    dt and alphas compute the same stage inputs."""
    a = _gradient(64, 12, 5)
    b = _gradient(64, 12, 5, keep_stages=True)
    assert torch.equal(a[4], b[4])
    assert torch.equal(a[5], b[5])


def test_kept_stages_at_1024():
    """The adjoint workload's size with kept stage inputs (0.3 GB per step): the gradient of 40
    steps equals the checkpointed one bit for bit."""
    a = _gradient(1024, 40, 20)[4]
    b = _gradient(1024, 40, 20, keep_stages=True)[4]
    assert torch.equal(a, b)
