"""Pins of the oracle's derivatives (adjoint conventions: the step sizes and the LF coefficients of
every stage held at recorded values).

The operator is strongly curved at the scale of 1e-6 relative perturbations (the nonlinear
weights respond to the smoothness indicators on the scale of eps = 1e-10): plain central
differences with a 1e-6 step carry 1e-3 errors here and fall off exactly as step^2.  The
differences below are therefore fourth-order (Richardson: (8 (f(e) - f(-e)) - (f(2e) - f(-2e))) / 12e)
with e = 1e-7.

* forward mode (dual numbers through the templated oracle) against central differences of the
  plain FP64 operator;
* reverse mode (per-face and per-cell tapes) against forward mode: the dot-product identity
  <mu, J delta> = <J^T mu, delta> for one stage;
* the gradient of J = 1/2 sum rho(T)^2 dx dy over several SSP-RK3 steps (adjoint steps backwards
  through recorded states) against central differences of J in the same replay mode.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W


def _cases():
    S1, dx, dy = W.euler2d_random(12, 10, 21, "jumps")
    S2, dx2, dy2 = W.euler2d_random(11, 13, 22, "smooth")
    S3, dx3 = W.euler1d_random(17, 23, "jumps")
    S4, dx4, _ = W.scalar_random(2, 9, 8, 24, "smooth")
    S5, dx5, dy5 = W.euler2d_random(11, 9, 25, "jumps")
    return [
        (O.make_cfg(2, O.EULER, 12, 10, dx=dx, dy=dy), S1),
        (O.make_cfg(2, O.EULER, 11, 13, dx=dx2, dy=dy2, bc=O.BC_TRANSMISSIVE), S2),
        (O.make_cfg(1, O.EULER, 17, dx=dx3, bc=O.BC_TRANSMISSIVE), S3),
        (O.make_cfg(2, O.BURGERS, 9, 8, dx=dx4, dy=dx4), S4),
        (O.make_cfg(2, O.EULER, 11, 9, dx=dx5, dy=dy5, bc=O.BC_REFLECTIVE), S5),
    ]


@pytest.mark.parametrize("case", [1, 3])
def test_jvp_matches_central_differences(case):
    """Smooth data only: on the blocky data (random derivative noise inside constant blocks) the
    weights sit where tau / (beta + eps) has curvature of order 1/eps^2 and no practical step
    resolves it; there the reverse mode is pinned by the dot-product identity alone."""
    cfg, S = _cases()[case]
    alpha = O.max_wavespeed(cfg, S)
    rng = np.random.default_rng(case)
    delta = rng.normal(size=S.shape) * np.abs(S).max(axis=(2, 3), keepdims=True)
    jM, jL = O.stage_jvp(cfg, S, alpha, delta)
    eps = 1e-7
    f = lambda e: O.rhs(cfg, S + e * delta, alpha=alpha)
    (L1, M1), (L2, M2), (L3, M3), (L4, M4) = f(eps), f(-eps), f(2 * eps), f(-2 * eps)
    fdL = (8 * (L1 - L2) - (L3 - L4)) / (12 * eps)
    fdM = (8 * (M1 - M2) - (M3 - M4)) / (12 * eps)
    assert np.abs(jL - fdL).max() <= 1e-6 * np.abs(fdL).max()
    assert np.abs(jM - fdM).max() <= 1e-6 * np.abs(fdM).max()


@pytest.mark.parametrize("case", range(5))
def test_vjp_dot_product_identity(case):
    cfg, S = _cases()[case]
    alpha = O.max_wavespeed(cfg, S)
    rng = np.random.default_rng(10 + case)
    delta = rng.normal(size=S.shape)
    muM = rng.normal(size=S.shape)
    muL = rng.normal(size=S.shape)
    jM, jL = O.stage_jvp(cfg, S, alpha, delta)
    lam = O.stage_vjp(cfg, S, alpha, muM, muL)
    lhs = np.vdot(muM, jM) + np.vdot(muL, jL)
    rhs = np.vdot(lam, delta)
    scale = np.abs(muM * jM).sum() + np.abs(muL * jL).sum()
    assert abs(lhs - rhs) <= 1e-13 * scale, (lhs, rhs)


def _J(S, dx, dy):
    return 0.5 * np.sum(S[0, 0] ** 2) * dx * dy


def test_multistep_gradient_matches_central_differences():
    """32^2 grid, 3 steps; each direction scaled per plane.  The fourth-order difference is taken
    at two steps (1e-7, 5e-8) and the closer one must be within 1e-6 (truncation error falls and
    rounding error grows as the step shrinks; the better of the two is the estimate)."""
    n, nsteps = 32, 3
    S0, dx, dy = W.euler2d_adjoint_init(n, seed=4000)
    cfg = O.make_cfg(2, O.EULER, n, n, dx=dx, dy=dy)
    # forward pass: record dt and alpha, keep the state at every step
    states = [S0]
    dts, alphas = [], []
    S = S0
    for _ in range(nsteps):
        S, d, a = O.steps_record(cfg, S, 1)
        states.append(S)
        dts.append(d[0])
        alphas.append(a[0])
    # backward pass
    lam = np.zeros_like(S)
    lam[0, 0] = states[-1][0, 0] * dx * dy
    for k in range(nsteps - 1, -1, -1):
        lam = O.adjoint_step(cfg, states[k], dts[k], alphas[k], lam)
    rng = np.random.default_rng(5000)
    dts, alphas = np.array(dts), np.array(alphas)
    for _ in range(4):
        d = rng.normal(size=S0.shape) * np.abs(S0).max(axis=(2, 3), keepdims=True)
        f = lambda e: _J(O.steps_replay(cfg, S0 + e * d, dts, alphas), dx, dy)
        ad = np.vdot(lam, d)
        err = min(abs(ad - (8 * (f(e) - f(-e)) - (f(2 * e) - f(-2 * e))) / (12 * e)) for e in (1e-7, 5e-8))
        assert err <= 1e-6 * abs(ad), (ad, err)
