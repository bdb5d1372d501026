"""Parity of the extended CUDA kernels (hweno_create_ex) with the oracle's variants.

Variants: v^+/- with the nonlinear weights, the D-terms of Eq. (Cd-2), the per-cell
characteristic decomposition (R2), the gravity source of Eq. (euler2d-s), per-side boundary types
with fixed-state sides.  Bars as for the plain scheme: one stage (L, M) and one step within 1e-12
relative max-norm per plane, 100 smooth steps within 1e-10, discontinuous runs within ten times
the oracle's own one-ulp rounding envelope.
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

SYS = {"advection": O.ADVECTION, "burgers": O.BURGERS, "euler": O.EULER}
P, T, R, F = O.BC_PERIODIC, O.BC_TRANSMISSIVE, O.BC_REFLECTIVE, O.BC_FIXED
VW, CD2, R2 = O.FLAG_V_WEIGHTED, O.FLAG_CD2, O.FLAG_R2
AST, ALOC = O.FLAG_ALPHA_STEP, O.FLAG_ALPHA_LOCAL
ALL = VW | CD2 | R2


def rel_planes(a, b):
    nf, nc = b.shape[0], b.shape[1]
    a = a.reshape(nf * nc, -1)
    b = b.reshape(nf * nc, -1)
    den = np.maximum(np.abs(b).max(axis=1), 1e-300)
    return (np.abs(a - b).max(axis=1) / den).max()


def rel_l1_planes(a, b):
    """Per (field, component) plane: sum |a - b| / sum |b| (the plain sum where b's plane is zero)."""
    nf, nc = b.shape[0], b.shape[1]
    a = a.reshape(nf * nc, -1)
    b = b.reshape(nf * nc, -1)
    num = np.abs(a - b).sum(axis=1)
    den = np.abs(b).sum(axis=1)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)


def make_state(dim, system, nx, ny, kind, seed):
    if system == "euler":
        if dim == 1:
            S, dx = W.euler1d_random(nx, seed, kind)
            return S, dx, dx
        return W.euler2d_random(nx, ny, seed, kind)
    return W.scalar_random(dim, nx, ny, seed, kind)


def fixed_states(S, dim):
    """Fixed-side states near the data (mean of the adjacent boundary row, slightly moved)."""
    U = S[0]
    out = {0: U[:, :, 0].mean(axis=1) * 1.05, 1: U[:, :, -1].mean(axis=1) * 0.97}
    if dim == 2:
        out[2] = U[:, 0, :].mean(axis=1) * 1.02
        out[3] = U[:, -1, :].mean(axis=1) * 0.99
    return out


def pair(dim, system, nx, ny, S, dx, dy, flags=0, sides=(P, P, P, P), grav=0.0, fixed=None, gamma=1.4,
         ax=0.8, ay=-0.6):
    cfg = O.make_cfg(dim, SYS[system], nx, ny, dx=dx, dy=dy, gamma=gamma, ax=ax, ay=ay, flags=flags,
                     grav=grav, sides=sides, fixed=fixed)
    s = Solver(dim, system, nx, ny, dx=dx, dy=dy, gamma=gamma, ax=ax, ay=ay, flags=flags, grav=grav,
               sides=sides, fixed=fixed)
    s.set_state(S)
    return cfg, s


CASES = [
    # dim, system, nx, ny, flags, sides
    (1, "burgers", 64, 1, VW, (P, P, P, P)),
    (1, "burgers", 50, 1, VW | CD2, (T, F, P, P)),
    (2, "advection", 29, 23, CD2, (F, T, P, P)),
    (1, "euler", 133, 1, VW, (P, P, P, P)),
    (1, "euler", 130, 1, CD2, (T, T, P, P)),
    (1, "euler", 97, 1, R2, (P, P, P, P)),
    (1, "euler", 96, 1, R2, (T, R, P, P)),
    (1, "euler", 61, 1, ALL, (F, R, P, P)),
    (1, "euler", 6, 1, R2, (R, F, P, P)),
    (2, "euler", 37, 29, VW, (P, P, P, P)),
    (2, "euler", 33, 21, CD2, (T, T, R, R)),
    (2, "euler", 37, 29, R2, (P, P, P, P)),
    (2, "euler", 33, 21, R2, (T, T, T, T)),
    (2, "euler", 31, 26, R2, (R, R, F, F)),
    (2, "euler", 30, 27, ALL, (F, T, R, F)),
    (2, "euler", 6, 9, ALL, (R, R, F, F)),
    (2, "euler", 35, 22, 0, (F, R, P, P)),
    (1, "burgers", 47, 1, ALOC, (T, F, P, P)),
    (1, "euler", 88, 1, ALOC, (F, R, P, P)),
    (2, "euler", 33, 21, ALOC, (P, P, P, P)),
    (2, "euler", 30, 27, ALOC | R2, (R, R, F, F)),
    (2, "euler", 29, 24, AST | ALL, (T, F, R, R)),
]


@pytest.mark.parametrize("kind", ["smooth", "jumps"])
@pytest.mark.parametrize("dim,system,nx,ny,flags,sides", CASES)
def test_rhs_parity(dim, system, nx, ny, flags, sides, kind):
    S, dx, dy = make_state(dim, system, nx, ny, kind, seed=nx * 11 + ny)
    fixed = fixed_states(S, dim) if F in sides else None
    cfg, s = pair(dim, system, nx, ny, S, dx, dy, flags=flags, sides=sides, fixed=fixed)
    L, M = s.rhs()
    Lo, Mo = O.rhs(cfg, S)
    assert rel_planes(L.cpu().numpy(), Lo) <= 1e-12
    assert rel_planes(M.cpu().numpy(), Mo) <= 1e-12


@pytest.mark.parametrize("dim,system,nx,ny,flags,sides", CASES)
def test_one_step_parity(dim, system, nx, ny, flags, sides):
    S, dx, dy = make_state(dim, system, nx, ny, "jumps", seed=nx * 13 + ny)
    fixed = fixed_states(S, dim) if F in sides else None
    cfg, s = pair(dim, system, nx, ny, S, dx, dy, flags=flags, sides=sides, fixed=fixed)
    dt = O.cfl_dt(cfg, S, 0.6)
    s.step(dt)
    ref = O.steps(cfg, S, dt, 1)
    assert rel_planes(s.state.cpu().numpy(), ref) <= 1e-12


@pytest.mark.parametrize("flags", [0, R2, ALL])
def test_gravity_rhs_and_step_parity(flags):
    """Example 4.11's set-up (gamma = 5/3, g = 1, reflective sides, fixed bottom and top) with a
    small smooth x-velocity added (with u = 0 and P independent of x the x-momentum planes are zero
    exactly and hold nothing but each side's rounding), and a hydrostatic column."""
    S, dx, dy, fixed = W.rayleigh_taylor(24, 40)
    x = (np.arange(24) + 0.5) * dx
    y = (np.arange(40) + 0.5) * dy
    S[0, 1] += 0.05 * S[0, 0] * np.sin(8 * np.pi * x)[None, :] * np.cos(2 * np.pi * y)[:, None]
    S[1, 1] += 0.05 * S[0, 0] * 8 * np.pi * np.cos(8 * np.pi * x)[None, :] * np.cos(2 * np.pi * y)[:, None]
    sides = (R, R, F, F)
    cfg, s = pair(2, "euler", 24, 40, S, dx, dy, flags=flags, sides=sides, grav=1.0, fixed=fixed, gamma=5.0 / 3.0)
    L, M = s.rhs()
    Lo, Mo = O.rhs(cfg, S)
    # the y-momentum rate is a near-balance of -dP/dy against g rho (terms a hundred times its
    # size), so its rounding is measured by the oracle's own one-ulp envelope
    envL, envM = _stage_envelope(cfg, S, Lo, Mo)
    assert rel_planes(L.cpu().numpy(), Lo) <= max(1e-12, 10.0 * envL)
    assert rel_planes(M.cpu().numpy(), Mo) <= max(1e-12, 10.0 * envM)
    dt = O.cfl_dt(cfg, S, 0.6)
    s.step(dt)
    ref = O.steps(cfg, S, dt, 1)
    env1 = max(rel_planes(O.steps(cfg, _ulp(S, sd), dt, 1), ref) for sd in range(3))
    assert rel_planes(s.state.cpu().numpy(), ref) <= max(1e-12, 10.0 * env1)
    Sh, dxh, dyh = W.hydrostatic_column(12, 30)
    fx = {2: Sh[0, :, 0, 0], 3: Sh[0, :, -1, 0]}
    cfg, s = pair(2, "euler", 12, 30, Sh, dxh, dyh, flags=flags, sides=(P, P, F, F), grav=1.0, fixed=fx)
    L, _ = s.rhs()
    Lo, _ = O.rhs(cfg, Sh)
    L = L.cpu().numpy()
    # away from the fixed ends both sides balance to round-off; near them they agree per plane
    assert np.abs(L[:, :, 3:-3]).max() <= 1e-10
    assert np.abs(L - Lo).max() <= 1e-12 * max(np.abs(Lo).max(), 1.0)


def _ulp(S, seed):
    """S with every entry moved by one unit in the last place, random signs."""
    sign = np.random.default_rng(100 + seed).choice([-1.0, 1.0], S.shape)
    return S * (1.0 + sign * 2.0 ** -52)


def _stage_envelope(cfg, S, Lo, Mo, seeds=3):
    """How far the oracle's own L and M move when S moves by one ulp."""
    eL = eM = 0.0
    for sd in range(seeds):
        L1, M1 = O.rhs(cfg, _ulp(S, sd))
        eL, eM = max(eL, rel_planes(L1, Lo)), max(eM, rel_planes(M1, Mo))
    return eL, eM


def _l1_envelope(cfg, S, ref, nsteps, seeds=4):
    """Per plane, the largest relative L1 drift of the oracle over four runs from inputs moved by one
    ulp (a plane that holds only rounding, such as the x-momentum of a column at rest in x, drifts
    by its own size, so it is measured against its own noise)."""
    env = np.zeros(ref.shape[0] * ref.shape[1])
    for sd in range(seeds):
        sign = np.random.default_rng(100 + sd).choice([-1.0, 1.0], S.shape)
        out, _, _ = O.run(cfg, S * (1.0 + sign * 2.0 ** -52), 0.0, 0.6, 1.0, max_steps=nsteps)
        env = np.maximum(env, rel_l1_planes(out, ref))
    return env


def _gpu_steps(s, n):
    s.set_time(0.0, 0.0)
    for _ in range(n):
        s.step(0.0)
    return s.state.cpu().numpy()


@pytest.mark.parametrize("flags", [R2, ALL, AST, ALOC, AST | ALOC | R2])
def test_hundred_smooth_steps(flags):
    S, dx, dy = W.euler2d_smooth(40, 32)
    cfg, s = pair(2, "euler", 40, 32, S, dx, dy, flags=flags)
    out = _gpu_steps(s, 100)
    ref, n, _ = O.run(cfg, S, 0.0, 0.6, 1.0, max_steps=100)
    assert n == 100
    assert rel_planes(out, ref) <= 1e-10


@pytest.mark.parametrize("flags", [0, R2, AST | ALOC])
@pytest.mark.parametrize("nsteps", [20, 100])
def test_rayleigh_taylor_run(flags, nsteps):
    """Example 4.11 at 16 x 64: the discontinuous interface amplifies rounding, so every plane is
    compared in the relative L1 norm against ten times its largest drift over four oracle runs from
    one-ulp perturbed inputs (or 1e-10)."""
    S, dx, dy, fixed = W.rayleigh_taylor(16)
    cfg, s = pair(2, "euler", 16, 64, S, dx, dy, flags=flags, sides=(R, R, F, F), grav=1.0, fixed=fixed,
                  gamma=5.0 / 3.0)
    out = _gpu_steps(s, nsteps)
    ref, n, _ = O.run(cfg, S, 0.0, 0.6, 1.0, max_steps=nsteps)
    assert n == nsteps
    env = _l1_envelope(cfg, S, ref, nsteps)
    err = rel_l1_planes(out, ref)
    print("Rayleigh-Taylor", flags, nsteps, "L1 per plane", err.max(), "envelope", env.max())
    assert np.all(err <= np.maximum(1e-10, 10.0 * env)), (err, env)
    # the total mass of both sides agrees to round-off
    assert abs(out[0, 0].sum() - ref[0, 0].sum()) <= 1e-12 * np.abs(ref[0, 0]).sum()
