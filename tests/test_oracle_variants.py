"""Pins of the oracle's scheme variants and extensions (no GPU).

* Eq. (Cd-2): re-derived with sympy from the Hermite interpolant (Pc2) it comes from, and exact
  for quintic fluxes;
* v^+/- with the nonlinear weights: reduces to p0' where the weights are linear, and to the slope
  of the smooth sub-stencil at a jump;
* every variant keeps fifth order on the smooth 1D Euler problem of Example 4.2;
* the gravity source of Eq. (euler2d-s): its value on uniform flow and the balance of a
  hydrostatic column (the discrete pressure gradient of a linear pressure is exact);
* fixed-state sides: one stage equals that of a larger grid whose extra cells hold the state;
* the adjoint identity with all of the above switched on;
* the Rayleigh-Taylor set-up of Example 4.11 runs.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

sp = pytest.importorskip("sympy")


# ------------------------------------------------------------------------------------------------
# Eq. (Cd-2)

def test_cd2_matches_degree5_hermite_pc2():
    """Eqs. (Pc2), (Cd-2), (DfDh): D-terms from the degree-5 interpolant with h at x_i, x_{i+1}."""
    x, h = sp.symbols("x h", positive=True)
    f = sp.symbols("f0:4")
    h0, h1 = sp.symbols("h0 h1")
    c = sp.symbols("c0:6")
    P = sum(c[k] * x ** k for k in range(6))
    nodes = [-h, 0, h, 2 * h]
    eqs = [P.subs(x, nodes[q]) - f[q] for q in range(4)]
    eqs += [sp.diff(P, x).subs(x, 0) - h0, sp.diff(P, x).subs(x, h) - h1]
    P = P.subs(sp.solve(eqs, c))
    xh = h / 2
    Df = -sp.Rational(1, 24) * h ** 2 * sp.diff(P, x, 2).subs(x, xh) + \
        sp.Rational(7, 5760) * h ** 4 * sp.diff(P, x, 4).subs(x, xh)
    Dh = -sp.Rational(1, 24) * h ** 2 * sp.diff(P, x, 3).subs(x, xh) + \
        sp.Rational(7, 5760) * h ** 4 * sp.diff(P, x, 5).subs(x, xh)
    fDf = sp.lambdify((h,) + f + (h0, h1), Df, "math")
    fDh = sp.lambdify((h,) + f + (h0, h1), Dh, "math")
    rng = np.random.default_rng(14)
    for _ in range(50):
        hh = float(rng.uniform(0.01, 1.0))
        ff = rng.normal(size=4)
        hv = rng.normal(size=2)
        got = O.dterms(ff, hv, hh, form=2)
        ref = (fDf(hh, *ff, *hv), fDh(hh, *ff, *hv))
        sc = 1 + np.abs(ff).max() + hh * np.abs(hv).max()
        assert abs(got[0] - ref[0]) <= 1e-13 * sc
        assert abs(got[1] - ref[1]) <= 1e-12 * sc / hh


def test_cd2_exact_for_quintic_flux():
    """For a degree-5 flux the interpolant is the flux itself, so D(f) and D(h) are the truncated
    series -(1/24) dx^2 f'' + (7/5760) dx^4 f'''' (and the same for f') at the midpoint."""
    rng = np.random.default_rng(15)
    for _ in range(20):
        a = rng.normal(size=6)
        dx, x0 = float(rng.uniform(0.05, 0.5)), float(rng.uniform(-1, 1))
        p = np.polynomial.Polynomial(a)
        xs = x0 + dx * np.arange(-1, 3)
        Df, Dh = O.dterms(p(xs), p.deriv()(xs[1:3]), dx, form=2)
        xm = x0 + 0.5 * dx
        ef = -dx ** 2 / 24 * p.deriv(2)(xm) + 7 * dx ** 4 / 5760 * p.deriv(4)(xm)
        eh = -dx ** 2 / 24 * p.deriv(3)(xm) + 7 * dx ** 4 / 5760 * p.deriv(5)(xm)
        assert abs(Df - ef) <= 1e-12 * (1 + np.abs(a).sum())
        assert abs(Dh - eh) <= 1e-10 * (1 + np.abs(a).sum())


# ------------------------------------------------------------------------------------------------
# v^+/- with the nonlinear weights

def test_v_weighted_equals_linear_value_on_linear_data():
    """On linear data all three smoothness indicators are (h s)^2, tau = 0 and the weights are
    the linear weights; the weighted combination of (p0', p1', p2') then collapses to p0' = s."""
    rng = np.random.default_rng(16)
    for _ in range(20):
        s, b, h = rng.normal(), rng.normal(), float(rng.uniform(0.01, 0.2))
        u = b + s * h * np.array([-1.0, 0.0, 1.0])
        lin = O.stencil(u, [s, s], h)
        w = O.stencil(u, [s, s], h, v_weighted=True)
        assert abs(w["v_minus"] - s) <= 1e-12 * (1 + abs(s))
        assert abs(w["v_plus"] - s) <= 1e-12 * (1 + abs(s))
        assert abs(w["v_minus"] - lin["v_minus"]) <= 1e-12 * (1 + abs(s))
        assert w["u_minus"] == lin["u_minus"]


def test_v_weighted_takes_the_smooth_slope_at_a_jump():
    """u = (0, 0, 1) with zero derivatives: the left sub-stencil {i-1, i} is flat, the weights
    pick it, and v^- is its slope 0 (up to eps/tau), while the linear p0' is 21/(16 h)."""
    h = 0.01
    lin = O.stencil([0.0, 0.0, 1.0], [0.0, 0.0], h)
    w = O.stencil([0.0, 0.0, 1.0], [0.0, 0.0], h, v_weighted=True)
    assert abs(lin["v_minus"] - 21.0 / 16.0 / h) <= 1e-12 / h
    assert abs(w["v_minus"]) <= 1e-6 / h
    # and the mirror: u = (1, 0, 0) -> v^+ at x_{i-1/2} from the flat right sub-stencil
    w2 = O.stencil([1.0, 0.0, 0.0], [0.0, 0.0], h, v_weighted=True)
    assert abs(w2["v_plus"]) <= 1e-6 / h


# ------------------------------------------------------------------------------------------------
# fifth order for every variant (Example 4.2, dt ~ dx^(5/3))

def _euler1d_error(n, flags):
    S, dx = W.euler1d_smooth(n)
    cfg = O.make_cfg(1, O.EULER, n, dx=dx, flags=flags)
    out, _, t = O.run(cfg, S, 2.0, 0.6, 5.0 / 3.0)
    ex, _ = W.euler1d_smooth(n, t=2.0)
    return np.abs(out[0, 0] - ex[0, 0]).mean()


@pytest.mark.parametrize("flags", [O.FLAG_V_WEIGHTED, O.FLAG_CD2, O.FLAG_R2,
                                   O.FLAG_V_WEIGHTED | O.FLAG_CD2 | O.FLAG_R2])
def test_variants_keep_fifth_order_euler1d(flags):
    e40, e80 = _euler1d_error(40, flags), _euler1d_error(80, flags)
    base80 = _euler1d_error(80, 0)
    assert np.log2(e40 / e80) >= 4.6, (e40, e80)
    assert e80 <= 3.0 * base80, (e80, base80)


def test_r2_changes_euler_faces_but_not_scalar_ones():
    S, dx = W.euler1d_smooth(32)
    L1, M1 = O.rhs(O.make_cfg(1, O.EULER, 32, dx=dx), S)
    L2, M2 = O.rhs(O.make_cfg(1, O.EULER, 32, dx=dx, flags=O.FLAG_R2), S)
    assert np.array_equal(M1, M2)          # the modified derivative already uses the cell's basis
    d = np.abs(L1 - L2).max()
    assert 0 < d <= 1e-3 * np.abs(L1).max()
    Sb, dxb = W.burgers_1d(40)
    La, _ = O.rhs(O.make_cfg(1, O.BURGERS, 40, dx=dxb), Sb)
    Lb, _ = O.rhs(O.make_cfg(1, O.BURGERS, 40, dx=dxb, flags=O.FLAG_R2), Sb)
    assert np.array_equal(La, Lb)


# ------------------------------------------------------------------------------------------------
# gravity source, Eq. (euler2d-s)

def test_gravity_source_on_uniform_flow():
    """Uniform flow: every flux difference vanishes, so L is the source itself,
    (0, 0, g rho, g rho nu) for U and zero for the (zero) derivatives."""
    n, g = 12, 0.7
    rho, u, v, p, gam = 1.3, 0.4, -0.6, 2.1, 1.4
    one = np.ones((n, n))
    zero = 0 * one
    U, _ = W.euler_from_primitive_2d(rho * one, u * one, v * one, p * one, zero, zero, zero, zero, gam)
    S = np.stack([U, 0 * U, 0 * U])
    cfg = O.make_cfg(2, O.EULER, n, n, dx=0.1, dy=0.1, gamma=gam, grav=g)
    L, M = O.rhs(cfg, S)
    ref = np.zeros_like(S)
    ref[0, 2] = g * rho
    ref[0, 3] = g * rho * v
    assert np.abs(L - ref).max() <= 1e-12


def test_ssp_rk3_integrates_the_gravity_source_exactly():
    """Uniform flow with gravity stays uniform, so at every stage L is the source alone: rho nu grows
    linearly and E quadratically in time.  That system is nilpotent, so a third-order Runge-Kutta
    step (Eqs. fully-hweno, 2Dfully-hweno) integrates it exactly: one step and ten steps equal the
    closed form rho nu(t) = rho nu_0 + g rho t, E(t) = E_0 + g (rho nu_0 t + g rho t^2 / 2) to
    round-off, and the derivative fields stay zero.  A wrong stage coefficient breaks the t^2 term."""
    n, g = 8, 0.7
    rho, u, v, p, gam = 1.3, 0.4, -0.6, 2.1, 1.4
    one = np.ones((n, n))
    zero = 0 * one
    U, _ = W.euler_from_primitive_2d(rho * one, u * one, v * one, p * one, zero, zero, zero, zero, gam)
    S0 = np.stack([U, 0 * U, 0 * U])
    cfg = O.make_cfg(2, O.EULER, n, n, dx=0.1, dy=0.1, gamma=gam, grav=g)
    E0 = p / (gam - 1.0) + 0.5 * rho * (u * u + v * v)
    dt = 0.013
    for nsteps in (1, 10):
        S = O.steps(cfg, S0, dt, nsteps)
        t = dt * nsteps
        exact = (rho, rho * u, rho * v + g * rho * t, E0 + g * (rho * v * t + 0.5 * g * rho * t * t))
        for k, val in enumerate(exact):
            assert np.abs(S[0, k] - val).max() <= 1e-13 * max(1.0, abs(val)), (nsteps, k)
        assert np.abs(S[1:]).max() == 0.0


def test_gravity_balances_a_hydrostatic_column():
    """Constant density, P = p0 + g rho0 y: the scheme differentiates the linear pressure exactly,
    so away from the fixed top and bottom (whose ghost values are constant) L vanishes to
    round-off, for U and for both derivative fields.  Without gravity the same cells keep the
    uncompensated -dP/dy = -g rho0 in the y-momentum."""
    nx, ny, g, rho0 = 8, 24, 1.0, 1.5
    S, dx, dy = W.hydrostatic_column(nx, ny, rho0=rho0, g=g)
    bottom = S[0, :, 0, 0]
    top = S[0, :, -1, 0]
    sides = (O.BC_PERIODIC, O.BC_PERIODIC, O.BC_FIXED, O.BC_FIXED)
    fixed = {2: bottom, 3: top}
    cfg = O.make_cfg(2, O.EULER, nx, ny, dx=dx, dy=dy, grav=g, sides=sides, fixed=fixed)
    L, _ = O.rhs(cfg, S)
    inner = (slice(None), slice(None), slice(3, ny - 3), slice(None))
    assert np.abs(L[inner]).max() <= 1e-10
    cfg0 = O.make_cfg(2, O.EULER, nx, ny, dx=dx, dy=dy, sides=sides, fixed=fixed)
    L0, _ = O.rhs(cfg0, S)
    assert np.abs(L0[0, 2, 3:ny - 3] + g * rho0).max() <= 1e-10


# ------------------------------------------------------------------------------------------------
# fixed-state sides

def test_fixed_sides_equal_a_padded_grid():
    """A side of type BC_FIXED behaves as two more cells holding the state with zero derivatives:
    one stage (same alpha) on the n-cell grid equals the interior of an (n+4)-cell grid padded
    with those cells (the stencils of the interior cells never reach the big grid's own ghosts)."""
    rng = np.random.default_rng(17)
    nx, ny = 14, 11
    S, dx, dy = W.euler2d_random(nx, ny, 33, "smooth")
    fx_lo = S[0, :, :, 0].mean(axis=1) * (1 + 0.1 * rng.random(4))
    fy_hi = S[0, :, -1, :].mean(axis=1) * (1 + 0.1 * rng.random(4))
    sides = (O.BC_FIXED, O.BC_TRANSMISSIVE, O.BC_PERIODIC, O.BC_PERIODIC)
    cfg = O.make_cfg(2, O.EULER, nx, ny, dx=dx, dy=dy, sides=sides, fixed={0: fx_lo})
    alpha = O.max_wavespeed(cfg, S)
    L, M = O.rhs(cfg, S, alpha=alpha)
    big = np.zeros((3, 4, ny, nx + 2))
    big[..., 2:] = S
    big[0, :, :, :2] = fx_lo[:, None, None]
    cfgb = O.make_cfg(2, O.EULER, nx + 2, ny, dx=dx, dy=dy,
                      sides=(O.BC_TRANSMISSIVE, O.BC_TRANSMISSIVE, O.BC_PERIODIC, O.BC_PERIODIC))
    Lb, Mb = O.rhs(cfgb, big, alpha=alpha)
    assert np.abs(L - Lb[..., 2:]).max() <= 1e-12 * np.abs(L).max()
    assert np.abs(M - Mb[..., 2:]).max() <= 1e-12 * np.abs(M).max()
    # the same along y (top side fixed), with x periodic
    sides = (O.BC_PERIODIC, O.BC_PERIODIC, O.BC_TRANSMISSIVE, O.BC_FIXED)
    cfg = O.make_cfg(2, O.EULER, nx, ny, dx=dx, dy=dy, sides=sides, fixed={3: fy_hi})
    L, M = O.rhs(cfg, S, alpha=alpha)
    big = np.zeros((3, 4, ny + 2, nx))
    big[..., :ny, :] = S
    big[0, :, ny:, :] = fy_hi[:, None, None]
    cfgb = O.make_cfg(2, O.EULER, nx, ny + 2, dx=dx, dy=dy,
                      sides=(O.BC_PERIODIC, O.BC_PERIODIC, O.BC_TRANSMISSIVE, O.BC_TRANSMISSIVE))
    Lb, Mb = O.rhs(cfgb, big, alpha=alpha)
    assert np.abs(L - Lb[..., :ny, :]).max() <= 1e-12 * np.abs(L).max()
    assert np.abs(M - Mb[..., :ny, :]).max() <= 1e-12 * np.abs(M).max()


def test_uniform_state_matching_fixed_sides_is_steady():
    n = 10
    U = np.array([1.2, 0.3, -0.2, 3.0])
    S = np.zeros((3, 4, n, n))
    S[0] = U[:, None, None]
    cfg = O.make_cfg(2, O.EULER, n, n, dx=0.1, dy=0.1, sides=(O.BC_FIXED,) * 4,
                     fixed={k: U for k in range(4)})
    L, _ = O.rhs(cfg, S)
    assert np.abs(L).max() <= 1e-13


def test_invalid_extensions_rejected():
    with pytest.raises(ValueError):  # gravity outside 2D Euler
        O.state_size(O.make_cfg(1, O.EULER, 16, grav=1.0))
    with pytest.raises(ValueError):  # periodic on one side only
        O.state_size(O.make_cfg(2, O.EULER, 8, 8, sides=(O.BC_PERIODIC, O.BC_FIXED, 0, 0)))
    with pytest.raises(ValueError):
        O.state_size(O.make_cfg(2, O.EULER, 8, 8, flags=32))


# ------------------------------------------------------------------------------------------------
# adjoint identity and the Rayleigh-Taylor set-up

def test_vjp_dot_product_identity_with_extensions():
    S, dx, dy, fixed = W.rayleigh_taylor(8, 12)
    cfg = O.make_cfg(2, O.EULER, 8, 12, dx=dx, dy=dy, gamma=5.0 / 3.0, grav=1.0,
                     sides=(O.BC_REFLECTIVE, O.BC_REFLECTIVE, O.BC_FIXED, O.BC_FIXED), fixed=fixed,
                     flags=O.FLAG_V_WEIGHTED | O.FLAG_CD2 | O.FLAG_R2)
    alpha = O.max_wavespeed(cfg, S)
    rng = np.random.default_rng(18)
    delta, muM, muL = (rng.normal(size=S.shape) for _ in range(3))
    jM, jL = O.stage_jvp(cfg, S, alpha, delta)
    lam = O.stage_vjp(cfg, S, alpha, muM, muL)
    lhs = np.vdot(muM, jM) + np.vdot(muL, jL)
    scale = np.abs(muM * jM).sum() + np.abs(muL * jL).sum()
    assert abs(lhs - np.vdot(lam, delta)) <= 1e-13 * scale


def test_rayleigh_taylor_runs():
    """Example 4.11 at 16 x 64 for 40 steps: finite, positive density and pressure, and the heavy
    fluid starts to fall where v < 0 (x near 0 and 0.25)."""
    S, dx, dy, fixed = W.rayleigh_taylor(16)
    cfg = O.make_cfg(2, O.EULER, 16, 64, dx=dx, dy=dy, gamma=5.0 / 3.0, grav=1.0,
                     sides=(O.BC_REFLECTIVE, O.BC_REFLECTIVE, O.BC_FIXED, O.BC_FIXED), fixed=fixed)
    out, n, t = O.run(cfg, S, 0.0, 0.6, 1.0, max_steps=40)
    assert n == 40 and np.isfinite(out).all()
    rho = out[0, 0]
    p = (5.0 / 3.0 - 1) * (out[0, 3] - 0.5 * (out[0, 1] ** 2 + out[0, 2] ** 2) / rho)
    assert rho.min() > 0.9 and p.min() > 0.9


def _mirror(S):
    """x -> -x on a periodic 1D Euler state: cells reversed, rho u and the derivatives of rho, E
    change sign (U: (+, -, +), V = U_x: (-, +, -))."""
    sU = np.array([1.0, -1.0, 1.0])[:, None, None]
    R = S[..., ::-1].copy()
    R[0] *= sU
    R[1] *= -sU
    return R


@pytest.mark.parametrize("flags", [0, O.FLAG_V_WEIGHTED, O.FLAG_CD2, O.FLAG_R2,
                                   O.FLAG_V_WEIGHTED | O.FLAG_CD2 | O.FLAG_R2])
@pytest.mark.parametrize("kind", ["smooth", "jumps"])
def test_operator_commutes_with_mirroring(flags, kind):
    """The scheme has no preferred direction: the operator of the mirrored state is the mirrored
    operator.  This pins which cell supplies which basis (each side of a face uses the centre of
    its own stencil under R2; the Roe average is symmetric) and the mirror image taken for u^+."""
    n = 30
    S, dx = W.euler1d_random(n, 41, kind)
    cfg = O.make_cfg(1, O.EULER, n, dx=dx, flags=flags)
    L, M = O.rhs(cfg, S)
    Lm, Mm = O.rhs(cfg, _mirror(S))
    for a, b in ((Lm, _mirror(L)), (Mm, _mirror(M))):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("dim", [1, 2])
def test_characteristic_bases_agree_when_the_weights_are_linear(dim):
    """With linear weights (eps far above every smoothness indicator) the interpolation is linear
    in its data, so it commutes with any projection: the Roe basis at the face (default) and the
    centre cells' bases (R2) give the same face states, and those are the componentwise ones.
    This pins the pairing of every projection with its back projection."""
    if dim == 1:
        S, dx = W.euler1d_random(24, 51, "jumps")
        dy = dx
        nx, ny = 24, 1
    else:
        S, dx, dy = W.euler2d_random(14, 11, 52, "jumps")
        nx, ny = 14, 11
    kw = dict(dx=dx, dy=dy, eps=1e30, bc=O.BC_TRANSMISSIVE)
    L1, M1 = O.rhs(O.make_cfg(dim, O.EULER, nx, ny, **kw), S)
    L2, M2 = O.rhs(O.make_cfg(dim, O.EULER, nx, ny, flags=O.FLAG_R2, **kw), S)
    for a, b in ((L1, L2), (M1, M2)):
        assert np.abs(a - b).max() <= 1e-11 * np.abs(a).max()
    # and with real weights on blocky data they differ
    L3, _ = O.rhs(O.make_cfg(dim, O.EULER, nx, ny, dx=dx, dy=dy, bc=O.BC_TRANSMISSIVE), S)
    L4, _ = O.rhs(O.make_cfg(dim, O.EULER, nx, ny, dx=dx, dy=dy, bc=O.BC_TRANSMISSIVE, flags=O.FLAG_R2), S)
    assert np.abs(L3 - L4).max() > 1e-10 * np.abs(L3).max()


# ------------------------------------------------------------------------------------------------
# LF coefficient scope (global per stage by default; per step; local per face)

def _three_region_1d(n, fast):
    """1D Euler: left state | right state with a jump at the middle face, both with the same
    |u| + c (same u; rho and P scaled together keep c), and (if fast) a region of large wavespeed
    far from the jump."""
    rho = np.where(np.arange(n) < n // 2, 1.0, 0.4)
    u = np.full(n, 0.2)
    p = np.where(np.arange(n) < n // 2, 1.0, 0.4)
    if fast:
        u[-6:] = 30.0
    zero = np.zeros(n)
    U, V = W.euler_from_primitive_1d(rho, u, p, zero, zero, zero)
    S = np.zeros((2, 3, 1, n))
    S[0, :, 0] = U
    return S


def test_local_alpha_is_the_adjacent_cells_maximum():
    """Local LF: at a face the coefficient is max(|u| + c) of its two adjacent cells, whatever the
    rest of the grid holds.  Near the jump every cell has the same |u| + c, so there the local
    operator on data with a far, fast region equals the global operator on the same data without
    that region (whose global maximum is that common value)."""
    n = 40
    S3, S2 = _three_region_1d(n, True), _three_region_1d(n, False)
    cfg_loc = O.make_cfg(1, O.EULER, n, dx=0.05, bc=O.BC_TRANSMISSIVE, flags=O.FLAG_ALPHA_LOCAL)
    cfg_glob = O.make_cfg(1, O.EULER, n, dx=0.05, bc=O.BC_TRANSMISSIVE)
    L3, _ = O.rhs(cfg_loc, S3)
    L2, _ = O.rhs(cfg_glob, S2)
    near = slice(n // 2 - 3, n // 2 + 3)
    assert np.abs(L3[..., near] - L2[..., near]).max() <= 1e-13 * np.abs(L2[..., near]).max()
    # and the global coefficient (set by the fast region) dissipates more there
    L3g, _ = O.rhs(cfg_glob, S3)
    assert np.abs(L3g[..., near] - L2[..., near]).max() > 1e-3 * np.abs(L2[..., near]).max()


def test_alpha_held_for_the_step_equals_a_replay_with_stage_one_alphas():
    S, dx, dy = W.euler2d_random(12, 10, 53, "jumps")
    cfg = O.make_cfg(2, O.EULER, 12, 10, dx=dx, dy=dy, flags=O.FLAG_ALPHA_STEP)
    out, dts, alphas = O.steps_record(cfg, S, 3)
    assert np.array_equal(alphas[:, 2:4], alphas[:, 0:2]) and np.array_equal(alphas[:, 4:6], alphas[:, 0:2])
    base = O.make_cfg(2, O.EULER, 12, 10, dx=dx, dy=dy)
    rep = O.steps_replay(base, S, dts, alphas)
    assert np.array_equal(out, rep)
    # the default scheme recomputes alpha at every stage, which differs on this data
    _, _, a_def = O.steps_record(base, S, 3)
    assert not np.array_equal(a_def[:, 2:4], a_def[:, 0:2])


@pytest.mark.parametrize("flags", [O.FLAG_ALPHA_STEP, O.FLAG_ALPHA_LOCAL, O.FLAG_ALPHA_LOCAL | O.FLAG_R2])
def test_alpha_modes_keep_fifth_order_euler1d(flags):
    e40, e80 = _euler1d_error(40, flags), _euler1d_error(80, flags)
    assert np.log2(e40 / e80) >= 4.6, (e40, e80)
