"""Pins of the oracle's building blocks against sympy re-derivations from their defining
conditions: the Hermite candidates of Eq. (HWEp0) evaluated as in Eqs. (Pxi), (P'xi), (limiter-p),
the smoothness indicators of Eq. (GHYZ), and the degree-5 central Hermite interpolant of Eq. (Pc)
behind Eqs. (Cd-1), (DfDh)."""
import numpy as np
import pytest

import oracle as O

sp = pytest.importorskip("sympy")


def _hermite_candidates():
    """p0 (degree 4: five conditions of Eq. HWEp0), p1, p2 on x_i = 0 with spacing h."""
    x, h = sp.symbols("x h", positive=True)
    um, u0, up, vm, vp = sp.symbols("um u0 up vm vp")
    c = sp.symbols("c0:5")
    p0 = sum(c[k] * x ** k for k in range(5))
    eqs = [p0.subs(x, -h) - um, p0.subs(x, 0) - u0, p0.subs(x, h) - up,
           sp.diff(p0, x).subs(x, -h) - vm, sp.diff(p0, x).subs(x, h) - vp]
    p0 = p0.subs(sp.solve(eqs, c))
    p1 = um + (u0 - um) * (x + h) / h
    p2 = u0 + (up - u0) * x / h
    return x, h, (um, u0, up, vm, vp), (sp.expand(p0), p1, p2)


def _beta(p, x, h, degree):
    """Eq. (GHYZ): sum over alpha of int_{I_i} h^(2 alpha - 1) (d^alpha p / dx^alpha)^2 dx."""
    return sum(sp.integrate(h ** (2 * a - 1) * sp.diff(p, x, a) ** 2, (x, -h / 2, h / 2))
               for a in range(1, degree + 1))


@pytest.fixture(scope="module")
def candidates():
    x, h, syms, (p0, p1, p2) = _hermite_candidates()
    ex = {
        "p0": p0.subs(x, h / 2), "p1": p1.subs(x, h / 2), "p2": p2.subs(x, h / 2),
        "dp0_half": sp.diff(p0, x).subs(x, h / 2),
        "dp0_c": sp.diff(p0, x).subs(x, 0), "dp1_c": sp.diff(p1, x).subs(x, 0),
        "dp2_c": sp.diff(p2, x).subs(x, 0),
        "p0_left": p0.subs(x, -h / 2), "dp0_left": sp.diff(p0, x).subs(x, -h / 2),
        "beta0": _beta(p0, x, h, 4), "beta1": _beta(p1, x, h, 1), "beta2": _beta(p2, x, h, 1),
    }
    args = (h,) + syms
    return {k: sp.lambdify(args, v, "math") for k, v in ex.items()}


def test_candidates_and_indicators_match_sympy(candidates):
    rng = np.random.default_rng(11)
    for _ in range(50):
        h = float(rng.uniform(0.01, 1.0))
        u = rng.normal(size=3)
        v = rng.normal(size=2) * rng.choice([0.1, 1.0, 10.0])
        o = O.stencil(u, v, h, gamma0=0.95, d0=0.9, eps=1e-10)
        a = (h, u[0], u[1], u[2], v[0], v[1])
        ref = {k: f(*a) for k, f in candidates.items()}
        scale = 1.0 + np.abs(u).max() + h * np.abs(v).max()
        for got, key in ((o["p"][0], "p0"), (o["p"][1], "p1"), (o["p"][2], "p2")):
            assert abs(got - ref[key]) <= 1e-13 * scale
        assert abs(o["dp0_half"] - ref["dp0_half"]) <= 1e-12 * scale / h
        for l, key in enumerate(("dp0_c", "dp1_c", "dp2_c")):
            assert abs(o["dp_center"][l] - ref[key]) <= 1e-12 * scale / h
        for l in range(3):
            assert abs(o["beta"][l] - ref[f"beta{l}"]) <= 1e-12 * scale ** 2


def test_mirror_uses_the_reflected_stencil(candidates):
    """With linear weights (huge eps), u^+_{i-1/2} is p0(x_{i-1/2}) and v^+ is p0'(x_{i-1/2})."""
    rng = np.random.default_rng(12)
    for _ in range(20):
        h = float(rng.uniform(0.05, 0.5))
        u = rng.normal(size=3)
        v = rng.normal(size=2)
        o = O.stencil(u, v, h, eps=1e300)
        a = (h, u[0], u[1], u[2], v[0], v[1])
        assert abs(o["u_plus"] - candidates["p0_left"](*a)) <= 1e-13 * (1 + np.abs(u).max())
        assert abs(o["v_plus"] - candidates["dp0_left"](*a)) <= 1e-12 * (1 + np.abs(u).max()) / h
        assert abs(o["u_minus"] - candidates["p0"](*a)) <= 1e-13 * (1 + np.abs(u).max())


def test_dterms_match_degree5_hermite():
    """Eqs. (Pc), (Cd-1), (DfDh): D-terms from the unique degree-5 Hermite interpolant P."""
    x, h = sp.symbols("x h", positive=True)
    f = sp.symbols("f0:4")
    hm, h2 = sp.symbols("hm h2")
    c = sp.symbols("c0:6")
    P = sum(c[k] * x ** k for k in range(6))
    nodes = [-h, 0, h, 2 * h]  # x_{i-1}, x_i, x_{i+1}, x_{i+2}
    eqs = [P.subs(x, nodes[q]) - f[q] for q in range(4)]
    eqs += [sp.diff(P, x).subs(x, -h) - hm, sp.diff(P, x).subs(x, 2 * h) - h2]
    P = P.subs(sp.solve(eqs, c))
    xh = h / 2
    Df = -sp.Rational(1, 24) * h ** 2 * sp.diff(P, x, 2).subs(x, xh) + \
        sp.Rational(7, 5760) * h ** 4 * sp.diff(P, x, 4).subs(x, xh)
    Dh = -sp.Rational(1, 24) * h ** 2 * sp.diff(P, x, 3).subs(x, xh) + \
        sp.Rational(7, 5760) * h ** 4 * sp.diff(P, x, 5).subs(x, xh)
    fDf = sp.lambdify((h,) + f + (hm, h2), Df, "math")
    fDh = sp.lambdify((h,) + f + (hm, h2), Dh, "math")
    rng = np.random.default_rng(13)
    for _ in range(50):
        hh = float(rng.uniform(0.01, 1.0))
        ff = rng.normal(size=4)
        hv = rng.normal(size=2)
        got = O.dterms(ff, hv, hh)
        ref = (fDf(hh, *ff, *hv), fDh(hh, *ff, *hv))
        sc = 1 + np.abs(ff).max() + hh * np.abs(hv).max()
        assert abs(got[0] - ref[0]) <= 1e-13 * sc
        assert abs(got[1] - ref[1]) <= 1e-12 * sc / hh




def test_beta0_as_two_completed_squares():
    """The kernels evaluate beta0 (Eq. GHYZ) as S1 (sv + N1 du)^2 + T1 du^2 + S2 (dv + N2 d2)^2
    + T2 d2^2 with du = u_{i+1} - u_{i-1}, d2 = u_{i+1} - 2 u_i + u_{i-1}, sv = h (v_{i-1} +
    v_{i+1}), dv = h (v_{i-1} - v_{i+1}): each pair of the explicit linear forms (a1 + a3/4 with a3;
    a2 + 63/130 a4 with a4), with its weights, is one quadratic form s X^2 + 2 q X Y + r Y^2 =
    s (X + (q/s) Y)^2 + (det/s) Y^2.  Exact in rationals against the integral definition."""
    x, h, (um, u0, up, vm, vp), (p0, _, _) = _hermite_candidates()
    beta0 = sp.expand(_beta(p0, x, h, 4))
    R = sp.Rational

    def pair(f, wf, k, wk):
        s = wf * f[0] ** 2 + wk * k[0] ** 2
        q = wf * f[0] * f[1] + wk * k[0] * k[1]
        m = f[0] * k[1] - f[1] * k[0]
        return s, q / s, wf * wk * m * m / s

    S1, N1, T1 = pair((R(-3, 16), R(11, 16)), 1, (R(1, 4), R(-1, 4)), R(781, 20))
    S2, N2, T2 = pair((R(67, 520), R(197, 260)), R(13, 3), (R(-1, 4), R(-1, 2)), R(1421461, 2275))
    du, d2 = up - um, up - 2 * u0 + um
    sv, dv = h * (vm + vp), h * (vm - vp)
    squares = S1 * (sv + N1 * du) ** 2 + T1 * du ** 2 + S2 * (dv + N2 * d2) ** 2 + T2 * d2 ** 2
    assert sp.simplify(sp.expand(squares) - beta0) == 0
    assert T1 == R(781, 3169) and T1 > 0 and T2 > 0 and S1 > 0 and S2 > 0
