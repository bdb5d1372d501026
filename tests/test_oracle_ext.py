"""Pins of the oracle's extended-precision evaluation (long double: 64-bit significand on x86-64,
113-bit on AArch64), the reference the GPU path's rounding is measured against at full size.

  * it computes the same scheme: the HWENO-I accuracy tables of Sec. 4 (1D and 2D Euler, 1D and 2D
    Burgers) to the printed digits, and the FP64 oracle within that oracle's own rounding envelope;
  * it carries the extra precision through the whole operator: for linear advection the scheme is
    invariant under u -> u + C in exact arithmetic (the candidates of Eqs. (Pxi) and the
    combination of Eq. (interp) reproduce constants, the indicators, slopes, D-terms of Eq. (Cd-1)
    and the conservative difference see only differences), so L(u + C) - L(u) is rounding alone;
    with C = 1024 the FP64 evaluation's share is about ulp(1024)/h, and the extended one must be
    smaller by at least 2^6 (it is 2^11 or more smaller if no value is rounded to double on the way).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_error_tables.json")


def _close_to_printed(value, printed):
    e = math.floor(math.log10(abs(printed)))
    return abs(value - printed) <= 2.5 * 10.0 ** (e - 3)


def _rel_planes(a, b, nplanes):
    a, b = a.reshape(nplanes, -1), b.reshape(nplanes, -1)
    return np.abs(a - b).max(axis=1) / np.maximum(np.abs(b).max(axis=1), 1e-300)


def test_ext_has_more_significand_bits():
    assert O.ext_mantissa_bits() >= 64


def test_ext_paper_table_euler1d():
    with open(GOLD) as f:
        rows = json.load(f)["euler1d"]["rows"]
    for n, l1, linf in rows[:2]:
        S, dx = W.euler1d_smooth(n)
        cfg = O.make_cfg(1, O.EULER, n, dx=dx)
        out, _, _ = O.run_ext(cfg, S, 2.0, 0.6, 5.0 / 3.0)
        ex, _ = W.euler1d_smooth(n, t=2.0)
        e = np.abs(out[0, 0] - ex[0, 0])
        assert _close_to_printed(e.mean(), l1), (n, e.mean(), l1)
        assert _close_to_printed(e.max(), linf), (n, e.max(), linf)


def test_ext_paper_table_euler2d():
    with open(GOLD) as f:
        n, l1, linf = json.load(f)["euler2d"]["rows"][0]
    S, dx, dy = W.euler2d_smooth(n, mu=1.0, nu=1.0)
    cfg = O.make_cfg(2, O.EULER, n, n, dx=dx, dy=dy)
    out, _, _ = O.run_ext(cfg, S, 2.0, 0.6, 5.0 / 3.0)
    ex, _, _ = W.euler2d_smooth(n, t=2.0, mu=1.0, nu=1.0)
    e = np.abs(out[0, 0] - ex[0, 0])
    assert _close_to_printed(e.mean(), l1), (n, e.mean(), l1)
    assert _close_to_printed(e.max(), linf), (n, e.max(), linf)


def _offset_data(dim, n, C):
    """Smooth periodic data u, v = u_x (, w = u_y) with u rounded so that u + C is exact."""
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    if dim == 1:
        u = 0.6 * np.sin(2 * np.pi * x) + 0.3 * np.cos(6 * np.pi * x)
        v = 0.6 * 2 * np.pi * np.cos(2 * np.pi * x) - 0.3 * 6 * np.pi * np.sin(6 * np.pi * x)
        u = (u + C) - C
        return np.stack([u, v])[:, None, :], h
    X, Y = np.meshgrid(x, x, indexing="xy")
    u = 0.6 * np.sin(2 * np.pi * (X + 2 * Y)) + 0.2 * np.cos(2 * np.pi * X)
    v = 0.6 * 2 * np.pi * np.cos(2 * np.pi * (X + 2 * Y)) - 0.2 * 2 * np.pi * np.sin(2 * np.pi * X)
    w = 0.6 * 4 * np.pi * np.cos(2 * np.pi * (X + 2 * Y))
    u = (u + C) - C
    return np.stack([u, v, w])[:, None, :, :], h


@pytest.mark.parametrize("dim", [1, 2])
def test_ext_offset_invariance(dim):
    C = 1024.0
    n = 64 if dim == 1 else 48
    S, h = _offset_data(dim, n, C)
    cfg = O.make_cfg(dim, O.ADVECTION, n, n, dx=h, dy=h, ax=0.7, ay=-0.4, eps=1e-6)
    SC = S.copy()
    SC[0] = SC[0] + C
    assert np.array_equal(SC[0] - C, S[0])  # the offset data are exact doubles
    nf = S.shape[0]
    L0, M0 = O.rhs_ext(cfg, S)
    L1, M1 = O.rhs_ext(cfg, SC)
    Ld0, Md0 = O.rhs(cfg, S)
    Ld1, Md1 = O.rhs(cfg, SC)
    scale = np.abs(L0).max()
    dev_ext = np.abs(L1 - L0).max() / scale
    dev_64 = np.abs(Ld1 - Ld0).max() / scale
    print("offset invariance: FP64", dev_64, "extended", dev_ext)
    assert dev_64 > 1e-13  # FP64 rounding of the offset values is visible
    assert dev_ext <= dev_64 / 64, (dev_ext, dev_64)
    # the modified derivatives are invariant too
    dm_ext = np.abs(M1[1:] - M0[1:]).max() / np.abs(M0[1:]).max()
    dm_64 = np.abs(Md1[1:] - Md0[1:]).max() / np.abs(M0[1:]).max()
    assert dm_ext <= max(dm_64 / 64, 1e-17), (dm_ext, dm_64)
    assert nf == (2 if dim == 1 else 3)


def test_ext_against_fp64_within_rounding():
    """One stage and ten steps of 2D Euler (smooth wave, 48^2): the FP64 oracle differs from the
    extended evaluation by less than the FP64 oracle's own one-ulp input-perturbation drift."""
    n = 48
    S, dx, dy = W.euler2d_smooth(n)
    cfg = O.make_cfg(2, O.EULER, n, n, dx=dx, dy=dy)
    sign = np.random.default_rng(5).choice([-1.0, 1.0], S.shape)
    P = S * (1.0 + sign * 2.0 ** -52)
    L, M = O.rhs(cfg, S)
    Le, Me = O.rhs_ext(cfg, S)
    Lp, Mp = O.rhs(cfg, P)
    assert (_rel_planes(L, Le, 12) <= np.maximum(_rel_planes(Lp, L, 12), 1e-15)).all()
    assert (_rel_planes(M, Me, 12) <= np.maximum(_rel_planes(Mp, M, 12), 1e-15)).all()
    out, k, t = O.run(cfg, S, 0.0, 0.6, 1.0, max_steps=10)
    oute, ke, te = O.run_ext(cfg, S, 0.0, 0.6, 1.0, max_steps=10)
    outp, _, _ = O.run(cfg, P, 0.0, 0.6, 1.0, max_steps=10)
    assert k == ke == 10 and abs(t - te) <= 1e-15 * t
    err, env = _rel_planes(out, oute, 12), _rel_planes(outp, out, 12)
    print("10 steps: FP64 against extended", err.max(), "one-ulp drift", env.max())
    assert (err <= np.maximum(2 * env, 1e-15)).all(), (err, env)


def test_ext_paper_table_burgers():
    """The scalar code paths in extended precision: the HWENO-I columns of the 1D and 2D Burgers
    tables of Sec. 4 (first rows) to the printed digits."""
    with open(GOLD) as f:
        tables = json.load(f)
    for n, l1, linf in tables["burgers1d"]["rows"][:2]:
        S, dx = W.burgers_1d(n)
        cfg = O.make_cfg(1, O.BURGERS, n, dx=dx)
        out, _, _ = O.run_ext(cfg, S, 0.5, 0.6, 5.0 / 3.0)
        ex, _ = W.burgers_1d(n, t=0.5)
        e = np.abs(out[0, 0] - ex[0, 0])
        assert _close_to_printed(e.mean() / (2 * np.pi), l1), (n, e.mean(), l1)
        assert _close_to_printed(e.max(), linf), (n, e.max(), linf)
    n, l1, linf = tables["burgers2d"]["rows"][0]
    S, dx = W.burgers_2d(n)
    cfg = O.make_cfg(2, O.BURGERS, n, n, dx=dx, dy=dx)
    out, _, _ = O.run_ext(cfg, S, 0.5, 0.6, 5.0 / 3.0)
    ex, _ = W.burgers_2d(n, t=0.5)
    e = np.abs(out[0, 0] - ex[0, 0])
    assert _close_to_printed(e.mean(), l1), (n, e.mean(), l1)
    assert _close_to_printed(e.max(), linf), (n, e.max(), linf)
