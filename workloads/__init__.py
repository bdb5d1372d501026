"""Seeded synthetic inputs for the HWENO-I solvers (CPU oracle and CUDA library alike).

This module holds no part of the numerical method: it only builds initial states (conserved
variables and their exact spatial derivatives on cell centres), exact solutions of the smooth test
problems, and the stop time of the seeded Riemann problems.  Both the oracle tests and the CUDA
tests/bench draw their inputs from here.

State layout (shared convention): float64 array of shape (nfield, ncomp, ny, nx), x fastest.
nfield = 2 in 1D (U, V = U_x) and 3 in 2D (U, V = U_x, W = U_y); ncomp = 1 (scalar), 3 (1D Euler)
or 4 (2D Euler, U = (rho, rho*mu, rho*nu, E)).  1D states have ny = 1.

Test problems of the paper (Sec. 4) used here: 1D Burgers on [-pi, pi] (Example 4.1), 1D Euler
smooth wave on [0, 2] (Example 4.2), 2D Burgers on [-2pi, 2pi]^2 (Example 4.5), 2D Euler smooth
wave on [0, 2]^2 (Example 4.6).  The EOS is E = P/(gamma-1) + rho |vel|^2 / 2.
"""
from __future__ import annotations

import math

import numpy as np


def centres(n: int, a: float, b: float) -> np.ndarray:
    dx = (b - a) / n
    return a + (np.arange(n) + 0.5) * dx


# ----------------------------------------------------------------------------------------------
# scalar problems

def advection_1d(n: int, a: float = 0.0, b: float = 2.0, t: float = 0.0, speed: float = 1.0):
    """u = 0.5 + sin(pi (x - s t)) on [a, b]; returns (state, dx)."""
    x = centres(n, a, b)
    xi = x - speed * t
    S = np.zeros((2, 1, 1, n))
    S[0, 0, 0] = 0.5 + np.sin(np.pi * xi)
    S[1, 0, 0] = np.pi * np.cos(np.pi * xi)
    return S, (b - a) / n


def advection_2d(nx: int, ny: int, ax: float = 1.0, ay: float = 1.0, t: float = 0.0,
                 a: float = 0.0, b: float = 2.0):
    """u = 0.5 + sin(pi (x + y - (ax+ay) t)) on [a, b]^2."""
    x = centres(nx, a, b)[None, :]
    y = centres(ny, a, b)[:, None]
    ph = np.pi * (x - ax * t + y - ay * t)
    S = np.zeros((3, 1, ny, nx))
    S[0, 0] = 0.5 + np.sin(ph)
    S[1, 0] = np.pi * np.cos(ph)
    S[2, 0] = np.pi * np.cos(ph)
    return S, (b - a) / nx, (b - a) / ny


def burgers_1d_exact(x: np.ndarray, t: float):
    """u(x, t) of u_t + (u^2/2)_x = 0 with u0 = 0.5 + sin x (Example 4.1), before shocks form.
    Solves u = 0.5 + sin(x - u t) by Newton's method."""
    u = 0.5 + np.sin(x)
    for _ in range(100):
        g = u - 0.5 - np.sin(x - u * t)
        dg = 1.0 + t * np.cos(x - u * t)
        du = g / dg
        u = u - du
        if np.max(np.abs(du)) < 1e-15:
            break
    ux = np.cos(x - u * t) / (1.0 + t * np.cos(x - u * t))
    return u, ux


def burgers_1d(n: int, t: float = 0.0):
    x = centres(n, -np.pi, np.pi)
    u, ux = burgers_1d_exact(x, t)
    S = np.zeros((2, 1, 1, n))
    S[0, 0, 0] = u
    S[1, 0, 0] = ux
    return S, 2 * np.pi / n


def burgers_2d(n: int, t: float = 0.0):
    """u_t + (u^2/2)_x + (u^2/2)_y = 0, u0 = 0.5 + sin((x+y)/2) on [-2pi, 2pi]^2 (Example 4.5).
    Along characteristics u is constant: u = 0.5 + sin((x + y - 2 u t)/2)."""
    x = centres(n, -2 * np.pi, 2 * np.pi)[None, :]
    y = centres(n, -2 * np.pi, 2 * np.pi)[:, None]
    s = np.broadcast_to(x + y, (n, n))
    u = 0.5 + np.sin(s / 2)
    for _ in range(100):
        g = u - 0.5 - np.sin((s - 2 * u * t) / 2)
        dg = 1.0 + t * np.cos((s - 2 * u * t) / 2)
        du = g / dg
        u = u - du
        if np.max(np.abs(du)) < 1e-15:
            break
    ux = 0.5 * np.cos((s - 2 * u * t) / 2) / (1.0 + t * np.cos((s - 2 * u * t) / 2))
    S = np.zeros((3, 1, n, n))
    S[0, 0] = u
    S[1, 0] = ux
    S[2, 0] = ux
    return S, 4 * np.pi / n


# ----------------------------------------------------------------------------------------------
# Euler: conserved variables and derivatives from primitive fields and their derivatives

def euler_from_primitive_1d(rho, u, p, rho_x, u_x, p_x, gamma=1.4):
    E = p / (gamma - 1) + 0.5 * rho * u * u
    U = np.stack([rho, rho * u, E])
    V = np.stack([rho_x, rho_x * u + rho * u_x,
                  p_x / (gamma - 1) + 0.5 * rho_x * u * u + rho * u * u_x])
    return U, V


def euler_from_primitive_2d(rho, u, v, p, d_rho, d_u, d_v, d_p, gamma=1.4):
    """(U, dU) for one derivative direction; d_* are the primitive derivatives."""
    E = p / (gamma - 1) + 0.5 * rho * (u * u + v * v)
    U = np.stack([rho, rho * u, rho * v, E])
    dU = np.stack([d_rho, d_rho * u + rho * d_u, d_rho * v + rho * d_v,
                   d_p / (gamma - 1) + 0.5 * d_rho * (u * u + v * v) + rho * (u * d_u + v * d_v)])
    return U, dU


def euler1d_smooth(n: int, t: float = 0.0, gamma: float = 1.4, mu: float = 1.0):
    """rho = 1 + 0.2 sin(pi (x - mu t)), velocity mu, P = 1 on [0, 2] (Example 4.2)."""
    x = centres(n, 0.0, 2.0)
    ph = np.pi * (x - mu * t)
    rho = 1 + 0.2 * np.sin(ph)
    rx = 0.2 * np.pi * np.cos(ph)
    one, zero = np.ones(n), np.zeros(n)
    U, V = euler_from_primitive_1d(rho, mu * one, one, rx, zero, zero, gamma)
    S = np.zeros((2, 3, 1, n))
    S[0, :, 0] = U
    S[1, :, 0] = V
    return S, 2.0 / n


def euler2d_smooth(nx: int, ny: int = None, t: float = 0.0, mu: float = 0.7, nu: float = 0.3,
                   gamma: float = 1.4):
    """rho = 1 + 0.2 sin(pi (x + y - (mu+nu) t)), velocity (mu, nu), P = 1 on [0, 2]^2 (the smooth
    wave of Example 4.6 with a general constant velocity)."""
    ny = nx if ny is None else ny
    x = centres(nx, 0.0, 2.0)[None, :]
    y = centres(ny, 0.0, 2.0)[:, None]
    ph = np.pi * (x + y - (mu + nu) * t)
    rho = 1 + 0.2 * np.sin(ph)
    dr = 0.2 * np.pi * np.cos(ph)
    one, zero = np.ones((ny, nx)), np.zeros((ny, nx))
    U, V = euler_from_primitive_2d(rho, mu * one, nu * one, one, dr, zero, zero, zero, gamma)
    _, W = euler_from_primitive_2d(rho, mu * one, nu * one, one, dr, zero, zero, zero, gamma)
    S = np.zeros((3, 4, ny, nx))
    S[0], S[1], S[2] = U, V, W
    return S, 2.0 / nx, 2.0 / ny


def euler2d_quadrants(nx: int, ny: int = None, seed: int = 2000, gamma: float = 1.4):
    """Four piecewise-constant quadrant states on [0, 2]^2 split at (1, 1); rho, P ~ U[0.1, 2],
    velocities ~ U[-1, 1]; derivatives zero.  Quadrant order: (x<1,y<1), (x>=1,y<1), (x<1,y>=1),
    (x>=1,y>=1)."""
    ny = nx if ny is None else ny
    rng = np.random.Generator(np.random.PCG64(seed))
    rho = rng.uniform(0.1, 2.0, 4)
    p = rng.uniform(0.1, 2.0, 4)
    u = rng.uniform(-1.0, 1.0, 4)
    v = rng.uniform(-1.0, 1.0, 4)
    x = centres(nx, 0.0, 2.0)[None, :]
    y = centres(ny, 0.0, 2.0)[:, None]
    q = (x >= 1.0).astype(int) + 2 * (y >= 1.0).astype(int)
    zero = np.zeros((ny, nx))
    U, _ = euler_from_primitive_2d(rho[q], u[q], v[q], p[q], zero, zero, zero, zero, gamma)
    S = np.zeros((3, 4, ny, nx))
    S[0] = U
    return S, 2.0 / nx, 2.0 / ny


def euler2d_random(nx: int, ny: int, seed: int, kind: str = "smooth", gamma: float = 1.4):
    """Seeded test states on [0,2]^2 for parity: 'smooth' = a few random Fourier modes on a
    positive background with exact derivatives; 'jumps' = random blocks of constant states with
    random derivative noise (discontinuous data, large derivative values)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = centres(nx, 0.0, 2.0)[None, :]
    y = centres(ny, 0.0, 2.0)[:, None]
    if kind == "smooth":
        fields = []
        for base, amp in ((1.0, 0.3), (0.3, 0.4), (-0.2, 0.4), (1.0, 0.3)):
            f = np.full((ny, nx), base)
            fx = np.zeros((ny, nx))
            fy = np.zeros((ny, nx))
            for _ in range(3):
                kx, ky = rng.integers(-3, 4, 2)
                ph0 = rng.uniform(0, 2 * np.pi)
                a = amp / 3 * rng.uniform(0.5, 1.0)
                arg = np.pi * (kx * x + ky * y) + ph0
                f = f + a * np.sin(arg)
                fx = fx + a * np.pi * kx * np.cos(arg)
                fy = fy + a * np.pi * ky * np.cos(arg)
            fields.append((f, fx, fy))
        (r, rx, ry), (u, ux, uy), (v, vx, vy), (p, px, py) = fields
        U, V = euler_from_primitive_2d(r, u, v, p, rx, ux, vx, px, gamma)
        _, W = euler_from_primitive_2d(r, u, v, p, ry, uy, vy, py, gamma)
    else:
        bx = rng.integers(2, 6)
        by = rng.integers(2, 6)
        ix = np.minimum((x / 2.0 * bx).astype(int), bx - 1)
        iy = np.minimum((y / 2.0 * by).astype(int), by - 1)
        blk = np.broadcast_to(iy * bx + ix, (ny, nx))
        nb = bx * by
        r = rng.uniform(0.2, 3.0, nb)[blk]
        p = rng.uniform(0.2, 3.0, nb)[blk]
        u = rng.uniform(-1.0, 1.0, nb)[blk]
        v = rng.uniform(-1.0, 1.0, nb)[blk]
        zero = np.zeros((ny, nx))
        U, _ = euler_from_primitive_2d(r, u, v, p, zero, zero, zero, zero, gamma)
        V = rng.normal(0.0, 1.0, (4, ny, nx))
        W = rng.normal(0.0, 1.0, (4, ny, nx))
    S = np.zeros((3, 4, ny, nx))
    S[0], S[1], S[2] = U, V, W
    return S, 2.0 / nx, 2.0 / ny


def euler1d_random(n: int, seed: int, kind: str = "smooth", gamma: float = 1.4):
    """Seeded 1D Euler test states on [-5, 5] for parity (see euler2d_random)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = centres(n, -5.0, 5.0)
    if kind == "smooth":
        fields = []
        for base, amp in ((1.0, 0.3), (0.2, 0.4), (1.0, 0.3)):
            f = np.full(n, base)
            fx = np.zeros(n)
            for _ in range(3):
                k = rng.integers(1, 5)
                ph0 = rng.uniform(0, 2 * np.pi)
                a = amp / 3 * rng.uniform(0.5, 1.0)
                f = f + a * np.sin(np.pi * k * x / 5 + ph0)
                fx = fx + a * np.pi * k / 5 * np.cos(np.pi * k * x / 5 + ph0)
            fields.append((f, fx))
        (r, rx), (u, ux), (p, px) = fields
        U, V = euler_from_primitive_1d(r, u, p, rx, ux, px, gamma)
    else:
        nb = rng.integers(3, 9)
        blk = np.minimum(((x + 5) / 10 * nb).astype(int), nb - 1)
        r = rng.uniform(0.2, 3.0, nb)[blk]
        p = rng.uniform(0.2, 3.0, nb)[blk]
        u = rng.uniform(-1.0, 1.0, nb)[blk]
        zero = np.zeros(n)
        U, _ = euler_from_primitive_1d(r, u, p, zero, zero, zero, gamma)
        V = rng.normal(0.0, 1.0, (3, n))
    S = np.zeros((2, 3, 1, n))
    S[0, :, 0] = U
    S[1, :, 0] = V
    return S, 10.0 / n


# ----------------------------------------------------------------------------------------------
# Seeded 1D Euler Riemann problems on [-5, 5] with transmissive boundaries

def _riemann_star(rl, ul, pl, rr, ur, pr, gamma):
    """Pressure and velocity in the star region of the exact Riemann solver (Newton iteration on
    the pressure function, textbook form)."""
    cl, cr = math.sqrt(gamma * pl / rl), math.sqrt(gamma * pr / rr)

    def fk(p, rk, pk, ck):
        if p > pk:  # shock
            A = 2.0 / ((gamma + 1) * rk)
            B = (gamma - 1) / (gamma + 1) * pk
            q = math.sqrt(A / (p + B))
            return (p - pk) * q, q * (1 - 0.5 * (p - pk) / (p + B))
        pr_ = (p / pk) ** ((gamma - 1) / (2 * gamma))  # rarefaction
        return 2 * ck / (gamma - 1) * (pr_ - 1), 1.0 / (rk * ck) * (p / pk) ** (-(gamma + 1) / (2 * gamma))

    p = max(1e-8, 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr))
    for _ in range(100):
        f1, d1 = fk(p, rl, pl, cl)
        f2, d2 = fk(p, rr, pr, cr)
        pn = p - (f1 + f2 + ur - ul) / (d1 + d2)
        pn = max(pn, 1e-10)
        if abs(pn - p) < 1e-14 * (pn + p):
            p = pn
            break
        p = pn
    f1, _ = fk(p, rl, pl, cl)
    f2, _ = fk(p, rr, pr, cr)
    u = 0.5 * (ul + ur) + 0.5 * (f2 - f1)
    return p, u


def riemann_wave_extent(rl, ul, pl, rr, ur, pr, gamma=1.4):
    """(leftmost, rightmost) wave speeds of the exact Riemann solution."""
    cl, cr = math.sqrt(gamma * pl / rl), math.sqrt(gamma * pr / rr)
    ps, us = _riemann_star(rl, ul, pl, rr, ur, pr, gamma)
    if ps > pl:
        sl = ul - cl * math.sqrt((gamma + 1) / (2 * gamma) * ps / pl + (gamma - 1) / (2 * gamma))
    else:
        sl = ul - cl
    if ps > pr:
        sr = ur + cr * math.sqrt((gamma + 1) / (2 * gamma) * ps / pr + (gamma - 1) / (2 * gamma))
    else:
        sr = ur + cr
    return sl, sr


def euler1d_riemann(n: int, seed: int, gamma: float = 1.4):
    """Seeded Riemann data on [-5, 5]: rho ~ U[0.1, 5], u ~ U[-1, 1], p ~ U[0.1, 10] on each side,
    jump at x0 ~ U[-2, 2], right density times (1 + 0.2 sin(k x)), k ~ {1..10}.  Derivatives are the
    exact derivatives of the smooth parts (zero on the constant left part).  A centre exactly at x0
    takes the left state.  Returns (state, dx, t_stop) with t_stop the time at which the fastest wave
    of the unperturbed Riemann problem has covered 80% of its distance to the boundary."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rl, rr = rng.uniform(0.1, 5.0, 2)
    ul, ur = rng.uniform(-1.0, 1.0, 2)
    pl, pr = rng.uniform(0.1, 10.0, 2)
    x0 = rng.uniform(-2.0, 2.0)
    k = int(rng.integers(1, 11))
    x = centres(n, -5.0, 5.0)
    right = x > x0
    rho = np.where(right, rr * (1 + 0.2 * np.sin(k * x)), rl)
    rx = np.where(right, rr * 0.2 * k * np.cos(k * x), 0.0)
    u = np.where(right, ur, ul)
    p = np.where(right, pr, pl)
    zero = np.zeros(n)
    U, V = euler_from_primitive_1d(rho, u, p, rx, zero, zero, gamma)
    S = np.zeros((2, 3, 1, n))
    S[0, :, 0] = U
    S[1, :, 0] = V
    sl, sr = riemann_wave_extent(rl, ul, pl, rr, ur, pr, gamma)
    tl = (x0 + 5.0) / -sl if sl < 0 else math.inf
    tr = (5.0 - x0) / sr if sr > 0 else math.inf
    t_stop = 0.8 * min(tl, tr)
    return S, 10.0 / n, t_stop


# ----------------------------------------------------------------------------------------------
# Batched uneven workload and the adjoint initial state

def batched_instances(seed: int = 3000, n1d: int = 256, n2d: int = 32):
    """Instance list of the batched sweep: n1d 1D Euler instances with N log-uniform in
    [128, 16384] and n2d 2D Euler grids with side in {128, 256, 512, 1024}.  Returns a list of
    dicts (dim, nx, ny, seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(n1d):
        n = int(round(math.exp(rng.uniform(math.log(128), math.log(16384)))))
        out.append({"dim": 1, "nx": n, "ny": 1, "seed": seed + k})
    sides = (128, 256, 512, 1024)
    for k in range(n2d):
        s = int(sides[rng.integers(0, 4)])
        out.append({"dim": 2, "nx": s, "ny": s, "seed": seed + n1d + k})
    return out


def euler2d_adjoint_init(n: int, seed: int = 4000, gamma: float = 1.4):
    """Smooth wave (velocity 0.7, 0.3) plus 8 seeded Fourier modes of amplitude 0.05/8 each in rho
    and in P; integer wave vectors in {-4..4}^2 without (0, 0), phases U[0, 2 pi)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = centres(n, 0.0, 2.0)[None, :]
    y = centres(n, 0.0, 2.0)[:, None]
    ph = np.pi * (x + y)
    rho = 1 + 0.2 * np.sin(ph)
    rx = 0.2 * np.pi * np.cos(ph)
    ry = rx.copy()
    p = np.ones((n, n))
    px = np.zeros((n, n))
    py = np.zeros((n, n))
    for target in ("rho", "p"):
        for _ in range(8):
            while True:
                kx, ky = rng.integers(-4, 5, 2)
                if kx != 0 or ky != 0:
                    break
            phase = rng.uniform(0, 2 * np.pi)
            a = 0.05 / 8
            arg = np.pi * (kx * x + ky * y) + phase
            if target == "rho":
                rho = rho + a * np.sin(arg)
                rx = rx + a * np.pi * kx * np.cos(arg)
                ry = ry + a * np.pi * ky * np.cos(arg)
            else:
                p = p + a * np.sin(arg)
                px = px + a * np.pi * kx * np.cos(arg)
                py = py + a * np.pi * ky * np.cos(arg)
    one, zero = np.ones((n, n)), np.zeros((n, n))
    U, V = euler_from_primitive_2d(rho, 0.7 * one, 0.3 * one, p, rx, zero, zero, px, gamma)
    _, W = euler_from_primitive_2d(rho, 0.7 * one, 0.3 * one, p, ry, zero, zero, py, gamma)
    S = np.zeros((3, 4, n, n))
    S[0], S[1], S[2] = U, V, W
    return S, 2.0 / n, 2.0 / n


def scalar_random(dim: int, nx: int, ny: int, seed: int, kind: str = "smooth"):
    """Seeded scalar test states on [0, 2] (x [0, 2]): 'smooth' = a few random Fourier modes with
    exact derivatives; 'jumps' = random piecewise-constant blocks with random derivative noise."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ny = ny if dim == 2 else 1
    x = centres(nx, 0.0, 2.0)[None, :]
    y = centres(ny, 0.0, 2.0)[:, None] if dim == 2 else np.zeros((1, 1))
    nf = dim + 1
    S = np.zeros((nf, 1, ny, nx))
    if kind == "smooth":
        f = np.full((ny, nx), 0.5)
        fx = np.zeros((ny, nx))
        fy = np.zeros((ny, nx))
        for _ in range(3):
            kx = rng.integers(-3, 4)
            ky = rng.integers(-3, 4) if dim == 2 else 0
            ph0 = rng.uniform(0, 2 * np.pi)
            a = rng.uniform(0.2, 0.5)
            arg = np.pi * (kx * x + ky * y) + ph0
            f = f + a * np.sin(arg)
            fx = fx + a * np.pi * kx * np.cos(arg)
            fy = fy + a * np.pi * ky * np.cos(arg)
        S[0, 0], S[1, 0] = f, fx
        if dim == 2:
            S[2, 0] = fy
    else:
        nb = int(rng.integers(3, 8))
        ix = np.minimum((x / 2.0 * nb).astype(int), nb - 1)
        iy = np.minimum((y / 2.0 * nb).astype(int), nb - 1) if dim == 2 else 0
        blk = np.broadcast_to(iy * nb + ix, (ny, nx))
        S[0, 0] = rng.uniform(-1.0, 2.0, nb * nb)[blk]
        for f in range(1, nf):
            S[f, 0] = rng.normal(0.0, 1.0, (ny, nx))
    return S, 2.0 / nx, 2.0 / ny


def batched_states(instances, gamma: float = 1.4):
    """Initial states of the batched sweep: 1D instances take the seeded Riemann data (transmissive
    boundaries), 2D instances alternate between the smooth wave and the four-quadrant data (by seed
    parity, periodic boundaries).  Returns a list of (desc, state) with desc as hweno_desc fields."""
    out = []
    for inst in instances:
        if inst["dim"] == 1:
            S, dx, _ = euler1d_riemann(inst["nx"], inst["seed"], gamma)
            out.append(({"dim": 1, "nx": inst["nx"], "ny": 1, "dx": dx, "dy": dx, "bc": "transmissive",
                         "gamma": gamma}, S))
        else:
            n = inst["nx"]
            if inst["seed"] % 2 == 0:
                S, dx, dy = euler2d_smooth(n)
            else:
                S, dx, dy = euler2d_quadrants(n, seed=inst["seed"])
            out.append(({"dim": 2, "nx": n, "ny": n, "dx": dx, "dy": dy, "bc": "periodic", "gamma": gamma}, S))
    return out


def blast_wave_1d(n: int, gamma: float = 1.4, p_mid: float = 0.01):
    """Woodward-Colella blast wave on [0, 1] (Example 4.4): rho = 1, u = 0, P = 1000 / p_mid / 100 on
    [0, 0.1), [0.1, 0.9), [0.9, 1]; derivatives zero.  Reflective walls at both ends.

    p_mid = 0.01 is the printed problem.  The scheme without a positivity safeguard loses it in
    the first stage: the central D-term of the momentum flux at the face next to the 1e5
    pressure jump moves the first low-pressure node with a kinetic energy above its internal
    energy.  p_mid = 1 keeps the geometry, the wall reflections and the interaction of the two
    blasts, with a pressure ratio of 1e3."""
    x = centres(n, 0.0, 1.0)
    p = np.where(x < 0.1, 1000.0, np.where(x < 0.9, p_mid, 100.0))
    one, zero = np.ones(n), np.zeros(n)
    U, _ = euler_from_primitive_1d(one, zero, p, zero, zero, zero, gamma)
    S = np.zeros((2, 3, 1, n))
    S[0, :, 0] = U
    return S, 1.0 / n


def rayleigh_taylor(nx: int, ny: int = None, gamma: float = 5.0 / 3.0):
    """Rayleigh-Taylor instability of Example 4.11 on [0, 0.25] x [0, 1] (gravity g = 1 along +y):
    rho = 2, P = 2y + 1 below y = 1/2; rho = 1, P = y + 1.5 above; u = 0,
    v = -0.025 c cos(8 pi x) with c = sqrt(gamma P / rho).  Derivatives are the exact derivatives of
    each side's smooth expressions (the interface is a jump).  Reflective walls left and right;
    the bottom and top hold the fixed states (2, 0, 0, 1) and (1, 0, 0, 2.5).
    Returns (S, dx, dy, fixed) with fixed = {2: U_bottom, 3: U_top} in conserved variables."""
    ny = 4 * nx if ny is None else ny
    x = centres(nx, 0.0, 0.25)[None, :] * np.ones((ny, 1))
    y = centres(ny, 0.0, 1.0)[:, None] * np.ones((1, nx))
    low = y < 0.5
    rho = np.where(low, 2.0, 1.0)
    p = np.where(low, 2.0 * y + 1.0, y + 1.5)
    p_y = np.where(low, 2.0, 1.0)
    c = np.sqrt(gamma * p / rho)
    c_y = 0.5 * gamma * p_y / (rho * c)
    cosx, sinx = np.cos(8 * np.pi * x), np.sin(8 * np.pi * x)
    v = -0.025 * c * cosx
    v_x = 0.025 * c * 8 * np.pi * sinx
    v_y = -0.025 * c_y * cosx
    zero = np.zeros_like(x)
    U, V = euler_from_primitive_2d(rho, zero, v, p, zero, zero, v_x, zero, gamma)
    _, Wd = euler_from_primitive_2d(rho, zero, v, p, zero, zero, v_y, p_y, gamma)
    S = np.stack([U, V, Wd])
    fixed = {2: [2.0, 0.0, 0.0, 1.0 / (gamma - 1)], 3: [1.0, 0.0, 0.0, 2.5 / (gamma - 1)]}
    return S, 0.25 / nx, 1.0 / ny, fixed


def hydrostatic_column(nx: int, ny: int, rho0: float = 1.5, p0: float = 2.0, g: float = 1.0,
                       gamma: float = 1.4):
    """Fluid at rest with constant density and P = p0 + g rho0 y on [0, 1]^2 (exact derivatives):
    the pressure gradient balances the gravity source of Eq. (euler2d-s)."""
    x = centres(nx, 0.0, 1.0)[None, :] * np.ones((ny, 1))
    y = centres(ny, 0.0, 1.0)[:, None] * np.ones((1, nx))
    rho = rho0 * np.ones_like(x)
    p = p0 + g * rho0 * y
    zero = np.zeros_like(x)
    U, V = euler_from_primitive_2d(rho, zero, zero, p, zero, zero, zero, zero, gamma)
    _, Wd = euler_from_primitive_2d(rho, zero, zero, p, zero, zero, zero, g * rho0 * np.ones_like(x), gamma)
    return np.stack([U, V, Wd]), 1.0 / nx, 1.0 / ny
