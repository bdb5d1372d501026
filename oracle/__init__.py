"""ctypes wrapper of the HWENO-I CPU oracle (``hweno_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` are its only users.  The product package never imports this module and this module
never imports the product package.

The oracle follows the paper (Xie, Tao, Jiao, Zhang, arXiv 2411.11229) step by step in FP64:
Sec. 2.1 (HWENO interpolation and limiter), Sec. 2.2 (central Hermite D-terms), Eqs. (flux-1d),
(flux-LF), (fully-hweno), Sec. 3 (2D, Eq. mixed) and the characteristic-decomposition remarks.
The ``*_ext`` functions evaluate the same formulas in long double (the exact value that the rounding
of an FP64 evaluation is measured against).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hweno_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ADVECTION, BURGERS, EULER = 0, 1, 2
BC_PERIODIC, BC_TRANSMISSIVE, BC_REFLECTIVE, BC_FIXED = 0, 1, 2, 3
# scheme variants: v^+/- with the nonlinear weights, D-terms of Eq. (Cd-2), characteristic
# decomposition with the eigenvectors of each side's centre cell, LF coefficients held for the
# whole step, local LF coefficients (per face)
FLAG_V_WEIGHTED, FLAG_CD2, FLAG_R2, FLAG_ALPHA_STEP, FLAG_ALPHA_LOCAL = 1, 2, 4, 8, 16


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-O2, no FMA contraction) into oracle/liboracle.so."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-pthread",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Cfg(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("system", ctypes.c_int32), ("nx", ctypes.c_int32),
                ("ny", ctypes.c_int32), ("bc", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("gamma", ctypes.c_double),
                ("gamma0", ctypes.c_double), ("d0", ctypes.c_double), ("eps", ctypes.c_double),
                ("ax", ctypes.c_double), ("ay", ctypes.c_double), ("grav", ctypes.c_double),
                ("side", ctypes.c_int32 * 4), ("fixed", (ctypes.c_double * 4) * 4)]


def make_cfg(dim, system, nx, ny=1, dx=1.0, dy=1.0, gamma=1.4, bc=BC_PERIODIC, gamma0=None, d0=0.9,
             eps=1e-10, ax=1.0, ay=1.0, flags=0, grav=0.0, sides=None, fixed=None) -> Cfg:
    """Scheme parameters; gamma0 defaults to 0.95 (1D) / 0.99 (2D) and d0 to 0.9 (Sec. 4).

    bc applies to every side unless ``sides`` gives the four types (x-low, x-high, y-low, y-high);
    ``fixed`` maps a side index to the conserved state held in its ghost cells (BC_FIXED).
    grav: g of the gravity source of Eq. (euler2d-s) (2D Euler)."""
    if gamma0 is None:
        gamma0 = 0.95 if dim == 1 else 0.99
    c = Cfg(dim, system, nx, ny if dim == 2 else 1, bc, flags, dx, dy if dim == 2 else dx, gamma,
            gamma0, d0, eps, ax, ay, grav)
    for k, t in enumerate(sides if sides is not None else (bc,) * 4):
        c.side[k] = t
    for k, U in (fixed or {}).items():
        for j, u in enumerate(U):
            c.fixed[k][j] = float(u)
    return c


_P = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            CP = ctypes.POINTER(Cfg)
            L.oracle_set_threads.argtypes = [ctypes.c_int]
            L.oracle_set_threads.restype = ctypes.c_int
            L.oracle_state_size.argtypes = [CP]
            L.oracle_state_size.restype = ctypes.c_longlong
            L.oracle_max_wavespeed.argtypes = [CP, _P, _P, _P]
            L.oracle_rhs.argtypes = [CP, _P, _P, _P]
            L.oracle_rhs_alpha.argtypes = [CP, _P, ctypes.c_double, ctypes.c_double, _P, _P]
            L.oracle_rhs_cells.argtypes = [CP, _P, ctypes.c_double, ctypes.c_double, ctypes.c_longlong,
                                           ctypes.POINTER(ctypes.c_longlong), _P, _P]
            L.oracle_steps.argtypes = [CP, _P, ctypes.c_double, ctypes.c_int]
            L.oracle_cfl_dt.argtypes = [CP, _P, ctypes.c_double, ctypes.c_double]
            L.oracle_cfl_dt.restype = ctypes.c_double
            L.oracle_run.argtypes = [CP, _P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_longlong, _P]
            L.oracle_run.restype = ctypes.c_longlong
            L.oracle_ext_mantissa_bits.argtypes = []
            L.oracle_ext_mantissa_bits.restype = ctypes.c_int
            L.oracle_rhs_ext.argtypes = [CP, _P, _P, _P]
            L.oracle_rhs_cells_ext.argtypes = [CP, _P, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong),
                                               _P, _P]
            L.oracle_run_ext.argtypes = [CP, _P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_longlong, _P]
            L.oracle_run_ext.restype = ctypes.c_longlong
            L.oracle_count_flops.argtypes = [CP, ctypes.POINTER(ctypes.c_longlong)]
            L.oracle_count_stencil.argtypes = [ctypes.POINTER(ctypes.c_longlong)]
            L.oracle_stage_vjp.argtypes = [CP, _P, ctypes.c_double, ctypes.c_double, _P, _P, _P]
            L.oracle_stage_jvp.argtypes = [CP, _P, ctypes.c_double, ctypes.c_double, _P, _P, _P]
            L.oracle_steps_record.argtypes = [CP, _P, ctypes.c_int, ctypes.c_double, _P, _P]
            L.oracle_steps_replay.argtypes = [CP, _P, ctypes.c_int, _P, _P]
            L.oracle_adjoint_step.argtypes = [CP, _P, ctypes.c_double, _P, _P, _P]
            L.oracle_stencil.argtypes = [_P, _P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int, _P]
            L.oracle_dterms.argtypes = [_P, _P, ctypes.c_double, _P]
            L.oracle_dterms2.argtypes = [_P, _P, ctypes.c_double, _P]
            L.oracle_euler_flux.argtypes = [CP, ctypes.c_int, _P, _P]
            L.oracle_euler_jacobian.argtypes = [CP, ctypes.c_int, _P, _P]
            L.oracle_euler_eigen.argtypes = [CP, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P]
            _lib = L
    return _lib


def set_threads(n: int = 0) -> int:
    """Threads the operator runs on (0: all hardware threads, the default; 1: one).  Lines of a
    sweep and values of an update are split over the threads; the results are the same bit for bit
    for every thread count.  Returns the count the next calls use."""
    return int(lib().oracle_set_threads(int(n)))


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_P)


def _check(rc):
    if rc != 0:
        raise ValueError(f"oracle call failed ({rc})")


def state_size(cfg: Cfg) -> int:
    n = lib().oracle_state_size(ctypes.byref(cfg))
    if n < 0:
        raise ValueError("invalid configuration")
    return int(n)


def max_wavespeed(cfg: Cfg, S: np.ndarray):
    S = np.ascontiguousarray(S, dtype=np.float64)
    ax, ay = np.zeros(1), np.zeros(1)
    _check(lib().oracle_max_wavespeed(ctypes.byref(cfg), _ptr(S), _ptr(ax), _ptr(ay)))
    return float(ax[0]), float(ay[0])


def rhs(cfg: Cfg, S: np.ndarray, alpha=None):
    """(L(S), M(S)) of one stage; M = (U, V~, W~).  Arrays have the state's shape."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    assert S.size == state_size(cfg)
    L = np.zeros_like(S)
    M = np.zeros_like(S)
    if alpha is None:
        _check(lib().oracle_rhs(ctypes.byref(cfg), _ptr(S), _ptr(L), _ptr(M)))
    else:
        _check(lib().oracle_rhs_alpha(ctypes.byref(cfg), _ptr(S), float(alpha[0]), float(alpha[1]),
                                      _ptr(L), _ptr(M)))
    return L, M


def rhs_cells(cfg: Cfg, S: np.ndarray, idx, alpha):
    """L and M at the cells with flat indices idx (j*nx + i); arrays [ncell, field, comp]."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    nf = 2 if cfg.dim == 1 else 3
    m = S.size // (nf * cfg.nx * cfg.ny)
    L = np.zeros((idx.size, nf, m))
    M = np.zeros((idx.size, nf, m))
    _check(lib().oracle_rhs_cells(ctypes.byref(cfg), _ptr(S), float(alpha[0]), float(alpha[1]), idx.size,
                                  idx.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), _ptr(L), _ptr(M)))
    return L, M


def steps(cfg: Cfg, S: np.ndarray, dt: float, nsteps: int = 1) -> np.ndarray:
    out = np.array(S, dtype=np.float64, copy=True, order="C")
    _check(lib().oracle_steps(ctypes.byref(cfg), _ptr(out), float(dt), int(nsteps)))
    return out


def cfl_dt(cfg: Cfg, S: np.ndarray, cfl: float = 0.6, dx_pow: float = 1.0) -> float:
    S = np.ascontiguousarray(S, dtype=np.float64)
    return float(lib().oracle_cfl_dt(ctypes.byref(cfg), _ptr(S), float(cfl), float(dx_pow)))


def run(cfg: Cfg, S: np.ndarray, t_end: float, cfl: float = 0.6, dx_pow: float = 1.0,
        max_steps: int = 0):
    """CFL time stepping to t_end (last step clamped).  Returns (state, steps, t)."""
    out = np.array(S, dtype=np.float64, copy=True, order="C")
    t = np.zeros(1)
    n = lib().oracle_run(ctypes.byref(cfg), _ptr(out), float(t_end), float(cfl), float(dx_pow),
                         int(max_steps), _ptr(t))
    if n < 0:
        raise ValueError("oracle run failed")
    return out, int(n), float(t[0])


def ext_mantissa_bits() -> int:
    """Significand bits of the extended-precision evaluation (64 on x86-64, 113 on AArch64)."""
    return int(lib().oracle_ext_mantissa_bits())


def rhs_ext(cfg: Cfg, S: np.ndarray):
    """rhs() with every value computed from the data held in long double (the LF coefficients from
    S); the scheme's coefficients are the same double constants.  Results rounded to double."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    assert S.size == state_size(cfg)
    L = np.zeros_like(S)
    M = np.zeros_like(S)
    _check(lib().oracle_rhs_ext(ctypes.byref(cfg), _ptr(S), _ptr(L), _ptr(M)))
    return L, M


def rhs_cells_ext(cfg: Cfg, S: np.ndarray, idx):
    """rhs_cells() in long double, with the LF coefficients of the whole of S; [ncell, field, comp]."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    nf = 2 if cfg.dim == 1 else 3
    m = S.size // (nf * cfg.nx * cfg.ny)
    L = np.zeros((idx.size, nf, m))
    M = np.zeros((idx.size, nf, m))
    _check(lib().oracle_rhs_cells_ext(ctypes.byref(cfg), _ptr(S), idx.size,
                                      idx.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), _ptr(L), _ptr(M)))
    return L, M


def run_ext(cfg: Cfg, S: np.ndarray, t_end: float, cfl: float = 0.6, dx_pow: float = 1.0,
            max_steps: int = 0):
    """run() with the state held in long double between steps.  Returns (state, steps, t)."""
    out = np.array(S, dtype=np.float64, copy=True, order="C")
    t = np.zeros(1)
    n = lib().oracle_run_ext(ctypes.byref(cfg), _ptr(out), float(t_end), float(cfl), float(dx_pow),
                             int(max_steps), _ptr(t))
    if n < 0:
        raise ValueError("oracle run failed")
    return out, int(n), float(t[0])


def count_flops(cfg: Cfg) -> dict:
    """Floating-point operation counts of the scheme as the oracle writes it, with nontrivial
    operands (see the C source): per face, per cell and direction, and per cell-step."""
    out = (ctypes.c_longlong * 6)()
    _check(lib().oracle_count_flops(ctypes.byref(cfg), out))
    keys = ("face", "nodal_per_dir", "modified_derivative_per_dir", "wavespeed_per_dir",
            "update", "per_cell_step")
    return dict(zip(keys, [int(v) for v in out]))


def count_stencil() -> dict:
    """Operation counts of one scalar HWENO stencil: the face part (u^-, v^-), the face part with the
    weighted derivative, and the cell part (v~)."""
    out = (ctypes.c_longlong * 3)()
    _check(lib().oracle_count_stencil(out))
    return {"face": int(out[0]), "face_v_weighted": int(out[1]), "cell": int(out[2])}


def stage_vjp(cfg: Cfg, S, alpha, muM, muL):
    """(dM/dS)^T muM + (dL/dS)^T muL at S with the LF coefficients alpha = (ax, ay) held fixed."""
    S, muM, muL = (np.ascontiguousarray(a, dtype=np.float64) for a in (S, muM, muL))
    lam = np.zeros_like(S)
    _check(lib().oracle_stage_vjp(ctypes.byref(cfg), _ptr(S), float(alpha[0]), float(alpha[1]), _ptr(muM),
                                  _ptr(muL), _ptr(lam)))
    return lam


def stage_jvp(cfg: Cfg, S, alpha, delta):
    """(dM/dS delta, dL/dS delta) at S with alpha held fixed (forward-mode derivatives)."""
    S, delta = (np.ascontiguousarray(a, dtype=np.float64) for a in (S, delta))
    jM, jL = np.zeros_like(S), np.zeros_like(S)
    _check(lib().oracle_stage_jvp(ctypes.byref(cfg), _ptr(S), float(alpha[0]), float(alpha[1]), _ptr(delta),
                                  _ptr(jM), _ptr(jL)))
    return jM, jL


def steps_record(cfg: Cfg, S, nsteps: int, cfl: float = 0.6):
    """nsteps CFL steps; returns (state, dts[nsteps], alphas[nsteps, 6])."""
    out = np.array(S, dtype=np.float64, copy=True, order="C")
    dts = np.zeros(nsteps)
    alphas = np.zeros((nsteps, 6))
    _check(lib().oracle_steps_record(ctypes.byref(cfg), _ptr(out), int(nsteps), float(cfl), _ptr(dts),
                                     _ptr(alphas)))
    return out, dts, alphas


def steps_replay(cfg: Cfg, S, dts, alphas):
    """Steps with the given step sizes and per-stage LF coefficients."""
    out = np.array(S, dtype=np.float64, copy=True, order="C")
    dts = np.ascontiguousarray(dts, dtype=np.float64)
    alphas = np.ascontiguousarray(alphas, dtype=np.float64)
    _check(lib().oracle_steps_replay(ctypes.byref(cfg), _ptr(out), int(dts.size), _ptr(dts), _ptr(alphas)))
    return out


def adjoint_step(cfg: Cfg, Sn, dt: float, alpha6, lam_in):
    """(dS^{n+1}/dS^n)^T lam_in for one SSP-RK3 step with fixed dt and per-stage alpha."""
    Sn, lam_in = (np.ascontiguousarray(a, dtype=np.float64) for a in (Sn, lam_in))
    alpha6 = np.ascontiguousarray(alpha6, dtype=np.float64)
    lam = np.zeros_like(Sn)
    _check(lib().oracle_adjoint_step(ctypes.byref(cfg), _ptr(Sn), float(dt), _ptr(alpha6), _ptr(lam_in),
                                     _ptr(lam)))
    return lam


def stencil(u3, v2, dx, gamma0=0.95, d0=0.9, eps=1e-10, v_weighted=False) -> dict:
    """All intermediates of one HWENO stencil (Sec. 2.1); v_weighted: the FLAG_V_WEIGHTED variant
    of v^+/-."""
    u3 = np.ascontiguousarray(u3, dtype=np.float64)
    v2 = np.ascontiguousarray(v2, dtype=np.float64)
    out = np.zeros(22)
    _check(lib().oracle_stencil(_ptr(u3), _ptr(v2), float(dx), float(gamma0), float(d0), float(eps),
                                int(bool(v_weighted)), _ptr(out)))
    return {"p": out[0:3], "dp0_half": out[3], "dp_center": out[4:7], "beta": out[7:10],
            "tau": out[10], "omega_g": out[11:14], "omega_d": out[14:17], "u_minus": out[17],
            "v_minus": out[18], "v_mod": out[19], "u_plus": out[20], "v_plus": out[21]}


def dterms(f4, h2, dx, form: int = 1):
    """(D(f), D(h)) of Eq. (DfDh) from f_{i-1..i+2} and, for form 1 (Eq. Cd-1), h_{i-1}, h_{i+2};
    for form 2 (Eq. Cd-2), h_i, h_{i+1}."""
    f4 = np.ascontiguousarray(f4, dtype=np.float64)
    h2 = np.ascontiguousarray(h2, dtype=np.float64)
    out = np.zeros(2)
    fn = lib().oracle_dterms if form == 1 else lib().oracle_dterms2
    _check(fn(_ptr(f4), _ptr(h2), float(dx), _ptr(out)))
    return float(out[0]), float(out[1])


def euler_flux(cfg: Cfg, direction: int, U):
    U = np.ascontiguousarray(U, dtype=np.float64)
    F = np.zeros_like(U)
    _check(lib().oracle_euler_flux(ctypes.byref(cfg), int(direction), _ptr(U), _ptr(F)))
    return F


def euler_jacobian(cfg: Cfg, direction: int, U):
    U = np.ascontiguousarray(U, dtype=np.float64)
    m = U.size
    A = np.zeros(m * m)
    _check(lib().oracle_euler_jacobian(ctypes.byref(cfg), int(direction), _ptr(U), _ptr(A)))
    return A.reshape(m, m)


def euler_eigen(cfg: Cfg, direction: int, UL, UR=None):
    """(R, L, (u, v, H, c)) at the Roe average of UL, UR, or at the cell state UL if UR is None."""
    UL = np.ascontiguousarray(UL, dtype=np.float64)
    which = 1 if UR is None else 0
    UR = UL if UR is None else np.ascontiguousarray(UR, dtype=np.float64)
    m = UL.size
    Rm, Lm, st = np.zeros(m * m), np.zeros(m * m), np.zeros(4)
    _check(lib().oracle_euler_eigen(ctypes.byref(cfg), int(direction), which, _ptr(UL), _ptr(UR),
                                    _ptr(Rm), _ptr(Lm), _ptr(st)))
    return Rm.reshape(m, m), Lm.reshape(m, m), st
