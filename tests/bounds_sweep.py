"""Every family of entry points over ragged grids (down to 5 cells a side), every boundary type and
the scheme variants, on the library the environment selects (HWENO_BOUNDS_CHECK=1: the
bounds-checked build), with the results saved to the .npz file named on the command line.  With
the bounds-checked build it first runs the check's self-test and at the end prints the count of
out-of-range indices.  Run by tests/test_gpu_bounds.py as a child process, once per library.
"""
import ctypes
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import workloads as W  # noqa: E402
from paper_2411_11229_gb300 import Batch, Solver  # noqa: E402
from paper_2411_11229_gb300 import _capi as C  # noqa: E402

P, T, R, F = C.HWENO_BC_PERIODIC, C.HWENO_BC_TRANSMISSIVE, C.HWENO_BC_REFLECTIVE, C.HWENO_BC_FIXED
VW, CD2, R2 = C.HWENO_FLAG_V_WEIGHTED, C.HWENO_FLAG_CD2, C.HWENO_FLAG_R2
AST, ALOC = C.HWENO_FLAG_ALPHA_STEP, C.HWENO_FLAG_ALPHA_LOCAL
BCN = {P: "periodic", T: "transmissive", R: "reflective"}


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _state(dim, system, nx, ny, kind, seed):
    if system == "euler":
        if dim == 1:
            S, dx = W.euler1d_random(nx, seed, kind)
            return S, dx, dx
        return W.euler2d_random(nx, ny, seed, kind)
    return W.scalar_random(dim, nx, ny, seed, kind)


def _fixed(S, dim):
    U = S[0]
    out = {0: U[:, :, 0].mean(axis=1) * 1.05, 1: U[:, :, -1].mean(axis=1) * 0.97}
    if dim == 2:
        out[2] = U[:, 0, :].mean(axis=1) * 1.02
        out[3] = U[:, -1, :].mean(axis=1) * 0.99
    return out


def plain(res):
    for dim, sizes in ((1, [(5, 1), (6, 1), (13, 1)]), (2, [(5, 5), (6, 9), (13, 7)])):
        for system in ("advection", "burgers", "euler"):
            for bc in (P, T, R) if system == "euler" else (P, T):
                for nx, ny in sizes:
                    for kind in ("smooth", "jumps"):
                        S, dx, dy = _state(dim, system, nx, ny, kind, seed=nx * 7 + ny)
                        s = Solver(dim, system, nx, ny, dx=dx, dy=dy, bc=BCN[bc])
                        s.set_state(S)
                        key = f"plain_{dim}_{system}_{bc}_{nx}_{ny}_{kind}"
                        L, M = s.rhs()
                        res[key + "_L"], res[key + "_M"] = L.cpu().numpy(), M.cpu().numpy()
                        res[key + "_a"] = np.array(s.max_wavespeed())
                        s.set_time(0.0, 0.0)
                        s.step(0.0, 2)
                        res[key + "_S2"] = s.state.cpu().numpy()
                        s.close()


def variants(res):
    cases = [(1, "burgers", 6, 1, VW | CD2, (T, F, P, P), 0.0), (1, "euler", 6, 1, R2, (R, F, P, P), 0.0),
             (1, "euler", 7, 1, VW | CD2 | R2, (F, R, P, P), 0.0), (1, "euler", 9, 1, ALOC, (F, R, P, P), 0.0),
             (2, "advection", 6, 5, CD2, (F, T, P, P), 0.0), (2, "euler", 6, 9, VW | CD2 | R2, (R, R, F, F), 0.0),
             (2, "euler", 7, 5, ALOC | R2, (F, T, R, F), 0.0), (2, "euler", 5, 6, AST | VW | CD2 | R2, (T, F, R, R), 0.0),
             (2, "euler", 6, 8, R2, (R, R, F, F), 1.0), (2, "euler", 5, 7, 0, (F, R, P, P), 1.0)]
    for dim, system, nx, ny, flags, sides, grav in cases:
        for kind in ("smooth", "jumps"):
            S, dx, dy = _state(dim, system, nx, ny, kind, seed=nx * 11 + ny)
            fixed = _fixed(S, dim) if F in sides else None
            s = Solver(dim, system, nx, ny, dx=dx, dy=dy, flags=flags, sides=sides, fixed=fixed, grav=grav,
                       ax=0.8, ay=-0.6)
            s.set_state(S)
            key = f"var_{dim}_{system}_{nx}_{ny}_{flags}_{'_'.join(map(str, sides))}_{grav}_{kind}"
            L, M = s.rhs()
            res[key + "_L"], res[key + "_M"] = L.cpu().numpy(), M.cpu().numpy()
            s.set_time(0.0, 0.0)
            s.step(0.0, 2)
            res[key + "_S2"] = s.state.cpu().numpy()
            s.close()


def adjoint(res):
    lib = C.load()
    for dim, nx, ny in ((1, 5, 1), (1, 12, 1), (2, 5, 6), (2, 9, 7)):
        for bc in (P, T, R):
            if dim == 2:
                S, dx, dy = W.euler2d_random(nx, ny, nx + ny, "jumps")
            else:
                S, dx = W.euler1d_random(nx, nx + ny, "jumps")
                dy = dx
            s = Solver(dim, "euler", nx, ny, dx=dx, dy=dy, bc=BCN[bc])
            s.set_state(S)
            aws = torch.empty(int(lib.hweno_adjoint_workspace_bytes(s.h)), dtype=torch.uint8, device="cuda")
            rng = np.random.default_rng(nx * 3 + ny)
            dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
            Sd, mM, mL = dev(S), dev(rng.normal(size=S.shape)), dev(rng.normal(size=S.shape))
            al = dev(np.array(s.max_wavespeed()))
            lam = torch.empty_like(Sd)
            C.check(lib.hweno_stage_vjp(s.h, _ptr(Sd), _ptr(al), _ptr(mM), _ptr(mL), _ptr(lam), _ptr(aws)),
                    "hweno_stage_vjp")
            key = f"adj_{dim}_{bc}_{nx}_{ny}"
            res[key + "_vjp"] = lam.cpu().numpy()
            # a recorded CFL step with its stage inputs, then both adjoint step forms
            rec = torch.empty(7, dtype=torch.float64, device="cuda")
            S1, S2 = torch.empty_like(Sd), torch.empty_like(Sd)
            s.set_time(0.0, 0.0)
            s.step_stages(S1, S2)
            s.record(rec)
            dt, a6 = float(rec[0].item()), rec[1:].contiguous()
            lam_in = dev(rng.normal(size=S.shape))
            res[key + "_step"] = s.adjoint_step(Sd, dt, a6, lam_in).cpu().numpy()
            res[key + "_stages"] = s.adjoint_step_stages(Sd, S1, S2, dt, a6, lam_in).cpu().numpy()
            s.close()


def batch(res):
    items = []
    for n, seed, bc in ((5, 1, "transmissive"), (37, 2, "periodic"), (11, 3, "reflective")):
        S, dx = W.euler1d_random(n, seed, "jumps")
        items.append(({"dim": 1, "nx": n, "dx": dx, "bc": bc}, S))
    for (nx, ny), seed, bc in (((5, 6), 4, "periodic"), ((19, 7), 5, "reflective"), ((6, 13), 6, "transmissive")):
        S, dx, dy = W.euler2d_random(nx, ny, seed, "jumps")
        items.append(({"dim": 2, "nx": nx, "ny": ny, "dx": dx, "dy": dy, "bc": bc}, S))
    b = Batch([d for d, _ in items])
    for i, (_, S) in enumerate(items):
        b.set_state(i, S)
    b.set_time(0.0)
    b.step(2)
    b.tune()
    b.step(1)
    b.step_plain(1)
    b.sync()
    for i in range(len(items)):
        res[f"batch_{i}"] = b.view(i).cpu().numpy()
    b.close()


def static(res):
    lib = C.load()
    sysn = {"advection": C.HWENO_ADVECTION, "burgers": C.HWENO_BURGERS, "euler": C.HWENO_EULER}
    for dim, nx, ny in ((1, 5, 1), (2, 6, 5)):
        for system in ("advection", "burgers", "euler"):
            S, dx, dy = _state(dim, system, nx, ny, "jumps", seed=nx + 5 * ny)
            Sd = torch.as_tensor(S, device="cuda").contiguous()
            L, M = torch.empty_like(Sd), torch.empty_like(Sd)
            st = torch.cuda.current_stream()
            C.check(lib.hweno_rhs_static(dim, sysn[system], nx, ny, dx, dy, 1.4, C.HWENO_BC_TRANSMISSIVE, None,
                                         _ptr(Sd), _ptr(L), _ptr(M), ctypes.c_void_p(st.cuda_stream)),
                    "hweno_rhs_static")
            torch.cuda.synchronize()
            res[f"static_{dim}_{system}_L"], res[f"static_{dim}_{system}_M"] = L.cpu().numpy(), M.cpu().numpy()


def run_to_time(res):
    S, dx = W.euler1d_random(7, 9, "jumps")
    s = Solver(1, "euler", 7, dx=dx, bc="reflective")
    s.set_state(S)
    s.run(0.05)
    res["run_1d"] = s.state.cpu().numpy()
    s.close()


def main(out):
    lib = C.load()
    checked = C.bounds_checked()
    if checked:
        st = int(lib.hweno_bounds_selftest())
        print(f"bounds: selftest {st}")
        assert st == 1, st
    res = {}
    for part in (plain, variants, adjoint, batch, static, run_to_time):
        part(res)
    torch.cuda.synchronize()
    np.savez(out, **res)
    if checked:
        where = ctypes.c_int()
        n = int(lib.hweno_bounds_status(ctypes.byref(where)))
        print(f"bounds: out-of-range {n} first at {where.value}")
    print(f"arrays {len(res)}")


if __name__ == "__main__":
    main(sys.argv[1])
