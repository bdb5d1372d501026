"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element.

Bars (FP64): one stage (L and M of the spatial operator) within 1e-12 relative max-norm per
plane; one SSP-RK3 step within 1e-12; 100 steps within 1e-10.  The relative max-norm of a plane
is max|gpu - oracle| / max|oracle| over that (field, component) plane.
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
BC = {"periodic": O.BC_PERIODIC, "transmissive": O.BC_TRANSMISSIVE, "reflective": O.BC_REFLECTIVE}


def rel_planes(a, b):
    nf, nc = b.shape[0], b.shape[1]
    a = a.reshape(nf * nc, -1)
    b = b.reshape(nf * nc, -1)
    den = np.maximum(np.abs(b).max(axis=1), 1e-300)
    return (np.abs(a - b).max(axis=1) / den).max()


def make_state(dim, system, nx, ny, kind, seed):
    if system == "euler":
        if dim == 1:
            S, dx = W.euler1d_random(nx, seed, kind)
            return S, dx, dx
        return W.euler2d_random(nx, ny, seed, kind)
    return W.scalar_random(dim, nx, ny, seed, kind)


def pair(dim, system, nx, ny, bc, S, dx, dy, **kw):
    cfg = O.make_cfg(dim, SYS[system], nx, ny, dx=dx, dy=dy, bc=BC[bc], ax=kw.get("ax", 1.0),
                     ay=kw.get("ay", 1.0))
    s = Solver(dim, system, nx, ny, dx=dx, dy=dy, bc=bc, ax=kw.get("ax", 1.0), ay=kw.get("ay", 1.0))
    s.set_state(S)
    return cfg, s


CASES = [
    (1, "advection", 37, 1, "periodic"),
    (1, "burgers", 64, 1, "periodic"),
    (1, "burgers", 50, 1, "transmissive"),
    (1, "euler", 133, 1, "periodic"),
    (1, "euler", 130, 1, "transmissive"),
    (1, "euler", 5, 1, "periodic"),
    (2, "advection", 29, 23, "periodic"),
    (2, "burgers", 31, 17, "periodic"),
    (2, "burgers", 19, 26, "transmissive"),
    (2, "euler", 37, 29, "periodic"),
    (2, "euler", 33, 21, "transmissive"),
    (2, "euler", 5, 7, "periodic"),
    (2, "euler", 130, 6, "transmissive"),
    (1, "euler", 130, 1, "reflective"),
    (1, "euler", 6, 1, "reflective"),
    (2, "euler", 33, 21, "reflective"),
    (2, "euler", 6, 9, "reflective"),
]


@pytest.mark.parametrize("kind", ["smooth", "jumps"])
@pytest.mark.parametrize("dim,system,nx,ny,bc", CASES)
def test_rhs_parity(dim, system, nx, ny, bc, kind):
    S, dx, dy = make_state(dim, system, nx, ny, kind, seed=nx * 7 + ny)
    cfg, s = pair(dim, system, nx, ny, bc, S, dx, dy, ax=0.8, ay=-0.6)
    L, M = s.rhs()
    Lo, Mo = O.rhs(cfg, S)
    assert rel_planes(L.cpu().numpy(), Lo) <= 1e-12
    assert rel_planes(M.cpu().numpy(), Mo) <= 1e-12
    ax, ay = s.max_wavespeed()
    oax, oay = O.max_wavespeed(cfg, S)
    assert abs(ax - oax) <= 1e-14 * oax and abs(ay - oay) <= 1e-14 * max(oay, 1e-300)


@pytest.mark.parametrize("kind", ["smooth", "jumps"])
@pytest.mark.parametrize("dim,system,nx,ny,bc", CASES)
def test_one_step_parity(dim, system, nx, ny, bc, kind):
    S, dx, dy = make_state(dim, system, nx, ny, kind, seed=nx * 5 + ny)
    cfg, s = pair(dim, system, nx, ny, bc, S, dx, dy)
    dt = O.cfl_dt(cfg, S, 0.6)
    s.step(dt)
    ref = O.steps(cfg, S, dt, 1)
    assert rel_planes(s.state.cpu().numpy(), ref) <= 1e-12


def _long_case(case):
    if case == "euler2d_smooth":
        S, dx, dy = W.euler2d_smooth(40, 32)
        return S, dx, dy, (2, "euler", 40, 32, "periodic")
    if case == "euler1d_smooth":
        S, dx = W.euler1d_smooth(96)
        return S, dx, dx, (1, "euler", 96, 1, "periodic")
    if case == "euler2d_jumps":
        S, dx, dy = W.euler2d_random(36, 28, 9, "jumps")
        return S, dx, dy, (2, "euler", 36, 28, "periodic")
    if case == "euler2d_quadrants":
        S, dx, dy = W.euler2d_quadrants(32, 32, seed=2000)
        return S, dx, dy, (2, "euler", 32, 32, "periodic")
    if case == "euler1d_riemann":
        S, dx, _ = W.euler1d_riemann(256, seed=1000)
        return S, dx, dx, (1, "euler", 256, 1, "transmissive")
    if case == "interacting_blasts":
        # Example 4.4's layout with the middle pressure 1 instead of 0.01 (the printed data loses
        # positivity in the first stage on both sides; the oracle's pins record why)
        S, dx = W.blast_wave_1d(400, p_mid=1.0)
        return S, dx, dx, (1, "euler", 400, 1, "reflective")
    if case == "euler2d_box":
        S, dx, dy = W.euler2d_quadrants(32, 28, seed=2001)
        return S, dx, dy, (2, "euler", 32, 28, "reflective")
    if case == "burgers2d":
        S, dx = W.burgers_2d(40)
        return S, dx, dx, (2, "burgers", 40, 40, "periodic")
    S, dx = W.advection_1d(160)
    return S, dx, dx, (1, "advection", 160, 1, "periodic")


def _gpu_steps(s, n):
    s.set_time(0.0, 0.0)
    for _ in range(n):
        s.step(0.0)
    return s.state.cpu().numpy()


@pytest.mark.parametrize("case", ["euler2d_smooth", "euler1d_smooth", "burgers2d", "advection1d"])
def test_hundred_steps_parity_smooth(case):
    """Smooth data: 100 CFL steps (dt computed on each side from its own state) within 1e-10."""
    S, dx, dy, (dim, system, nx, ny, bc) = _long_case(case)
    cfg, s = pair(dim, system, nx, ny, bc, S, dx, dy)
    out = _gpu_steps(s, 100)
    ref, n, t = O.run(cfg, S, 0.0, 0.6, 1.0, max_steps=100)
    assert n == 100
    _, tg = s.last_dt()
    assert abs(tg - t) <= 1e-12 * t
    assert rel_planes(out, ref) <= 1e-10


def rel_l1_planes(a, b):
    """Per (field, component) plane: sum |a - b| / sum |b| (the plain sum where b's plane is zero)."""
    nf, nc = b.shape[0], b.shape[1]
    a = a.reshape(nf * nc, -1)
    b = b.reshape(nf * nc, -1)
    num = np.abs(a - b).sum(axis=1)
    den = np.abs(b).sum(axis=1)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)


def _l1_envelope(cfg, S, ref, nsteps, seeds=(7, 8, 9, 10)):
    """Per plane, the largest relative L1 drift of the oracle itself over nsteps when its input is
    moved by one ulp (random signs), over four such runs: the rounding-noise envelope of the
    scheme on this data."""
    env = np.zeros(ref.shape[0] * ref.shape[1])
    for sd in seeds:
        sign = np.random.default_rng(100 + sd).choice([-1.0, 1.0], S.shape)
        out, _, _ = O.run(cfg, S * (1.0 + sign * 2.0 ** -52), 0.0, 0.6, 1.0, max_steps=nsteps)
        env = np.maximum(env, rel_l1_planes(out, ref))
    return env


@pytest.mark.parametrize("case", ["euler2d_jumps", "euler2d_quadrants", "euler1d_riemann", "interacting_blasts",
                                  "euler2d_box"])
@pytest.mark.parametrize("nsteps", [20, 100])
def test_long_run_parity_discontinuous(case, nsteps):
    """Discontinuous data over many steps: the scheme amplifies rounding differences (the oracle
    against itself with a one-ulp input perturbation drifts by up to 1e-2 in the max-norm after
    100 steps, where a shock moves by a fraction of a cell), so no implementation with another
    rounding order stays within a fixed bar.  Each (field, component) plane is compared in the
    relative L1 norm, against ten times the largest drift of that plane over four perturbed oracle
    runs (or 1e-10); the step count is exact and the conserved totals agree to round-off."""
    S, dx, dy, (dim, system, nx, ny, bc) = _long_case(case)
    cfg, s = pair(dim, system, nx, ny, bc, S, dx, dy)
    out = _gpu_steps(s, nsteps)
    ref, n, _ = O.run(cfg, S, 0.0, 0.6, 1.0, max_steps=nsteps)
    assert n == nsteps
    env = _l1_envelope(cfg, S, ref, nsteps)
    err = rel_l1_planes(out, ref)
    print(case, nsteps, "L1 per plane", err.max(), "envelope", env.max(), "max-norm", rel_planes(out, ref))
    assert np.all(err <= np.maximum(1e-10, 10.0 * env)), (err, env)
    # periodic: every component is conserved; reflective walls: mass and energy (the wall faces
    # carry no mass or energy flux by the mirror symmetry), not the momenta
    comps = {"periodic": range(out.shape[1]), "reflective": (0, out.shape[1] - 1)}.get(bc, ())
    for k in comps:
        tot = np.abs(ref[0, k]).sum()
        assert abs(out[0, k].sum() - ref[0, k].sum()) <= 1e-12 * tot


def test_run_to_end_time_clamps_last_step():
    """Config of the 1D advection workload: N = 160 on [0, 2] to T = 2 with CFL 0.6."""
    S, dx = W.advection_1d(160)
    cfg, s = pair(1, "advection", 160, 1, "periodic", S, dx, dx)
    n = s.run(2.0)
    ref, no, t = O.run(cfg, S, 2.0, 0.6)
    assert n == no
    dt, tg = s.last_dt()
    assert abs(tg - 2.0) < 1e-14
    assert rel_planes(s.state.cpu().numpy(), ref) <= 1e-10
    assert np.abs(s.state.cpu().numpy()[0] - S[0]).max() < 1e-4  # exact solution is the initial data


def test_constant_state_is_steady():
    S = np.zeros((3, 4, 16, 16))
    S[0, 0], S[0, 1], S[0, 2], S[0, 3] = 1.0, 0.3, -0.2, 2.5
    s = Solver(2, "euler", 16, 16, dx=0.1, dy=0.1)
    s.set_state(S)
    L, M = s.rhs()
    assert np.abs(L.cpu().numpy()).max() < 1e-13
    assert np.abs(M.cpu().numpy() - S).max() < 1e-15


def test_nonphysical_state_reported():
    S, dx, dy = W.euler2d_random(16, 16, 3, "smooth")
    S[0, 0, 5, 5] = -1.0  # negative density
    s = Solver(2, "euler", 16, 16, dx=dx, dy=dy)
    s.set_state(S)
    from paper_2411_11229_gb300._capi import HwenoError, HWENO_ENONPHYS
    with pytest.raises(HwenoError) as ei:
        s.max_wavespeed()
    assert ei.value.code == HWENO_ENONPHYS


def test_reciprocal_accuracy():
    """The library's reciprocal (hardware approximation + one third-order correction) against the
    correctly rounded 1/x: at most one unit in the last place over twenty decades."""
    import ctypes
    from paper_2411_11229_gb300 import _capi as C
    rng = np.random.default_rng(17)
    x = (rng.uniform(1.0, 2.0, 200000) * 10.0 ** rng.integers(-30, 30, 200000)) * rng.choice([-1, 1], 200000)
    xd = torch.as_tensor(x, device="cuda")
    rd = torch.empty_like(xd)
    C.check(C.load().hweno_selftest_rcp(ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(rd.data_ptr()),
                                        x.size, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)),
            "hweno_selftest_rcp")
    r = rd.cpu().numpy()
    exact = 1.0 / x
    ulps = np.abs(r - exact) / np.spacing(np.abs(exact))
    assert ulps.max() <= 1.0, ulps.max()


def test_fp64_peak_probe():
    """The FP64 issue probe (the measured peak of the ALU roofline) reports a rate between half of
    and the nominal rate of 2 DFMA per SM per clock at the maximum SM clock, and counts the DFMAs
    of its launch from its grid (eight blocks of 256 threads per SM, 8 chains x 2048 steps)."""
    import ctypes

    from paper_2411_11229_gb300 import _capi as C
    props = torch.cuda.get_device_properties(0)
    scratch = torch.zeros(4, dtype=torch.float64, device="cuda")
    rate, per = ctypes.c_double(), ctypes.c_double()
    C.check(C.load().hweno_selftest_fp64_peak(ctypes.c_void_p(scratch.data_ptr()), 3,
                                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                              ctypes.byref(rate), ctypes.byref(per)), "hweno_selftest_fp64_peak")
    assert per.value == props.multi_processor_count * 8 * 256 * 2048 * 8
    nominal = 2 * props.multi_processor_count * 2.07e9
    assert 0.5 * nominal < rate.value <= 1.02 * nominal, (rate.value, nominal)
    assert scratch[3].item() == 1e-3  # the sink was not written


@pytest.mark.parametrize("ext", [False, True, "r2"])
def test_run_matches_stepping_and_stops_at_the_end(ext):
    """hweno_run (graph-replayed chunks of 16 CFL steps) against one hweno_step call per step:
    bit for bit, with max_steps honoured exactly; steps issued after the end time leave the state
    unchanged.  ext: the Rayleigh-Taylor set-up of Example 4.11 through the extended kernels, also
    with the per-cell characteristic decomposition (whose stages add the ghost-state launch)."""
    if ext:
        S, dx, dy, fixed = W.rayleigh_taylor(12, 48)
        kw = dict(gamma=5.0 / 3.0, grav=1.0, sides=("reflective", "reflective", "fixed", "fixed"), fixed=fixed)
        if ext == "r2":
            kw["flags"] = O.FLAG_R2
        nx, ny, t_end = 12, 48, 0.1
    else:
        S, dx, dy = W.euler2d_smooth(24, 20)
        kw = {}
        nx, ny, t_end = 24, 20, 0.5
    a = Solver(2, "euler", nx, ny, dx=dx, dy=dy, **kw)
    b = Solver(2, "euler", nx, ny, dx=dx, dy=dy, **kw)
    a.set_state(S)
    b.set_state(S)
    n = a.run(t_end)
    b.set_time(0.0, t_end)
    m = 0
    while True:
        b.step(0.0)
        m += 1
        dt, t = b.last_dt()
        if t >= t_end:
            break
    assert n == m and n > 16
    assert torch.equal(a.state, b.state)
    _, ta = a.last_dt()
    assert ta == t_end
    before = a.state.clone()
    a.step(0.0, 3)
    dt, ta2 = a.last_dt()
    assert dt == 0.0 and ta2 == t_end and torch.equal(a.state, before)
    # max_steps: 37 steps of a run that would take more
    c = Solver(2, "euler", nx, ny, dx=dx, dy=dy, **kw)
    c.set_state(S)
    assert c.run(10.0, max_steps=37) == 37
    d = Solver(2, "euler", nx, ny, dx=dx, dy=dy, **kw)
    d.set_state(S)
    d.set_time(0.0, 10.0)
    d.step(0.0, 37)
    assert torch.equal(c.state, d.state)


@pytest.mark.parametrize("dim,system,bc", [(1, "advection", "periodic"), (1, "burgers", "transmissive"),
                                           (1, "euler", "reflective"), (2, "burgers", "periodic"),
                                           (2, "euler", "transmissive"), (2, "euler", "reflective")])
def test_uniform_state_is_steady(dim, system, bc):
    """The degenerate case of every smoothness indicator: a uniform state at rest (flowing where the
    boundary allows it) with zero derivatives.  All fluxes of a line are equal, so L is zero exactly
    and M = (U, 0, 0), on both sides; a step leaves the state as it is up to the rounding of the
    third stage's weights 1/3 and 2/3 (not binary fractions)."""
    nx, ny = 23, (17 if dim == 2 else 1)
    if system == "euler":
        nc = 3 if dim == 1 else 4
        U = np.array([1.3, 0.0, 2.7]) if dim == 1 else np.array([1.3, 0.0, 0.0, 2.7])
        if bc != "reflective":
            U[1] = 0.4
    else:
        nc, U = 1, np.array([0.7])
    S = np.zeros((dim + 1, nc, ny, nx))
    S[0] = U[:, None, None]
    cfg, s = pair(dim, system, nx, ny, bc, S, 0.1, 0.1)
    L, M = s.rhs()
    assert torch.count_nonzero(L).item() == 0
    assert np.array_equal(M.cpu().numpy(), S)
    Lo, Mo = O.rhs(cfg, S)
    assert not Lo.any() and np.array_equal(Mo, S)
    s.step(0.0)
    assert np.abs(s.state.cpu().numpy() - S).max() <= 1e-15 * np.abs(S).max()


def test_handle_on_its_own_stream_orders_with_the_callers():
    """A handle on a non-default stream: the input is produced on the caller's stream behind a
    long-running kernel, hweno_rhs runs on the handle's stream and the outputs are read on the
    caller's stream; the handle's state is filled and stepped the same way.  Without the waits
    between the two streams the kernels would read the input before it is written."""
    S, dx, dy = W.euler2d_random(37, 29, 3, "jumps")
    cfg = O.make_cfg(2, O.EULER, 37, 29, dx=dx, dy=dy)
    own = torch.cuda.Stream()
    s = Solver(2, "euler", 37, 29, dx=dx, dy=dy, stream=own)
    src = torch.as_tensor(S, device="cuda")
    torch.cuda._sleep(100_000_000)  # keeps the caller's stream busy for tens of milliseconds
    Sd = src * 1.0  # written on the caller's stream after the sleep
    L, M = s.rhs(Sd)
    Lo, Mo = O.rhs(cfg, S)
    assert rel_planes(L.cpu().numpy(), Lo) <= 1e-12
    assert rel_planes(M.cpu().numpy(), Mo) <= 1e-12
    dt = O.cfl_dt(cfg, S, 0.6)
    torch.cuda._sleep(100_000_000)
    s.set_state(src * 1.0)
    s.step(dt)
    out = s.state.cpu().numpy()  # read on the caller's stream
    assert rel_planes(out, O.steps(cfg, S, dt, 1)) <= 1e-12
