"""Oracle runs for process pools started with spawn (no torch, no CUDA in the workers)."""
import numpy as np

import oracle as O
import workloads as W


def riemann_run(args):
    """(n, seed, sign seed or None) -> the oracle's 1D Euler Riemann run to its stop time
    (state, steps, time); with a sign seed the input is first moved by one ulp (random signs)."""
    n, seed, psign = args
    S, dx, t_stop = W.euler1d_riemann(n, seed=seed)
    if psign is not None:
        sign = np.random.default_rng(psign).choice([-1.0, 1.0], S.shape)
        S = S * (1.0 + sign * 2.0 ** -52)
    cfg = O.make_cfg(1, O.EULER, n, dx=dx, bc=O.BC_TRANSMISSIVE)
    out, steps, t = O.run(cfg, S, t_stop, 0.6)
    return out, steps, t
