"""The oracle's threads change no bit of its results.

The oracle splits the lines of each sweep and the values of each update into contiguous chunks
over threads.  Every face flux, modified derivative and updated value is computed by one thread
from the same inputs in the same order as in a serial run, so any thread count must reproduce the
serial arrays exactly; a race or a chunk boundary that drops or repeats a line would show up here
as a difference (ragged sizes that do not divide by the thread counts, every system, boundary
and scheme variant).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W


@pytest.fixture(autouse=True)
def _restore_threads():
    yield
    O.set_threads(0)


def _cases():
    S, dx, dy = W.euler2d_random(37, 29, 5, "jumps")
    yield O.make_cfg(2, O.EULER, 37, 29, dx=dx, dy=dy), S
    yield O.make_cfg(2, O.EULER, 37, 29, dx=dx, dy=dy, bc=O.BC_REFLECTIVE), S
    yield O.make_cfg(2, O.EULER, 37, 29, dx=dx, dy=dy, flags=O.FLAG_R2 | O.FLAG_ALPHA_LOCAL), S
    S, dx, dy = W.euler2d_quadrants(33, 23, seed=2000)
    yield O.make_cfg(2, O.EULER, 33, 23, dx=dx, dy=dy, bc=O.BC_TRANSMISSIVE), S
    S, dx = W.euler1d_random(131, 3, "jumps")
    yield O.make_cfg(1, O.EULER, 131, dx=dx, bc=O.BC_TRANSMISSIVE), S
    S, dx, dy = W.scalar_random(2, 31, 17, 4, "jumps")
    yield O.make_cfg(2, O.BURGERS, 31, 17, dx=dx, dy=dy), S


@pytest.mark.parametrize("threads", [2, 3, 7, 16])
def test_threads_bit_identical(threads):
    for cfg, S in _cases():
        O.set_threads(1)
        L1, M1 = O.rhs(cfg, S)
        dt = O.cfl_dt(cfg, S, 0.6)
        S1 = O.steps(cfg, S, dt, 3)
        R1, n1, t1 = O.run(cfg, S, 0.0, 0.6, 1.0, max_steps=4)
        assert O.set_threads(threads) == threads
        L2, M2 = O.rhs(cfg, S)
        S2 = O.steps(cfg, S, dt, 3)
        R2, n2, t2 = O.run(cfg, S, 0.0, 0.6, 1.0, max_steps=4)
        assert np.array_equal(L1, L2) and np.array_equal(M1, M2)
        assert np.array_equal(S1, S2)
        assert np.array_equal(R1, R2) and n1 == n2 and t1 == t2


def test_threads_default_is_all_hardware_threads():
    import os
    assert O.set_threads(0) == (os.cpu_count() or 1)
