"""The bounds-checked build (libhweno_bounds.so, -DHWENO_BOUNDS_CHECK), in place of a memory checker:
its kernels check every cell, face, ghost-line and batch-instance index they form against the
extent of the arrays it addresses (an out-of-range index is counted and the access redirected to
element 0).  tests/bounds_sweep.py runs every family of entry points (stage operator, CFL steps,
scheme variants with every side type, stage VJP and both adjoint steps, the batched path with its
autotuner, the allocation-free operator, runs to a time) over ragged grids down to 5 cells a side,
once on each library, in child processes.  The checked build must record no out-of-range index
(and its self-test exactly one), and both builds must give the same results bit for bit (the
checks change no arithmetic).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

HERE = os.path.dirname(os.path.abspath(__file__))
SWEEP = os.path.join(HERE, "bounds_sweep.py")


def _sweep(out, checked):
    env = dict(os.environ)
    env.pop("HWENO_BOUNDS_CHECK", None)
    if checked:
        env["HWENO_BOUNDS_CHECK"] = "1"
    r = subprocess.run([sys.executable, SWEEP, str(out)], env=env, capture_output=True, text=True, timeout=1200,
                       cwd=os.path.dirname(HERE))
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    return r.stdout


def test_bounds_checked_build_sweep(tmp_path):
    log = _sweep(tmp_path / "checked.npz", True)
    print(log)
    assert "bounds: selftest 1" in log
    assert "bounds: out-of-range 0 " in log, log
    _sweep(tmp_path / "plain.npz", False)
    a = np.load(tmp_path / "checked.npz")
    b = np.load(tmp_path / "plain.npz")
    assert sorted(a.files) == sorted(b.files) and len(a.files) > 300
    # equal bit for bit, NaN where both are NaN (a few of the harshest ragged cases, discontinuous
    # data on 9 cells between a fixed and a reflective wall, break down within two steps, in the
    # oracle as well)
    differ = [k for k in a.files if not np.array_equal(a[k], b[k], equal_nan=True)]
    assert not differ, differ[:10]
