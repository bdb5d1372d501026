"""The benchmark's ncu-derived figures of the face kernel (DRAM bytes per face, FP64 pipe activity,
FP64 instructions per face) are the ones in the committed ncu summary of that kernel."""
import importlib.util
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_figures", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _row(text, label):
    m = re.search(r"^\| " + re.escape(label) + r"[^|]*\| ([0-9.]+)", text, re.M)
    assert m, label
    return float(m.group(1))


def test_face_figures_match_the_ncu_summary():
    b = _bench()
    if b.FACE_TRAFFIC_BYTES_PER_FACE is None:
        return  # the face kernel changed after its last capture: the bench reports no traffic
    with open(os.path.join(ROOT, "profiles", "k_face_euler2d_2048_full.md")) as fh:
        text = fh.read()
    assert b.FACE_TRAFFIC_BYTES_PER_FACE == _row(text, "DRAM bytes per face (read + write)")
    assert abs(b.FACE_FP64_PIPE_ACTIVE - _row(text, "FP64 pipe active") / 100.0) < 5e-4
    assert b.FACE_FP64_INSTR_PER_FACE == _row(text, "FP64 instructions per face")
