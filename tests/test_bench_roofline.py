"""bench.py's roofline accounting on CPU: the binary64 level-0 kernels' operation
counts per grid row (the formulation's binary64 operations, and the share the FP64
pipe executes once the explicit row's two additions and two inner FMAs run on the
integer pipe, which the library does where level 0 fills the GPU), and the
achieved rate derived from a kernel time."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_binary64_operations_per_row():
    # loop row 30 (coefficient 1, explicit row 6, RD 4, pivot 2, reciprocal 5, RU 12),
    # per block 46 in place of two loop rows; substitution 10 - 10/m
    assert bench.f64_ops_per_row("reduce_level0", 32, True) == pytest.approx(30 - 14 / 32)
    assert bench.f64_ops_per_row("substitute_level0", 32, True) == pytest.approx(10 - 10 / 32)
    assert bench.f64_ops_per_row("fused_level0", 32, True) == pytest.approx(39.25)
    assert bench.flops_per_row("fused_level0", "f64", 32, True) == pytest.approx(51 - 26 / 32 + 16 - 16 / 32)


@pytest.mark.parametrize("n,pipe_ops", [(1 << 24, 35.25), (4096, 39.25)])
def test_fp64_pipe_share_follows_the_librarys_rule(monkeypatch, n, pipe_ops):
    monkeypatch.setattr(bench, "FP64_MEASURED_OPS", 6.0e11)
    monkeypatch.setattr(bench, "FP64_PEAK_SOURCE", "test")
    monkeypatch.setattr(bench, "ncu_traffic", lambda *a, **k: None)
    ms = 1.2  # one launch of the fused kernel
    prof = {"fused_level0": (ms, 1), "reduce_level0": (0.0, 0), "substitute_level0": (0.0, 0)}
    r = bench.roofline(prof, n, "f64", {}, 32, True, 148)
    assert r["kernel"] == "fused_level0" and r["ops_per_row"] == pytest.approx(39.25)
    assert r["fp64_pipe"]["ops_per_row"] == pytest.approx(pipe_ops)
    assert r["achieved"] == pytest.approx(39.25 * n / (ms * 1e-3) / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 0.6)
    assert r["fp64_pipe"]["frac"] == pytest.approx(pipe_ops * n / (ms * 1e-3) / 1e12 / 0.6)
