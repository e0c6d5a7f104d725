"""The byte and operation counts behind bench.py's roofline fields: the
method's per-pass bytes of the measurement plan, the bytes this design's
passes move, the FP32 operation count of the pair residual, and the
residual schedule the line reports.  Host logic only (no GPU)."""
import importlib.util
import os
import sys

import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test",
                                                  os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    try:
        sys.argv = ["bench.py"]
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def _grid3(n=16):
    return W.Grid(W.CART3D, n, n, n, 1.0 / n)


def test_method_bytes_follow_the_measurement_plan(bench):
    """5 s per cell per field and sweep (s = 4 in FP32): a colour launch of
    the coupled sweep is half a sweep of both fields (20 B), a tiled launch
    a whole one (40 B), a residual pass of both fields 40 B, advection of
    both fields (4 + d) s."""
    g = _grid3()
    N = g.ncell
    assert bench.method_bytes("smooth_fine", g, 4) == 20 * N
    assert bench.method_bytes("smooth_tiled", g, 4) == 40 * N
    for kind in ("residual", "residual_fp32", "residual_incr"):
        assert bench.method_bytes(kind, g, 4) == 40 * N
    assert bench.method_bytes("advect", g, 4) == (4 + 3) * 4 * N
    assert bench.method_bytes("totals", g, 4) == 8 * N
    assert bench.method_bytes("forces", g, 4) == (2 + 3) * 4 * N
    # FP64: one colour of one field, 2.5 s
    assert bench.method_bytes("smooth_fine", g, 8) == 2.5 * 8 * N


def test_design_bytes_of_the_fp32_passes(bench):
    """The arrays each pass of this design reads and writes, per cell of a
    3D grid: the tiled sweep 40 B (its design meets the method's), the pair
    and FP32 residual passes 80 B, the incremental pass 72 B (no state or x*
    reads)."""
    g = _grid3()
    N = g.ncell
    assert bench.algorithmic_bytes("smooth_tiled", g, 4) == 40 * N
    assert bench.algorithmic_bytes("residual", g, 4) == 80 * N
    assert bench.algorithmic_bytes("residual_fp32", g, 4) == 80 * N
    assert bench.algorithmic_bytes("residual_incr", g, 4) == 72 * N
    # the state-update colour launch of the tiled path reads and writes the
    # state besides the colour's own bytes
    assert (bench.algorithmic_bytes("smooth_fine", g, 4, 3, tiled=True)
            - bench.algorithmic_bytes("smooth_fine", g, 4, 3, tiled=False)) == \
        (32.0 - 32.0 / 5) * N


def test_pair_residual_operation_count(bench):
    """469.5 FP32 operations per interior 3D cell: per field six faces of 22
    and 32 for the centre term and scalings, 44 for the exchange, 70 for
    both residuals, 7 for u, v and the residuals' rounding, 7.5 for the red
    half-sweep (half the cells), 13 for the norms."""
    assert bench.PAIR_RESID_OPS_3D == 469.5


class _Opts:
    def __init__(self, fast, incr, tiled=1):
        self.fast_resid, self.incr_resid, self.tiled = fast, incr, tiled


@pytest.mark.parametrize("fast,incr,tiled,want", [
    (1, 1, 1, "then one pair pass, then incremental FP32 from it"),
    (2, 0, 1, "then pair passes"),
    (0, 1, 1, "pair passes, incremental FP32 from a small one"),
    (0, 0, 1, "pair passes"),
    (0, 1, 0, "pair passes"),
])
def test_residual_schedule_text(bench, fast, incr, tiled, want):
    text = bench.residual_schedule(_Opts(fast, incr, tiled), True)
    assert text.endswith(want), text
    assert bench.residual_schedule(_Opts(fast, incr, tiled), False) == "pair arithmetic"
