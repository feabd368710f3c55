"""The benchmark's algorithmic-work model: bytes per cell that each level-0 kernel family must move
across HBM, and the float64 operations it must execute, stated here from the fields each kernel reads
and writes (float32 fields 4 B per cell, float64 8 B, coarse fields a quarter of the cells in 2D)."""
import math
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

B32, B64, QUARTER = 4.0, 8.0, 0.25


def _bytes(family, level, inner=1):
    bound, work, unit = bench.kernel_work(family, level, inner)
    assert bound == "hbm" and unit == "B"
    return work


def test_pre_smoothing_zero_start():
    # f in; u out; R(u), R(r) out on the coarse grid
    assert _bytes("smooth", 0, 1) == B32 + B32 + 2 * QUARTER * B32


@pytest.mark.parametrize("inner", [1, 2, 3])
def test_pre_smoothing_averages_its_launches(inner):
    zero = B32 + B32 + 2 * QUARTER * B32
    nonzero = zero + B32  # the later cycles of a refinement step also read u
    assert math.isclose(_bytes("smooth", 0, inner), (zero + (inner - 1) * nonzero) / inner)


def test_pre_smoothing_coarser_levels():
    # u, R(r) in; the tau right-hand side f and u out; R(u), R(r) out
    assert _bytes("smooth", 1) == 4 * B32 + 2 * QUARTER * B32


def test_post_smoothing():
    # u, f, coarse u in; u out
    assert _bytes("prolong", 0) == 3 * B32 + QUARTER * B32


def test_post_smoothing_with_float64_update():
    # u, f, coarse u in; float64 u read and written in the L2; no float32 u written
    assert _bytes("update", 0) == 2 * B32 + QUARTER * B32 + 2 * B64


def test_refinement_residual():
    # float64 u, b in; float32 r out; 2 FMAs on the FP64 pipe per cell
    assert _bytes("ir", 0) == 2 * B64 + B32
    assert bench.fp64_work("ir") == 4.0
    assert bench.fp64_work("update") == 1.0
    assert bench.fp64_work("smooth") is None


def test_unknown_family_has_no_model():
    assert bench.kernel_work("coarse", 6) == (None, None, None)
