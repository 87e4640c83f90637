"""The algorithmic byte model of the level-0 sweep class in bench.py: the method's per-unit
figures (12 B per regular cell, 16 x 12 B + 2 x 20 x 4 B per irregular row) for a plain sweep,
and the per-launch average once a solve's zero-start sweeps (no iterate read) and its sweeps
that also update the FP64 solution are in the class."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_plain_sweeps_use_the_method_figures():
    byts, reg_b, irr_b = bench.sweep_class_bytes(4_877_864, 36_356, 90, 0, 3, 3, 0)
    assert reg_b == 12.0 and irr_b == 352.0
    assert byts == pytest.approx(4_877_864 * 12 + 36_356 * 352)       # 71.3 MB on the star 4096^2


def test_zero_start_and_folded_update_are_averaged():
    # 6 outer iterations of 3 V-cycles with nu1 = nu2 = 3: 90 launches, 6 of them start from
    # zero (8 B per regular cell), 6 also read and write u_hat (12 + 16 B per regular cell)
    _, reg_b, irr_b = bench.sweep_class_bytes(1000, 10, 90, 6, 3, 3, 0)
    assert reg_b == pytest.approx((78 * 12 + 6 * 8 + 6 * 28) / 90)
    assert reg_b == pytest.approx(12.8)
    assert irr_b == pytest.approx(352 + 16 * 6 / 90)


def test_no_zero_start_with_fmg_or_without_presmoothing_and_no_fold_with_one_postsweep():
    assert bench.sweep_class_bytes(1000, 10, 90, 6, 3, 3, 1)[1] == pytest.approx((90 * 12 + 6 * 16) / 90)
    assert bench.sweep_class_bytes(1000, 10, 90, 6, 0, 3, 0)[1] == pytest.approx((90 * 12 + 6 * 16) / 90)
    assert bench.sweep_class_bytes(1000, 10, 90, 6, 3, 1, 0) == pytest.approx(
        (1000 * (90 * 12 - 6 * 4) / 90 + 10 * 352, (90 * 12 - 6 * 4) / 90, 352))
