"""The parity measures themselves (CPU): what they accept and what they reject.

The GPU tests lean on these functions, so a measure that passed a wrong
result would void them: a GPU value that is not finite where the oracle's
is finite and the point is valid must fail, the mask check must fail in
both directions, and the error must be the stated normwise quantity.
"""
import numpy as np
import pytest

import oracle
from parity_util import (check_mask, field_error, mhat_error, sample_grid_indices,
                         singular_within)


def test_mhat_error_is_the_stated_normwise_quantity():
    mo = np.array([1.0, -2.0, 0.5, 3.0])
    s0 = np.array([4.0, 1.0, 2.0, 0.5])
    a_y = np.array([10.0, 3.0, 5.0, 20.0])
    assert mhat_error(mo, mo, s0, a_y) == 0.0
    mg = mo.copy()
    mg[2] += 1e-3
    assert mhat_error(mg, mo, s0, a_y) == pytest.approx(2.0 * 1e-3 / 20.0, rel=1e-12)


def test_mhat_error_fails_on_a_gpu_nan_at_a_valid_point():
    mo = np.array([1.0, 2.0, 3.0])
    s0 = np.ones(3)
    a_y = np.ones(3)
    for bad in (np.nan, np.inf, -np.inf):
        mg = mo.copy()
        mg[1] = bad
        assert mhat_error(mg, mo, s0, a_y) == float("inf")
        # a masked (invalid) point is not compared
        assert mhat_error(mg, mo, s0, a_y, valid=np.array([True, False, True])) == 0.0
    # where the oracle itself is not finite (a singular system) the point is skipped
    mo2 = mo.copy()
    mo2[1] = np.nan
    mg = mo.copy()
    mg[1] = np.nan
    assert mhat_error(mg, mo2, s0, a_y) == 0.0


def test_check_mask_fails_in_both_directions():
    s0 = np.array([10.0, 5.0, 1.0, 0.0101, 0.0099, 0.001])
    smax = 10.0                                     # threshold rho * smax = 0.01
    good = np.array([1, 1, 1, 1, 0, 0], dtype=np.uint8)
    check_mask(good, s0, smax, rho=1e-3, margin=0.05)       # within the margin: either
    check_mask(np.array([1, 1, 1, 0, 1, 0]), s0, smax, rho=1e-3, margin=0.05)
    with pytest.raises(AssertionError, match="dense points masked"):
        check_mask(np.array([1, 0, 1, 1, 0, 0]), s0, smax, rho=1e-3, margin=0.05)
    with pytest.raises(AssertionError, match="sparse points unmasked"):
        check_mask(np.array([1, 1, 1, 1, 0, 1]), s0, smax, rho=1e-3, margin=0.05)
    # a dense point singular within the bar may be masked
    check_mask(np.array([1, 0, 1, 1, 0, 0]), s0, smax, rho=1e-3, margin=0.05,
               singular=np.array([0, 1, 0, 0, 0, 0], dtype=bool))


def test_field_error_is_normwise():
    o = np.array([1.0, -4.0, 2.0])
    g = o + np.array([0.0, 3e-6, -1e-6])
    a = np.array([2.0, 8.0, 4.0])
    assert field_error(g, o, a, 0.5) == pytest.approx(3e-6 / (8.0 * 0.5), rel=1e-9)


def test_singular_within_flags_a_one_sample_local_linear_system():
    # one sample under the kernel: the local-linear system of eq. 3 has rank 1
    H = np.diag([0.01 ** 2, 0.01 ** 2])
    x = np.array([[0.5, 0.5], [0.9, 0.9], [0.1, 0.9]])
    q = np.array([[0.5, 0.5], [0.5001, 0.5], [0.7, 0.7]])
    s = oracle.moment_sums(x, np.ones((1, 3)), H, 2, q)[:, 0, :]
    eps = 1e-5 * s[:, 0].max()
    flags = singular_within(s, H, 2, 1, eps)
    assert flags[0] and flags[1]
    # a well-posed system (many samples under a wide kernel) is not flagged
    rng = np.random.default_rng(3)
    xw = rng.random((400, 2))
    Hw = np.diag([0.1 ** 2, 0.1 ** 2])
    sw = oracle.moment_sums(xw, np.ones((1, 400)), Hw, 2, np.array([[0.5, 0.5]]))[:, 0, :]
    assert not singular_within(sw, Hw, 2, 1, 1e-5 * sw[:, 0].max())[0]
    # NW: only an (almost) empty kernel is singular
    assert list(singular_within(s[:, :1], H, 2, 0, eps)) == [False, False, True]


def test_sample_grid_indices_are_unique_in_range_and_keep_the_corners():
    idx = sample_grid_indices((64, 48), 100, seed=5)
    assert idx[0] == 0 and idx[-1] == 64 * 48 - 1
    assert len(np.unique(idx)) == len(idx) and 100 <= len(idx) <= 102
    assert np.array_equal(sample_grid_indices((4, 4), 100), np.arange(16))
