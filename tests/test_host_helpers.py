"""Host-side helpers of the binding (no GPU): the candidate bandwidth lists of
Sec. 4 (get_hList) and the dstd selection rule of Table 1."""
import os

import numpy as np
import pytest

from paper_2204_07716_gb300 import fkreg

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_bandwidth_list_reproduces_the_printed_bessel_values():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "get_hlist_bessel.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert rows
    for n, lo, hi, sp, idx, val in rows:
        H = fkreg.bandwidth_list(int(n), [(float(lo), float(hi))], sp)
        assert H.shape == (int(n), 1, 1)
        sig = np.sqrt(H[:, 0, 0])
        assert sig[0] == pytest.approx(float(lo)) and sig[-1] == pytest.approx(float(hi))
        assert round(sig[int(idx) - 1], 6 if float(val) < 0.1 else 5) == pytest.approx(float(val))


def test_bandwidth_list_two_axes_is_every_combination():
    # the bivariate example of Sec. 4: 10 values on one axis, 20 on the other
    H = fkreg.bandwidth_list([10, 20], [(0.01, 1.0), (0.1, 1.0)], "lin")
    assert H.shape == (200, 2, 2)
    assert np.all(H[:, 0, 1] == 0) and np.all(H[:, 1, 0] == 0)
    s0, s1 = np.sqrt(H[:, 0, 0]), np.sqrt(H[:, 1, 1])
    assert np.allclose(s0[:20], 0.01) and np.allclose(s1[:20], np.linspace(0.1, 1.0, 20))
    assert np.allclose(s0[::20], np.linspace(0.01, 1.0, 10))
    assert len({(round(a, 12), round(b, 12)) for a, b in zip(s0, s1)}) == 200
    with pytest.raises(fkreg.FkregError):
        fkreg.bandwidth_list([10], [(0.01, 1.0), (0.1, 1.0)])
    with pytest.raises(fkreg.FkregError):
        fkreg.bandwidth_list(5, [(0.0, 1.0)])


def test_select_bandwidth_dstd_rule():
    assert fkreg.select_bandwidth([5.0, 3.0, 2.0, 2.0, 4.0]) == 3      # ties: the later one
    assert fkreg.select_bandwidth([5.0, 2.0, 2.1, 9.0]) == 1
    s = float(np.std([5.0, 2.0, 2.1, 9.0]))
    assert fkreg.select_bandwidth([5.0, 2.0, 2.1, 9.0], 0.15 / s) == 2
    assert fkreg.select_bandwidth([float("nan"), 3.0, 1.0, float("nan")]) == 2
