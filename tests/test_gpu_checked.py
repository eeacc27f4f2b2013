"""The checked build (libfkreg_checked.so, FKREG_CHECKED).

Its kernels range-check their index arithmetic (sort scatter, spreading tile
and flush, interpolation window and field reads, grid solve, direct-sum bin
ranges) and report a failed check through the plan's error word; nothing
traps.  Each test runs in a child process that loads the checked library
(FKREG_CHECKED=1): small parity cases of every kernel family pass with no
check failing, and the one deliberately out-of-range checked access of
fkreg_check_selftest (inside the error-word region, so it cannot leave the
workspace) is reported with its site and index.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2204_07716_gb300 import build
    build.build(checked=True)


def run_child(args, timeout=900):
    env = dict(os.environ, FKREG_CHECKED="1")
    return subprocess.run([sys.executable] + args, cwd=ROOT, env=env, capture_output=True,
                          text=True, timeout=timeout)


# small cases of each kernel family, through the checked library
CASES = [
    "tests/test_gpu_parity.py::test_sort_is_bit_exact",
    "tests/test_gpu_parity.py::test_fp64_tol12_all_dims",
    "tests/test_gpu_parity.py::test_fp32_tol6_all_dims",
    "tests/test_gpu_parity.py::test_full_bandwidth_matrix",
    "tests/test_gpu_parity.py::test_fp32_df_sweep",
    "tests/test_gpu_parity.py::test_variance_pass",
    "tests/test_gpu_parity.py::test_compact_kernel_direct_path",
    "tests/test_gpu_parity.py::test_empty_and_single_sample",
    "tests/test_gpu_gauss_direct.py::test_gaussian_direct_against_oracle",
    "tests/test_gpu_step.py::test_timed_step_reduced_n_every_output",
]


def test_checked_build_passes_parity_cases():
    r = run_child(["-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "gpu"] + CASES)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]


SELFTEST = r'''
import numpy as np, torch
from paper_2204_07716_gb300 import fkreg, inputs
assert fkreg.CHECKED and fkreg.load().fkreg_checked_build() == 1
w = inputs.random_small(5, 2, 2000, 16, 1, [0.05], precision="f64", tol=1e-12)
p = fkreg.Plan(2, 1, w.grid_n, w.lo, w.hi, w.H, max_n=w.n, tol=w.tol, precision="f64")
p.set_points(torch.tensor(w.x, device="cuda"))
p.sync()
p.check_selftest()
try:
    p.sync()
    raise SystemExit("the failed check was not reported")
except fkreg.FkregError as e:
    assert "site 15, index 20" in str(e), str(e)
# the word is cleared by the report: the plan works on
out = p.smooth(torch.tensor(w.y, device="cuda"), want=("mhat_grid",))
p.sync()
assert torch.isfinite(out["mhat_grid"]).any()
print("selftest ok")
'''


def test_failed_check_is_reported():
    r = run_child(["-c", SELFTEST], timeout=300)
    assert r.returncode == 0 and "selftest ok" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
