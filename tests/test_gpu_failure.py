"""The failure path of the bounded device waits, made to run out on purpose.

The at-sample kernels stage each bin's field window in shared memory with
bulk copies and wait for them with a bounded number of polls.  With the
plan's wait limit at 0 every such wait gives up at once: the kernel records
a timeout in the error word, waits (with the full budget) for the copies
still in flight and returns, so the context stays usable.  fkreg_sync_status
must report FKREG_ERR_TIMEOUT, and the next call with the default limit must
give the normal results.  No fault, trap or hang is involved: the copies are
valid and complete; only the waits stop early.
"""
import numpy as np
import pytest

from paper_2204_07716_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2204_07716_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


@pytest.mark.parametrize("prec,d", [("f32", 2), ("f64", 2), ("f32", 1)])
def test_a_wait_that_runs_out_reports_a_timeout_and_the_plan_recovers(prec, d):
    from paper_2204_07716_gb300.fkreg import FkregError, Plan
    tol = 1e-6 if prec == "f32" else 1e-12
    w = inputs.random_small(160 + d, d, 20_000, {1: 200, 2: 32}[d], 1, [0.04], precision=prec,
                            tol=tol)
    # 1-D: an explicit tile, so the fine grid is split into bins with windows
    # (the automatic 1-D tile is the whole grid, which needs no staging)
    p = Plan(d, 1, w.grid_n, w.lo, w.hi, w.H, max_n=w.n, max_probes=2, tol=tol, precision=prec,
             tile=64 if d == 1 else 0)
    dt = torch.float32 if prec == "f32" else torch.float64
    p.set_points(torch.tensor(w.x, dtype=dt))
    y = torch.tensor(w.y, dtype=dt)
    ref = p.df(y, 2, seed=3, want=("mhat_at_x",))
    p.sync()
    ref = {k: v.clone() for k, v in ref.items()}
    p.set_wait_limit(0)
    p.df(y, 2, seed=3, want=("mhat_at_x",))
    with pytest.raises(FkregError, match="TIMEOUT"):
        p.sync()
    p.set_wait_limit(-1)
    out = p.df(y, 2, seed=3, want=("mhat_at_x",))
    p.sync()                                   # no error left behind
    rt = 1e-5 if prec == "f32" else 1e-12
    a, b = out["mhat_at_x"], ref["mhat_at_x"]
    assert torch.allclose(a, b, rtol=rt, atol=rt * float(b.abs().max()))
    assert torch.allclose(out["trace"], ref["trace"], rtol=rt)
    # the forward grid path has no staged waits: a zero limit leaves it alone
    p.set_wait_limit(0)
    g = p.smooth(y, want=("mhat_grid",))
    p.sync()
    assert torch.isfinite(g["mhat_grid"]).any()
    p.set_wait_limit(-1)
