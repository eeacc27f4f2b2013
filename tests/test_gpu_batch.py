"""Uneven batch of independent problems in one captured CUDA graph: results
equal the standalone plans', one problem checked against the FP64 oracle,
per-problem latencies from the device timer, the tile autotuner, and one
plan's whole step captured as a graph (StepGraph)."""
import numpy as np
import pytest

import oracle
from paper_2204_07716_gb300 import inputs
from parity_util import mhat_error, sample_grid_indices

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2204_07716_gb300 import build
    build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def problem_kwargs(w, tile=0):
    return dict(d=w.d, order=1, grid_n=w.grid_n, lo=w.lo, hi=w.hi, H=w.H, max_n=w.n, tol=w.tol,
                precision="f32", y_complex=True, tile=tile)


def test_batch_graph_matches_standalone_plans_and_oracle():
    from paper_2204_07716_gb300.fkreg import Batch, Plan
    ws = inputs.uneven(n_problems=8, scale=0.01, gmax=256)
    probs = [problem_kwargs(w) for w in ws]
    xs = [torch.tensor(w.x, dtype=torch.float32, device="cuda") for w in ws]
    ys = [torch.tensor(w.y[0], dtype=torch.complex64, device="cuda") for w in ws]
    yv = [torch.view_as_real(y).contiguous() for y in ys]
    batch = Batch(probs)
    outs = batch.capture(xs, yv, variance=True)
    batch.launch()
    batch.launch()
    torch.cuda.synchronize()
    lat = batch.latencies()
    assert np.all(lat > 0) and np.all(np.isfinite(lat))
    for i, w in enumerate(ws):
        p = Plan(**problem_kwargs(w))
        p.set_points(xs[i])
        ref = p.smooth(ys[i], want=("mhat_grid", "mask", "mhat_at_x"))
        s2 = p.variance(ys[i], ref["mhat_at_x"])
        p.sync()
        assert torch.equal(outs[i]["mask"], ref["mask"])
        m = ref["mask"].bool()
        a, b = outs[i]["mhat_grid"][0, 0][m[0]], ref["mhat_grid"][0, 0][m[0]]
        assert torch.allclose(a, b, rtol=1e-4, atol=1e-5 * float(b.abs().max()))
        a, b = outs[i]["mhat_at_x"], ref["mhat_at_x"]
        assert torch.allclose(a, b, rtol=1e-4, atol=1e-5 * float(b.abs().max()))
        a, b = outs[i]["sigma2"][0, 0][m[0]], s2[0, 0][m[0]]
        assert torch.allclose(a, b, rtol=1e-3, atol=1e-5 * float(b.abs().max()))
    # one problem against the oracle (sampled grid points, both parts of y)
    w = ws[int(np.argmax([v.n for v in ws]))]
    i = ws.index(w)
    x32 = w.x.astype(np.float32).astype(np.float64)
    y32 = w.y[0].astype(np.complex64).astype(np.complex128)
    gp = oracle.grid_points(w.grid_n, w.lo, w.hi)
    idx = sample_grid_indices(w.grid_n, 200, seed=3)
    mg = outs[i]["mhat_grid"][0, 0].reshape(-1).cpu().numpy()[idx]
    mask = outs[i]["mask"][0].reshape(-1).cpu().numpy()[idx].astype(bool)
    for part, yy, gg in (("re", y32.real, mg.real), ("im", y32.imag, mg.imag)):
        r = oracle.smooth_at(x32, yy[None], w.H[0], 1, gp[idx])
        ay = oracle.scale_field(x32, yy[None], w.H[0], gp[idx])[:, 0]
        assert mhat_error(gg, r["mhat"][:, 0], r["s"][:, 0], ay, mask) < 1e-5, part
    # its conditional-variance pass (eq. 23) from the batch's own m-hat(x_i):
    # r_i = |y_i - mhat(x_i)|^2 smoothed with the same bandwidth
    mx = outs[i]["mhat_at_x"][0, 0].cpu().numpy()
    rr = np.abs(w.y[0].astype(np.complex64) - mx).astype(np.float64) ** 2
    ov = oracle.smooth_at(x32, rr[None], w.H[0], 1, gp[idx])
    ar = oracle.scale_field(x32, rr[None], w.H[0], gp[idx])[:, 0]
    s2 = outs[i]["sigma2"][0, 0].reshape(-1).cpu().numpy()[idx]
    assert np.all(np.isnan(s2[~mask]))
    assert mhat_error(s2, ov["mhat"][:, 0], ov["s"][:, 0], ar, mask) < 1e-5


def test_autotuner_picks_a_candidate():
    from paper_2204_07716_gb300.fkreg import autotune_tile
    w = inputs.ll2d(n=100_000)
    kw = dict(d=2, order=1, grid_n=w.grid_n, lo=w.lo, hi=w.hi, H=w.H, max_n=w.n, tol=1e-6,
              precision="f32")
    x = torch.tensor(w.x, dtype=torch.float32, device="cuda")
    y = torch.tensor(w.y, dtype=torch.float32, device="cuda")
    t = autotune_tile(kw, x, y, candidates=(8, 16, 32))
    assert t in (8, 16, 32)


def test_step_graph_replays_the_eager_step():
    # set_points + df (device probes) + variance captured as one CUDA graph:
    # a replay after new data is copied into the input buffers gives the eager
    # step's results on that data (FP64; the spreading's atomic order may
    # differ between runs, so the comparison allows rounding)
    from paper_2204_07716_gb300.fkreg import Plan, StepGraph
    w = inputs.random_small(150, 2, 3000, 28, 1, [0.06], precision="f64", tol=1e-12)
    p = Plan(2, 1, w.grid_n, w.lo, w.hi, w.H, max_n=w.n, n_rhs=1, max_probes=4, tol=1e-12,
             precision="f64")
    x = torch.tensor(w.x, device="cuda")
    y = torch.tensor(w.y, device="cuda")

    def step():
        p.set_points(x)
        o = p.df(y, 4, seed=5, want=("mhat_grid", "mask", "mhat_at_x"))
        return o, p.variance(y, o["mhat_at_x"])

    g = StepGraph(step)
    g2 = inputs.random_small(151, 2, 3000, 28, 1, [0.06], precision="f64", tol=1e-12)
    x.copy_(torch.tensor(g2.x))
    y.copy_(torch.tensor(g2.y))
    g.replay()
    go, gs2 = g.outputs
    eo, es2 = step()
    torch.cuda.synchronize()
    p.sync()
    for a, b in ((go["mhat_grid"], eo["mhat_grid"]), (go["mhat_at_x"], eo["mhat_at_x"]),
                 (gs2, es2), (go["gcv"], eo["gcv"]), (go["trace"], eo["trace"])):
        a, b = torch.nan_to_num(a), torch.nan_to_num(b)
        assert torch.allclose(a, b, rtol=1e-11, atol=1e-12 * float(b.abs().max()))
    assert torch.equal(go["mask"], eo["mask"])
    # and it differs from the first data set's result (the buffers were read)
    y.copy_(torch.tensor(w.y))
    x.copy_(torch.tensor(w.x))
    g.replay()
    torch.cuda.synchronize()
    assert not torch.allclose(torch.nan_to_num(go["mhat_grid"]), torch.nan_to_num(eo["mhat_grid"]))
