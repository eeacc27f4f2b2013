"""Parity of the timed step itself with the FP64 oracle.

The step is bench.py's headline step, called through the same functions:
the bin sort, fkreg_df with y and 10 probes drawn on the device (FP32
fields, tol 1e-6), and the conditional-variance pass (eq. 23), captured once
as a CUDA graph and replayed.  Two shapes:

* a reduced-N run of the same recipe (N = 80,000, above the size at which the
  grid branch forks onto its own stream; the same 256 x 256 grid and launch
  templates as the timed step), compared on every grid point and every
  sample: m-hat on the grid and its mask, m-hat(x_i), RSS, the Girard and
  Hutchinson traces of Sec. 2.1 with the oracle's copy of the probe
  generator, the exact trace, GCV (eq. 22) and sigma^2 of eq. 23;
* the full step (N = 10^6) against the oracle's cutoff sums: the mask at
  every grid point, m-hat and sigma^2 at sampled grid points, m-hat(x_i) at
  sampled samples, and RSS / GCV against the step's own outputs.

Bars: the FP32 bar of 1e-5 on the normwise errors of parity_util; scalars
with the bar scaled as in the error definitions (a trace by
sum_p sum_i |z_pi| |(S z_p)_i|).  The m-hat errors are weighted by
1 / ||S~^-1 e_1||_1 (parity_util.effective_weight), which is s_0 up to a small
factor where the local-linear system is well posed; the reduced-N sample
leaves some grid points with too few samples under the kernel for that,
and there the weight tracks the amplification of the field error.  The
plain s_0 weight is checked on the well-posed points (weight >= s_0 / 4).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2204_07716_gb300 import inputs
from parity_util import check_mask, effective_weight, mhat_error, singular_within

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BAR = 1e-5
SEED = 4242


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2204_07716_gb300 import build
    build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def run_step(w):
    """The headline step on workload w, captured as a graph and replayed once."""
    import bench
    from paper_2204_07716_gb300.fkreg import StepGraph
    plan = bench.ll2d_plan(w, torch.device("cuda", torch.cuda.current_device()))
    x = torch.tensor(w.x, dtype=torch.float32, device="cuda")
    y = torch.tensor(w.y, dtype=torch.float32, device="cuda")
    g = StepGraph(lambda: bench.ll2d_step(plan, x, y, SEED))
    g.replay()
    torch.cuda.synchronize()
    plan.sync()
    out, s2 = g.outputs
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["sigma2"] = s2.cpu().numpy()
    return plan, res


def seen(w):
    return (w.x.astype(np.float32).astype(np.float64),
            w.y.astype(np.float32).astype(np.float64))


def test_timed_step_reduced_n_every_output():
    import bench
    w = inputs.ll2d(n=80_000)
    plan, r = run_step(w)
    x, y = seen(w)
    H = w.H[0]
    n = w.n
    gp = oracle.grid_points(w.grid_n, w.lo, w.hi)
    # grid: m-hat and the mask, every point
    og = oracle.smooth_at(x, y, H, 1, gp, cutoff=True)
    ay = oracle.scale_field(x, y, H, gp, cutoff=True)[:, 0]
    mask = r["mask"][0].reshape(-1).astype(bool)
    s0 = og["s"][:, 0]
    sing = singular_within(og["s"], H, 2, 1, BAR * s0.max())
    check_mask(mask, s0, s0.max(), singular=sing)
    mg = r["mhat_grid"][0, 0].reshape(-1)
    assert np.all(np.isnan(mg[~mask]))
    wg = effective_weight(og["s"], H, 2, 1)
    posed = wg >= 0.25 * s0
    assert mhat_error(mg, og["mhat"][:, 0], wg, ay, mask) < BAR
    assert mhat_error(mg, og["mhat"][:, 0], s0, ay, mask & posed) < BAR
    # samples: y and the 10 probes of the device generator, every sample
    z = oracle.probes(SEED, bench.N_PROBES, n, "f32").astype(np.float64)
    ox = oracle.smooth_at(x, np.concatenate([y, z]), H, 1, x, cutoff=True)
    ayx = oracle.scale_field(x, y, H, x, cutoff=True)[:, 0]
    mx = r["mhat_at_x"][0, 0]
    assert np.all(np.isfinite(mx))
    wx = effective_weight(ox["s"], H, 2, 1)
    assert mhat_error(mx, ox["mhat"][:, 0], wx, ayx) < BAR
    assert mhat_error(mx, ox["mhat"][:, 0], ox["s"][:, 0], ayx, wx >= 0.25 * ox["s"][:, 0]) < BAR
    # RSS: the device's sum of its own residuals, and the oracle's RSS within
    # the change the m-hat error allows
    res_g = y[0] - mx.astype(np.float64)
    res_o = y[0] - ox["mhat"][:, 0]
    rss = float(r["rss"][0, 0])
    assert rss == pytest.approx(float(np.sum(res_g ** 2)), rel=1e-6)
    dm = np.abs(mx - ox["mhat"][:, 0])
    assert abs(rss - np.sum(res_o ** 2)) <= 2 * np.sum(np.abs(res_o) * dm) + np.sum(dm ** 2) + \
        1e-6 * rss
    # traces (Sec. 2.1) with the oracle's S z_p
    Sz = ox["mhat"][:, 1:].T
    f = oracle.fmc_trace(x, z, H, 1, Sw=Sz)
    scale = np.sum(np.abs(z) * np.abs(Sz)) / bench.N_PROBES
    girard, hutch, exact = (float(v) for v in r["trace"][0])
    assert abs(hutch - f["hutchinson"]) <= BAR * scale
    gscale = n * np.mean(np.sum(np.abs(z) * np.abs(Sz), axis=1) / f["ww"])
    assert abs(girard - f["girard"]) <= BAR * gscale
    tr = oracle.kernel(H, np.zeros(2)) * float(np.sum(ox["sinv11"]))
    assert exact == pytest.approx(tr, rel=BAR)
    # GCV (eq. 22): the device's value from its own RSS and trace, and the
    # oracle's within the errors of both
    gcv = float(r["gcv"][0, 0])
    assert gcv == pytest.approx(oracle.gcv(rss, n, girard), rel=1e-12)
    g_o = oracle.gcv(float(np.sum(res_o ** 2)), n, f["girard"])
    rel = abs(rss - np.sum(res_o ** 2)) / rss + 2 * abs(girard - f["girard"]) / (n - girard)
    assert abs(gcv - g_o) <= (rel + 1e-9) * g_o
    # sigma^2 of eq. 23 on the grid from the device's m-hat(x_i)
    rr = ((w.y[0].astype(np.float32) - mx) ** 2).astype(np.float64)
    ov = oracle.smooth_at(x, rr[None], H, 1, gp, cutoff=True)
    ar = oracle.scale_field(x, rr[None], H, gp, cutoff=True)[:, 0]
    s2 = r["sigma2"][0, 0].reshape(-1)
    assert np.all(np.isnan(s2[~mask]))
    assert mhat_error(s2, ov["mhat"][:, 0], wg, ar, mask) < BAR
    assert mhat_error(s2, ov["mhat"][:, 0], s0, ar, mask & posed) < BAR


def test_timed_step_full_size_sampled():
    w = inputs.ll2d()
    plan, r = run_step(w)
    x, y = seen(w)
    H = w.H[0]
    n = w.n
    gp = oracle.grid_points(w.grid_n, w.lo, w.hi)
    # the mask at every grid point against the oracle's s_0 (and its local
    # systems, for the points it may mask as singular)
    sf = oracle.moment_sums(x, np.ones((1, n)), H, 2, gp, cutoff=True)[:, 0, :]
    s0 = sf[:, 0]
    mask = r["mask"][0].reshape(-1).astype(bool)
    check_mask(mask, s0, s0.max(), singular=singular_within(sf, H, 2, 1, BAR * s0.max()))
    # m-hat and sigma^2 at sampled grid points (the corners included)
    rng = np.random.default_rng(11)
    gi = np.unique(np.concatenate([rng.choice(gp.shape[0], 300, replace=False),
                                   [0, gp.shape[0] - 1]]))
    og = oracle.smooth_at(x, y, H, 1, gp[gi], cutoff=True)
    ay = oracle.scale_field(x, y, H, gp, cutoff=True)[:, 0]     # normwise: the whole grid's
    mg = r["mhat_grid"][0, 0].reshape(-1)
    assert np.all(np.isnan(mg[~mask]))
    wg = effective_weight(og["s"], H, 2, 1)
    assert mhat_error(mg[gi], og["mhat"][:, 0], wg, ay, mask[gi]) < BAR
    assert mhat_error(mg[gi], og["mhat"][:, 0], og["s"][:, 0], ay, mask[gi] & (wg >= 0.25 * og["s"][:, 0])) < BAR
    mx = r["mhat_at_x"][0, 0]
    assert np.all(np.isfinite(mx))
    rr = ((w.y[0].astype(np.float32) - mx) ** 2).astype(np.float64)
    ov = oracle.smooth_at(x, rr[None], H, 1, gp[gi], cutoff=True)
    ar = oracle.scale_field(x, rr[None], H, gp, cutoff=True)[:, 0]
    s2 = r["sigma2"][0, 0].reshape(-1)
    assert mhat_error(s2[gi], ov["mhat"][:, 0], wg, ar, mask[gi]) < BAR
    # m-hat(x_i) at sampled samples
    si = rng.choice(n, 400, replace=False)
    ox = oracle.smooth_at(x, y, H, 1, x[si], cutoff=True)
    ayx = oracle.scale_field(x, y, H, x[si], cutoff=True)[:, 0]
    wx = effective_weight(ox["s"], H, 2, 1)
    assert mhat_error(mx[si], ox["mhat"][:, 0], wx, ayx) < BAR
    assert mhat_error(mx[si], ox["mhat"][:, 0], ox["s"][:, 0], ayx, wx >= 0.25 * ox["s"][:, 0]) < BAR
    # RSS is the sum of the device's own squared residuals; GCV follows
    # from RSS and the Girard trace (eq. 22)
    rss = float(r["rss"][0, 0])
    assert rss == pytest.approx(float(np.sum((y[0] - mx.astype(np.float64)) ** 2)), rel=1e-6)
    girard = float(r["trace"][0, 0])
    assert 0 < girard < n and math.isfinite(float(r["trace"][0, 2]))
    assert float(r["gcv"][0, 0]) == pytest.approx(oracle.gcv(rss, n, girard), rel=1e-12)
