"""Bandwidth sweeps with a Fourier period per group of bandwidths.

A sweep runs one plan per contiguous group of the bandwidth list, each with
the period its own bandwidths' tails need.  The results are checked against
the oracle (they approximate the same sums at the same tolerance) and
against plans made for the groups' sub-lists (the same computation, equal
up to the summation order of FP32 atomics).
"""
import numpy as np
import pytest

import oracle
from paper_2204_07716_gb300 import inputs
from parity_util import mhat_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2204_07716_gb300 import build
    build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def as_seen(w):
    return (w.x.astype(np.float32).astype(np.float64),
            w.y.astype(np.float32).astype(np.float64))


def reduced():
    return inputs.nw3d_df(n=30_000, grid=16, n_bw=6, n_probes=4)


def sweep_for(w, n_probes, max_groups=2):
    from paper_2204_07716_gb300.fkreg import Sweep
    return Sweep(w.d, w.order, w.grid_n, w.lo, w.hi, w.H, max_n=w.n, n_rhs=w.y.shape[0],
                 max_probes=n_probes, tol=w.tol, precision=w.precision, max_groups=max_groups)


def test_sweep_against_oracle():
    w = reduced()
    p = sweep_for(w, 4)
    first, geoms = p.groups()
    assert len(first) >= 3, first
    # the narrow group's period is shorter than the wide group's
    assert geoms[0]["period"][0] < geoms[-1]["period"][0]
    z = w.probes
    p.set_points(torch.tensor(w.x, dtype=torch.float32))
    out = p.df(torch.tensor(w.y, dtype=torch.float32), 4, probes=torch.tensor(z),
               want=("mhat_grid", "mask", "moments", "mhat_at_x"))
    p.sync()
    x, y = as_seen(w)
    z32 = z.astype(np.float32).astype(np.float64)
    gp = oracle.grid_points(w.grid_n, w.lo, w.hi)
    c = np.concatenate([np.ones((1, w.n)), y, np.abs(y)])
    for b in range(w.n_bw):
        H = w.H[b]
        m = oracle.moment_sums(x, c, H, 0, gp)[:, :, 0]
        mask = out["mask"][b].reshape(-1).cpu().numpy().astype(bool)
        mg = out["mhat_grid"][b, 0].reshape(-1).cpu().numpy()
        assert mhat_error(mg, m[:, 1] / m[:, 0], m[:, 0], m[:, 2], mask) < 1e-5, b
        mx = oracle.moment_sums(x, c, H, 0, x[:500])[:, :, 0]
        got = out["mhat_at_x"][b, 0].cpu().numpy()[:500]
        assert mhat_error(got, mx[:, 1] / mx[:, 0], mx[:, 0], mx[:, 2]) < 1e-5, b
        Sz = oracle.apply_smoother(x, z32, H, 0).T
        f = oracle.fmc_trace(x, z32, H, 0, Sw=Sz)
        scale = np.sum(np.abs(z32) * np.abs(Sz)) / 4
        assert abs(out["trace"][b, 1].item() - f["hutchinson"]) <= 1e-5 * scale, b
        assert out["trace"][b, 2].item() == pytest.approx(oracle.trace_exact(x, H, 0), rel=1e-5)


def test_sweep_equals_group_plans():
    from paper_2204_07716_gb300.fkreg import Plan
    w = reduced()
    p = sweep_for(w, 4)
    first, _ = p.groups()
    x = torch.tensor(w.x, dtype=torch.float32)
    y = torch.tensor(w.y, dtype=torch.float32)
    p.set_points(x)
    out = p.df(y, 4, seed=5, want=("mhat_grid", "mask", "mhat_at_x", "moments"))
    s2 = p.variance(y, out["mhat_at_x"])
    p.sync()
    for g in range(len(first) - 1):
        b0, b1 = first[g], first[g + 1]
        q = Plan(w.d, w.order, w.grid_n, w.lo, w.hi, w.H[b0:b1], max_n=w.n, max_probes=4,
                 tol=w.tol, precision=w.precision)
        q.set_points(x)
        o = q.df(y, 4, seed=5, want=("mhat_grid", "mask", "mhat_at_x", "moments"))
        v = q.variance(y, o["mhat_at_x"])
        q.sync()
        # the same computation; FP32 global atomics (the tile flush of the
        # spreading) make the summation order, and so the last bits, vary
        # from run to run
        ma, mb = out["mask"][b0:b1], o["mask"]
        assert int((ma != mb).sum()) <= 2, g
        both = (ma != 0) & (mb != 0)
        # ratios of grid sums: compared with the s_0 weight, as in the
        # oracle comparisons
        s0 = o["moments"][:, 0:1].double().expand_as(o["mhat_grid"])
        for k, a, b in (("mhat_grid", out["mhat_grid"][b0:b1], o["mhat_grid"]),
                        ("sigma2", s2[b0:b1], v)):
            sel = both.unsqueeze(1).expand_as(a)
            a, b, wgt = a.double()[sel], b.double()[sel], s0[sel]
            err = (wgt * (a - b).abs()).sum() / (wgt * b.abs()).sum()
            assert err.item() <= 1e-5, (g, k, err.item())
        a, b = out["mhat_at_x"][b0:b1].double(), o["mhat_at_x"].double()
        err = (a - b).abs().sum() / b.abs().sum()
        assert err.item() <= 1e-5, (g, "mhat_at_x", err.item())
        np.testing.assert_allclose(out["trace"][b0:b1].cpu().numpy(), o["trace"].cpu().numpy(),
                                   rtol=1e-5)
        np.testing.assert_allclose(out["gcv"][b0:b1].cpu().numpy(), o["gcv"].cpu().numpy(),
                                   rtol=1e-5)


def test_sweep_variance_against_oracle():
    w = reduced()
    p = sweep_for(w, 0)
    x32 = torch.tensor(w.x, dtype=torch.float32)
    y32 = torch.tensor(w.y, dtype=torch.float32)
    p.set_points(x32)
    out = p.smooth(y32, want=("mhat_at_x", "mask"))
    s2 = p.variance(y32, out["mhat_at_x"])
    p.sync()
    x, y = as_seen(w)
    gp = oracle.grid_points(w.grid_n, w.lo, w.hi)
    for b in (0, w.n_bw - 1):
        mh = out["mhat_at_x"][b, 0].cpu().numpy().astype(np.float64)
        r = (y[0] - mh) ** 2
        m = oracle.moment_sums(x, np.concatenate([np.ones((1, w.n)), r[None]]), w.H[b], 0,
                               gp)[:, :, 0]
        mask = out["mask"][b].reshape(-1).cpu().numpy().astype(bool)
        got = s2[b, 0].reshape(-1).cpu().numpy()
        assert mhat_error(got, m[:, 1] / m[:, 0], m[:, 0], m[:, 1], mask) < 1e-5, b


def test_single_group_is_a_plan():
    w = reduced()
    p = sweep_for(w, 0, max_groups=1)
    first, geoms = p.groups()
    assert first == [0, w.n_bw]
    p.set_points(torch.tensor(w.x, dtype=torch.float32))
    out = p.smooth(torch.tensor(w.y, dtype=torch.float32), want=("mhat_grid",))
    p.sync()
    assert out["mhat_grid"].shape == (w.n_bw, 1) + tuple(w.grid_n)


def test_sweep_backward_and_log_variance_equal_group_plans():
    # the GCV gradient of a bandwidth and the log-variance pass through a
    # sweep equal the calls on the plan of that bandwidth's group
    from paper_2204_07716_gb300 import fkreg
    from paper_2204_07716_gb300.fkreg import Plan, Sweep
    g = np.random.Generator(np.random.PCG64(123))
    n = 50_000
    x = g.random((n, 2))
    y = np.cos(4 * x[:, 0]) * x[:, 1] + 0.1 * g.standard_normal(n)
    H = np.array([np.eye(2) * s * s for s in (0.006, 0.01, 0.06, 0.1)])
    kw = dict(max_n=n, max_probes=4, tol=1e-6, precision="f32", flags=fkreg.FKREG_WANT_BACKWARD)
    sw = Sweep(2, 1, (64, 64), (0.0, 0.0), (1.0, 1.0), H, max_groups=2, **kw)
    first, _ = sw.groups()
    assert len(first) == 3, first
    xt = torch.tensor(x, dtype=torch.float32)
    yt = torch.tensor(y, dtype=torch.float32)
    z = torch.tensor(g.standard_normal((4, n)), dtype=torch.float32)
    sw.set_points(xt)
    o = sw.smooth(yt, want=("mhat_grid", "mask", "mhat_at_x"))
    lv = sw.log_variance(yt, o["mhat_at_x"])
    sw.sync()
    grads = {b: sw.backward(yt, 4, probes=z, b=b) for b in (1, 3)}
    sw.sync()
    for gi in range(2):
        b0, b1 = first[gi], first[gi + 1]
        p = Plan(2, 1, (64, 64), (0.0, 0.0), (1.0, 1.0), H[b0:b1], **kw)
        p.set_points(xt)
        op = p.smooth(yt, want=("mhat_grid", "mask", "mhat_at_x"))
        lp = p.log_variance(yt, op["mhat_at_x"])
        p.sync()
        np.testing.assert_allclose(lv["kappa"][b0:b1].cpu().numpy(), lp["kappa"].cpu().numpy(),
                                   rtol=1e-5)
        a = lv["v_at_x"][b0:b1].double().cpu().numpy()
        bref = lp["v_at_x"].double().cpu().numpy()
        assert np.sum(np.abs(a - bref)) <= 1e-5 * np.sum(np.abs(bref)), gi
        for b in (1, 3):
            if not b0 <= b < b1:
                continue
            r = p.backward(yt, 4, probes=z, b=b - b0)
            p.sync()
            assert grads[b]["gcv"].item() == pytest.approx(r["gcv"].item(), rel=1e-5)
            # FP32 fine grids are sums of atomic adds in no fixed order, so two
            # runs of one call differ by rounding; a component that is a small
            # difference of large terms (the weak direction of this y) carries
            # that rounding relative to the gradient's size: normwise, as dy
            dl_a = grads[b]["dlogh"].cpu().numpy()
            dl_b = r["dlogh"].cpu().numpy()
            assert np.max(np.abs(dl_a - dl_b)) <= 1e-4 * np.max(np.abs(dl_b)), (b, dl_a, dl_b)
            dy_a, dy_b = grads[b]["dy"].double(), r["dy"].double()
            assert (dy_a - dy_b).abs().sum().item() <= 1e-4 * dy_b.abs().sum().item()
