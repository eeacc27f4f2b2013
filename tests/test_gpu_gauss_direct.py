"""The Gaussian kernel by direct sums (FKREG_KERNEL_GAUSSIAN_DIRECT).

Direct sums over the samples within Mahalanobis distance R of each point,
R^2 = 2 ln(10 / tol), so that every dropped term is below tol / 10 of
K_H(0).  Checked against the oracle's untruncated Gaussian sums (eqs. 3, 9,
11 at the grid points and at the samples, the exact and Monte-Carlo traces
of Sec. 2.1, the variance pass of eq. 23), against the NUFFT path on the same
problem, and inside a sweep that picks direct sums for its narrow group.
"""
import numpy as np
import pytest

import oracle
from paper_2204_07716_gb300 import inputs
from parity_util import check_mask, mhat_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BAR = {("f64", 1e-12): 1e-10, ("f32", 1e-6): 1e-5}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2204_07716_gb300 import build
    build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def plan_for(w, n_probes=0, **kw):
    from paper_2204_07716_gb300.fkreg import Plan
    return Plan(w.d, w.order, w.grid_n, w.lo, w.hi, w.H, max_n=max(w.n, 1), n_rhs=w.y.shape[0],
                max_probes=n_probes, tol=w.tol, precision=w.precision, **kw)


def as_seen(w):
    if w.precision == "f32":
        return (w.x.astype(np.float32).astype(np.float64),
                w.y.astype(np.float32).astype(np.float64))
    return w.x, w.y


@pytest.mark.parametrize("d,order,prec,sig,grid,full_h", [
    (1, 1, "f64", 0.01, 200, False), (2, 1, "f64", 0.012, 60, True),
    (2, 0, "f32", 0.008, 90, False), (3, 0, "f32", 0.03, 16, False),
    (2, 2, "f64", 0.03, 40, False)])
def test_gaussian_direct_against_oracle(d, order, prec, sig, grid, full_h):
    tol = 1e-12 if prec == "f64" else 1e-6
    w = inputs.random_small(150 + 3 * d + order, d, 3000, grid, order, [sig], precision=prec,
                            tol=tol, full_h=full_h)
    p = plan_for(w, n_probes=2, kernel="gaussian_direct")
    p.set_points(torch.tensor(w.x))
    z = oracle.probes(21, 2, w.n)
    out = p.df(torch.tensor(w.y), 2, probes=torch.tensor(z),
               want=("mhat_grid", "mask", "mhat_at_x"))
    p.sync()
    bar = BAR[(prec, tol)]
    x, y = as_seen(w)
    H = w.H[0]
    gp = oracle.grid_points(w.grid_n, w.lo, w.hi)
    r = oracle.smooth_at(x, y, H, order, gp)
    ay = oracle.scale_field(x, y, H, gp)[:, 0]
    mask = out["mask"][0].reshape(-1).cpu().numpy().astype(bool)
    s0 = r["s"][:, 0]
    check_mask(mask, s0, s0.max())
    mg = out["mhat_grid"][0, 0].reshape(-1).cpu().numpy()
    assert mhat_error(mg, r["mhat"][:, 0], s0, ay, mask) < bar
    rx = oracle.smooth_at(x, y, H, order, x)
    ayx = oracle.scale_field(x, y, H, x)[:, 0]
    mh = out["mhat_at_x"][0, 0].cpu().numpy()
    assert mhat_error(mh, rx["mhat"][:, 0], rx["s"][:, 0], ayx) < bar
    rel = 1e-9 if prec == "f64" else 1e-4
    k0 = oracle.kernel(H, np.zeros(d))
    assert out["trace"][0, 2].item() == pytest.approx(k0 * np.nansum(rx["sinv11"]), rel=rel)
    sz = oracle.smooth_at(x, z, H, order, x)["mhat"]
    girard = w.n * np.mean([float(z[k] @ sz[:, k]) / float(z[k] @ z[k]) for k in range(2)])
    assert out["trace"][0, 0].item() == pytest.approx(girard, rel=rel)


def test_gaussian_direct_equals_nufft():
    # the same Gaussian smoother by both paths (FP64, tol 1e-12)
    w = inputs.random_small(171, 2, 5000, 50, 1, [0.02, 0.035], precision="f64", tol=1e-12)
    outs = []
    for kern in ("gaussian", "gaussian_direct"):
        p = plan_for(w, kernel=kern)
        p.set_points(torch.tensor(w.x))
        o = p.smooth(torch.tensor(w.y), want=("mhat_grid", "mask", "moments", "mhat_at_x"))
        p.sync()
        outs.append(o)
    a, b = outs
    for bw in range(2):
        s0 = b["moments"][bw, 0].reshape(-1).cpu().numpy()
        mask = a["mask"][bw].reshape(-1).cpu().numpy().astype(bool) & \
            b["mask"][bw].reshape(-1).cpu().numpy().astype(bool)
        ma = a["mhat_grid"][bw, 0].reshape(-1).cpu().numpy()
        mb = b["mhat_grid"][bw, 0].reshape(-1).cpu().numpy()
        err = np.sum(s0[mask] * np.abs(ma[mask] - mb[mask])) / np.sum(s0[mask] * np.abs(mb[mask]))
        assert err < 1e-10, bw
        xa = a["mhat_at_x"][bw, 0].cpu().numpy()
        xb = b["mhat_at_x"][bw, 0].cpu().numpy()
        assert np.sum(np.abs(xa - xb)) / np.sum(np.abs(xb)) < 1e-10, bw


def test_sweep_picks_direct_sums_for_narrow_bandwidths():
    from paper_2204_07716_gb300.fkreg import Sweep
    g = np.random.Generator(np.random.PCG64(4711))
    n = 200_000
    x = g.random((n, 2))
    y = np.sin(5 * x[:, 0]) * np.cos(3 * x[:, 1]) + 0.1 * g.standard_normal(n)
    sig = [0.0015, 0.003, 0.05]
    H = np.array([np.eye(2) * s * s for s in sig])
    p = Sweep(2, 0, (100, 100), (0.0, 0.0), (1.0, 1.0), H, max_n=n, max_probes=0, tol=1e-6,
              precision="f32", max_groups=3)
    first, geoms, kern = p.groups(with_kernels=True)
    assert kern[0] == "gaussian_direct" and kern[-1] == "gaussian", (first, kern)
    x32 = torch.tensor(x, dtype=torch.float32)
    y32 = torch.tensor(y, dtype=torch.float32)
    p.set_points(x32)
    out = p.smooth(y32, want=("mhat_grid", "mask", "mhat_at_x"))
    s2 = p.variance(y32, out["mhat_at_x"])
    p.sync()
    xs = x.astype(np.float32).astype(np.float64)
    ys = y.astype(np.float32).astype(np.float64)[None]
    gp = oracle.grid_points((100, 100), (0.0, 0.0), (1.0, 1.0))
    si = g.choice(n, 2000, replace=False)
    for b in range(3):
        r = oracle.smooth_at(xs, ys, H[b], 0, gp, cutoff=True)
        ay = oracle.scale_field(xs, ys, H[b], gp, cutoff=True)[:, 0]
        mask = out["mask"][b].reshape(-1).cpu().numpy().astype(bool)
        mg = out["mhat_grid"][b, 0].reshape(-1).cpu().numpy()
        assert mhat_error(mg, r["mhat"][:, 0], r["s"][:, 0], ay, mask) < 1e-5, b
        rx = oracle.smooth_at(xs, ys, H[b], 0, xs[si], cutoff=True)
        ayx = oracle.scale_field(xs, ys, H[b], xs[si], cutoff=True)[:, 0]
        mh = out["mhat_at_x"][b, 0].cpu().numpy()
        assert mhat_error(mh[si], rx["mhat"][:, 0], rx["s"][:, 0], ayx) < 1e-5, b
        rr = ((y.astype(np.float32) - mh) ** 2).astype(np.float64)[None]
        rv = oracle.smooth_at(xs, rr, H[b], 0, gp, cutoff=True)
        ar = oracle.scale_field(xs, rr, H[b], gp, cutoff=True)[:, 0]
        got = s2[b, 0].reshape(-1).cpu().numpy()
        assert mhat_error(got, rv["mhat"][:, 0], rv["s"][:, 0], ar, mask) < 1e-5, b
