"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars (normwise errors defined in parity_util):
  FP64, tol 1e-12 -> 1e-10;  FP64, tol 1e-9 -> 1e-8;  FP32, tol 1e-6 -> 1e-5.
Bin counts and permutations are compared bit for bit.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2204_07716_gb300 import inputs
from parity_util import (check_mask, field_error, field_scale_sigma, mhat_error,
                         sample_grid_indices)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BAR = {("f64", 1e-12): 1e-10, ("f64", 1e-9): 1e-8, ("f32", 1e-6): 1e-5}


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
    """x, y exactly as the device sees them (rounded to the plan precision)."""
    if w.precision == "f32":
        x = w.x.astype(np.float32).astype(np.float64)
        y = w.y.astype(np.complex64 if np.iscomplexobj(w.y) else np.float32)
        y = y.astype(np.complex128 if np.iscomplexobj(w.y) else np.float64)
        return x, y
    return w.x, w.y


def check_grid(w, out, b=0, idx=None, bar=None, cutoff=False):
    """Compare mhat, the mask and the moment fields on (a subset of) the grid.

    With a subset the mask threshold needs max_g s_0 over the whole grid:
    the GPU's s_0 grid gives the location of the maximum and the oracle's
    s_0 there (checked against the GPU's) gives its value.
    """
    bar = bar or BAR[(w.precision, w.tol)]
    x, y = as_seen(w)
    H = w.H[b]
    gp = oracle.grid_points(w.grid_n, w.lo, w.hi)
    full = idx is None
    if full:
        idx = np.arange(gp.shape[0])
    q = gp[idx]
    r = oracle.smooth_at(x, y, H, w.order, q, cutoff=cutoff)
    a1 = oracle.scale_field(x, np.ones((1, w.n)), H, q, cutoff=cutoff)[:, 0]
    ay = oracle.scale_field(x, y, H, q, cutoff=cutoff)
    mg = out["mhat_grid"][b].reshape(y.shape[0], -1).cpu().numpy()[:, idx]
    mask = out["mask"][b].reshape(-1).cpu().numpy()[idx].astype(bool)
    errs = {}
    for rr in range(y.shape[0]):
        errs[f"mhat{rr}"] = mhat_error(mg[rr], r["mhat"][:, rr], r["s"][:, 0], ay[:, rr], mask)
    if "moments" in out:
        mom = out["moments"][b].reshape(out["moments"].shape[1], -1).cpu().numpy()[:, idx]
        ex = oracle.monomials(w.d, 2 * w.order)
        for f in range(r["s"].shape[1]):
            errs[f"s{f}"] = field_error(mom[f], r["s"][:, f], a1, field_scale_sigma(H, ex[f]))
        for rr in range(y.shape[0]):
            for f in range(r["t"].shape[2]):
                g = mom[r["s"].shape[1] + rr * r["t"].shape[2] + f]
                errs[f"t{rr}_{f}"] = field_error(g, r["t"][:, rr, f], ay[:, rr],
                                                 field_scale_sigma(H, ex[f]))
    # the density mask, both ways, against the oracle's s_0
    if full:
        s0max = np.max(r["s"][:, 0])
    else:
        assert "moments" in out, "a sampled grid check needs the GPU's s_0 grid"
        s0g = out["moments"][b, 0].reshape(-1).cpu().numpy().astype(np.float64)
        am = int(np.argmax(s0g))
        s0max = float(oracle.moment_sums(x, np.ones((1, w.n)), H, 0, gp[am:am + 1],
                                         cutoff=cutoff)[0, 0, 0])
        assert abs(s0g[am] - s0max) <= 1e-4 * s0max
    check_mask(mask, r["s"][:, 0], s0max)
    worst = max(errs.values())
    assert worst <= bar, {k: f"{v:.2e}" for k, v in errs.items()}
    return errs


# ---------------------------------------------------------------- sorting ----
def cpu_keys(x, geom, precision):
    """Sort keys of the bin rule (bin, then window centre inside the bin)."""
    ft = np.float32 if precision == "f32" else np.float64
    d = x.shape[1]
    w = geom["w"]
    tile, nbins = geom["tile"], geom["nbins"]
    bins = np.zeros(x.shape[0], dtype=np.int64)
    local = np.zeros(x.shape[0], dtype=np.int64)
    cells, nb = 1, 1
    for j in range(d):
        xp = (x[:, j].astype(ft) - ft(0.0)).astype(ft)
        u = (xp * ft(geom["inv_h"][j])).astype(ft)
        c = np.floor(u).astype(np.int64)
        c = np.clip(c, 0, geom["nf"][j] - 1)
        b = c // tile[j]
        e = np.ceil((u - ft(0.5 * w)).astype(ft)).astype(np.int64) + w // 2 - b * tile[j]
        e = np.clip(e, 0, tile[j])
        bins = bins * nbins[j] + b
        local = local * (tile[j] + 1) + np.where(local & 1, tile[j] - e, e)   # serpentine
        cells *= tile[j] + 1
        nb *= nbins[j]
    kb = int(np.ceil(np.log2(cells))) if cells > 1 else 0
    bb = int(np.ceil(np.log2(nb))) if nb > 1 else 0
    if bb + kb > 32:
        return bins, bins
    return (bins << kb) | local, bins


@pytest.mark.parametrize("case", ["d1", "d2clip", "d2full", "d3", "dups", "one"])
def test_sort_is_bit_exact(case):
    if case == "d1":
        w = inputs.nw1d()
    elif case == "d2clip":
        w = inputs.ll2d(n=200_000)
    elif case == "d2full":
        w = inputs.ll2d()          # the bench's size: 19-bit keys, two 10-bit passes
    elif case == "d3":
        w = inputs.random_small(1, 3, 50_000, 16, 0, [0.05], precision="f32", tol=1e-6)
    elif case == "dups":
        w = inputs.random_small(2, 2, 30_000, 32, 1, [0.03], precision="f32", tol=1e-6)
        w.x[::3] = w.x[0]          # many identical locations
        w.x[1::7, 0] = 1.0         # points on the upper boundary
    else:
        w = inputs.random_small(3, 2, 1, 16, 0, [0.1])
    p = plan_for(w)
    p.set_points(torch.tensor(w.x))
    perm, bstart = p.get_sort()
    p.sync()
    key, bins = cpu_keys(w.x, p.geom, w.precision)
    ref = np.argsort(key, kind="stable")
    assert np.array_equal(perm.cpu().numpy().astype(np.int64), ref)
    nb = int(np.prod(p.geom["nbins"]))
    counts = np.bincount(bins, minlength=nb)
    ref_start = np.concatenate([[0], np.cumsum(counts)])
    assert np.array_equal(bstart.cpu().numpy().astype(np.int64), ref_start)
    assert bstart.cpu().numpy()[-1] == w.n


# ------------------------------------------------------------ grid parity ----
def smooth(w, want=("mhat_grid", "mask", "moments")):
    p = plan_for(w)
    p.set_points(torch.tensor(w.x))
    out = p.smooth(torch.tensor(w.y), want=want)
    p.sync()
    return p, out


def test_nw1d_fp64_full():
    # 1-D Nadaraya-Watson, N = 10^4, 256 grid points, FP64, tol 1e-9
    w = inputs.nw1d()
    _, out = smooth(w)
    check_grid(w, out)


def test_nw1d_fp64_tol12():
    w = inputs.nw1d(tol=1e-12)
    _, out = smooth(w)
    check_grid(w, out)


@pytest.mark.parametrize("d,order,grid,sig", [(1, 1, 200, 0.01), (2, 0, 40, 0.03), (2, 1, 40, 0.03),
                                              (3, 0, 12, 0.06), (3, 1, 12, 0.07), (1, 2, 200, 0.01),
                                              (2, 2, 40, 0.03)])
def test_fp64_tol12_all_dims(d, order, grid, sig):
    w = inputs.random_small(10 + d + order, d, 3000, grid, order, [sig], precision="f64", tol=1e-12)
    _, out = smooth(w)
    check_grid(w, out)


@pytest.mark.parametrize("d,order,grid,sig", [(1, 0, 300, 0.01), (2, 1, 64, 0.02), (3, 0, 16, 0.05),
                                              (3, 1, 16, 0.06), (2, 2, 64, 0.03)])
def test_fp32_tol6_all_dims(d, order, grid, sig):
    w = inputs.random_small(20 + d + order, d, 20_000, grid, order, [sig], precision="f32", tol=1e-6)
    _, out = smooth(w)
    check_grid(w, out)


@pytest.mark.parametrize("order", [1, 2])
def test_full_bandwidth_matrix(order):
    w = inputs.random_small(31, 2, 4000, 40, order, [0.04], precision="f64", tol=1e-12, full_h=True)
    _, out = smooth(w)
    check_grid(w, out)


def test_bandwidth_sweep_with_narrow_kernels():
    # narrow bandwidths fold the spectrum onto the grid lattice (modes > L)
    w = inputs.random_small(32, 1, 5000, 64, 0, np.logspace(-2.5, -1, 5), precision="f64", tol=1e-12)
    p, out = smooth(w)
    g = p.geom
    for b in range(w.n_bw):
        check_grid(w, out, b=b)


def test_stacked_and_complex_responses():
    w = inputs.random_small(33, 1, 3000, 80, 1, [0.03], precision="f64", tol=1e-12, n_rhs=3)
    _, out = smooth(w)
    check_grid(w, out)
    # complex y = (re, im) smoothed as two real responses
    wc = inputs.random_small(34, 2, 3000, 32, 1, [0.05], precision="f64", tol=1e-12)
    yc = wc.y[0] + 1j * np.sin(5 * wc.x[:, 1])
    from paper_2204_07716_gb300.fkreg import Plan
    p = Plan(2, 1, wc.grid_n, wc.lo, wc.hi, wc.H, max_n=wc.n, n_rhs=1, tol=1e-12,
             precision="f64", y_complex=True)
    p.set_points(torch.tensor(wc.x))
    out = p.smooth(torch.tensor(yc), want=("mhat_grid", "mask"))
    p.sync()
    mg = out["mhat_grid"][0, 0].reshape(-1).cpu().numpy()
    for part, yy in (("re", yc.real), ("im", yc.imag)):
        wr = inputs.Workload("c", 2, wc.x, yy[None], wc.grid_n, wc.lo, wc.hi, wc.H, 1, 1e-12, "f64")
        o2 = {"mhat_grid": torch.tensor((mg.real if part == "re" else mg.imag).reshape((1, 1) + wc.grid_n)),
              "mask": out["mask"]}
        check_grid(wr, o2)


def test_complex_locations():
    # Sec. 4.4: complex points z smoothed over the plane as (Re z, Im z), with
    # complex responses; grid, at-sample values and prediction at complex points
    from paper_2204_07716_gb300.fkreg import Plan, predict
    wc = inputs.complex_log2d()
    z = wc.x[:, 0] + 1j * wc.x[:, 1]
    p = Plan(2, 1, wc.grid_n, wc.lo, wc.hi, wc.H, max_n=wc.n, n_rhs=1, tol=1e-12,
             precision="f64", y_complex=True)
    p.set_points(torch.tensor(z))
    out = p.smooth(torch.tensor(wc.y[0]), want=("mhat_grid", "mask", "mhat_at_x"))
    p.sync()
    mg = out["mhat_grid"][0, 0].reshape(-1).cpu().numpy()
    for part in ("re", "im"):
        yy = wc.y[0].real if part == "re" else wc.y[0].imag
        wr = inputs.Workload("c", 2, wc.x, yy[None], wc.grid_n, wc.lo, wc.hi, wc.H, 1, 1e-12, "f64")
        o2 = {"mhat_grid": torch.tensor((mg.real if part == "re" else mg.imag).reshape((1, 1) + wc.grid_n)),
              "mask": out["mask"]}
        check_grid(wr, o2)
    ro = oracle.smooth_at(wc.x, np.stack([wc.y[0].real, wc.y[0].imag]), wc.H[0], 1, wc.x)
    ay = oracle.scale_field(wc.x, np.stack([wc.y[0].real, wc.y[0].imag]), wc.H[0], wc.x)
    mh = out["mhat_at_x"][0, 0].cpu().numpy()
    assert mhat_error(mh.real, ro["mhat"][:, 0], ro["s"][:, 0], ay[:, 0]) < 1e-10
    assert mhat_error(mh.imag, ro["mhat"][:, 1], ro["s"][:, 0], ay[:, 1]) < 1e-10
    # prediction at complex points equals prediction at their (re, im) pairs
    g = torch.nan_to_num(out["mhat_grid"][0, 0].real.contiguous())
    zq = torch.tensor(z[:50])
    a = predict(g, wc.grid_n, wc.lo, wc.hi, zq, "linear")
    b = predict(g, wc.grid_n, wc.lo, wc.hi, torch.tensor(wc.x[:50]), "linear")
    p.sync()
    assert torch.equal(a, b)


def test_ll2d_full_size_sampled():
    # 2-D local linear, N = 10^6, 256^2 grid, FP32, tol 1e-6 (sampled grid points)
    w = inputs.ll2d()
    _, out = smooth(w)
    idx = sample_grid_indices(w.grid_n, 300, seed=1)
    check_grid(w, out, idx=idx, cutoff=True)


# --------------------------------------------------------- sample parity ----
def test_at_samples_rss_and_exact_trace():
    w = inputs.random_small(40, 2, 3000, 32, 1, [0.05], precision="f64", tol=1e-12)
    p = plan_for(w, n_probes=1)
    p.set_points(torch.tensor(w.x))
    z = oracle.probes(7, 1, w.n)
    out = p.df(torch.tensor(w.y), 1, probes=torch.tensor(z), want=("mhat_at_x",))
    p.sync()
    r = oracle.smooth_at(w.x, w.y, w.H[0], 1, w.x)
    ay = oracle.scale_field(w.x, w.y, w.H[0], w.x)
    mh = out["mhat_at_x"][0, 0].cpu().numpy()
    assert mhat_error(mh, r["mhat"][:, 0], r["s"][:, 0], ay[:, 0]) < 1e-10
    rss_o = float(np.sum((w.y[0] - r["mhat"][:, 0]) ** 2))
    assert out["rss"][0, 0].item() == pytest.approx(rss_o, rel=1e-9)
    tr_o = oracle.trace_exact(w.x, w.H[0], 1)
    assert out["trace"][0, 2].item() == pytest.approx(tr_o, rel=1e-9)


@pytest.mark.parametrize("d,order", [(1, 0), (2, 1), (3, 0), (1, 2), (2, 2)])
def test_df_and_gcv_with_given_probes(d, order):
    grid = {1: 64, 2: 24, 3: 10}[d]
    w = inputs.random_small(50 + d, d, 2500, grid, order, [0.04, 0.08], precision="f64", tol=1e-12)
    npb = 4
    z = oracle.probes(11, npb, w.n)
    p = plan_for(w, n_probes=npb)
    p.set_points(torch.tensor(w.x))
    out = p.df(torch.tensor(w.y), npb, probes=torch.tensor(z), want=())
    p.sync()
    for b in range(w.n_bw):
        Sz = oracle.apply_smoother(w.x, z, w.H[b], order).T
        f = oracle.fmc_trace(w.x, z, w.H[b], order, Sw=Sz)
        scale = np.sum(np.abs(z) * np.abs(Sz)) / npb
        assert abs(out["trace"][b, 1].item() - f["hutchinson"]) <= 1e-10 * scale
        assert out["trace"][b, 0].item() == pytest.approx(f["girard"], rel=1e-9)
        m = oracle.apply_smoother(w.x, w.y, w.H[b], order)[:, 0]
        rss = float(np.sum((w.y[0] - m) ** 2))
        assert out["rss"][b, 0].item() == pytest.approx(rss, rel=1e-9)
        assert out["gcv"][b, 0].item() == pytest.approx(oracle.gcv(rss, w.n, f["girard"]), rel=1e-8)


def test_device_probes_follow_the_counter_generator():
    w = inputs.random_small(60, 1, 4000, 64, 0, [0.03], precision="f64", tol=1e-12)
    p = plan_for(w, n_probes=3)
    p.set_points(torch.tensor(w.x))
    a = p.df(torch.tensor(w.y), 3, seed=12345, want=())
    tr_dev = a["trace"].cpu().numpy().copy()
    z = oracle.probes(12345, 3, w.n)
    b = p.df(torch.tensor(w.y), 3, probes=torch.tensor(z), want=())
    p.sync()
    np.testing.assert_allclose(tr_dev, b["trace"].cpu().numpy(), rtol=1e-12)


def test_fp32_device_probes_follow_the_single_precision_generator():
    w = inputs.random_small(61, 2, 20_000, 32, 1, [0.04], precision="f32", tol=1e-6)
    p = plan_for(w, n_probes=3)
    p.set_points(torch.tensor(w.x))
    a = p.df(torch.tensor(w.y), 3, seed=777, want=())
    tr_dev = a["trace"].cpu().numpy().copy()
    z = oracle.probes(777, 3, w.n, precision="f32")
    b = p.df(torch.tensor(w.y), 3, probes=torch.tensor(z), want=())
    p.sync()
    np.testing.assert_allclose(tr_dev[:, :2], b["trace"].cpu().numpy()[:, :2], rtol=1e-5)


def test_fp32_df_sweep():
    w = inputs.nw3d_df(n=30_000, grid=16, n_bw=4, n_probes=4)
    z = w.probes
    p = plan_for(w, n_probes=4)
    p.set_points(torch.tensor(w.x))
    out = p.df(torch.tensor(w.y), 4, probes=torch.tensor(z), want=())
    p.sync()
    x, y = as_seen(w)
    z32 = z.astype(np.float32).astype(np.float64)
    for b in range(w.n_bw):
        Sz = oracle.apply_smoother(x, z32, w.H[b], 0).T
        f = oracle.fmc_trace(x, z32, w.H[b], 0, Sw=Sz)
        scale = np.sum(np.abs(z32) * np.abs(Sz)) / 4
        assert abs(out["trace"][b, 1].item() - f["hutchinson"]) <= 1e-5 * scale
        tr = oracle.trace_exact(x, w.H[b], 0)
        assert out["trace"][b, 2].item() == pytest.approx(tr, rel=1e-5)


def test_nw3d_df_full_size_sampled():
    # the 3-D DF sweep at its full size (N = 4e6, 64^3 grid, 16 bandwidths,
    # y + 32 device probes, FP32, tol 1e-6), run as the bench runs it (a
    # Sweep with a period per group of bandwidths): per bandwidth, m-hat and
    # the mask at 512 sampled grid points and m-hat(x_i) at 16 sampled samples
    # against the oracle's cutoff sums
    from paper_2204_07716_gb300.fkreg import Sweep
    w = inputs.nw3d_df()
    p = Sweep(w.d, w.order, w.grid_n, w.lo, w.hi, w.H, max_n=w.n, n_rhs=1,
              max_probes=w.n_probes, tol=w.tol, precision=w.precision)
    first, _ = p.groups()
    assert len(first) == 3, first
    p.set_points(torch.tensor(w.x, dtype=torch.float32))
    out = p.df(torch.tensor(w.y, dtype=torch.float32), w.n_probes, seed=17,
               want=("mhat_grid", "mask", "moments", "mhat_at_x"))
    p.sync()
    x, y = as_seen(w)
    gp = oracle.grid_points(w.grid_n, w.lo, w.hi)
    rng = np.random.default_rng(21)
    gi = rng.choice(gp.shape[0], 512, replace=False)
    c = np.concatenate([np.ones((1, w.n)), y, np.abs(y)])
    for b in range(w.n_bw):
        H = w.H[b]
        s0g = out["moments"][b, 0].reshape(-1).cpu().numpy().astype(np.float64)
        am = int(np.argmax(s0g))
        m = oracle.moment_sums(x, c, H, 0, np.concatenate([gp[gi], gp[am:am + 1]]),
                               cutoff=True)[:, :, 0]
        s0max = m[-1, 0]
        assert abs(s0g[am] - s0max) <= 1e-4 * s0max
        m = m[:-1]
        mask = out["mask"][b].reshape(-1).cpu().numpy().astype(bool)[gi]
        check_mask(mask, m[:, 0], s0max)
        mg = out["mhat_grid"][b, 0].reshape(-1).cpu().numpy()[gi]
        mo = m[:, 1] / m[:, 0]
        assert mhat_error(mg, mo, m[:, 0], m[:, 2], mask) < 1e-5, b
        si = rng.choice(w.n, 16, replace=False)
        mx = oracle.moment_sums(x, c, H, 0, x[si], cutoff=True)[:, :, 0]
        got = out["mhat_at_x"][b, 0].cpu().numpy()[si]
        assert mhat_error(got, mx[:, 1] / mx[:, 0], mx[:, 0], mx[:, 2]) < 1e-5, b


# --------------------------------------------------------- variance pass ----
def test_variance_pass():
    w = inputs.random_small(70, 1, 3000, 100, 1, [0.04], precision="f64", tol=1e-12)
    p = plan_for(w)
    p.set_points(torch.tensor(w.x))
    out = p.smooth(torch.tensor(w.y), want=("mhat_at_x",))
    s2 = p.variance(torch.tensor(w.y), out["mhat_at_x"])
    p.sync()
    mh = out["mhat_at_x"][0, 0].cpu().numpy()
    gp = oracle.grid_points(w.grid_n, w.lo, w.hi)
    ro = oracle.variance_pass(w.x, w.y, mh[None], w.H[0], gp, order=1)
    r = (w.y[0] - mh) ** 2
    s0 = oracle.moment_sums(w.x, np.ones((1, w.n)), w.H[0], 0, gp)[:, 0, 0]
    ar = oracle.scale_field(w.x, r[None], w.H[0], gp)[:, 0]
    valid = s0 >= 2e-3 * s0.max()
    assert mhat_error(s2[0, 0].cpu().numpy(), ro[:, 0], s0, ar, valid) < 1e-10


@pytest.mark.parametrize("d,order,prec,tol,bar", [(1, 1, "f64", 1e-12, 1e-10),
                                                  (2, 1, "f64", 1e-12, 1e-10),
                                                  (2, 0, "f64", 1e-12, 1e-10),
                                                  (2, 1, "f32", 1e-6, 1e-5)])
def test_log_variance(d, order, prec, tol, bar):
    # eqs. 24-26 against the oracle, with the device's mhat(x_i) as the
    # common input so the comparison isolates the log-variance step
    grid = {1: 100, 2: 24}[d]
    w = inputs.random_small(71 + d + 3 * order, d, 3000, grid, order, [0.05], precision=prec,
                            tol=tol)
    p = plan_for(w)
    p.set_points(torch.tensor(w.x))
    out = p.smooth(torch.tensor(w.y), want=("mhat_at_x",))
    lv = p.log_variance(torch.tensor(w.y), out["mhat_at_x"])
    p.sync()
    x, y = as_seen(w)
    mh = out["mhat_at_x"][0, 0].cpu().numpy().astype(np.float64)
    gp = oracle.grid_points(w.grid_n, w.lo, w.hi)
    ro = oracle.log_variance(x, y, mh[None], w.H[0], gp, order=order)
    ell = np.log((y[0] - mh) ** 2 + 1.0 / w.n)
    s0 = oracle.moment_sums(x, np.ones((1, w.n)), w.H[0], 0, gp)[:, 0, 0]
    al = oracle.scale_field(x, ell[None], w.H[0], gp)[:, 0]
    valid = s0 >= 2e-3 * s0.max()
    vg = lv["v_grid"][0, 0].cpu().numpy().reshape(-1)
    assert mhat_error(vg, ro["v_grid"][:, 0], s0, al, valid) < bar
    sx = oracle.moment_sums(x, np.ones((1, w.n)), w.H[0], 0, x)[:, 0, 0]
    alx = oracle.scale_field(x, ell[None], w.H[0], x)[:, 0]
    vx = lv["v_at_x"][0, 0].cpu().numpy()
    assert mhat_error(vx, ro["v_at_x"][:, 0], sx, alx) < bar
    kappa = lv["kappa"][0, 0].item()
    assert kappa == pytest.approx(ro["kappa"][0], rel=10 * bar)
    s2 = lv["sigma2"][0, 0].cpu().numpy().reshape(-1)
    ok = valid & np.isfinite(s2)
    np.testing.assert_allclose(s2[ok], np.exp(vg[ok]) / kappa, rtol=1e-5 if prec == "f32" else 1e-12)
    assert np.all(s2[ok] > 0)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_interval_eq28(prec):
    # eq. 28 on the grid estimate and the log-variance sigma^2 of one smooth
    w = inputs.random_small(77, 2, 3000, 20, 1, [0.06], precision=prec,
                            tol=1e-12 if prec == "f64" else 1e-6)
    p = plan_for(w)
    p.set_points(torch.tensor(w.x))
    out = p.smooth(torch.tensor(w.y), want=("mhat_grid", "mhat_at_x"))
    s2 = p.log_variance(torch.tensor(w.y), out["mhat_at_x"])["sigma2"]
    from paper_2204_07716_gb300.fkreg import interval
    for alpha in (0.05, 0.2):
        lo, hi = interval(out["mhat_grid"], s2, alpha)
        p.sync()
        lo_o, hi_o = oracle.interval(out["mhat_grid"].cpu().numpy(), s2.cpu().numpy(), alpha)
        rt = 1e-13 if prec == "f64" else 2e-6
        np.testing.assert_allclose(lo.cpu().numpy(), lo_o, rtol=rt, atol=rt, equal_nan=True)
        np.testing.assert_allclose(hi.cpu().numpy(), hi_o, rtol=rt, atol=rt, equal_nan=True)
    # a scalar variance (homoscedastic model) broadcast over the grid
    lo, hi = interval(out["mhat_grid"], torch.tensor(0.04, dtype=out["mhat_grid"].dtype,
                                                     device=out["mhat_grid"].device), 0.05)
    np.testing.assert_allclose((hi - lo).cpu().numpy(), 2 * 1.959963984540054 * 0.2,
                               rtol=1e-6 if prec == "f32" else 1e-14)


@pytest.mark.parametrize("d,prec", [(1, "f64"), (2, "f64"), (2, "f32"), (3, "f64")])
def test_predict_at_new_points(d, prec):
    # the grid estimate carried to new points, linear and cubic, against the
    # oracle's interpolation of the same grid values
    grid = {1: 60, 2: 20, 3: 8}[d]
    w = inputs.random_small(90 + d, d, 3000, grid, 1, [0.08], precision=prec,
                            tol=1e-12 if prec == "f64" else 1e-6)
    p = plan_for(w)
    p.set_points(torch.tensor(w.x))
    out = p.smooth(torch.tensor(w.y), want=("mhat_grid",))
    rng = np.random.default_rng(5 + d)
    xq = rng.random((500, d)) * 1.2 - 0.1          # some queries outside the box
    xq[:3] = 0.0
    xq[3:6] = 1.0
    from paper_2204_07716_gb300.fkreg import predict
    dt = torch.float32 if prec == "f32" else torch.float64
    g = out["mhat_grid"]
    gh = g.reshape(1, -1).cpu().numpy().astype(np.float64)
    for method in ("linear", "cubic"):
        v = predict(g, w.grid_n, w.lo, w.hi, torch.tensor(xq, dtype=dt, device=g.device), method)
        p.sync()
        xr = xq.astype(np.float32).astype(np.float64) if prec == "f32" else xq
        ref = oracle.predict(gh, w.grid_n, w.lo, w.hi, xr, method)[0]
        got = v.reshape(-1).cpu().numpy()
        ok = np.isfinite(ref)
        assert np.array_equal(np.isfinite(got), ok)
        rt = 1e-12 if prec == "f64" else 1e-5
        np.testing.assert_allclose(got[ok], ref[ok], rtol=rt, atol=rt * np.max(np.abs(gh[np.isfinite(gh)])))


@pytest.mark.parametrize("kernel,d,order,prec", [("epanechnikov", 1, 1, "f64"),
                                                  ("uniform", 2, 0, "f64"),
                                                  ("triangle", 2, 1, "f64"),
                                                  ("biweight", 2, 2, "f64"),
                                                  ("triweight", 3, 1, "f64"),
                                                  ("epanechnikov", 2, 1, "f32")])
def test_compact_kernel_direct_path(kernel, d, order, prec):
    # compact kernels: exact direct sums on the grid and at the samples
    grid = {1: 80, 2: 30, 3: 12}[d]
    sig = {1: 0.05, 2: 0.09, 3: 0.2}[d]
    w = inputs.random_small(120 + d + order, d, 3000, grid, order, [sig], precision=prec,
                            tol=1e-12 if prec == "f64" else 1e-6)
    p = plan_for(w, n_probes=1, kernel=kernel)
    p.set_points(torch.tensor(w.x))
    z = oracle.probes(9, 1, w.n)
    out = p.df(torch.tensor(w.y), 1, probes=torch.tensor(z),
               want=("mhat_grid", "mask", "moments", "mhat_at_x"))
    p.sync()
    bar = BAR[(w.precision, w.tol)]
    x, y = as_seen(w)
    H = w.H[0]
    gp = oracle.grid_points(w.grid_n, w.lo, w.hi)
    r = oracle.smooth_at_compact(x, y, H, order, gp, kernel)
    a1 = oracle.moment_sums_compact(x, np.ones((1, w.n)), H, 0, gp, kernel)[:, 0, 0]
    ay = oracle.moment_sums_compact(x, np.abs(y), H, 0, gp, kernel)[:, 0, 0]
    mask = out["mask"][0].reshape(-1).cpu().numpy().astype(bool)
    mg = out["mhat_grid"][0, 0].reshape(-1).cpu().numpy()
    assert mhat_error(mg, r["mhat"][:, 0], r["s"][:, 0], ay, mask) < bar
    mom = out["moments"][0].reshape(out["moments"].shape[1], -1).cpu().numpy()
    ex = oracle.monomials(w.d, 2 * order)
    for f in range(r["s"].shape[1]):
        assert field_error(mom[f], r["s"][:, f], a1, field_scale_sigma(H, ex[f])) < bar
    # at the samples: mhat, RSS, the exact trace and the Monte-Carlo trace
    rx = oracle.smooth_at_compact(x, y, H, order, x, kernel)
    ayx = oracle.moment_sums_compact(x, np.abs(y), H, 0, x, kernel)[:, 0, 0]
    mh = out["mhat_at_x"][0, 0].cpu().numpy()
    assert mhat_error(mh, rx["mhat"][:, 0], rx["s"][:, 0], ayx) < bar
    k0 = float(oracle.compact_profile(kernel, d, 0.0)) / math.sqrt(np.linalg.det(H))
    tr_exact = k0 * np.nansum(rx["sinv11"])
    rel = 1e-9 if prec == "f64" else 1e-4
    assert out["trace"][0, 2].item() == pytest.approx(tr_exact, rel=rel)
    sz = oracle.smooth_at_compact(x, z, H, order, x, kernel)["mhat"][:, 0]
    girard = w.n * float(z[0] @ sz) / float(z[0] @ z[0])
    assert out["trace"][0, 0].item() == pytest.approx(girard, rel=rel)


@pytest.mark.parametrize("kernel,full_h,prec", [("epanechnikov", True, "f64"),
                                                 ("biweight", False, "f64"),
                                                 ("triangle", True, "f32")])
def test_compact_probes_and_variance(kernel, full_h, prec):
    # several probes (strengths in more than one chunk of four), a correlated
    # H (no row cut) or a diagonal one (rows cut to the ellipse), a sample
    # cluster denser than one warp per bin, and the variance pass of eq. 23
    n_pr = 6
    w = inputs.random_small(131 + int(full_h), 2, 4000, 26, 1, [0.08], precision=prec,
                            tol=1e-12 if prec == "f64" else 1e-6, full_h=full_h)
    g = np.random.Generator(np.random.PCG64(77))
    w.x[:600] = 0.5 + 0.01 * g.standard_normal((600, 2))
    p = plan_for(w, n_probes=n_pr, kernel=kernel)
    p.set_points(torch.tensor(w.x))
    z = oracle.probes(13, n_pr, w.n)
    out = p.df(torch.tensor(w.y), n_pr, probes=torch.tensor(z), want=("mhat_at_x",))
    s2 = p.variance(torch.tensor(w.y), out["mhat_at_x"])
    p.sync()
    bar = BAR[(w.precision, w.tol)]
    x, y = as_seen(w)
    H = w.H[0]
    rx = oracle.smooth_at_compact(x, y, H, 1, x, kernel)
    ayx = oracle.moment_sums_compact(x, np.abs(y), H, 0, x, kernel)[:, 0, 0]
    mh = out["mhat_at_x"][0, 0].cpu().numpy()
    assert mhat_error(mh, rx["mhat"][:, 0], rx["s"][:, 0], ayx) < bar
    sz = oracle.smooth_at_compact(x, z, H, 1, x, kernel)["mhat"]
    girard = w.n * np.mean([float(z[k] @ sz[:, k]) / float(z[k] @ z[k]) for k in range(n_pr)])
    rel = 1e-9 if prec == "f64" else 1e-4
    assert out["trace"][0, 0].item() == pytest.approx(girard, rel=rel)
    # variance: the same smoother applied to r_i = (y_i - mhat(x_i))^2 on the grid,
    # with the device's mhat(x_i) as the common input
    r = (y[0] - mh.astype(np.float64)) ** 2
    if prec == "f32":
        r = ((w.y[0].astype(np.float32) - mh) ** 2).astype(np.float64)
    gp = oracle.grid_points(w.grid_n, w.lo, w.hi)
    ro = oracle.smooth_at_compact(x, r, H, 1, gp, kernel)
    ar = oracle.moment_sums_compact(x, np.abs(r), H, 0, gp, kernel)[:, 0, 0]
    s0 = ro["s"][:, 0]
    valid = s0 >= 2e-3 * s0.max()
    assert mhat_error(s2[0, 0].reshape(-1).cpu().numpy(), ro["mhat"][:, 0], s0, ar, valid) < bar


def test_compact_full_size_sampled():
    # the ll2d_epan bench step's configuration: N = 10^6 clustered samples,
    # 256^2 grid, Epanechnikov, FP32, y + 10 device probes; grid values on
    # sampled grid points and at-sample values on sampled samples against the
    # oracle's direct sums (the Girard trace is checked through the probes'
    # smoother in the small cases)
    w = inputs.ll2d()
    p = plan_for(w, n_probes=10, kernel="epanechnikov")
    p.set_points(torch.tensor(w.x))
    out = p.df(torch.tensor(w.y), 10, seed=3, want=("mhat_grid", "mask", "mhat_at_x"))
    p.sync()
    bar = BAR[(w.precision, w.tol)]
    x, y = as_seen(w)
    H = w.H[0]
    half = 1.01 * np.sqrt(np.diag(H))

    ex = [tuple(e) for e in oracle.monomials(2, 2)]
    lin = [(0, 0), (1, 0), (0, 1)]
    dsc = np.diag([1.0, 1.0 / np.sqrt(H[0, 0]), 1.0 / np.sqrt(H[1, 1])])

    def ref(q):
        # the oracle's direct sums over the samples of the query's support box
        # (every sample outside it has weight exactly 0), and the condition
        # number of the scaled local-linear system S of eq. 3
        mh, s0, ay, cond = [], [], [], []
        for qq in q:
            sel = np.all(np.abs(x - qq) <= half, axis=1)
            r = oracle.smooth_at_compact(x[sel], y[:, sel], H, 1, qq[None], "epanechnikov")
            a = oracle.moment_sums_compact(x[sel], np.abs(y[:, sel]), H, 0, qq[None],
                                           "epanechnikov")
            sf = r["s"][0]
            S = np.array([[sf[ex.index((u[0] + v[0], u[1] + v[1]))] for v in lin] for u in lin])
            mh.append(r["mhat"][0, 0])
            s0.append(sf[0])
            ay.append(a[0, 0, 0])
            cond.append(np.linalg.cond(dsc @ S @ dsc) if sf[0] > 0 else np.inf)
        return np.array(mh), np.array(s0), np.array(ay), np.array(cond)

    # Fewer than three samples in a support make S singular: m-hat is not
    # defined there and any value the rounding gives is as right as another,
    # so parity is taken where S is well-posed and the rest need only be NaN
    # or finite (both are)
    idx = sample_grid_indices(w.grid_n, 200, seed=4)
    rm, rs, ra, rc = ref(oracle.grid_points(w.grid_n, w.lo, w.hi)[idx])
    mask = out["mask"][0].reshape(-1).cpu().numpy()[idx].astype(bool)
    mg = out["mhat_grid"][0, 0].reshape(-1).cpu().numpy()[idx]
    posed = rc < 1e8
    assert posed.sum() > 100
    assert np.all(np.isfinite(mg[mask & posed]))
    assert mhat_error(mg, rm, rs, ra, mask & posed) < bar
    si = np.random.default_rng(5).choice(w.n, 200, replace=False)
    rm, rs, ra, rc = ref(x[si])
    mh = out["mhat_at_x"][0, 0].cpu().numpy()[si]
    posed = rc < 1e8
    assert np.all(np.isfinite(mh[posed]))
    assert mhat_error(mh[posed], rm[posed], rs[posed], ra[posed]) < bar


# ------------------------------------------------------------ edge cases ----
def test_empty_and_single_sample():
    w = inputs.random_small(80, 2, 1, 20, 0, [0.1], precision="f64", tol=1e-12)
    p = plan_for(w)
    p.set_points(torch.zeros((0, 2), dtype=torch.float64))
    out = p.smooth(torch.zeros((1, 0), dtype=torch.float64), want=("mhat_grid", "mask"))
    p.sync()
    assert out["mask"].sum().item() == 0
    assert torch.isnan(out["mhat_grid"]).all()
    p.set_points(torch.tensor(w.x))
    out = p.smooth(torch.tensor([[2.5]], dtype=torch.float64), want=("mhat_grid", "mask"))
    p.sync()
    m = out["mhat_grid"][0, 0][out["mask"][0].bool()]
    assert m.numel() > 0
    assert torch.allclose(m, torch.full_like(m, 2.5), rtol=1e-9)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_compact_empty_and_single_sample(prec):
    # direct path: no samples (everything masked) and one sample, whose NW
    # estimate is its own response inside its support (up to the rounding of
    # t / s) and masked (NaN) outside it; so is its at-sample value
    w = inputs.random_small(82, 2, 1, 20, 0, [0.12], precision=prec,
                            tol=1e-12 if prec == "f64" else 1e-6)
    dt = torch.float64 if prec == "f64" else torch.float32
    p = plan_for(w, kernel="epanechnikov")
    p.set_points(torch.zeros((0, 2), dtype=dt))
    out = p.smooth(torch.zeros((1, 0), dtype=dt), want=("mhat_grid", "mask"))
    p.sync()
    assert out["mask"].sum().item() == 0
    assert torch.isnan(out["mhat_grid"]).all()
    p.set_points(torch.tensor(w.x, dtype=dt))
    out = p.smooth(torch.tensor([[2.5]], dtype=dt), want=("mhat_grid", "mask", "mhat_at_x"))
    p.sync()
    gp = oracle.grid_points(w.grid_n, w.lo, w.hi)
    x = w.x.astype(np.float32).astype(np.float64) if prec == "f32" else w.x
    z = (gp - x[0]) / 0.12
    inside = np.sum(z * z, axis=1) < 0.999
    outside = np.sum(z * z, axis=1) > 1.001
    mask = out["mask"][0].reshape(-1).cpu().numpy().astype(bool)
    mg = out["mhat_grid"][0, 0].reshape(-1).cpu().numpy()
    assert inside.sum() > 10 and mask[inside].all() and not mask[outside].any()
    rt = 1e-12 if prec == "f64" else 1e-6
    np.testing.assert_allclose(mg[inside], 2.5, rtol=rt)
    assert np.isnan(mg[outside]).all()
    assert out["mhat_at_x"][0, 0, 0].item() == pytest.approx(2.5, rel=rt)


def test_points_outside_the_box_are_flagged():
    from paper_2204_07716_gb300.fkreg import FkregError
    w = inputs.random_small(81, 1, 100, 20, 0, [0.1], precision="f64", tol=1e-12)
    w.x[5, 0] = 1.5
    w.x[9, 0] = float("nan")
    p = plan_for(w)
    p.set_points(torch.tensor(w.x))
    with pytest.raises(FkregError, match="DEVICE"):
        p.sync()
    p.sync()   # the error word was cleared
