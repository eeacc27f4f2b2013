"""Gradients of the smoothed grid (fkreg_backward_grid) and the autograd
wrappers, on the GPU through the C ABI.

* The grid estimate's vector-Jacobian product (eqs. 3, 9, 11) against the
  oracle's analytic gradient and against central finite differences of the
  GPU forward (FP64, tol 1e-12).
* fkreg.smooth_grid and fkreg.gcv under torch.autograd equal the plan calls
  they wrap, for float64 and float32 inputs; GCV against central differences
  in log sigma (eq. 22).
* The FP32 GCV backward on a reduced form of the 2-D GCV workload against the
  oracle's analytic GCV gradient.
"""
import numpy as np
import pytest

import oracle
from paper_2204_07716_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2204_07716_gb300 import build
    build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def fd_pair(f, eps=1e-4):
    """Central difference and its Richardson extrapolation (4 D(eps) - D(2 eps)) / 3."""
    d1 = (f(eps) - f(-eps)) / (2 * eps)
    d2 = (f(2 * eps) - f(-2 * eps)) / (4 * eps)
    return d1, (4 * d1 - d2) / 3


def grid_problem(seed, d, n, order, sig, grid, nrhs=1):
    # samples inside [0.1, 0.9], the grid box [0.05, 0.95]: every grid point
    # has samples under its kernel and x +/- eps stays in the box
    rng = np.random.default_rng(500 + seed)
    x = 0.1 + 0.8 * rng.random((n, d))
    y = np.stack([np.cos(3 * x.sum(axis=1) + r) + 0.2 * rng.standard_normal(n)
                  for r in range(nrhs)])
    return dict(x=x, y=y, sig=np.asarray(sig, dtype=np.float64), order=order, d=d,
                grid_n=(grid,) * d, lo=(0.05,) * d, hi=(0.95,) * d)


def gpu_grid(pb, gbar, prec="f64", want=("dlogh", "dy", "dx"), x=None, y=None, sig=None):
    from paper_2204_07716_gb300.fkreg import FKREG_WANT_BACKWARD, Plan
    x = pb["x"] if x is None else x
    y = pb["y"] if y is None else y
    sig = pb["sig"] if sig is None else sig
    H = np.diag(sig ** 2)[None]
    p = Plan(pb["d"], pb["order"], pb["grid_n"], pb["lo"], pb["hi"], H, max_n=x.shape[0],
             n_rhs=y.shape[0], tol=1e-12 if prec == "f64" else 1e-6, precision=prec,
             flags=FKREG_WANT_BACKWARD)
    dt = torch.float64 if prec == "f64" else torch.float32
    p.set_points(torch.tensor(x, dtype=dt))
    out = p.smooth(torch.tensor(y, dtype=dt), want=("mhat_grid", "mask"))
    mh = out["mhat_grid"][0].cpu().numpy().reshape(y.shape[0], -1)
    mask = out["mask"][0].cpu().numpy().reshape(-1).astype(bool)
    g = {}
    if want:
        g = p.backward_grid(torch.tensor(y, dtype=dt), torch.tensor(gbar, dtype=dt), b=0, want=want)
        g = {k: v.cpu().numpy() for k, v in g.items()}
    p.sync()
    return mh, mask, g


@pytest.mark.parametrize("d,order,nrhs", [(1, 0, 1), (1, 1, 2), (2, 1, 1), (2, 0, 1)])
def test_grid_vjp_matches_oracle_gradient(d, order, nrhs):
    pb = grid_problem(10 * d + order, d, 300, order, [0.07, 0.09][:d], {1: 40, 2: 14}[d], nrhs)
    M = int(np.prod(pb["grid_n"]))
    gbar = np.random.default_rng(3).standard_normal((nrhs, M))
    mh, mask, g = gpu_grid(pb, gbar)
    assert mask.all()
    q = oracle.grid_points(pb["grid_n"], pb["lo"], pb["hi"])
    ref = oracle.estimate_vjp(pb["x"], pb["y"], pb["sig"], order, q, gbar)
    np.testing.assert_allclose(g["dlogh"], ref["dlogsigma"], rtol=1e-8, atol=1e-10)
    scale = np.max(np.abs(ref["dY"]))
    assert np.max(np.abs(g["dy"] - ref["dY"])) <= 1e-8 * scale
    scale = np.max(np.abs(ref["dx"]))
    assert np.max(np.abs(g["dx"] - ref["dx"])) <= 1e-8 * scale


@pytest.mark.parametrize("d,order", [(1, 1), (2, 1)])
def test_grid_vjp_matches_finite_differences(d, order):
    pb = grid_problem(30 + d, d, 250, order, [0.08, 0.1][:d], {1: 30, 2: 12}[d])
    M = int(np.prod(pb["grid_n"]))
    gbar = np.random.default_rng(8).standard_normal((1, M))
    _, mask, g = gpu_grid(pb, gbar)
    assert mask.all()

    def L(**kw):
        mh, _, _ = gpu_grid(pb, gbar, want=(), **kw)
        return float(np.sum(gbar * mh))

    for j in range(d):
        def f(e, j=j):
            s = pb["sig"].copy()
            s[j] *= np.exp(e)
            return L(sig=s)
        fd, rich = fd_pair(f)
        assert g["dlogh"][j] == pytest.approx(rich, rel=1e-7, abs=1e-10)
    rng = np.random.default_rng(9)
    v = rng.standard_normal(pb["y"].shape)
    fd, rich = fd_pair(lambda e: L(y=pb["y"] + e * v))
    assert float(np.sum(g["dy"] * v)) == pytest.approx(rich, rel=1e-7)
    V = rng.standard_normal(pb["x"].shape)
    fd, rich = fd_pair(lambda e: L(x=pb["x"] + e * V))
    assert float(np.sum(g["dx"] * V)) == pytest.approx(rich, rel=1e-7)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_smooth_grid_autograd_equals_the_plan_backward(prec):
    from paper_2204_07716_gb300 import fkreg
    pb = grid_problem(41, 2, 2000, 1, [0.06, 0.08], 20)
    dt = torch.float64 if prec == "f64" else torch.float32
    x = torch.tensor(pb["x"], dtype=dt, device="cuda", requires_grad=True)
    y = torch.tensor(pb["y"][0], dtype=dt, device="cuda", requires_grad=True)
    ls = torch.tensor(np.log(pb["sig"]), dtype=dt, device="cuda", requires_grad=True)
    # a smooth positive functional of the grid (a random-sign one, tested in
    # FP64 above, cancels so strongly that FP32 rounding dominates d/dlog sigma)
    gg = np.linspace(0.0, 1.0, 20)
    gw = 1.0 + 0.5 * np.sin(3 * gg)[:, None] * np.cos(2 * gg)[None, :]
    gbar = torch.tensor(gw, dtype=dt, device="cuda").reshape(1, 20, 20)
    m = fkreg.smooth_grid(x, y, ls, pb["grid_n"], pb["lo"], pb["hi"], order=1, precision=prec)
    assert m.shape == (1, 20, 20) and m.dtype == dt
    loss = torch.sum(torch.nan_to_num(m) * gbar)
    gx, gy, gl = torch.autograd.grad(loss, (x, y, ls))
    _, _, ref = gpu_grid(pb, gbar.reshape(1, -1).cpu().numpy(), prec=prec,
                         x=pb["x"], y=pb["y"])
    # two FP32 runs differ by the order of the spreading's float atomics
    rt = 1e-12 if prec == "f64" else 1e-4
    np.testing.assert_allclose(gl.cpu().numpy(), ref["dlogh"], rtol=rt, atol=rt)
    np.testing.assert_allclose(gy.cpu().numpy(), ref["dy"][0], rtol=rt,
                               atol=rt * np.max(np.abs(ref["dy"])))
    np.testing.assert_allclose(gx.cpu().numpy(), ref["dx"], rtol=rt,
                               atol=rt * np.max(np.abs(ref["dx"])))
    # the FP32 form stays within its tolerance of the FP64 one
    if prec == "f32":
        _, _, r64 = gpu_grid(pb, gbar.reshape(1, -1).cpu().numpy().astype(np.float64))
        for k in ("dy", "dx"):
            err = np.max(np.abs(ref[k] - r64[k])) / np.max(np.abs(r64[k]))
            assert err < 2e-4, (k, err)
        np.testing.assert_allclose(ref["dlogh"], r64["dlogh"], rtol=2e-4)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_gcv_autograd_equals_the_plan_backward_and_finite_differences(prec):
    from paper_2204_07716_gb300 import fkreg
    from paper_2204_07716_gb300.fkreg import FKREG_WANT_BACKWARD, Plan
    pb = grid_problem(43, 2, 1500, 1, [0.07, 0.09], 16)
    dt = torch.float64 if prec == "f64" else torch.float32
    tol = 1e-12 if prec == "f64" else 1e-6
    x = torch.tensor(pb["x"], dtype=dt, device="cuda", requires_grad=True)
    y = torch.tensor(pb["y"][0], dtype=dt, device="cuda", requires_grad=True)
    ls = torch.tensor(np.log(pb["sig"]), dtype=dt, device="cuda", requires_grad=True)
    kw = dict(order=1, n_probes=4, seed=21, precision=prec, tol=tol)
    g = fkreg.gcv(x, y, ls, pb["grid_n"], pb["lo"], pb["hi"], **kw)
    gx, gy, gl = torch.autograd.grad(3.0 * g, (x, y, ls))
    sig = np.exp(ls.detach().cpu().numpy().astype(np.float64))   # the bandwidth gcv() used
    p = Plan(2, 1, pb["grid_n"], pb["lo"], pb["hi"], np.diag(sig ** 2)[None], max_n=1500,
             max_probes=4, tol=tol, precision=prec, flags=FKREG_WANT_BACKWARD)
    p.set_points(torch.tensor(pb["x"], dtype=dt))
    ref = p.backward(torch.tensor(pb["y"][0], dtype=dt), 4, seed=21)
    p.sync()
    # the same call twice; FP32 runs differ by the order of the float atomics
    rt = 1e-10 if prec == "f64" else 1e-4
    assert float(g.detach()) == pytest.approx(ref["gcv"].item(), rel=rt / 10)
    np.testing.assert_allclose(gl.cpu().numpy(), 3.0 * ref["dlogh"].cpu().numpy(), rtol=rt)
    np.testing.assert_allclose(gy.cpu().numpy(), 3.0 * ref["dy"].cpu().numpy(), rtol=rt,
                               atol=rt * float(ref["dy"].abs().max()))
    np.testing.assert_allclose(gx.cpu().numpy(), 3.0 * ref["dx"].cpu().numpy(), rtol=rt,
                               atol=rt * float(ref["dx"].abs().max()))
    if prec == "f64":
        for j in range(2):
            def f(e, j=j):
                s = np.log(pb["sig"])
                s[j] += e
                return float(fkreg.gcv(torch.tensor(pb["x"]), torch.tensor(pb["y"][0]),
                                       torch.tensor(s), pb["grid_n"], pb["lo"], pb["hi"], **kw))
            fd, rich = fd_pair(f)
            assert float(gl[j]) / 3.0 == pytest.approx(rich, rel=1e-7)


def test_gcv_backward_fp32_reduced_workload_against_the_oracle_gradient():
    # the 2-D GCV workload's recipe at N = 4000 on a 64^2 grid, FP32 (tol
    # 1e-6), against the oracle's analytic gradient of eq. 22 with the same
    # (float32) probes
    from paper_2204_07716_gb300.fkreg import FKREG_WANT_BACKWARD, Plan
    w = inputs.ll2d_gcv(n=4000, grid=64, n_probes=4)
    sig = np.array([0.04, 0.05])          # a few samples under each kernel at this N
    z = oracle.probes(5, 4, w.n, "f32").astype(np.float64)
    x32 = w.x.astype(np.float32).astype(np.float64)
    y32 = w.y[0].astype(np.float32).astype(np.float64)
    p = Plan(2, 1, w.grid_n, w.lo, w.hi, np.diag(sig ** 2)[None], max_n=w.n, max_probes=4,
             tol=1e-6, precision="f32", flags=FKREG_WANT_BACKWARD)
    p.set_points(torch.tensor(x32, dtype=torch.float32))
    g = p.backward(torch.tensor(y32, dtype=torch.float32), 4,
                   probes=torch.tensor(z, dtype=torch.float32))
    p.sync()
    ref = oracle.gcv_grad(x32, y32, z, sig, 1)
    assert g["gcv"].item() == pytest.approx(ref["gcv"], rel=1e-5)
    np.testing.assert_allclose(g["dlogh"].cpu().numpy(), ref["dlogsigma"], rtol=5e-4)
    for k, rk in (("dy", "dy"), ("dx", "dx")):
        got = g[k].cpu().numpy().astype(np.float64)
        err = np.max(np.abs(got - ref[rk])) / np.max(np.abs(ref[rk]))
        assert err < 5e-4, (k, err)
