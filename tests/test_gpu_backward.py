"""Hand-written backward of GCV (eq. 22): gradients with respect to log h, y
and x, checked against central finite differences (step 1e-4, FP64) of the
GPU forward and of the FP64 oracle's direct-sum GCV with the same probes."""
import numpy as np
import pytest

import oracle
from paper_2204_07716_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2204_07716_gb300 import build
    build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def problem(seed, d, n, order, sig, prec="f64", tol=1e-12):
    w = inputs.random_small(seed, d, n, 16, order, [sig] * d if np.isscalar(sig) else [sig],
                            precision=prec, tol=tol)
    w.x = 0.1 + 0.8 * w.x           # interior, so x +/- eps stays in the box
    sig = np.broadcast_to(np.asarray(sig, dtype=np.float64), (d,))
    w.H = np.diag(sig ** 2)[None]
    return w


def gpu_gcv_and_grad(w, z, sig, want=("dlogh", "dy", "dx")):
    from paper_2204_07716_gb300.fkreg import FKREG_WANT_BACKWARD, Plan
    H = np.diag(np.asarray(sig, dtype=np.float64) ** 2)
    p = Plan(w.d, w.order, w.grid_n, w.lo, w.hi, H, max_n=w.n, max_probes=z.shape[0], tol=w.tol,
             precision=w.precision, flags=FKREG_WANT_BACKWARD)
    dt = torch.float64 if w.precision == "f64" else torch.float32
    p.set_points(torch.tensor(w.x, dtype=dt))
    out = p.backward(torch.tensor(w.y[0], dtype=dt), z.shape[0], probes=torch.tensor(z, dtype=dt),
                     want=want)
    p.sync()
    return {k: v.cpu().numpy() for k, v in out.items()}


def fd_pair(f, eps=EPS):
    """Central difference at step eps and its Richardson extrapolation
    (4 D(eps) - D(2 eps)) / 3, which removes the O(eps^2) truncation term."""
    d1 = (f(eps) - f(-eps)) / (2 * eps)
    d2 = (f(2 * eps) - f(-2 * eps)) / (4 * eps)
    return d1, (4 * d1 - d2) / 3


def oracle_gcv(x, y, z, H, order):
    S_y = oracle.apply_smoother(x, y[None], H, order)[:, 0]
    rss = float(np.sum((y - S_y) ** 2))
    f = oracle.fmc_trace(x, z, H, order)
    return oracle.gcv(rss, x.shape[0], f["girard"])


@pytest.mark.parametrize("d,order", [(1, 0), (1, 1), (2, 1)])
def test_backward_matches_finite_differences(d, order):
    sig = [0.07, 0.09][:d]
    w = problem(90 + d + order, d, 300, order, sig)
    z = oracle.probes(5, 3, w.n)
    g = gpu_gcv_and_grad(w, z, sig)
    rng = np.random.default_rng(7)

    def gcv_at(x, y, s):
        ww = problem(90 + d + order, d, 300, order, sig)
        ww.x, ww.y = x, y
        return gpu_gcv_and_grad(ww, z, s, want=())["gcv"][0]

    # log-bandwidth
    for j in range(d):
        def f(e, j=j):
            s = list(sig)
            s[j] *= np.exp(e)
            return gcv_at(w.x, w.y, s)
        fd, rich = fd_pair(f)
        assert g["dlogh"][j] == pytest.approx(fd, rel=1e-4)
        assert g["dlogh"][j] == pytest.approx(rich, rel=1e-7, abs=1e-12)
    # responses and sample locations, along random directions
    v = rng.standard_normal(w.n)
    fd, rich = fd_pair(lambda e: gcv_at(w.x, w.y + e * v[None], sig))
    assert float(g["dy"] @ v) == pytest.approx(fd, rel=1e-4)
    assert float(g["dy"] @ v) == pytest.approx(rich, rel=1e-7)
    V = rng.standard_normal((w.n, d))
    fd, rich = fd_pair(lambda e: gcv_at(w.x + e * V, w.y, sig))
    assert float(np.sum(g["dx"] * V)) == pytest.approx(fd, rel=1e-4)
    assert float(np.sum(g["dx"] * V)) == pytest.approx(rich, rel=1e-7)


def test_backward_matches_oracle_gradient():
    # the oracle's GCV with the same probes, differentiated by central differences
    d, order = 2, 1
    sig = [0.08, 0.1]
    w = problem(97, d, 250, order, sig)
    z = oracle.probes(9, 3, w.n)
    g = gpu_gcv_and_grad(w, z, sig)
    H = np.diag(np.asarray(sig) ** 2)
    assert g["gcv"][0] == pytest.approx(oracle_gcv(w.x, w.y[0], z, H, order), rel=1e-9)
    for j in range(d):
        def f(e, j=j):
            s = np.array(sig)
            s[j] *= np.exp(e)
            return oracle_gcv(w.x, w.y[0], z, np.diag(s ** 2), order)
        fd, rich = fd_pair(f)
        assert g["dlogh"][j] == pytest.approx(fd, rel=1e-4)
        assert g["dlogh"][j] == pytest.approx(rich, rel=1e-7)
    rng = np.random.default_rng(3)
    # per-component checks on a few samples
    for i in rng.choice(w.n, size=4, replace=False):
        def fy(e, i=i):
            yy = w.y[0].copy()
            yy[i] += e
            return oracle_gcv(w.x, yy, z, H, order)
        fd, rich = fd_pair(fy)
        assert g["dy"][i] == pytest.approx(rich, rel=1e-6, abs=1e-11)
        for a in range(d):
            def fx(e, i=i, a=a):
                xx = w.x.copy()
                xx[i, a] += e
                return oracle_gcv(xx, w.y[0], z, H, order)
            fd, rich = fd_pair(fx)
            assert g["dx"][i, a] == pytest.approx(rich, rel=1e-6, abs=1e-10)


def test_backward_fp32_close_to_fp64():
    sig = [0.03, 0.04]
    w64 = problem(98, 2, 20_000, 1, sig)
    z = oracle.probes(11, 4, w64.n)
    g64 = gpu_gcv_and_grad(w64, z, sig)
    w32 = problem(98, 2, 20_000, 1, sig, prec="f32", tol=1e-6)
    w32.x = w64.x.astype(np.float32).astype(np.float64)
    w32.y = w64.y.astype(np.float32).astype(np.float64)
    w64.x, w64.y = w32.x, w32.y
    g64 = gpu_gcv_and_grad(w64, z.astype(np.float32).astype(np.float64), sig)
    g32 = gpu_gcv_and_grad(w32, z.astype(np.float32).astype(np.float64), sig)
    assert g32["gcv"][0] == pytest.approx(g64["gcv"][0], rel=1e-5)
    np.testing.assert_allclose(g32["dlogh"], g64["dlogh"], rtol=2e-4)
    for k in ("dy", "dx"):
        err = np.max(np.abs(g32[k] - g64[k])) / np.max(np.abs(g64[k]))
        assert err < 2e-4, (k, err)
