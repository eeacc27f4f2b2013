"""The seeded input generators follow their stated recipes (CPU).

Every GPU test and the benchmark draw their samples from ``inputs``; these
checks pin each family to the workload it stands for: sizes, boxes, grids,
bandwidth lists, orders and precisions, the sample distributions, and the
noise level of the responses (model of eq. 1, y = m(x) + sigma(x) eps).
The same call returns the same bytes.
"""
import inspect
import math

import numpy as np
import pytest

from paper_2204_07716_gb300 import inputs


def defaults(fn):
    return {k: v.default for k, v in inspect.signature(fn).parameters.items()}


def test_nw1d_recipe():
    assert defaults(inputs.nw1d)["n"] == 10_000
    w = inputs.nw1d()
    assert (w.d, w.order, w.precision, w.tol, w.grid_n) == (1, 0, "f64", 1e-9, (256,))
    np.testing.assert_allclose(w.H, [[[0.02 ** 2]]])
    assert w.x.shape == (10_000, 1) and 0.0 <= w.x.min() and w.x.max() <= 1.0
    assert abs(w.x.mean() - 0.5) < 0.01
    eps = w.y[0] - np.sin(2 * np.pi * w.x[:, 0])
    assert abs(eps.std() - 0.3) < 0.01 and abs(eps.mean()) < 0.01


def test_ll2d_recipe():
    assert defaults(inputs.ll2d)["n"] == 1_000_000
    w = inputs.ll2d(n=300_000)
    assert (w.d, w.order, w.precision, w.tol, w.grid_n) == (2, 1, "f32", 1e-6, (256, 256))
    np.testing.assert_allclose(w.H[0], np.diag([0.01 ** 2, 0.015 ** 2]))
    assert w.x.min() >= 0.0 and w.x.max() <= 1.0
    # an equal mixture of N((0.3,0.3)), N((0.7,0.4)), N((0.5,0.75)), sd 0.1:
    # the mean of the mixture and the share near each centre
    np.testing.assert_allclose(w.x.mean(axis=0), [0.5, 1.45 / 3], atol=5e-3)
    for c in ([0.3, 0.3], [0.7, 0.4], [0.5, 0.75]):
        near = np.mean(np.sum((w.x - c) ** 2, axis=1) < 0.05 ** 2)
        # an isotropic N(c, 0.1^2) puts 1 - exp(-1/8) of its mass within 0.05
        assert near == pytest.approx((1 - math.exp(-0.125)) / 3, rel=0.1)
    m = np.sin(4 * w.x[:, 0]) * np.cos(3 * w.x[:, 1])
    eps = (w.y[0] - m) / (0.1 + 0.2 * w.x[:, 0])
    assert abs(eps.std() - 1.0) < 0.01 and abs(eps.mean()) < 0.01


def test_nw3d_df_recipe():
    dflt = defaults(inputs.nw3d_df)
    assert (dflt["n"], dflt["n_probes"], dflt["n_bw"]) == (4_000_000, 32, 16)
    w = inputs.nw3d_df(n=100_000, n_probes=2)
    assert (w.d, w.order, w.precision, w.tol, w.grid_n) == (3, 0, "f32", 1e-6, (64, 64, 64))
    sig = np.sqrt(w.H[:, 0, 0])
    np.testing.assert_allclose(sig, np.logspace(-2, -1, 16), rtol=1e-12)
    for b in range(16):
        np.testing.assert_allclose(w.H[b], np.eye(3) * sig[b] ** 2)
    assert w.x.min() >= 0.0 and w.x.max() <= 1.0
    np.testing.assert_allclose(w.x.mean(axis=0), 0.5, atol=5e-3)
    m = np.exp(-np.sum((w.x - 0.5) ** 2, axis=1) / 0.05)
    assert abs((w.y[0] - m).std() - 0.2) < 0.005
    assert w.probes.shape == (2, 100_000)
    assert abs(w.probes.std() - 1.0) < 0.01


def test_ll2d_gcv_recipe():
    dflt = defaults(inputs.ll2d_gcv)
    assert (dflt["n"], dflt["n_probes"], dflt["grid"]) == (2_000_000, 10, 512)
    w = inputs.ll2d_gcv(n=100_000, n_probes=1)
    assert (w.d, w.order, w.precision, w.tol, w.grid_n) == (2, 1, "f32", 1e-6, (512, 512))
    np.testing.assert_allclose(w.H[0], np.diag([0.01 ** 2, 0.015 ** 2]))
    x1, x2 = w.x[:, 0], w.x[:, 1]
    m = x1 ** 2 - x2 + 0.5 * np.sin(8 * x1 * x2)
    assert abs((w.y[0] - m).std() - 0.1) < 0.003


def test_uneven_recipe():
    ws = inputs.uneven()
    assert len(ws) == 64
    dims = {w.d for w in ws}
    assert dims == {1, 2}
    ns = np.array([w.n for w in ws])
    assert ns.min() >= 1_000 and ns.max() <= 1_000_000
    # log-uniform sizes: the log spans most of [log 1e3, log 1e6]
    assert np.log10(ns).max() - np.log10(ns).min() > 2.0
    for w in ws[:8]:
        assert all(128 <= g <= 1024 for g in w.grid_n) and len(w.grid_n) == w.d
        assert np.iscomplexobj(w.y) and w.order == 1 and w.precision == "f32"
        assert w.x.min() >= 0.0 and w.x.max() <= 1.0
        f = 0.4 + 18.8 * w.x[:, 0]                 # the frequency axis, [0.4, 19.2]
        # |y| ~ 1 / (1 + f) up to the complex noise of sd 0.05 per part
        assert np.median(np.abs(np.abs(w.y[0]) - 1 / (1 + f))) < 0.06


def test_generators_are_deterministic():
    a, b = inputs.ll2d(n=1000), inputs.ll2d(n=1000)
    assert a.x.tobytes() == b.x.tobytes() and a.y.tobytes() == b.y.tobytes()
    u, v = inputs.uneven(n_problems=3, scale=0.01), inputs.uneven(n_problems=3, scale=0.01)
    assert all(p.x.tobytes() == q.x.tobytes() and p.y.tobytes() == q.y.tobytes()
               for p, q in zip(u, v))
