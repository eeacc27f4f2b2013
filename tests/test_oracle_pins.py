"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a library
routine (scipy's Gaussian density, numpy least squares), a closed form, an
invariant, derivatives of the density, brute force on tiny inputs, or values
the paper prints.  A dropped term, a wrong sign, H in place of H^-1 or a
transposed operand in the oracle fails at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_spd(rng, d, scale):
    A = rng.standard_normal((d, d))
    H = A @ A.T + d * np.eye(d)
    return H * (scale ** 2 / np.mean(np.diag(H)))


def test_monomial_order_is_combinations_with_replacement():
    for d in (1, 2, 3):
        for deg in range(0, 5):
            e = oracle.monomials(d, deg)
            expect = []
            for k in range(deg + 1):
                for tup in itertools.combinations_with_replacement(range(d), k):
                    v = [0] * d
                    for a in tup:
                        v[a] += 1
                    expect.append(v)
            assert e.tolist() == expect
            assert oracle.nmono(d, deg) == math.comb(d + deg, deg)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_single_point_numerator_is_the_gaussian_density(d):
    # eq. 9 with one sample: t_0(g) = K_H(x_1 - g) y_1, K_H the N(0, H) density
    rng = np.random.default_rng(1 + d)
    H = rand_spd(rng, d, 0.1)
    x = rng.random((1, d))
    y = np.array([[1.7]])
    q = rng.random((20, d))
    t = oracle.moment_sums(x, y, H, 0, q)[:, 0, 0]
    ref = 1.7 * stats.multivariate_normal(mean=x[0], cov=H).pdf(q)
    np.testing.assert_allclose(t, ref, rtol=1e-13)


@pytest.mark.parametrize("d", [1, 2])
def test_scale_field_is_the_absolute_strength_sum(d):
    # the natural size a(q) = sum_i K_H(x_i - q) |c_i| that normalises every
    # field error: scipy's density times |c|, for strengths of both signs
    rng = np.random.default_rng(15 + d)
    H = rand_spd(rng, d, 0.12)
    x = rng.random((30, d))
    c = np.stack([rng.standard_normal(30), np.ones(30)])
    q = rng.random((9, d))
    a = oracle.scale_field(x, c, H, q)
    K = np.stack([stats.multivariate_normal(mean=x[i], cov=H).pdf(q) for i in range(30)], axis=1)
    np.testing.assert_allclose(a, K @ np.abs(c).T, rtol=1e-12)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_first_and_second_moments_are_density_derivatives(d):
    # grad_q s_0 = H^-1 s_(1) and H (grad grad^T s_0) H = s_(2) - H s_0, where
    # s_(1), s_(2) are the first and second moments of (x_i - q).  This pins the
    # sign (x_i - q) of eq. 4 and the exponent bookkeeping independently of eq. 9.
    rng = np.random.default_rng(10 + d)
    H = rand_spd(rng, d, 0.15)
    x = rng.random((40, d))
    q = rng.random((3, d))
    ones = np.ones((1, 40))
    m = oracle.moment_sums(x, ones, H, 2, q)[:, 0, :]
    ex = oracle.monomials(d, 2)
    first = [int(np.where((ex == np.eye(d, dtype=int)[j]).all(1))[0][0]) for j in range(d)]

    def s0(p):
        return oracle.moment_sums(x, ones, H, 0, p[None])[0, 0, 0]

    h = 1e-4
    for k in range(q.shape[0]):
        grad = np.zeros(d)
        hess = np.zeros((d, d))
        for a in range(d):
            ea = np.eye(d)[a] * h
            grad[a] = (s0(q[k] + ea) - s0(q[k] - ea)) / (2 * h)
            for b in range(d):
                eb = np.eye(d)[b] * h
                hess[a, b] = (s0(q[k] + ea + eb) - s0(q[k] + ea - eb)
                              - s0(q[k] - ea + eb) + s0(q[k] - ea - eb)) / (4 * h * h)
        s1 = m[k, first]
        np.testing.assert_allclose(H @ grad, s1, rtol=1e-6, atol=1e-7 * np.abs(s1).max())
        S2 = np.zeros((d, d))
        for a in range(d):
            for b in range(d):
                e = np.zeros(d, dtype=int)
                e[a] += 1
                e[b] += 1
                S2[a, b] = m[k, int(np.where((ex == e).all(1))[0][0])]
        np.testing.assert_allclose(H @ hess @ H + H * m[k, 0], S2,
                                   rtol=1e-4, atol=1e-5 * np.abs(S2).max())


@pytest.mark.parametrize("d,order", [(1, 0), (2, 0), (3, 0), (1, 1), (2, 1), (3, 1)])
def test_constant_response_is_returned(d, order):
    rng = np.random.default_rng(20 + d + 3 * order)
    x = rng.random((60, d))
    H = rand_spd(rng, d, 0.2)
    q = rng.random((15, d))
    r = oracle.smooth_at(x, np.full((1, 60), -2.5), H, order, q)
    np.testing.assert_allclose(r["mhat"], -2.5, rtol=1e-12)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_local_linear_reproduces_linear_m(d):
    rng = np.random.default_rng(30 + d)
    x = rng.random((80, d))
    H = rand_spd(rng, d, 0.2)
    a, b = 0.7, rng.standard_normal(d)
    y = a + x @ b
    q = rng.random((25, d))
    r = oracle.smooth_at(x, y[None], H, 1, q)
    np.testing.assert_allclose(r["mhat"][:, 0], a + q @ b, rtol=1e-10, atol=1e-11)
    # NW does not reproduce a sloped line (boundary bias, Sec. 1): it must differ
    r0 = oracle.smooth_at(x, y[None], H, 0, q)
    assert np.max(np.abs(r0["mhat"][:, 0] - (a + q @ b))) > 1e-3


@pytest.mark.parametrize("d", [1, 2, 3])
def test_local_linear_reproduces_linear_m_where_the_solve_pivots(d):
    # query points well outside the sample cloud: a first moment of eq. 3's
    # system exceeds s_0 (|sum_i K (x_i - q)_a| > sum_i K), so the elimination
    # swaps rows; local linear still reproduces a line exactly there
    rng = np.random.default_rng(80 + d)
    n = 60
    x = rng.random((n, d))
    H = rand_spd(rng, d, 1.0)          # wide enough that far queries see the samples
    a, b = 0.3, rng.standard_normal(d)
    y = a + x @ b
    q = 3.0 + rng.random((10, d))
    r = oracle.smooth_at(x, y[None], H, 1, q)
    first = r["s"][:, 1:d + 1]          # monomial order: 1, then z_1 .. z_d
    assert np.all(np.max(np.abs(first), axis=1) > r["s"][:, 0])
    np.testing.assert_allclose(r["mhat"][:, 0], a + q @ b, rtol=1e-9, atol=1e-10)


@pytest.mark.parametrize("d", [1, 2])
def test_local_quadratic_reproduces_quadratic_m(d):
    # order 2 (the paper's LQ): exact for any quadratic m, where LL is not
    rng = np.random.default_rng(35 + d)
    x = rng.random((90, d))
    H = rand_spd(rng, d, 0.2)
    a, b = 0.4, rng.standard_normal(d)
    C = rng.standard_normal((d, d))
    C = C + C.T
    y = a + x @ b + np.einsum("ni,ij,nj->n", x, C, x)
    q = rng.random((25, d))
    r = oracle.smooth_at(x, y[None], H, 2, q)
    np.testing.assert_allclose(r["mhat"][:, 0], a + q @ b + np.einsum("ni,ij,nj->n", q, C, q),
                               rtol=1e-9, atol=1e-10)
    r1 = oracle.smooth_at(x, y[None], H, 1, q)
    assert np.max(np.abs(r1["mhat"][:, 0] - r["mhat"][:, 0])) > 1e-3


@pytest.mark.parametrize("d", [1, 2, 3])
def test_local_linear_equals_weighted_least_squares(d):
    # eq. 2 minimised directly with numpy's least-squares routine
    rng = np.random.default_rng(40 + d)
    n = 50
    x = rng.random((n, d))
    H = rand_spd(rng, d, 0.25)
    y = np.sin(4 * x[:, 0]) + rng.standard_normal(n) * 0.1
    q = rng.random((6, d))
    r = oracle.smooth_at(x, y[None], H, 1, q)
    for k in range(q.shape[0]):
        z = x - q[k]
        w = stats.multivariate_normal(mean=np.zeros(d), cov=H).pdf(z).reshape(-1)
        D = np.hstack([np.ones((n, 1)), z])
        sw = np.sqrt(w)[:, None]
        beta = np.linalg.lstsq(D * sw, y * sw[:, 0], rcond=None)[0]
        np.testing.assert_allclose(r["mhat"][k, 0], beta[0], rtol=1e-9, atol=1e-12)
    # NW is the weighted mean
    r0 = oracle.smooth_at(x, y[None], H, 0, q)
    for k in range(q.shape[0]):
        w = stats.multivariate_normal(mean=np.zeros(d), cov=H).pdf(x - q[k]).reshape(-1)
        np.testing.assert_allclose(r0["mhat"][k, 0], np.sum(w * y) / np.sum(w), rtol=1e-12)


@pytest.mark.parametrize("d,order", [(1, 0), (2, 0), (1, 1), (2, 1), (3, 1)])
def test_smoother_diagonal_and_trace_match_explicit_matrix(d, order):
    # Build S column by column by smoothing unit vectors, compare diag(S)
    rng = np.random.default_rng(50 + d + order)
    n = 30
    x = rng.random((n, d))
    H = rand_spd(rng, d, 0.3)
    S = oracle.apply_smoother(x, np.eye(n), H, order)   # S[i, j] = (S e_j)_i
    np.testing.assert_allclose(np.diag(S), oracle.smoother_diag(x, H, order), rtol=1e-10)
    np.testing.assert_allclose(np.trace(S), oracle.trace_exact(x, H, order), rtol=1e-10)
    np.testing.assert_allclose(S.sum(axis=1), 1.0, rtol=1e-10)     # rows reproduce constants
    if order == 0:
        s0 = oracle.moment_sums(x, np.ones((1, n)), H, 0, x)[:, 0, 0]
        k0 = stats.multivariate_normal(mean=np.zeros(d), cov=H).pdf(np.zeros(d))
        np.testing.assert_allclose(np.diag(S), k0 / s0, rtol=1e-12)


def test_single_sample_trace_is_one():
    for d in (1, 2, 3):
        x = np.full((1, d), 0.4)
        assert abs(oracle.trace_exact(x, np.eye(d) * 0.01, 0) - 1.0) < 1e-14


def test_gcv_vanishes_for_reproduced_response():
    rng = np.random.default_rng(7)
    x = rng.random((40, 2))
    y = 1.0 - 2.0 * x[:, 0] + 0.5 * x[:, 1]
    H = np.diag([0.05, 0.08])
    m = oracle.apply_smoother(x, y[None], H, 1)[:, 0]
    rss = float(np.sum((y - m) ** 2))
    assert rss < 1e-20
    tr = oracle.trace_exact(x, H, 1)
    assert oracle.gcv(rss, 40, tr) < 1e-20
    # eq. 22 on a hand-made case
    assert oracle.gcv(8.0, 4, 2.0) == pytest.approx((8.0 / 4) / (0.5 ** 2))


def test_fmc_trace_is_unbiased():
    # Sec. 2.1: E[w^T S w] = tr(S) for w ~ N(0, I); mean over 3000 probes lies
    # within 4 standard errors of the exact trace.
    rng = np.random.default_rng(99)
    n = 200
    x = rng.random((n, 1))
    H = np.array([[0.03 ** 2]])
    S = oracle.apply_smoother(x, np.eye(n), H, 0)
    exact = np.trace(S)
    assert exact == pytest.approx(oracle.trace_exact(x, H, 0), rel=1e-10)
    w = oracle.probes(12345, 3000, n)
    r = oracle.fmc_trace(x, w, H, 0, Sw=(S @ w.T).T)
    se = np.std(r["wSw"]) / math.sqrt(3000)
    assert abs(r["hutchinson"] - exact) < 4 * se
    assert abs(r["girard"] - exact) < 4 * se * 1.5


def test_probe_generator_is_standard_normal():
    z = oracle.probes(2024, 4, 50_000)
    for p in range(4):
        assert stats.kstest(z[p], "norm").pvalue > 1e-4
        assert abs(z[p].mean()) < 5 / math.sqrt(50_000)
        assert abs(z[p].var() - 1) < 0.03
    c = np.corrcoef(z)
    assert np.max(np.abs(c - np.eye(4))) < 0.02
    z32 = oracle.probes(2024, 2, 50_000, precision="f32")
    assert z32.dtype == np.float32
    for p in range(2):
        assert stats.kstest(z32[p].astype(np.float64), "norm").pvalue > 1e-4
    # Box-Muller pairs: probes 2j and 2j+1 share the radius r, and r^2 of a pair
    # of independent standard normals is exponential with mean 2
    r2 = z[0] ** 2 + z[1] ** 2
    assert stats.kstest(r2, "expon", args=(0, 2)).pvalue > 1e-4
    # an odd count draws the cosine of its last pair: the first probes agree
    z3 = oracle.probes(2024, 3, 50_000)
    np.testing.assert_array_equal(z3, z[:3])
    # the single-precision variant draws from the same counters (24-bit uniforms)
    assert np.corrcoef(z[0], z32[0].astype(np.float64))[0, 1] > 0.999
    # SplitMix64 is a bijection on 64-bit words: no collisions on a run of counters
    outs = {oracle.splitmix64(k) for k in range(5000)}
    assert len(outs) == 5000


def test_get_hlist_reproduces_printed_bessel_values():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "get_hlist_bessel.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert rows
    for n, lo, hi, sp, idx, val in rows:
        h = oracle.get_hlist(int(n), float(lo), float(hi), sp)
        assert round(h[int(idx) - 1], 6 if float(val) < 0.1 else 5) == pytest.approx(float(val), abs=1e-12)
    # original-scale h = normalised h * std(x): the two printed pairs share the ratio
    assert 0.26178 / 0.046416 == pytest.approx(0.72843 / 0.12915, rel=1e-4)


def test_select_h_dstd_rule():
    g = [5.0, 3.0, 2.0, 2.0, 4.0]
    assert oracle.select_h(g, 0.0) == 3          # ties go to the larger h
    assert oracle.select_h([5.0, 2.0, 2.1, 9.0], 0.0) == 1
    # relaxed: anything within dstd*std of the min qualifies, the largest h wins
    s = float(np.std([5.0, 2.0, 2.1, 9.0]))
    assert oracle.select_h([5.0, 2.0, 2.1, 9.0], 0.15 / s) == 2
    assert oracle.select_h([5.0, 2.0, 2.1, 9.0], 0.05 / s) == 1


def test_variance_pass_reproduces_constant_and_linear_residuals():
    rng = np.random.default_rng(5)
    x = rng.random((70, 2))
    y = rng.standard_normal(70)
    q = rng.random((10, 2))
    H = np.diag([0.1 ** 2, 0.12 ** 2])
    m = y - 0.3 * np.sign(rng.standard_normal(70))      # |y - m|^2 == 0.09
    v = oracle.variance_pass(x, y[None], m[None], H, q)
    np.testing.assert_allclose(v[:, 0], 0.09, rtol=1e-12)
    r = 0.5 + x[:, 0] - 0.25 * x[:, 1]                  # |y - m|^2 linear in x
    v = oracle.variance_pass(x, np.sqrt(r)[None], np.zeros((1, 70)), H, q)
    np.testing.assert_allclose(v[:, 0], 0.5 + q[:, 0] - 0.25 * q[:, 1], rtol=1e-10)


def test_log_variance_closed_forms():
    # eqs. 24-26 on residuals with known structure
    rng = np.random.default_rng(6)
    n = 80
    x = rng.random((n, 2))
    q = rng.random((12, 2))
    H = np.diag([0.1 ** 2, 0.12 ** 2])
    y = rng.standard_normal(n)
    # constant squared residual c: v = log(c + 1/N), kappa = (c + 1/N) / c,
    # sigma^2 = c exactly
    c = 0.09
    m = y - 0.3 * np.sign(rng.standard_normal(n))
    out = oracle.log_variance(x, y[None], m[None], H, q)
    np.testing.assert_allclose(out["v_grid"][:, 0], np.log(c + 1.0 / n), rtol=1e-12)
    assert out["kappa"][0] == pytest.approx((c + 1.0 / n) / c, rel=1e-12)
    np.testing.assert_allclose(out["sigma2"][:, 0], c, rtol=1e-12)
    # log(r + 1/N) linear in x: local linear reproduces v at q and at the
    # samples, so kappa = 1 / (1 - mean(exp(-v_i)) / N)
    def v_true(p):
        return -1.0 + 0.8 * p[:, 0] - 0.5 * p[:, 1]
    r = np.exp(v_true(x)) - 1.0 / n
    out = oracle.log_variance(x, np.sqrt(r)[None], np.zeros((1, n)), H, q)
    np.testing.assert_allclose(out["v_grid"][:, 0], v_true(q), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(out["v_at_x"][:, 0], v_true(x), rtol=1e-10, atol=1e-12)
    kappa = 1.0 / (1.0 - np.mean(np.exp(-v_true(x))) / n)
    assert out["kappa"][0] == pytest.approx(kappa, rel=1e-12)
    np.testing.assert_allclose(out["sigma2"][:, 0], np.exp(v_true(q)) / kappa, rtol=1e-10)


def test_interval_eq28():
    # 95 % two-sided normal quantile is the textbook 1.959963984540054; a
    # 68.27 % interval is one standard deviation wide on each side
    lo, hi = oracle.interval(np.array([1.0, -2.0]), np.array([4.0, 0.25]), 0.05)
    np.testing.assert_allclose(hi - np.array([1.0, -2.0]), 1.959963984540054 * np.array([2.0, 0.5]),
                               rtol=1e-14)
    np.testing.assert_allclose(lo + hi, 2 * np.array([1.0, -2.0]), rtol=1e-15)
    lo, hi = oracle.interval(np.zeros(1), np.ones(1), 1 - 0.6826894921370859)
    assert hi[0] == pytest.approx(1.0, rel=1e-12)
    lo, hi = oracle.interval(np.zeros(1), -np.ones(1), 0.05)
    assert np.isnan(lo[0]) and np.isnan(hi[0])


@pytest.mark.parametrize("d", [1, 2, 3])
def test_predict_reproduces_polynomials(d):
    # multilinear interpolation is exact for affine functions (also when it
    # extends past the box); cubic convolution with Keys' boundary rows is
    # exact for quadratics anywhere in the box and returns node values at nodes
    rng = np.random.default_rng(60 + d)
    grid_n = (9, 7, 6)[:d]
    lo, hi = (0.0, -1.0, 0.5)[:d], (2.0, 1.0, 1.5)[:d]
    gp = oracle.grid_points(grid_n, lo, hi)
    b = rng.standard_normal(d)
    C = rng.standard_normal((d, d))
    C = C + C.T
    aff = 0.3 + gp @ b
    quad = 0.3 + gp @ b + np.einsum("ni,ij,nj->n", gp, C, gp)
    xin = np.asarray(lo) + rng.random((40, d)) * (np.asarray(hi) - np.asarray(lo))
    xin[:4] = np.asarray(lo)            # on the lower edge
    xin[4:8] = np.asarray(hi)           # on the upper edge
    xout = np.asarray(lo) - 0.3 + rng.random((10, d)) * (np.asarray(hi) - np.asarray(lo) + 0.6)
    lin = oracle.predict(aff[None], grid_n, lo, hi, np.vstack([xin, xout]), "linear")
    np.testing.assert_allclose(lin[0], 0.3 + np.vstack([xin, xout]) @ b, rtol=1e-12, atol=1e-12)
    cub = oracle.predict(quad[None], grid_n, lo, hi, xin, "cubic")
    np.testing.assert_allclose(cub[0], 0.3 + xin @ b + np.einsum("ni,ij,nj->n", xin, C, xin),
                               rtol=1e-11, atol=1e-11)
    node = oracle.predict(np.sin(3 * gp.sum(axis=1))[None], grid_n, lo, hi, gp[::5], "cubic")
    np.testing.assert_allclose(node[0], np.sin(3 * gp[::5].sum(axis=1)), rtol=1e-13, atol=1e-14)
    assert np.all(np.isnan(oracle.predict(quad[None], grid_n, lo, hi, np.asarray(lo)[None] - 0.1,
                                          "cubic")))
    # multilinear against scipy's regular-grid interpolator
    from scipy.interpolate import RegularGridInterpolator
    axes = [np.linspace(lo[j], hi[j], grid_n[j]) for j in range(d)]
    f = np.cos(gp.sum(axis=1))
    ref = RegularGridInterpolator(axes, f.reshape(grid_n))(xin)
    np.testing.assert_allclose(oracle.predict(f[None], grid_n, lo, hi, xin, "linear")[0], ref,
                               rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("name", oracle.COMPACT_KERNELS)
def test_compact_kernels_are_densities(name):
    from scipy import integrate
    v1 = integrate.quad(lambda u: float(oracle.compact_profile(name, 1, u * u)), -1, 1,
                        points=[0.0], epsabs=1e-13)[0]
    assert v1 == pytest.approx(1.0, rel=1e-9)
    v2 = integrate.dblquad(lambda b, a: float(oracle.compact_profile(name, 2, a * a + b * b)),
                           -1, 1, lambda a: -math.sqrt(1 - a * a), lambda a: math.sqrt(1 - a * a),
                           epsabs=1e-11, epsrel=1e-10)[0]
    assert v2 == pytest.approx(1.0, rel=1e-7)
    assert float(oracle.compact_profile(name, 2, 1.0001)) == 0.0


@pytest.mark.parametrize("name", oracle.COMPACT_KERNELS)
def test_compact_kernel_smoothing(name):
    rng = np.random.default_rng(70)
    x = rng.random((400, 2))
    H = np.diag([0.2 ** 2, 0.25 ** 2])
    q = 0.2 + 0.6 * rng.random((12, 2))
    # a constant is returned, local linear reproduces a line
    r = oracle.smooth_at_compact(x, np.full((1, 400), 1.5), H, 0, q, name)
    np.testing.assert_allclose(r["mhat"][:, 0], 1.5, rtol=1e-12)
    b = np.array([0.7, -0.4])
    r = oracle.smooth_at_compact(x, (0.2 + x @ b)[None], H, 1, q, name)
    np.testing.assert_allclose(r["mhat"][:, 0], 0.2 + q @ b, rtol=1e-10, atol=1e-12)
    # the density sum counts exactly the samples inside the ellipse, weighted
    z = x - q[0]
    u2 = z[:, 0] ** 2 / 0.04 + z[:, 1] ** 2 / 0.0625
    s0 = oracle.moment_sums_compact(x, np.ones((1, 400)), H, 0, q[:1], name)[0, 0, 0]
    ref = np.sum(oracle.compact_profile(name, 2, u2[u2 <= 1])) / (0.2 * 0.25)
    assert s0 == pytest.approx(ref, rel=1e-12)
    if name == "uniform":
        # NW with the uniform kernel is the plain mean of y over the ellipse
        y = rng.standard_normal(400)
        r = oracle.smooth_at_compact(x, y[None], H, 0, q[:1], name)
        assert r["mhat"][0, 0] == pytest.approx(np.mean(y[u2 <= 1]), rel=1e-12)


@pytest.mark.parametrize("name", ["epanechnikov", "triweight"])
def test_compact_kernel_full_bandwidth_matrix(name):
    # a correlated H: the support is the rotated ellipse z^T H^-1 z <= 1 and
    # the scale is |H|^-1/2; the moment sums equal brute-force weighted sums
    # over the samples inside it, and the first moments change sign with z
    rng = np.random.default_rng(71)
    x = rng.random((300, 2))
    H = np.array([[0.04, 0.018], [0.018, 0.02]])
    q = np.array([[0.45, 0.55]])
    z = x - q[0]
    u2 = np.einsum("ia,ab,ib->i", z, np.linalg.inv(H), z)
    w = oracle.compact_profile(name, 2, u2) / math.sqrt(np.linalg.det(H))
    y = rng.standard_normal(300)
    m = oracle.moment_sums_compact(x, np.stack([np.ones(300), y]), H, 2, q, name)[0]
    ex = [tuple(e) for e in oracle.monomials(2, 2)]
    for f, e in enumerate(ex):
        mono = z[:, 0] ** e[0] * z[:, 1] ** e[1]
        assert m[0, f] == pytest.approx(np.sum(w * mono), rel=1e-12, abs=1e-14)
        assert m[1, f] == pytest.approx(np.sum(w * mono * y), rel=1e-11, abs=1e-13)
    assert np.sum(u2 <= 1) > 10 and np.sum((u2 > 1) & (np.abs(z).max(axis=1) < 0.2)) > 0


def test_kde_integrates_to_one():
    # eq. 8: s_0 / N is a density (Gaussian K has unit mass)
    rng = np.random.default_rng(3)
    x = 0.3 + 0.4 * rng.random((25, 2))
    H = np.diag([0.03 ** 2, 0.02 ** 2])
    g = oracle.grid_points((201, 201), (0, 0), (1, 1))
    s0 = oracle.moment_sums(x, np.ones((1, 25)), H, 0, g)[:, 0, 0]
    assert np.sum(s0) * (1 / 200) ** 2 / 25 == pytest.approx(1.0, rel=1e-6)


def test_grid_points_eq6():
    g = oracle.grid_points((3, 5), (0.0, -1.0), (1.0, 1.0))
    assert g.shape == (15, 2)
    np.testing.assert_allclose(g[:5, 1], [-1, -0.5, 0, 0.5, 1])
    np.testing.assert_allclose(g[::5, 0], [0, 0.5, 1])


# ------------------------------------------------------------ cutoff mode ----
@pytest.mark.parametrize("d,deg", [(1, 2), (2, 2), (2, 4), (3, 2)])
def test_cutoff_sums_equal_the_full_sums(d, deg):
    # the cell-list sums leave out only pairs with K_H < 1e-18 K_H(0): on small
    # inputs they equal the plain O(N) sums of eq. 9 to rounding, with a
    # correlated H, clustered samples and queries inside and outside the box
    rng = np.random.default_rng(300 + d + deg)
    H = rand_spd(rng, d, 0.04)
    x = np.concatenate([rng.random((1500, d)), 0.5 + 0.01 * rng.standard_normal((500, d))])
    c = np.stack([np.ones(x.shape[0]), rng.standard_normal(x.shape[0])])
    q = np.concatenate([rng.random((60, d)), rng.random((20, d)) * 1.6 - 0.3])
    full = oracle.moment_sums(x, c, H, deg, q)
    cut = oracle.moment_sums(x, c, H, deg, q, cutoff=True)
    scale = oracle.moment_sums(x, np.abs(c), H, 0, q)[:, :, :1]      # sum of |terms| per point
    sig = np.sqrt(np.max(np.diag(H)))
    expo = oracle.monomials(d, deg).sum(axis=1)
    # pointwise inside the sample cloud, normwise (against the largest sum of
    # |terms|) at the queries outside it, where every term is tiny
    ref = scale * sig ** expo[None, None, :]
    err_in = np.abs(cut - full)[:60] / ref[:60]
    err_all = np.abs(cut - full) / np.max(ref, axis=0, keepdims=True)
    assert np.max(err_in) < 1e-12
    assert np.max(err_all) < 1e-12


@pytest.mark.parametrize("d", [1, 2, 3])
def test_cutoff_neighbour_search_finds_every_pair(d):
    # with a small radius most pairs are cut: the cell-list sum must equal a
    # brute-force sum over exactly the pairs with z^T H^-1 z <= r2 (numpy, all
    # pairs), so a cell the search skipped would show up
    rng = np.random.default_rng(310 + d)
    H = rand_spd(rng, d, 0.08)
    n = 3000
    x = rng.random((n, d))
    y = rng.standard_normal(n)
    q = np.concatenate([rng.random((50, d)), x[:10]])
    r2 = 2.0
    L = oracle.lib()
    out = np.zeros((q.shape[0], 2, d + 1))
    c = np.ascontiguousarray(np.stack([np.ones(n), y]))
    rc = L.or_moment_sums_cutoff(d, n, oracle._dp(np.ascontiguousarray(x)), 2, oracle._dp(c),
                                 oracle._dp(np.ascontiguousarray(H)), 1, q.shape[0],
                                 oracle._dp(np.ascontiguousarray(q)), r2, oracle._dp(out), 0)
    assert rc == 0
    Hinv = np.linalg.inv(H)
    norm = 1.0 / math.sqrt((2 * math.pi) ** d * np.linalg.det(H))
    counts = []
    for k, qq in enumerate(q):
        z = x - qq
        e = np.einsum("ni,ij,nj->n", z, Hinv, z)
        inside = e <= r2
        counts.append(int(inside.sum()))
        kv = np.where(inside, norm * np.exp(-0.5 * e), 0.0)
        mono = np.concatenate([np.ones((n, 1)), z], axis=1)
        ref = np.stack([kv @ mono, (kv * y) @ mono])
        np.testing.assert_allclose(out[k], ref, rtol=1e-12, atol=1e-12 * max(np.abs(ref).max(), 1.0))
    counts = np.array(counts)
    assert np.mean((counts > 0) & (counts < n)) > 0.8 and np.all(counts[50:] > 0)


def test_cutoff_sums_without_neighbours_or_samples():
    H = np.diag([1e-4, 1e-4])
    x = np.array([[0.2, 0.2], [0.25, 0.2]])
    q = np.array([[0.9, 0.9], [0.2, 0.2]])
    m = oracle.moment_sums(x, np.ones((1, 2)), H, 2, q, cutoff=True)
    assert np.all(m[0] == 0.0)
    np.testing.assert_allclose(m[1], oracle.moment_sums(x, np.ones((1, 2)), H, 2, q[1:]) [0],
                               rtol=1e-14)
    e = oracle.moment_sums(np.zeros((0, 2)), np.ones((1, 0)), H, 1, q, cutoff=True)
    assert e.shape == (2, 1, 3) and np.all(e == 0.0)


def test_effective_weight_is_s0_for_nw_and_pins_the_error_bound():
    # parity_util.effective_weight: 1/||S~^-1 e_1||_1 equals s_0 for
    # Nadaraya-Watson, and bounds the m-hat change under a field perturbation
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    from parity_util import effective_weight
    rng = np.random.default_rng(77)
    H = np.diag([0.05 ** 2, 0.08 ** 2])
    x = rng.random((400, 2))
    q = rng.random((50, 2))
    y = rng.standard_normal((1, 400))
    s = oracle.moment_sums(x, np.ones((1, 400)), H, 0, q)[:, 0, :]
    np.testing.assert_allclose(effective_weight(s, H, 2, 0), s[:, 0], rtol=1e-14)
    r = oracle.smooth_at(x, y, H, 1, q)
    w = effective_weight(r["s"], H, 2, 1)
    assert np.all(w > 0) and np.all(w <= r["s"][:, 0] * (1 + 1e-12))
    # perturb the t-fields by delta (scaled basis): |dm| <= max|delta~| / w
    sig = np.sqrt(np.diag(H))
    delta = 1e-6 * rng.standard_normal(r["t"].shape)
    m2, _ = oracle.lpr_solve(2, 1, r["s"], r["t"] + delta)
    dt_scaled = np.abs(delta[:, 0, :] / np.array([1.0, sig[0], sig[1]]))
    assert np.all(np.abs(m2[:, 0] - r["mhat"][:, 0]) <= dt_scaled.max(axis=1) / w * (1 + 1e-9))


# ------------------------------------------------------- oracle gradients ----
def _fd(f, eps=1e-5):
    return (f(eps) - f(-eps)) / (2 * eps)


@pytest.mark.parametrize("d,order", [(1, 0), (1, 1), (2, 1), (2, 0)])
def test_estimate_vjp_matches_finite_differences_of_the_estimate(d, order):
    # the analytic gradient of sum_q gbar(q) mhat(q) against central
    # differences of the oracle's own estimates (eqs. 3, 9, 11)
    rng = np.random.default_rng(400 + 10 * d + order)
    n = 60
    x = rng.random((n, d))
    Y = np.stack([np.cos(3 * x.sum(axis=1)) + 0.1 * rng.standard_normal(n),
                  rng.standard_normal(n)])
    sig = np.array([0.12, 0.17][:d])
    q = rng.random((7, d)) * 0.8 + 0.1
    gbar = rng.standard_normal((2, 7))

    def L(xx, YY, s):
        H = np.diag(s ** 2)
        return float(np.sum(gbar * oracle.smooth_at(xx, YY, H, order, q)["mhat"].T))

    g = oracle.estimate_vjp(x, Y, sig, order, q, gbar)
    for j in range(d):
        def f(e, j=j):
            s = sig.copy()
            s[j] *= np.exp(e)
            return L(x, Y, s)
        assert g["dlogsigma"][j] == pytest.approx(_fd(f), rel=1e-6, abs=1e-9)
    for i in (0, 13, 41):
        for v in range(2):
            def fy(e, i=i, v=v):
                YY = Y.copy()
                YY[v, i] += e
                return L(x, YY, sig)
            assert g["dY"][v, i] == pytest.approx(_fd(fy), rel=1e-6, abs=1e-9)
        for a in range(d):
            def fx(e, i=i, a=a):
                xx = x.copy()
                xx[i, a] += e
                return L(xx, Y, sig)
            assert g["dx"][i, a] == pytest.approx(_fd(fx), rel=1e-6, abs=1e-8)


def test_estimate_vjp_at_the_samples_moves_the_query_points():
    # q = x: the estimate at each sample moves with the sample (target side)
    rng = np.random.default_rng(431)
    n, d = 40, 2
    x = rng.random((n, d))
    Y = np.sin(4 * x[:, :1].T) + 0.1 * rng.standard_normal((1, n))
    sig = np.array([0.15, 0.2])
    gbar = rng.standard_normal((1, n))

    def L(xx):
        return float(np.sum(gbar * oracle.smooth_at(xx, Y, np.diag(sig ** 2), 1, xx)["mhat"].T))

    g = oracle.estimate_vjp(x, Y, sig, 1, x, gbar, q_is_x=True)
    for i in (2, 17, 33):
        for a in range(d):
            def fx(e, i=i, a=a):
                xx = x.copy()
                xx[i, a] += e
                return L(xx)
            assert g["dx"][i, a] == pytest.approx(_fd(fx), rel=1e-6, abs=1e-8)


def test_gcv_grad_matches_finite_differences():
    # eq. 22 with fixed probes: the analytic gradient against central
    # differences of the oracle's GCV
    rng = np.random.default_rng(440)
    n, d = 50, 2
    x = rng.random((n, d))
    y = np.cos(3 * x.sum(axis=1)) + 0.2 * rng.standard_normal(n)
    w = oracle.probes(3, 2, n)
    sig = np.array([0.14, 0.18])

    def G(xx, yy, s):
        H = np.diag(s ** 2)
        m = oracle.apply_smoother(xx, yy[None], H, 1)[:, 0]
        f = oracle.fmc_trace(xx, w, H, 1)
        return oracle.gcv(float(np.sum((yy - m) ** 2)), n, f["girard"])

    g = oracle.gcv_grad(x, y, w, sig, 1)
    assert g["gcv"] == pytest.approx(G(x, y, sig), rel=1e-12)
    for j in range(d):
        def f(e, j=j):
            s = sig.copy()
            s[j] *= np.exp(e)
            return G(x, y, s)
        assert g["dlogsigma"][j] == pytest.approx(_fd(f), rel=1e-6, abs=1e-10)
    for i in (1, 22, 47):
        def fy(e, i=i):
            yy = y.copy()
            yy[i] += e
            return G(x, yy, sig)
        assert g["dy"][i] == pytest.approx(_fd(fy), rel=1e-6, abs=1e-10)
        for a in range(d):
            def fx(e, i=i, a=a):
                xx = x.copy()
                xx[i, a] += e
                return G(xx, y, sig)
            assert g["dx"][i, a] == pytest.approx(_fd(fx), rel=1e-6, abs=1e-9)
