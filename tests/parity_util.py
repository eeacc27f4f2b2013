"""Error measures for comparing the CUDA path with the FP64 oracle.

The paper states no error measure.  The NUFFT error is global and scales
with the l1 norm of the strengths, so a field is compared normwise against
its natural size (see the test tolerances):

* moment field s_g / t_g:   max_q |G(q) - O(q)| / (max_q a(q) * sigma^g),
  a(q) = sum_i K_H(x_i - q) |c_i| (c = 1 for s-fields, y for t-fields) and
  sigma^g = prod_j sigma_j^g_j the length scale of the moment.
* estimate mhat:            max_q s_0(q) |mhat_G(q) - mhat_O(q)| / max_q a_y(q),
  i.e. the error of the numerator t_0 that the estimate inherits; a plain
  relative error is undefined where mhat crosses zero and grows like
  tol / density in sparse regions for any tolerance-controlled method.

A point where the oracle's value is finite and the point is valid (not
masked) must be finite on the GPU too: mhat_error returns infinity there, so
a GPU NaN never hides behind the metric.  ``check_mask`` compares the GPU's
density mask with the oracle's s_0 in both directions.
"""
import numpy as np

import oracle


def field_scale_sigma(H, expo):
    sig = np.sqrt(np.diag(H))
    return float(np.prod(sig ** np.asarray(expo)))


def mhat_error(mg, mo, s0, a_y, valid=None):
    mg = np.asarray(mg, dtype=np.float64).reshape(-1)
    mo = np.asarray(mo, dtype=np.float64).reshape(-1)
    s0 = np.asarray(s0, dtype=np.float64).reshape(-1)
    ok = np.isfinite(mo)
    if valid is not None:
        ok &= np.asarray(valid).reshape(-1)
    if not ok.any():
        return 0.0
    if not np.all(np.isfinite(mg[ok])):
        return float("inf")
    return float(np.max(s0[ok] * np.abs(mg[ok] - mo[ok])) / np.max(np.abs(a_y)))


def check_mask(mask, s0_oracle, s0_max, rho=1e-3, margin=0.01):
    """The GPU's mask (s_0(g) >= rho max s_0) against the oracle's s_0.

    Points the oracle puts clearly above the threshold must be unmasked and
    points clearly below it masked; within ``margin`` of it either is right.
    """
    mask = np.asarray(mask).reshape(-1).astype(bool)
    s0 = np.asarray(s0_oracle, dtype=np.float64).reshape(-1)
    thr = rho * s0_max
    dense = s0 >= (1 + margin) * thr
    sparse = s0 <= (1 - margin) * thr
    assert np.all(mask[dense]), f"{int(np.sum(~mask[dense]))} dense points masked"
    assert not np.any(mask[sparse]), f"{int(np.sum(mask[sparse]))} sparse points unmasked"


def field_error(g, o, a, sigma_scale):
    g = np.asarray(g, dtype=np.float64).reshape(-1)
    o = np.asarray(o, dtype=np.float64).reshape(-1)
    return float(np.max(np.abs(g - o)) / (np.max(np.abs(a)) * sigma_scale))


def sample_grid_indices(grid_n, k, seed=0):
    M = int(np.prod(grid_n))
    rng = np.random.default_rng(seed)
    if k >= M:
        return np.arange(M)
    idx = rng.choice(M, size=k, replace=False)
    # always include the corners (boundary rows stress local-linear)
    idx = np.unique(np.concatenate([idx, [0, M - 1]]))
    return idx
