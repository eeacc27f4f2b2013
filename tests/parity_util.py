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


def check_mask(mask, s0_oracle, s0_max, rho=1e-3, margin=0.01, singular=None):
    """The GPU's mask (s_0(g) >= rho max s_0) against the oracle's s_0.

    Points the oracle puts clearly above the threshold must be unmasked and
    points clearly below it masked; within ``margin`` of it either is right.
    ``singular`` marks points whose local system of eq. 3 is singular within
    the field error the bar allows (``singular_within``): the GPU may mask
    those too (it masks a system whose determinant is not positive).
    """
    mask = np.asarray(mask).reshape(-1).astype(bool)
    s0 = np.asarray(s0_oracle, dtype=np.float64).reshape(-1)
    thr = rho * s0_max
    dense = s0 >= (1 + margin) * thr
    if singular is not None:
        dense &= ~np.asarray(singular).reshape(-1)
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


def scaled_system(s_fields, H, d, order):
    """The scaled local systems S~_ab = s_(a+b) / sigma^(a+b) of eq. 3, [nq, p, p]."""
    s_fields = np.asarray(s_fields, dtype=np.float64)
    ex2 = [tuple(e) for e in oracle.monomials(d, 2 * order)]
    ex1 = [tuple(e) for e in oracle.monomials(d, order)]
    sig = np.sqrt(np.diag(np.asarray(H, dtype=np.float64)))
    p = len(ex1)
    S = np.empty((s_fields.shape[0], p, p))
    for a, ea in enumerate(ex1):
        for b, eb in enumerate(ex1):
            e = tuple(u + v for u, v in zip(ea, eb))
            S[:, a, b] = s_fields[:, ex2.index(e)] / np.prod(sig ** np.asarray(e))
    return S


def effective_weight(s_fields, H, d, order):
    """1 / ||S~^-1 e_1||_1 per query point (0 where S~ is singular).

    m-hat = e_1^T S~^-1 t~ inherits a field error delta as
    |e_1^T S~^-1 delta| <= ||S~^-1 e_1||_1 max|delta|, so this weight is what
    s_0 is in the m-hat error of the module docstring: for Nadaraya-Watson
    (p = 1) it equals s_0, and for a well-posed local-linear system it is
    within a small factor of s_0.  Where the system is ill-conditioned (few
    samples under the kernel) it is much smaller than s_0: the field error is
    amplified there by any method whose fields carry a tolerance.
    """
    S = scaled_system(s_fields, H, d, order)
    nq, p = S.shape[0], S.shape[1]
    wgt = np.zeros(nq)
    det = np.linalg.det(S)
    ok = np.isfinite(det) & (det > 0)
    if ok.any():
        a = np.linalg.solve(S[ok], np.broadcast_to(np.eye(p)[:, :1], (int(ok.sum()), p, 1)))[..., 0]
        wgt[ok] = 1.0 / np.sum(np.abs(a), axis=1)
    return wgt


def singular_within(s_fields, H, d, order, eps_abs):
    """Points whose scaled local system S~ (eq. 3, S~_ab = s_(a+b) / sigma^(a+b))
    has a determinant that a change of eps_abs in every entry can make
    non-positive: det(S~) <= eps_abs * sum_ab |cofactor_ab(S~)|.

    s_fields [nq, nmono(d, 2 order)] are the oracle's s-fields; eps_abs is the
    absolute field error the parity bar allows on the scaled entries (the bar
    times the largest s_0).
    """
    s_fields = np.asarray(s_fields, dtype=np.float64)
    nq = s_fields.shape[0]
    if order == 0:
        return s_fields[:, 0] <= eps_abs
    S = scaled_system(s_fields, H, d, order)
    p = S.shape[1]
    det = np.linalg.det(S)
    cof = np.zeros(nq)
    for a in range(p):
        for b in range(p):
            minor = np.delete(np.delete(S, a, axis=1), b, axis=2)
            cof += np.abs(np.linalg.det(minor)) if p > 1 else 1.0
    return det <= eps_abs * cof
