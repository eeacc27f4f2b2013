"""FP64 oracle of the binned kernel smoother (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA path (``paper_2204_07716_gb300``) and never calls it.

The heavy lifting is the plain C library ``oracle.c`` (direct O(N) sums per
query point, Gaussian elimination in FP64).  This module adds the quantities
built on top of those sums, each written from its definition in the paper:

* ``grid_points``      the uniform grid of eq. 6, endpoints included.
* ``moment_sums``      s_g and t_a of eq. 9 at arbitrary query points; with
                       ``cutoff=True`` the pairs beyond the Mahalanobis radius
                       CUTOFF_R2 are left out (a cell list finds the rest),
                       which keeps N = 10^6 affordable.
* ``smooth_at``        mhat = e_1^T S^-1 t (eqs. 3, 10, 11) at query points.
* ``smoother_diag``    S_ii = K_H(0) [S(x_i)^-1]_11, the i-th diagonal entry of
                       the smoother matrix S of eq. 3 applied at the samples.
* ``trace_exact``      tr(S_h), the DF of eq. 22.
* ``fmc_trace``        Girard's fast Monte-Carlo estimate (Sec. 2.1) and the
                       Hutchinson mean of w_p^T S w_p.
* ``gcv``              eq. 22.
* ``estimate_vjp``     analytic gradient of sum_q gbar(q) mhat(q) (eqs. 3, 9,
                       11) with respect to the responses, the samples (and
                       the query points when they are the samples) and
                       log sigma_j of a diagonal H.
* ``gcv_grad``         analytic gradient of GCV (eq. 22) with fixed probes.
* ``variance_pass``    eq. 23: a local-linear smooth of squared residuals.
* ``log_variance``     eqs. 24-26: smooth of log(r + 1/N), kappa, sigma^2.
* ``interval``         eq. 28: mhat -/+ z_(1 - alpha/2) sqrt(variance).
* ``predict``          grid estimates at new points (multilinear with linear
                       extension; Keys cubic convolution), Sec. 1.1.
* ``compact_profile``, ``moment_sums_compact``, ``smooth_at_compact``
                       the compact kernels of Table 1 by direct sums.
* ``get_hlist``        the bandwidth list helper of Sec. 4.
* ``select_h``         the GCV argmin relaxed by ``dstd`` (Table 1).
* ``probes``           the counter-based Gaussian probe generator.
"""
from __future__ import annotations

import ctypes
import itertools
import math
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        L.or_nmono.argtypes = [ctypes.c_int, ctypes.c_int]
        L.or_nmono.restype = ctypes.c_int
        L.or_monomials.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.or_monomials.restype = ctypes.c_int
        L.or_kernel.argtypes = [ctypes.c_int, dp, dp]
        L.or_kernel.restype = ctypes.c_double
        L.or_moment_sums.argtypes = [ctypes.c_int, ctypes.c_int64, dp, ctypes.c_int, dp, dp,
                                     ctypes.c_int, ctypes.c_int64, dp, dp, ctypes.c_int]
        L.or_moment_sums.restype = ctypes.c_int
        L.or_moment_sums_cutoff.argtypes = [ctypes.c_int, ctypes.c_int64, dp, ctypes.c_int, dp,
                                            dp, ctypes.c_int, ctypes.c_int64, dp,
                                            ctypes.c_double, dp, ctypes.c_int]
        L.or_moment_sums_cutoff.restype = ctypes.c_int
        L.or_lpr_solve.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, dp, ctypes.c_int,
                                   dp, dp, dp]
        L.or_lpr_solve.restype = ctypes.c_int
        L.or_probes.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int64, dp]
        L.or_probes.restype = None
        L.or_probes_f32.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int64,
                                    ctypes.POINTER(ctypes.c_float)]
        L.or_probes_f32.restype = None
        L.or_splitmix64.argtypes = [ctypes.c_uint64]
        L.or_splitmix64.restype = ctypes.c_uint64
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def nmono(d: int, deg: int) -> int:
    return int(lib().or_nmono(d, deg))


def monomials(d: int, deg: int) -> np.ndarray:
    """Exponent table [nmono, d] in the oracle's (and the API's) order."""
    m = nmono(d, deg)
    e = np.zeros(m * d, dtype=np.int32)
    lib().or_monomials(d, deg, e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return e.reshape(m, d)


def kernel(H: np.ndarray, z: np.ndarray) -> float:
    H = _c64(H)
    z = _c64(z)
    return float(lib().or_kernel(H.shape[0], _dp(H), _dp(z)))


def grid_points(grid_n: Sequence[int], lo: Sequence[float], hi: Sequence[float]) -> np.ndarray:
    """All points of the eq. 6 grid, [prod(grid_n), d], last axis fastest.

    g_{k,j} = lo_j + k (hi_j - lo_j) / (M_j - 1), endpoints included.
    """
    axes = []
    for m, a, b in zip(grid_n, lo, hi):
        if m == 1:
            axes.append(np.array([a], dtype=np.float64))
        else:
            axes.append(a + np.arange(m, dtype=np.float64) * ((b - a) / (m - 1)))
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([g.reshape(-1) for g in mesh], axis=1)


# Mahalanobis radius of the cutoff mode: a skipped pair has
# K_H(z) < 1e-18 K_H(0), below the FP64 rounding of any sum near its centre.
CUTOFF_R2 = 2.0 * math.log(1e18)


def moment_sums(x: np.ndarray, c: np.ndarray, H: np.ndarray, deg: int,
                q: np.ndarray, nthreads: int = 0, cutoff: bool = False) -> np.ndarray:
    """s/t moment sums of eq. 9, [nq, nstr, nmono(d, deg)].

    ``c`` is [nstr, n] (use ones for the s-fields, y for the t-fields).
    ``cutoff=True`` skips the pairs with z^T H^-1 z > CUTOFF_R2 (found
    through a cell list); the result equals the full sum to rounding.
    """
    x = _c64(x)
    n, d = x.shape
    c = _c64(np.atleast_2d(c))
    q = _c64(np.atleast_2d(q))
    H = _c64(H)
    nm = nmono(d, deg)
    out = np.zeros((q.shape[0], c.shape[0], nm))
    if cutoff:
        rc = lib().or_moment_sums_cutoff(d, n, _dp(x), c.shape[0], _dp(c), _dp(H), deg,
                                         q.shape[0], _dp(q), CUTOFF_R2, _dp(out), nthreads)
    else:
        rc = lib().or_moment_sums(d, n, _dp(x), c.shape[0], _dp(c), _dp(H), deg,
                                  q.shape[0], _dp(q), _dp(out), nthreads)
    if rc != 0:
        raise ValueError(f"oracle moment sums failed ({rc}): H must be SPD, d in 1..3")
    return out


# ---- compact regression kernels (Table 1; Sec. 1 lists uniform, bi-weight,
# tri-weight, Epanechnikov) -------------------------------------------------
# Radial on the unit ball of u = H^(-1/2) z: K(u) = c_d k(|u|^2) for |u| <= 1,
# with c_d making K a density in d dimensions (V_d = unit-ball volume):
#   uniform      k = 1                 c_d = 1 / V_d
#   epanechnikov k = 1 - r^2           c_d = (d + 2) / (2 V_d)
#   triangle     k = 1 - r             c_d = (d + 1) / V_d
#   biweight     k = (1 - r^2)^2       c_d = (d + 2)(d + 4) / (8 V_d)
#   triweight    k = (1 - r^2)^3       c_d = (d + 2)(d + 4)(d + 6) / (48 V_d)
# and K_H(z) = |H|^(-1/2) K(H^(-1/2) z).
COMPACT_KERNELS = ("uniform", "epanechnikov", "triangle", "biweight", "triweight")


def compact_profile(name: str, d: int, r2: np.ndarray) -> np.ndarray:
    """c_d k(r^2) on |u| <= 1, 0 outside."""
    vd = {1: 2.0, 2: math.pi, 3: 4.0 * math.pi / 3.0}[d]
    r2 = np.asarray(r2, dtype=np.float64)
    inside = r2 <= 1.0
    if name == "uniform":
        k, c = np.ones_like(r2), 1.0 / vd
    elif name == "epanechnikov":
        k, c = 1.0 - r2, (d + 2) / (2.0 * vd)
    elif name == "triangle":
        k, c = 1.0 - np.sqrt(np.clip(r2, 0.0, None)), (d + 1) / vd
    elif name == "biweight":
        k, c = (1.0 - r2) ** 2, (d + 2) * (d + 4) / (8.0 * vd)
    elif name == "triweight":
        k, c = (1.0 - r2) ** 3, (d + 2) * (d + 4) * (d + 6) / (48.0 * vd)
    else:
        raise ValueError(name)
    return np.where(inside, c * k, 0.0)


def moment_sums_compact(x: np.ndarray, c: np.ndarray, H: np.ndarray, deg: int,
                        q: np.ndarray, kernel: str) -> np.ndarray:
    """Eq. 9 sums with a compact kernel, [nq, nstr, nmono(d, deg)] (direct, loops over q)."""
    x = _c64(x)
    n, d = x.shape
    c = _c64(np.atleast_2d(c))
    q = _c64(np.atleast_2d(q))
    H = _c64(H).reshape(d, d)
    Hinv = np.linalg.inv(H)
    scale = 1.0 / math.sqrt(np.linalg.det(H))
    ex = monomials(d, deg)
    out = np.zeros((q.shape[0], c.shape[0], ex.shape[0]))
    for k, qq in enumerate(q):
        z = x - qq
        r2 = np.einsum("ni,ij,nj->n", z, Hinv, z)
        wgt = scale * compact_profile(kernel, d, r2)
        mono = np.prod(z[:, None, :] ** ex[None, :, :], axis=2)      # [n, nm]
        out[k] = (c * wgt[None, :]) @ mono
    return out


def smooth_at_compact(x: np.ndarray, y: np.ndarray, H: np.ndarray, order: int,
                      q: np.ndarray, kernel: str) -> dict:
    """Local-polynomial estimate with a compact kernel (eqs. 3, 9), same outputs as smooth_at."""
    x = _c64(x)
    y = _c64(np.atleast_2d(y))
    d = x.shape[1]
    s = moment_sums_compact(x, np.ones((1, x.shape[0])), H, 2 * order, q, kernel)[:, 0, :]
    t = moment_sums_compact(x, y, H, order, q, kernel)
    mh, si = lpr_solve(d, order, s, t)
    return {"mhat": mh, "s": s, "t": t, "sinv11": si}


def lpr_solve(d: int, order: int, s: np.ndarray, t: np.ndarray):
    """mhat = e_1^T S^-1 t and [S^-1]_11 from moment sums (eqs. 3, 11).

    ``s`` [nq, nmono(d, 2 order)], ``t`` [nq, nrhs, nmono(d, order)].
    Returns (mhat [nq, nrhs], sinv11 [nq]).
    """
    s = _c64(s)
    t = _c64(t)
    nq = s.shape[0]
    nrhs = t.shape[1]
    mh = np.zeros((nq, nrhs))
    si = np.zeros(nq)
    lib().or_lpr_solve(d, order, nq, _dp(s), nrhs, _dp(t), _dp(mh), _dp(si))
    return mh, si


def smooth_at(x: np.ndarray, y: np.ndarray, H: np.ndarray, order: int,
              q: np.ndarray, nthreads: int = 0, cutoff: bool = False):
    """Local-polynomial estimate at query points q.

    Returns a dict with ``mhat`` [nq, nrhs], ``s`` [nq, ns] (s-fields),
    ``t`` [nq, nrhs, nt] (t-fields) and ``sinv11`` [nq].  ``cutoff`` as in
    ``moment_sums``.
    """
    x = _c64(x)
    d = x.shape[1]
    y = _c64(np.atleast_2d(y))
    nrhs = y.shape[0]
    ones = np.ones((1, x.shape[0]))
    s = moment_sums(x, ones, H, 2 * order, q, nthreads, cutoff)[:, 0, :]
    t = moment_sums(x, y, H, order, q, nthreads, cutoff)
    mh, si = lpr_solve(d, order, s, t)
    return {"mhat": mh, "s": s, "t": t, "sinv11": si}


def scale_field(x: np.ndarray, c: np.ndarray, H: np.ndarray, q: np.ndarray,
                nthreads: int = 0, cutoff: bool = False) -> np.ndarray:
    """a(q) = sum_i K_H(x_i - q) |c_i| : the natural size of a moment field."""
    return moment_sums(x, np.abs(np.atleast_2d(c)), H, 0, q, nthreads, cutoff)[:, :, 0]


def smoother_diag(x: np.ndarray, H: np.ndarray, order: int, idx=None,
                  nthreads: int = 0) -> np.ndarray:
    """S_ii for i in idx (all samples by default).

    With the smoother matrix of eq. 3 evaluated at q = x_i, row i is
    e_1^T S(x_i)^-1 D^T W and its i-th entry is K_H(0) [S(x_i)^-1]_11,
    because the i-th design row at q = x_i is e_1 (d(0) = (1, 0, ...)).
    """
    x = _c64(x)
    d = x.shape[1]
    q = x if idx is None else x[np.asarray(idx)]
    r = smooth_at(x, np.zeros((1, x.shape[0])), H, order, q, nthreads)
    return kernel(H, np.zeros(d)) * r["sinv11"]


def trace_exact(x: np.ndarray, H: np.ndarray, order: int, nthreads: int = 0) -> float:
    """tr(S_h) = sum_i S_ii (the DF in eq. 22)."""
    return float(np.sum(smoother_diag(x, H, order, None, nthreads)))


def apply_smoother(x: np.ndarray, v: np.ndarray, H: np.ndarray, order: int,
                   idx=None, nthreads: int = 0) -> np.ndarray:
    """(S_h v)_i at samples i in idx: the estimate of eq. 3 at q = x_i.

    ``v`` is [nrhs, n]; returns [len(idx), nrhs].
    """
    x = _c64(x)
    q = x if idx is None else x[np.asarray(idx)]
    return smooth_at(x, v, H, order, q, nthreads)["mhat"]


def fmc_trace(x: np.ndarray, w: np.ndarray, H: np.ndarray, order: int,
              Sw: Optional[np.ndarray] = None, nthreads: int = 0):
    """Fast Monte-Carlo DF (Sec. 2.1) with given probes w [np, n].

    Step iii: (1/N) tr(I - S) ~ mean_p w_p^T (w_p - S w_p) / (w_p^T w_p),
    hence tr(S) ~ N mean_p (w_p^T S w_p) / (w_p^T w_p)   (Girard).
    Also returns the Hutchinson estimate mean_p w_p^T S w_p and the per-probe
    numerators.
    """
    w = _c64(np.atleast_2d(w))
    n = w.shape[1]
    if Sw is None:
        Sw = apply_smoother(x, w, H, order, None, nthreads).T   # [np, n]
    num = np.sum(w * Sw, axis=1)
    den = np.sum(w * w, axis=1)
    return {"girard": float(n * np.mean(num / den)), "hutchinson": float(np.mean(num)),
            "wSw": num, "ww": den}


def gcv(rss: float, n: int, tr: float) -> float:
    """Eq. 22: (RSS / N) / (tr(I - S) / N)^2."""
    return (rss / n) / ((1.0 - tr / n) ** 2)


def estimate_vjp(x: np.ndarray, Y: np.ndarray, sigma, order: int, q: np.ndarray,
                 gbar: np.ndarray, q_is_x: bool = False) -> dict:
    """Analytic gradient of L = sum_q sum_v gbar[v, q] mhat_v(q) (eqs. 3, 9, 11).

    Y [V, n] responses, H = diag(sigma^2), q [nq, d] query points, gbar [V, nq].
    With z_j = x_j - q, K_j = K_H(z_j) and a = S^-1 e_1, beta_v = S^-1 t_v:
      dL/dt_(v,a) = gbar_v a_a,  dL/ds_g = -sum_(a+b = g) a_a sum_v gbar_v beta_(v,b),
    so each source j carries the weight function
      phi_j(z) = K_H(z) P_j(z),  P_j(z) = sum_g sbar_g z^g + sum_v Y_(v,j) sum_a tbar_(v,a) z^a,
    and
      dL/dY_(v,j)     = K_j sum_a tbar_(v,a) z_j^a
      dL/dx_j         = grad phi_j(z_j) = K_j (grad P_j(z_j) - P_j(z_j) H^-1 z_j)
      dL/dlog sigma_k = sum_j phi_j(z_j) (z_(j,k)^2 / sigma_k^2 - 1)
    (dK_H/dlog sigma_k = K_H (z_k^2 / sigma_k^2 - 1) for a diagonal H).  With
    q_is_x the query points are the samples themselves and also move with
    x: dL/dq_i = -sum_j grad phi_j(z_j) is added to dL/dx_i.  Query points whose
    system is singular contribute nothing.  Pure numpy, a loop over q: small
    inputs only.  Returns dY [V, n], dx [n, d], dlogsigma [d].
    """
    x = _c64(x)
    n, d = x.shape
    Y = _c64(np.atleast_2d(Y))
    V = Y.shape[0]
    q = _c64(np.atleast_2d(q))
    gbar = _c64(np.atleast_2d(gbar))
    sig = np.broadcast_to(np.asarray(sigma, dtype=np.float64), (d,)).copy()
    hinv = 1.0 / sig ** 2
    norm = 1.0 / math.sqrt((2 * math.pi) ** d * np.prod(sig ** 2))
    e2 = monomials(d, 2 * order)
    e1 = monomials(d, order)
    p = e1.shape[0]
    pair = [[[a, b] for a in range(p) for b in range(p)
             if np.array_equal(e1[a] + e1[b], e2[gi])] for gi in range(e2.shape[0])]
    sidx = np.array([[next(gi for gi in range(e2.shape[0]) if np.array_equal(e1[a] + e1[b], e2[gi]))
                      for b in range(p)] for a in range(p)])
    dY = np.zeros_like(Y)
    dx = np.zeros((n, d))
    dls = np.zeros(d)

    def mono(z, ex):
        return np.prod(z[:, None, :] ** ex[None, :, :], axis=2)          # [n, m]

    def dmono(z, ex):                                                     # [n, m, d]
        out = np.zeros((z.shape[0], ex.shape[0], d))
        for k in range(d):
            e = ex.copy()
            c = e[:, k].astype(np.float64)
            e[:, k] = np.maximum(e[:, k] - 1, 0)
            out[:, :, k] = c[None, :] * np.prod(z[:, None, :] ** e[None, :, :], axis=2)
        return out

    for qi, qq in enumerate(q):
        z = x - qq
        K = norm * np.exp(-0.5 * np.sum(z * z * hinv, axis=1))
        m2 = mono(z, e2)
        m1 = m2[:, : p]
        s = K @ m2
        S = s[sidx]
        try:
            Sinv = np.linalg.inv(S)
        except np.linalg.LinAlgError:
            continue
        if not np.all(np.isfinite(Sinv)):
            continue
        a = Sinv[:, 0]
        t = (Y * K[None, :]) @ m1                                        # [V, p]
        beta = t @ Sinv.T                                                 # [V, p]
        g = gbar[:, qi]
        tbar = g[:, None] * a[None, :]                                    # [V, p]
        bbar = g @ beta                                                   # [p]
        sbar = np.array([-sum(a[u] * bbar[v] for u, v in pr) for pr in pair])
        dY += K[None, :] * (tbar @ m1.T)
        P = m2 @ sbar + np.sum(Y * (tbar @ m1.T), axis=0)                 # [n]
        dP = np.einsum("nmk,m->nk", dmono(z, e2), sbar) + \
            np.einsum("vn,nmk,vm->nk", Y, dmono(z, e1), tbar)
        grad = K[:, None] * (dP - P[:, None] * z * hinv[None, :])         # [n, d]
        dx += grad
        if q_is_x:
            dx[qi] -= np.sum(grad, axis=0)
        dls += np.sum((K * P)[:, None] * (z * z * hinv[None, :] - 1.0), axis=0)
    return {"dY": dY, "dx": dx, "dlogsigma": dls}


def gcv_grad(x: np.ndarray, y: np.ndarray, w: np.ndarray, sigma, order: int) -> dict:
    """GCV (eq. 22) with the Girard trace of Sec. 2.1 over fixed probes w [np, n]
    and its analytic gradient with respect to y, x and log sigma_j (H = diag(sigma^2)).

    GCV = (RSS/N) / (1 - tr/N)^2 with RSS = sum_i (y_i - mhat_y(x_i))^2 and
    tr = (N/Np) sum_p w_p^T S w_p / w_p^T w_p.  The adjoints of the at-sample
    estimates are dGCV/dmhat_y(x_i) = -2 L_RSS (y_i - mhat_y(x_i)) and
    dGCV/dmhat_p(x_i) = L_tr (N/Np) w_pi / w_p^T w_p, L_RSS = (1/N)/(1 - tr/N)^2,
    L_tr = 2 (RSS/N) / (N (1 - tr/N)^3); estimate_vjp carries them to the
    parameters (the evaluation points are the samples), plus the explicit
    term 2 L_RSS (y_i - mhat_y(x_i)) of dGCV/dy_i.
    """
    x = _c64(x)
    n, d = x.shape
    y = _c64(y).reshape(-1)
    w = _c64(np.atleast_2d(w))
    npb = w.shape[0]
    H = np.diag(np.broadcast_to(np.asarray(sigma, dtype=np.float64), (d,)) ** 2)
    Y = np.concatenate([y[None], w])
    mh = smooth_at(x, Y, H, order, x)["mhat"].T                          # [1 + np, n]
    r = y - mh[0]
    rss = float(r @ r)
    ww = np.sum(w * w, axis=1)
    tr = n * float(np.mean(np.sum(w * mh[1:], axis=1) / ww))
    den = 1.0 - tr / n
    L_rss = (1.0 / n) / den ** 2
    L_tr = 2.0 * (rss / n) / (n * den ** 3)
    gbar = np.concatenate([(-2.0 * L_rss * r)[None], L_tr * (n / npb) * w / ww[:, None]])
    g = estimate_vjp(x, Y, np.sqrt(np.diag(H)), order, x, gbar, q_is_x=True)
    return {"gcv": (rss / n) / den ** 2, "dy": g["dY"][0] + 2.0 * L_rss * r,
            "dx": g["dx"], "dlogsigma": g["dlogsigma"]}


def variance_pass(x: np.ndarray, y: np.ndarray, mhat_at_x: np.ndarray,
                  H: np.ndarray, q: np.ndarray, order: int = 1, nthreads: int = 0) -> np.ndarray:
    """Eq. 23: sigma^2(q) = local-linear smooth of r_i = |y_i - mhat(x_i)|^2."""
    r = np.abs(np.atleast_2d(y) - np.atleast_2d(mhat_at_x)) ** 2
    return smooth_at(x, r, H, order, q, nthreads)["mhat"]


def log_variance(x: np.ndarray, y: np.ndarray, mhat_at_x: np.ndarray, H: np.ndarray,
                 q: np.ndarray, order: int = 1, nthreads: int = 0) -> dict:
    """Log-variance estimator of Sec. 3 (eqs. 24-26), real responses.

    r_i = (y_i - mhat(x_i))^2; v is the local-polynomial smooth of
    log(r_i + 1/N) (eq. 25), evaluated at the query points q and at the
    samples; kappa = [mean_i r_i exp(-v(x_i))]^-1; sigma^2(q) = exp(v(q)) /
    kappa (eq. 26).  Returns v_grid [nq, nrhs], v_at_x [n, nrhs], kappa [nrhs]
    and sigma2 [nq, nrhs].
    """
    x = _c64(x)
    n = x.shape[0]
    r = (np.atleast_2d(y) - np.atleast_2d(mhat_at_x)) ** 2
    ell = np.log(r + 1.0 / n)
    v_grid = smooth_at(x, ell, H, order, q, nthreads)["mhat"]
    v_x = smooth_at(x, ell, H, order, x, nthreads)["mhat"]
    kappa = 1.0 / np.mean(r.T * np.exp(-v_x), axis=0)
    return {"v_grid": v_grid, "v_at_x": v_x, "kappa": kappa, "sigma2": np.exp(v_grid) / kappa}


def interval(mhat: np.ndarray, var: np.ndarray, alpha: float = 0.05):
    """Pointwise interval of eq. 28: mhat -/+ z_(1 - alpha/2) sqrt(var).

    z is the standard normal quantile (scipy's ppf); var is the variance
    estimate the caller supplies (NaN where it is negative or not finite).
    """
    from scipy.stats import norm
    z = norm.ppf(1.0 - 0.5 * alpha)
    v = np.asarray(var, dtype=np.float64)
    sd = np.where(v >= 0, np.sqrt(np.where(v >= 0, v, 0.0)), np.nan)
    m = np.asarray(mhat, dtype=np.float64)
    return m - z * sd, m + z * sd


def _keys_weights(t: float, a: float = -0.5):
    """Cubic-convolution weights (Keys 1981) of the taps -1, 0, 1, 2 at offset t in [0, 1]."""
    def w(s):
        s = abs(s)
        if s <= 1:
            return (a + 2) * s ** 3 - (a + 3) * s ** 2 + 1
        if s < 2:
            return a * s ** 3 - 5 * a * s ** 2 + 8 * a * s - 4 * a
        return 0.0
    return [w(t + 1), w(t), w(1 - t), w(2 - t)]


def predict(grid_vals: np.ndarray, grid_n: Sequence[int], lo: Sequence[float],
            hi: Sequence[float], xq: np.ndarray, method: str = "linear") -> np.ndarray:
    """Values of a grid estimate at new points (the griddedInterpolant step of Sec. 1.1).

    grid_vals [count, M] on the eq. 6 lattice (last axis fastest); xq [nq, d].
    ``linear``: multilinear inside the box, extended linearly from the
    boundary cell outside.  ``cubic``: separable cubic convolution (Keys 1981,
    a = -1/2) with Keys' boundary rows f[-1] = 3f[0] - 3f[1] + f[2] (and the
    mirror at the top); NaN outside the box.  Returns [count, nq].
    Pure-Python loops: small cases only.
    """
    g = np.asarray(grid_vals, dtype=np.float64).reshape((-1,) + tuple(grid_n))
    xq = np.atleast_2d(np.asarray(xq, dtype=np.float64))
    d = xq.shape[1]
    out = np.empty((g.shape[0], xq.shape[0]))
    for qi, x in enumerate(xq):
        taps = []
        bad = False
        for j in range(d):
            M = grid_n[j]
            delta = (hi[j] - lo[j]) / (M - 1)
            u = (x[j] - lo[j]) / delta
            i = int(min(max(math.floor(u), 0), M - 2))
            t = u - i
            if method == "linear":
                taps.append([(i, 1 - t), (i + 1, t)])
            else:
                if u < 0 or u > M - 1:
                    bad = True
                ws = _keys_weights(min(max(t, 0.0), 1.0))
                taps.append([(i - 1 + k, ws[k]) for k in range(4)])
        if bad:
            out[:, qi] = np.nan
            continue
        val = np.zeros(g.shape[0])
        for combo in itertools.product(*taps):
            wgt = 1.0
            idx = []
            for j, (ii, wj) in enumerate(combo):
                wgt *= wj
                idx.append(ii)
            val += wgt * _grid_at(g, idx, grid_n)
        out[:, qi] = val
    return out


def _grid_at(g: np.ndarray, idx, grid_n) -> np.ndarray:
    """Grid values at a multi-index, with Keys' boundary rows at -1 and M."""
    for j, ii in enumerate(idx):
        M = grid_n[j]
        if ii == -1 or ii == M:
            sgn = 1 if ii == -1 else -1
            base = 0 if ii == -1 else M - 1
            parts = []
            for c, off in ((3, 0), (-3, 1), (1, 2)):
                jj = list(idx)
                jj[j] = base + sgn * off
                parts.append(c * _grid_at(g, jj, grid_n))
            return parts[0] + parts[1] + parts[2]
    return g[(slice(None),) + tuple(idx)]


def get_hlist(n: int, lo: float, hi: float, spacing: str = "log") -> np.ndarray:
    """Bandwidth candidates of Sec. 4 (get_hList): n values from lo to hi.

    ``log`` spacing is 10**linspace(log10 lo, log10 hi, n) (MATLAB logspace),
    ``lin`` is linspace(lo, hi, n).
    """
    if spacing == "log":
        return 10.0 ** np.linspace(math.log10(lo), math.log10(hi), n)
    return np.linspace(lo, hi, n)


def select_h(gcv_values: Sequence[float], dstd: float = 0.0) -> int:
    """Index of the selected bandwidth (Table 1, ``dstd``).

    Reading of the garbled rule: take the largest candidate (candidates in
    increasing order) whose GCV is within dstd * std(GCV) of the minimum;
    dstd = 0 is the plain argmin, ties resolved toward the larger bandwidth.
    """
    g = np.asarray(gcv_values, dtype=np.float64)
    thr = np.nanmin(g) + dstd * (np.nanstd(g) if dstd else 0.0)
    ok = np.where(g <= thr)[0]
    return int(ok.max())


def probes(seed: int, n_probes: int, n: int, precision: str = "f64") -> np.ndarray:
    """Counter-based Gaussian probes [n_probes, n] (SplitMix64 + Box-Muller).

    ``precision="f32"`` evaluates the single-precision variant (24-bit
    uniforms, float arithmetic) and returns float32 values.
    """
    if precision == "f32":
        out32 = np.zeros((n_probes, n), dtype=np.float32)
        lib().or_probes_f32(ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), n_probes, n,
                            out32.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
        return out32
    out = np.zeros((n_probes, n))
    lib().or_probes(ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), n_probes, n, _dp(out))
    return out


def splitmix64(z: int) -> int:
    return int(lib().or_splitmix64(ctypes.c_uint64(z & 0xFFFFFFFFFFFFFFFF)))
