"""Seeded synthetic workloads shaped like the paper's simulations.

This module only draws random inputs (sample locations, responses, probe
vectors and bandwidth lists).  It holds none of the smoother's arithmetic, so
the CUDA path and the FP64 oracle can both be fed from it without sharing any
of the method's code.

Every workload uses numpy's PCG64 generator seeded with
``220407716 + index`` (index = 1..5 for the five workload families below), so
the same call returns the same bytes on every machine.

Workload families (model of eq. 1, y = m(x) + sigma(x) * eps):

* ``nw1d``   1-D, x ~ U[0,1], y = sin(2 pi x) + 0.3 N(0,1), sigma_h = 0.02,
             256 grid points, Nadaraya-Watson (eqs. 7, 10), FP64, tol 1e-9.
* ``ll2d``   2-D, x from an equal mixture of three Gaussians (means
             (0.3,0.3), (0.7,0.4), (0.5,0.75), sd 0.1) clipped to [0,1]^2,
             y = sin(4 x1) cos(3 x2) + (0.1 + 0.2 x1) N(0,1),
             H = diag(0.01^2, 0.015^2), 256x256 grid, local linear (eq. 3).
* ``nw3d_df`` 3-D, x ~ U[0,1]^3, y = exp(-|x-0.5|^2/0.05) + 0.2 N(0,1),
             64^3 grid, NW, 32 Gaussian probes (Sec. 2.1), 16 isotropic
             bandwidths log-spaced 0.01..0.1.
* ``ll2d_gcv`` 2-D, x ~ U[0,1]^2, y = x1^2 - x2 + 0.5 sin(8 x1 x2) + 0.1 N,
             512^2 grid, local linear, H = diag(0.01^2, 0.015^2), 10 probes.
* ``uneven`` 64 independent problems (d in {1,2}), complex responses
             y = exp(i phi(f)) / (1 + f) + 0.05 (N + i N) with f the frequency
             in [0.4, 19.2] rescaled to [0,1], as in the EEG spectra of
             Sec. 4.4; N log-uniform in [1e3, 1e6], grids 128..1024 per axis.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

SEED_BASE = 220407716


@dataclasses.dataclass
class Workload:
    """One smoothing problem: samples, responses, grid and bandwidths."""

    name: str
    d: int
    x: np.ndarray            # [N, d] float64, inside the grid box
    y: np.ndarray            # [R, N] float64 (or complex128)
    grid_n: tuple            # points per axis, endpoints included (eq. 6)
    lo: tuple
    hi: tuple
    H: np.ndarray            # [n_bw, d, d] bandwidth matrices (SPD)
    order: int               # 0 = Nadaraya-Watson, 1 = local linear
    tol: float               # NUFFT tolerance
    precision: str           # "f32" or "f64"
    n_probes: int = 0
    probes: Optional[np.ndarray] = None   # [n_probes, N] float64 or None

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_bw(self) -> int:
        return int(self.H.shape[0])


def _rng(index: int, salt: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + index + 1000003 * salt))


def iso_bandwidths(sigmas, d: int) -> np.ndarray:
    """H = sigma^2 I for each per-axis standard deviation sigma."""
    s = np.asarray(sigmas, dtype=np.float64).reshape(-1)
    return np.stack([np.eye(d) * v * v for v in s])


def diag_bandwidth(sigmas) -> np.ndarray:
    s = np.asarray(sigmas, dtype=np.float64)
    return np.diag(s * s)[None]


def gaussian_probes(n_probes: int, n: int, seed: int) -> np.ndarray:
    """i.i.d. N(0,1) probe vectors w_p (Sec. 2.1 step i), [n_probes, n]."""
    g = np.random.Generator(np.random.PCG64(seed))
    return g.standard_normal((n_probes, n))


def nw1d(n: int = 10_000, grid: int = 256, sigma: float = 0.02,
         tol: float = 1e-9, precision: str = "f64") -> Workload:
    g = _rng(1)
    x = g.random((n, 1))
    y = np.sin(2 * np.pi * x[:, 0]) + 0.3 * g.standard_normal(n)
    return Workload("nw1d", 1, x, y[None], (grid,), (0.0,), (1.0,),
                    iso_bandwidths([sigma], 1), 0, tol, precision)


def ll2d(n: int = 1_000_000, grid: int = 256, sigmas=(0.01, 0.015),
         tol: float = 1e-6, precision: str = "f32", n_probes: int = 0) -> Workload:
    g = _rng(2)
    means = np.array([[0.3, 0.3], [0.7, 0.4], [0.5, 0.75]])
    comp = g.integers(0, 3, size=n)
    x = means[comp] + 0.1 * g.standard_normal((n, 2))
    x = np.clip(x, 0.0, 1.0)
    y = np.sin(4 * x[:, 0]) * np.cos(3 * x[:, 1]) + (0.1 + 0.2 * x[:, 0]) * g.standard_normal(n)
    w = Workload("ll2d", 2, x, y[None], (grid, grid), (0.0, 0.0), (1.0, 1.0),
                 diag_bandwidth(sigmas), 1, tol, precision, n_probes)
    if n_probes:
        w.probes = gaussian_probes(n_probes, n, SEED_BASE + 20)
    return w


def nw3d_df(n: int = 4_000_000, grid: int = 64, n_bw: int = 16,
            smin: float = 0.01, smax: float = 0.1, n_probes: int = 32,
            tol: float = 1e-6, precision: str = "f32") -> Workload:
    g = _rng(3)
    x = g.random((n, 3))
    r2 = np.sum((x - 0.5) ** 2, axis=1)
    y = np.exp(-r2 / 0.05) + 0.2 * g.standard_normal(n)
    sig = np.logspace(math.log10(smin), math.log10(smax), n_bw)
    w = Workload("nw3d_df", 3, x, y[None], (grid,) * 3, (0.0,) * 3, (1.0,) * 3,
                 iso_bandwidths(sig, 3), 0, tol, precision, n_probes)
    if n_probes:
        w.probes = gaussian_probes(n_probes, n, SEED_BASE + 30)
    return w


def ll2d_gcv(n: int = 2_000_000, grid: int = 512, sigmas=(0.01, 0.015),
             n_probes: int = 10, tol: float = 1e-6, precision: str = "f32") -> Workload:
    g = _rng(4)
    x = g.random((n, 2))
    y = (x[:, 0] ** 2 - x[:, 1] + 0.5 * np.sin(8 * x[:, 0] * x[:, 1])
         + 0.1 * g.standard_normal(n))
    w = Workload("ll2d_gcv", 2, x, y[None], (grid, grid), (0.0, 0.0), (1.0, 1.0),
                 diag_bandwidth(sigmas), 1, tol, precision, n_probes)
    if n_probes:
        w.probes = gaussian_probes(n_probes, n, SEED_BASE + 40)
    return w


def _smooth_phase(g: np.random.Generator):
    a = g.standard_normal(3) / np.arange(1, 4)
    b = g.random(3) * 2 * np.pi
    return lambda f: sum(a[k] * np.sin(2 * np.pi * (k + 1) * (f - 0.4) / 18.8 + b[k])
                         for k in range(3))


def uneven(n_problems: int = 64, nmin: float = 1e3, nmax: float = 1e6,
           gmin: int = 128, gmax: int = 1024, tol: float = 1e-6,
           scale: float = 1.0) -> List[Workload]:
    """Independent complex-valued LL problems of uneven size.

    ``scale`` multiplies every N (tests use a small scale).  The bandwidth per
    axis is max(1.06 std(x_j) N^(-1/(d+4)), 2.5 Delta_j) on the [0,1] scale.
    """
    g = _rng(5)
    out = []
    for p in range(n_problems):
        d = int(g.integers(1, 3))
        n = max(8, int(round(math.exp(g.uniform(math.log(nmin), math.log(nmax))) * scale)))
        gn = tuple(int(round(math.exp(g.uniform(math.log(gmin), math.log(gmax)))))
                   for _ in range(d))
        f = g.uniform(0.4, 19.2, size=n)
        x = np.empty((n, d))
        x[:, 0] = (f - 0.4) / 18.8
        if d == 2:
            x[:, 1] = g.random(n)
        phi = _smooth_phase(g)
        y = np.exp(1j * phi(f)) / (1 + f) + 0.05 * (g.standard_normal(n) + 1j * g.standard_normal(n))
        sig = []
        for j in range(d):
            delta = 1.0 / (gn[j] - 1)
            sig.append(max(1.06 * float(np.std(x[:, j])) * n ** (-1.0 / (d + 4)), 2.5 * delta))
        out.append(Workload(f"uneven{p}", d, x, y[None], gn, (0.0,) * d, (1.0,) * d,
                            diag_bandwidth(sig), 1, tol, "f32"))
    return out


def complex_log2d(n: int = 2500, grid: int = 24, sigma: float = 0.2) -> Workload:
    """Complex-location regression of Sec. 4.4: points z = x1 + i x2 with
    x1 ~ U[0.1, 2.1], x2 ~ U[-2, 2], complex responses log z plus noise of
    a tenth of the real and imaginary parts' spreads.  x holds (Re z, Im z);
    y[0] is the complex response."""
    g = _rng(6)
    x = np.column_stack([2.0 * g.random(n) + 0.1, 4.0 * g.random(n) - 2.0])
    z = x[:, 0] + 1j * x[:, 1]
    y = np.log(z)
    y = (y + 0.1 * np.std(y.real) * g.standard_normal(n)
         + 0.1j * np.std(y.imag) * g.standard_normal(n))
    return Workload("complex_log2d", 2, x, y[None], (grid, grid), (0.1, -2.0), (2.1, 2.0),
                    iso_bandwidths([sigma], 2), 1, 1e-12, "f64", 0)


def random_small(seed: int, d: int, n: int, grid, order: int, sigmas,
                 precision: str = "f64", tol: float = 1e-12, n_rhs: int = 1,
                 n_probes: int = 0, full_h: bool = False) -> Workload:
    """Small random problem for parity sweeps (x ~ U[0,1]^d, smooth y + noise).

    With ``full_h`` the bandwidth matrix gets a random off-diagonal correlation.
    """
    g = np.random.Generator(np.random.PCG64(SEED_BASE + 100 + seed))
    x = g.random((n, d))
    ys = []
    for r in range(n_rhs):
        ys.append(np.cos(3 * x.sum(axis=1) + r) + 0.2 * g.standard_normal(n))
    grid = tuple(grid) if hasattr(grid, "__len__") else (grid,) * d
    sig = np.asarray(sigmas, dtype=np.float64).reshape(-1)
    Hs = []
    for s in sig:
        H = np.eye(d) * s * s
        if full_h and d > 1:
            rho = 0.35
            for a in range(d):
                for b in range(d):
                    if a != b:
                        H[a, b] = rho * s * s
        Hs.append(H)
    w = Workload(f"small{seed}", d, x, np.stack(ys), grid, (0.0,) * d, (1.0,) * d,
                 np.stack(Hs), order, tol, precision, n_probes)
    if n_probes:
        w.probes = gaussian_probes(n_probes, n, SEED_BASE + 200 + seed)
    return w
