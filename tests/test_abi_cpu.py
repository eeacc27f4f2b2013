"""CPU-side checks of the C-ABI library: it loads, exports every declared
symbol, validates arguments, and its host planner is right.  No GPU needed."""
import ctypes
import math
import glob
import os
import re

import numpy as np
import pytest
from scipy import integrate

from paper_2204_07716_gb300 import build as fkbuild
from paper_2204_07716_gb300 import fkreg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    fkbuild.build()
    return fkreg.load()


def declared_symbols():
    names = set()
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(fkreg_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(fkreg.EXPORTS)


def test_checked_library_exports_the_same_symbols(lib):
    # the range-checked variant: same sources with FKREG_CHECKED, same ABI
    path = fkbuild.build(checked=True)
    chk = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(chk, name), name
    chk.fkreg_checked_build.restype = ctypes.c_int
    lib.fkreg_checked_build.restype = ctypes.c_int
    assert chk.fkreg_checked_build() == 1 and lib.fkreg_checked_build() == 0


def opts(**kw):
    base = dict(d=2, order=1, grid_n=(256, 256), lo=(0, 0), hi=(1, 1),
                H=np.diag([0.01 ** 2, 0.015 ** 2]), tol=1e-6)
    base.update(kw)
    return base


def test_geometry_covers_tail_and_spectrum(lib):
    g = fkreg.geometry(**opts())
    assert g["w"] == 7 and g["ns"] == 6 and g["nt"] == 3
    for j, sig in enumerate((0.01, 0.015)):
        delta = 1 / 255
        assert g["delta"][j] == pytest.approx(delta)
        # period covers the box plus the kernel tail (no wrap into the box)
        assert g["period"][j] >= 1.0 + 5.5 * sig
        assert g["period"][j] == pytest.approx(g["ldft"][j] * delta)
        # kept modes resolve the Gaussian multiplier to below tol
        kmax = g["modes"][j] // 2 - 1
        xi = kmax / g["period"][j]
        assert math.exp(-2 * math.pi ** 2 * sig ** 2 * xi ** 2) < 1e-6
        assert g["nf"][j] >= 2 * g["modes"][j] and g["nf"][j] % 2 == 0
        assert g["inv_h"][j] == pytest.approx(g["nf"][j] / g["period"][j], rel=1e-7)


@pytest.mark.parametrize("d,tol,order", [(d, t, o) for d in (1, 2, 3) for t in (1e-6, 1e-9, 1e-12)
                                          for o in (0, 1, 2) if not (d == 3 and o == 2)])
def test_geometry_invariants_across_configurations(lib, d, tol, order):
    # for every accepted plan: the period leaves room for the Gaussian tail to
    # fall below tol before it wraps into the box (exp(-r^2/2) < tol), the
    # largest kept mode's Gaussian multiplier is below tol, the fine grid is
    # oversampled by at least 2, the ES width follows tol, and a fine grid
    # beyond the size limit is refused as UNSUPPORTED, not planned
    need = math.sqrt(2 * math.log(1 / tol))
    for sig in (0.002, 0.005, 0.01, 0.03, 0.1, 0.3):
        for grid in (64, 256):
            kw = dict(d=d, order=order, grid_n=(grid,) * d, lo=(0.0,) * d, hi=(1.0,) * d,
                      H=np.eye(d) * sig * sig, tol=tol, precision="f64" if tol < 1e-7 else "f32")
            try:
                g = fkreg.geometry(**kw)
            except fkreg.FkregError as e:
                assert "UNSUPPORTED" in str(e) and d == 3 and sig < 0.005, (kw, e)
                continue
            assert g["w"] == math.ceil(math.log10(1 / tol)) + 1
            for j in range(d):
                P, K, nf = g["period"][j], g["modes"][j], g["nf"][j]
                assert (P - 1.0) / sig >= need, (kw, j, P)
                assert P == pytest.approx(g["ldft"][j] / (grid - 1))
                xi = (K // 2 - 1) / P
                assert math.exp(-2 * math.pi ** 2 * sig ** 2 * xi ** 2) < tol, (kw, j, K)
                assert nf >= 2 * K and nf % 2 == 0
                assert g["inv_h"][j] == pytest.approx(nf / P, rel=1e-7)


def test_direct_geometry_for_compact_kernels(lib):
    # compact kernels: bins on the output lattice (n_f = M), cells of the
    # grid spacing, a quarter of the widest support half-width per bin
    for sig, grid in ((0.01, 256), (0.08, 64), (0.3, 40)):
        g = fkreg.geometry(**opts(grid_n=(grid, grid), H=np.diag([sig ** 2, (1.5 * sig) ** 2]),
                                  kernel="epanechnikov"))
        for j in range(2):
            delta = 1.0 / (grid - 1)
            assert g["nf"][j] == grid
            assert g["inv_h"][j] == pytest.approx((grid - 1), rel=1e-7)
            rmax = 1.5 * sig / delta if j == 1 else sig / delta
            want = max(1, min(64, math.ceil(0.25 * rmax)))
            assert g["tile"][j] == min(want, grid)
            assert g["nbins"][j] == -(-grid // g["tile"][j])


def test_width_follows_tolerance(lib):
    for tol, w in ((1e-6, 7), (1e-9, 10), (1e-12, 13), (1e-3, 4)):
        assert fkreg.geometry(**opts(tol=tol))["w"] == w
    assert fkreg.geometry(**opts(tol=1e-6, spread_kernel="gauss"))["w"] == 14


def test_invalid_arguments_are_reported(lib):
    with pytest.raises(fkreg.FkregError, match="INVALID_ARG"):
        fkreg.geometry(**opts(H=np.array([[1.0, 2.0], [2.0, 1.0]]) * 1e-4))   # not SPD
    with pytest.raises(fkreg.FkregError, match="INVALID_ARG"):
        fkreg.geometry(**opts(order=3))
    with pytest.raises(fkreg.FkregError, match="INVALID_ARG"):
        fkreg.geometry(**opts(grid_n=(1, 256)))
    with pytest.raises(fkreg.FkregError, match="INVALID_ARG"):
        fkreg.geometry(**opts(tol=0.5))
    # the interval refuses alpha outside (0, 1) and bad precisions before any launch
    L = fkreg.load()
    for prec, alpha in ((0, 0.0), (0, 1.0), (1, -0.1), (7, 0.05)):
        assert L.fkreg_interval(prec, 4, None, None, alpha, None, None, None) == 1
    # prediction: bad method, dimension or grid sizes are refused before any launch
    gn = (ctypes.c_int64 * 2)(3, 3)
    lo2, hi2 = (ctypes.c_double * 2)(0, 0), (ctypes.c_double * 2)(1, 1)
    assert L.fkreg_predict(0, 2, gn, lo2, hi2, 1, None, 5, None, 2, None, None) == 1   # method
    assert L.fkreg_predict(0, 4, gn, lo2, hi2, 1, None, 5, None, 0, None, None) == 1   # dim
    assert L.fkreg_predict(0, 2, gn, lo2, hi2, 1, None, 5, None, 1, None, None) == 1   # cubic, M < 4
    assert L.fkreg_predict(0, 2, gn, lo2, hi2, 1, None, 0, None, 0, None, None) == 0   # nothing to do


@pytest.mark.parametrize("kind", ["es", "gauss"])
def test_spread_kernel_transform_matches_adaptive_quadrature(lib, kind):
    w = 7 if kind == "es" else 14
    beta = 2.30 * w if kind == "es" else 3 * math.pi / (4 * (w // 2))
    nf = 96
    ph = fkreg.spread_kernel_ft(kind, w, beta, nf, 24)

    def phi(z):
        if kind == "es":
            t = 2 * z / w
            return math.exp(beta * (math.sqrt(max(0.0, 1 - t * t)) - 1)) if abs(t) <= 1 else 0.0
        return math.exp(-beta * z * z) if abs(z) <= w / 2 else 0.0

    for k in range(24):
        ref = integrate.quad(lambda z: phi(z) * math.cos(2 * math.pi * k * z / nf), -w / 2, w / 2,
                             limit=400, epsabs=1e-15, epsrel=1e-13)[0]
        assert ph[k] == pytest.approx(ref, rel=1e-10, abs=1e-14)
