"""The device spreading kernel phi (Sec. 1.2) against its definition in FP64.

The FP32 form is built from the hardware reciprocal square root and base-2
exponential (one Newton step on the square root); the FP64 form from the
correctly rounded library functions.  The bound for FP32 follows from the
formula: the rounding of s = sqrt(1 - t^2) near 1 is amplified by beta in the
exponent, so a relative error of a few beta 2^-24 is what any FP32 evaluation
of exp(beta (s - 1)) has.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2204_07716_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def phi_ref(kind, w, beta, z):
    z = np.asarray(z, dtype=np.float64)
    if kind == "es":
        t = z * (2.0 / w)
        a = 1.0 - t * t
        return np.where(a > 0, np.exp(beta * (np.sqrt(np.maximum(a, 0.0)) - 1.0)), 0.0)
    return np.where(np.abs(z) <= 0.5 * w, np.exp(-beta * z * z), 0.0)


@pytest.mark.parametrize("kind,w,beta", [("es", 7, 16.1), ("es", 4, 9.2), ("es", 12, 27.6),
                                         ("es", 16, 36.8), ("gauss", 7, 1.13)])
def test_kernel_values(kind, w, beta):
    from paper_2204_07716_gb300 import fkreg
    rng = np.random.default_rng(w)
    z = np.concatenate([np.linspace(-0.5 * w - 0.5, 0.5 * w + 0.5, 200_001),
                        rng.uniform(-0.5 * w, 0.5 * w, 100_000), [0.0, 0.5 * w, -0.5 * w]])
    # FP64: the definition to rounding
    v64 = fkreg.spread_kernel_values(kind, w, beta, torch.tensor(z, device="cuda")).cpu().numpy()
    ref = phi_ref(kind, w, beta, z)
    # relative where the value is well conditioned in z (|2z/w| <= 0.968:
    # towards the edge the square root amplifies the rounding of z), absolute
    # against the peak value 1 everywhere
    core = np.abs(z) <= 0.484 * w
    np.testing.assert_allclose(v64[core], ref[core], rtol=1e-13, atol=0)
    np.testing.assert_allclose(v64, ref, rtol=0, atol=1e-14)
    # FP32: the same inputs as the device sees them (z and beta in float)
    z32 = z.astype(np.float32)
    b32 = float(np.float32(beta))
    v32 = fkreg.spread_kernel_values(kind, w, beta,
                                     torch.tensor(z32, device="cuda")).cpu().numpy()
    if kind == "es":
        # the device's t = fl(z fl(2 / w)), one IEEE product in float
        t32 = (z32 * np.float32(2.0 / w)).astype(np.float64)
        a = 1.0 - t32 * t32
        ref32 = np.where(a > 0, np.exp(b32 * (np.sqrt(np.maximum(a, 0.0)) - 1.0)), 0.0)
    else:
        ref32 = phi_ref(kind, w, b32, z32.astype(np.float64))
    inside = ref32 > 0
    assert np.all(v32[~inside] == 0)
    # largest magnitude of the exponent over the support
    xmax = b32 if kind == "es" else b32 * 0.25 * w * w
    core = inside & (np.abs(z32) <= 0.484 * w)
    rel = np.abs(v32[core].astype(np.float64) - ref32[core]) / ref32[core]
    assert rel.max() <= 8 * xmax * 2.0 ** -24 + 2.0 ** -20
    assert np.sqrt(np.mean(rel ** 2)) <= 2 * xmax * 2.0 ** -24 + 2.0 ** -22
    # absolute error against the peak value 1
    assert np.max(np.abs(v32.astype(np.float64) - ref32)) <= 2 * b32 * 2.0 ** -24 + 2.0 ** -22


def test_kernel_values_arguments():
    from paper_2204_07716_gb300 import fkreg
    with pytest.raises(fkreg.FkregError):
        fkreg.spread_kernel_values("es", 7, 16.1, torch.zeros(4, dtype=torch.int32, device="cuda"))
    L = fkreg.load()
    assert L.fkreg_spread_kernel_values(0, 1, 1.0, 0, 4, None, None, None) == 1
    assert L.fkreg_spread_kernel_values(0, 7, 1.0, 5, 4, None, None, None) == 1
    assert L.fkreg_spread_kernel_values(0, 7, 1.0, 0, 0, None, None, None) == 0
