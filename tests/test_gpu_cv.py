"""cv_fkreg (Sec. 4's one-call bandwidth selection) on the GPU.

float32 samples standardised on the device: every sample stays inside the
grid box in its own precision (the device flags one outside as an error),
and the chosen candidate's GCV and grid estimate agree with the same plan
run on the standardised samples by hand, and its GCV with the oracle's
(eq. 22) computed from the device's own trace.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2204_07716_gb300 import build
    build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


@pytest.mark.parametrize("d", [1, 2])
def test_cv_fkreg_float32_standardised(d):
    from paper_2204_07716_gb300 import fkreg
    rng = np.random.default_rng(31 + d)
    n = 20_000
    x = torch.tensor(rng.random((n, d)) * 20.0 + 3.0, dtype=torch.float32, device="cuda")
    y = torch.sin(x.sum(dim=1) / 4) + 0.1 * torch.randn(n, device="cuda")
    hl = fkreg.bandwidth_list(5, [(0.03, 0.3)] * d)
    r = fkreg.cv_fkreg(x if d > 1 else x[:, 0], y, hl, 48, order=1, standardize=True)
    p = r["plan"]
    p.sync()                        # no sample flagged outside the box
    def host(v):
        return torch.as_tensor(v).detach().double().cpu().numpy()
    gcv = host(r["gcv"]).reshape(-1)
    assert np.all(np.isfinite(gcv))
    k = int(r["index"])
    # GCV (eq. 22) from the device's RSS and Girard trace
    tr = host(r["trace"]).reshape(-1, 3)
    mh = host(r["mhat_at_x"])[0]
    rss = float(np.sum((y.double().cpu().numpy() - mh) ** 2))
    assert gcv[k] == pytest.approx(oracle.gcv(rss, n, tr[k, 0]), rel=1e-4)
    assert torch.isfinite(r["mhat_grid"]).any()
