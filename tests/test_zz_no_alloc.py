"""GPU test of the allocation-free bin sort (fkreg_bin_sort_static).

Callers that cannot allocate device memory while they run (a memory pool
that owns the whole device, a plug-in without an allocator) use this entry
point; its scratch is an array the library owns.  Its permutation and bin
offsets must equal numpy's stable argsort of the bin rule's keys (computed on
the CPU) and those of the workspace-based sort (fkreg_set_points +
fkreg_get_sort) bit for bit, on consecutive calls that reuse the array.
"""
import ctypes

import numpy as np
import pytest

from paper_2204_07716_gb300 import fkreg, inputs
from test_gpu_parity import cpu_keys

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_N = 1 << 18


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2204_07716_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def geometry_struct(w):
    o, keep = fkreg.make_opts(w.d, w.order, w.grid_n, w.lo, w.hi, w.H, tol=w.tol,
                              precision=w.precision)
    g = fkreg.Geometry()
    assert fkreg.load().fkreg_geometry_query(ctypes.byref(o), ctypes.byref(g)) == 0
    return g


def static_sort(w, x):
    L = fkreg.load()
    g = geometry_struct(w)
    n = int(x.shape[0])
    nb = int(np.prod(list(g.nbins)[: g.dim]))
    perm = torch.full((max(n, 1),), -1, dtype=torch.int32, device=x.device)
    bstart = torch.full((nb + 1,), -1, dtype=torch.int32, device=x.device)
    bad = torch.full((1,), -7, dtype=torch.int32, device=x.device)
    lo = (ctypes.c_double * 3)(*(list(w.lo) + [0.0] * (3 - w.d)))
    hi = (ctypes.c_double * 3)(*(list(w.hi) + [1.0] * (3 - w.d)))
    prec = fkreg.FKREG_F32 if w.precision == "f32" else fkreg.FKREG_F64
    st = L.fkreg_bin_sort_static(ctypes.byref(g), lo, hi, prec, n, ctypes.c_void_p(x.data_ptr()),
                                 ctypes.c_void_p(perm.data_ptr()), ctypes.c_void_p(bstart.data_ptr()),
                                 ctypes.c_void_p(bad.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, perm[:n].cpu().numpy(), bstart.cpu().numpy(), int(bad.item())


def workspace_sort(w, x):
    p = fkreg.Plan(w.d, w.order, w.grid_n, w.lo, w.hi, w.H, max_n=max(w.n, 1), tol=w.tol,
                   precision=w.precision)
    p.set_points(x)
    perm, bstart = p.get_sort()
    p.sync()
    return perm.cpu().numpy(), bstart.cpu().numpy()


def test_static_sort_equals_workspace_sort_on_consecutive_calls():
    wa = inputs.ll2d(n=200_000)
    wb = inputs.random_small(7, 3, 150_000, 16, 0, [0.05], precision="f64", tol=1e-12)
    xa = torch.tensor(wa.x, dtype=torch.float32, device="cuda")
    xb = torch.tensor(wb.x, dtype=torch.float64, device="cuda")
    ref_a = workspace_sort(wa, xa)
    ref_b = workspace_sort(wb, xb)
    for w, x, ref in ((wa, xa, ref_a), (wb, xb, ref_b), (wa, xa, ref_a)):
        st, perm, bstart, bad = static_sort(w, x)
        assert st == 0
        assert bad == 0
        # against the keys of the bin rule, computed on the CPU
        geom = geometry_struct(w).as_dict()
        key, bins = cpu_keys(w.x, geom, w.precision)
        assert np.array_equal(perm.astype(np.int64), np.argsort(key, kind="stable"))
        counts = np.bincount(bins, minlength=int(np.prod(geom["nbins"])))
        assert np.array_equal(bstart.astype(np.int64), np.concatenate([[0], np.cumsum(counts)]))
        # and against the workspace sort
        assert np.array_equal(perm, ref[0])
        assert np.array_equal(bstart, ref[1])
        assert bstart[-1] == w.n


def test_static_sort_limits_and_flag():
    w = inputs.random_small(8, 1, 1000, 64, 0, [0.02], precision="f64", tol=1e-9)
    x = torch.tensor(w.x, dtype=torch.float64, device="cuda")
    x[3, 0] = 2.0                                   # outside the grid box
    st, perm, bstart, bad = static_sort(w, x)
    assert st == 0 and bad == 1
    assert sorted(perm.tolist()) == list(range(w.n))
    # the flagged sample is sorted into the first bin along its axis
    pos = int(np.where(perm == 3)[0][0])
    assert bstart[0] <= pos < bstart[1]
    big = torch.zeros((MAX_N + 1, 1), dtype=torch.float64, device="cuda")
    st, *_ = static_sort(w, big)
    assert st == 1                                  # FKREG_ERR_INVALID_ARG, nothing launched
