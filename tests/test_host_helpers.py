"""Host-side logic of the binding (no GPU): the candidate bandwidth lists of
Sec. 4 (get_hList), the dstd selection rule of Table 1, the orchestration of
cv_fkreg and gcv, the sweep's split, and the marshalling of every plan call
(input checks, shapes, the entry point reached) against stand-in libraries."""
import ctypes
import os

import numpy as np
import pytest

from paper_2204_07716_gb300 import fkreg

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_bandwidth_list_reproduces_the_printed_bessel_values():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "get_hlist_bessel.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert rows
    for n, lo, hi, sp, idx, val in rows:
        H = fkreg.bandwidth_list(int(n), [(float(lo), float(hi))], sp)
        assert H.shape == (int(n), 1, 1)
        sig = np.sqrt(H[:, 0, 0])
        assert sig[0] == pytest.approx(float(lo)) and sig[-1] == pytest.approx(float(hi))
        assert round(sig[int(idx) - 1], 6 if float(val) < 0.1 else 5) == pytest.approx(float(val))


def test_bandwidth_list_two_axes_is_every_combination():
    # the bivariate example of Sec. 4: 10 values on one axis, 20 on the other
    H = fkreg.bandwidth_list([10, 20], [(0.01, 1.0), (0.1, 1.0)], "lin")
    assert H.shape == (200, 2, 2)
    assert np.all(H[:, 0, 1] == 0) and np.all(H[:, 1, 0] == 0)
    s0, s1 = np.sqrt(H[:, 0, 0]), np.sqrt(H[:, 1, 1])
    assert np.allclose(s0[:20], 0.01) and np.allclose(s1[:20], np.linspace(0.1, 1.0, 20))
    assert np.allclose(s0[::20], np.linspace(0.01, 1.0, 10))
    assert len({(round(a, 12), round(b, 12)) for a, b in zip(s0, s1)}) == 200
    with pytest.raises(fkreg.FkregError):
        fkreg.bandwidth_list([10], [(0.01, 1.0), (0.1, 1.0)])
    with pytest.raises(fkreg.FkregError):
        fkreg.bandwidth_list(5, [(0.0, 1.0)])


def test_select_bandwidth_dstd_rule():
    assert fkreg.select_bandwidth([5.0, 3.0, 2.0, 2.0, 4.0]) == 3      # ties: the later one
    assert fkreg.select_bandwidth([5.0, 2.0, 2.1, 9.0]) == 1
    s = float(np.std([5.0, 2.0, 2.1, 9.0]))
    assert fkreg.select_bandwidth([5.0, 2.0, 2.1, 9.0], 0.15 / s) == 2
    assert fkreg.select_bandwidth([float("nan"), 3.0, 1.0, float("nan")]) == 2


class _FakePlan:
    """Stands in for fkreg.Plan: records the arguments, returns outputs of the
    shapes the real plan returns, with a GCV curve whose minimum is known."""
    made = []

    def __init__(self, d, order, grid_n, lo, hi, H, max_n, n_rhs=1, max_probes=0, tol=1e-6,
                 precision="f32", y_complex=False, device=None, kernel="gaussian"):
        import torch
        self.args = dict(d=d, order=order, grid_n=list(grid_n), lo=list(lo), hi=list(hi),
                         H=np.array(H), max_n=max_n, n_rhs=n_rhs, max_probes=max_probes,
                         tol=tol, precision=precision, y_complex=y_complex, kernel=kernel)
        self.nb, self.grid = np.array(H).shape[0], tuple(grid_n)
        self.torch = torch
        _FakePlan.made.append(self)

    def set_points(self, x):
        self.x = x

    def df(self, y, n_probes, seed=0, want=()):
        t = self.torch
        nb, R, n = self.nb, self.args["n_rhs"], self.args["max_n"]
        g = t.tensor([(k - 2.0) ** 2 + 1.0 for k in range(nb)], dtype=t.float64)
        return {"gcv": t.stack([g] * R, dim=1), "trace": t.zeros((nb, 3), dtype=t.float64),
                "mhat_grid": t.arange(nb, dtype=t.float32).reshape(nb, 1, 1).expand(nb, R, int(np.prod(self.grid))).reshape((nb, R) + self.grid),
                "mask": t.ones((nb,) + self.grid, dtype=t.uint8),
                "mhat_at_x": t.zeros((nb, R, n))}

    def variance(self, y, mh):
        t = self.torch
        return t.full((self.nb, self.args["n_rhs"]) + self.grid, 7.0)

    def sync(self):
        pass


def test_cv_fkreg_orchestration(monkeypatch):
    torch = pytest.importorskip("torch")
    monkeypatch.setattr(fkreg, "Plan", _FakePlan)
    _FakePlan.made.clear()
    x = np.column_stack([np.linspace(0.2, 0.9, 50), np.linspace(-1.0, 3.0, 50)])
    y = np.sin(x[:, 0])
    H = fkreg.bandwidth_list(6, [(0.05, 0.5), (0.05, 0.5)])[:6]
    r = fkreg.cv_fkreg(x, y, H, 16, order=1, n_probes=4, variance=True)
    p = _FakePlan.made[-1]
    assert p.args["lo"] == pytest.approx([0.2, -1.0]) and p.args["hi"] == pytest.approx([0.9, 3.0])
    assert p.args["grid_n"] == [16, 16] and p.args["n_rhs"] == 1 and p.args["max_probes"] == 4
    assert r["index"] == 2 and np.array_equal(r["H"], H[2])
    assert r["mhat_grid"].shape == (1, 16, 16) and float(r["mhat_grid"][0, 0, 0]) == 2.0
    assert r["sigma2"].shape == (1, 16, 16) and r["gcv"].shape == (6,)
    # complex locations become the 2-D points (Re z, Im z)
    z = x[:, 0] + 1j * x[:, 1]
    fkreg.cv_fkreg(z, y, H, [16, 16])
    q = _FakePlan.made[-1]
    assert q.args["d"] == 2 and q.args["lo"] == pytest.approx([0.2, -1.0])


class _FakeBackwardPlan:
    """Stands in for fkreg.Plan in fkreg.gcv: returns known gradients."""
    made = []

    def __init__(self, d, order, grid_n, lo, hi, H, max_n, n_rhs=1, max_probes=0, tol=1e-6,
                 precision="f32", flags=0, device=None, **kw):
        import torch
        self.torch, self.d, self.n = torch, d, max_n
        self.args = dict(H=np.array(H), flags=flags, order=order, max_probes=max_probes)
        _FakeBackwardPlan.made.append(self)

    def set_points(self, x):
        self.x = x

    def backward(self, y, n_probes, seed=0, b=0):
        t = self.torch
        n, d = self.n, self.d
        return {"gcv": t.tensor([0.25], dtype=t.float64),
                "dlogh": t.arange(1, d + 1, dtype=t.float64),
                "dy": t.full((n,), 0.5, dtype=t.float32),
                "dx": t.arange(n * d, dtype=t.float32).reshape(n, d)}

    def sync(self):
        pass


def test_gcv_autograd_chains_the_backward(monkeypatch):
    torch = pytest.importorskip("torch")
    monkeypatch.setattr(fkreg, "Plan", _FakeBackwardPlan)
    x = torch.rand(20, 2, dtype=torch.float64, requires_grad=True)
    y = torch.rand(20, dtype=torch.float64, requires_grad=True)
    ls = torch.log(torch.tensor([0.1, 0.2], dtype=torch.float64)).requires_grad_()
    g = fkreg.gcv(x, y, ls, [16, 16], [0, 0], [1, 1], n_probes=4)
    (3.0 * g).backward()
    p = _FakeBackwardPlan.made[-1]
    assert p.args["flags"] & fkreg.FKREG_WANT_BACKWARD
    assert np.allclose(np.diag(p.args["H"][0]), [0.01, 0.04])
    assert float(g.detach()) == 0.25
    assert torch.allclose(ls.grad, torch.tensor([3.0, 6.0], dtype=torch.float64))
    assert torch.allclose(y.grad, torch.full((20,), 1.5, dtype=torch.float64))
    assert torch.allclose(x.grad, 3.0 * torch.arange(40, dtype=torch.float64).reshape(20, 2))


def test_cv_fkreg_standardises_x(monkeypatch):
    torch = pytest.importorskip("torch")
    monkeypatch.setattr(fkreg, "Plan", _FakePlan)
    _FakePlan.made.clear()
    rng = np.random.default_rng(4)
    x = rng.random(200) * 20.0
    y = np.sin(x)
    H = fkreg.bandwidth_list(10, [(0.01, 1.0)])
    r = fkreg.cv_fkreg(x, y, H, 100, order=0, standardize=True)
    p = _FakePlan.made[-1]
    sd = float(np.std(x, ddof=1))
    xs = p.x.numpy().reshape(-1)
    assert np.allclose(xs, x / sd)
    assert p.args["lo"][0] == pytest.approx(x.min() / sd) and p.args["hi"][0] == pytest.approx(x.max() / sd)
    # the printed Bessel example reports h on both scales: original = normalised * std(x)
    assert np.sqrt(r["H_original"][0, 0]) == pytest.approx(np.sqrt(r["H"][0, 0]) * sd)


def test_option_names_are_checked():
    H = np.diag([0.01, 0.02])
    base = dict(d=2, order=1, grid_n=(32, 32), lo=(0, 0), hi=(1, 1), H=H)
    for bad in (dict(kernel="gauss"), dict(spread_kernel="gaussian"), dict(precision="fp32")):
        with pytest.raises(fkreg.FkregError):
            fkreg.make_opts(**base, **bad)
    # Table 1 calls the uniform kernel "box"
    assert fkreg.make_opts(**base, kernel="box")[0].kernel == fkreg.make_opts(**base, kernel="uniform")[0].kernel


@pytest.mark.parametrize("box", [None, (-0.5, 21.0)])
def test_cv_fkreg_standardised_float32_samples_stay_in_the_box(monkeypatch, box):
    # the device keeps a sample only if lo <= x <= hi in the sample's own
    # precision (lo, hi rounded to it): every standardised float32 sample
    # passes that test, with the default box and with a given one
    torch = pytest.importorskip("torch")
    monkeypatch.setattr(fkreg, "Plan", _FakePlan)
    _FakePlan.made.clear()
    rng = np.random.default_rng(9)
    for trial in range(20):
        x = torch.tensor(rng.random(5000) * 20.0 + 1e-3 * trial, dtype=torch.float32)
        x[0], x[1] = x.min(), x.max()
        lo, hi = (None, None) if box is None else box
        fkreg.cv_fkreg(x, torch.sin(x), fkreg.bandwidth_list(4, [(0.05, 0.5)]), 64, lo=lo, hi=hi,
                       order=0, standardize=True)
        p = _FakePlan.made[-1]
        xs = p.x.reshape(-1)
        assert xs.dtype == torch.float32
        lo32 = np.float32(p.args["lo"][0])
        hi32 = np.float32(p.args["hi"][0])
        assert bool(torch.all(xs >= float(lo32))) and bool(torch.all(xs <= float(hi32)))
        sd = float(np.std(x.numpy().astype(np.float64), ddof=1))
        np.testing.assert_allclose(xs.numpy(), x.numpy().astype(np.float64) / sd, rtol=1e-6)


def test_sweep_split_of_the_3d_sweep():
    # sixteen bandwidths log-spaced over a decade: the narrow ones get their
    # own, shorter period and smaller fine grid; one bandwidth, or a list
    # whose members need the same period, stays one group
    from paper_2204_07716_gb300 import fkreg, inputs
    w = inputs.nw3d_df(n=10)
    kw = dict(d=3, order=0, grid_n=w.grid_n, lo=w.lo, hi=w.hi, n_rhs=1, max_probes=32,
              tol=1e-6, precision="f32")
    first, cost2 = fkreg.sweep_split(4_000_000, 2, H=w.H, **kw)
    assert len(first) == 3 and first[0] == 0 and first[-1] == 16 and 0 < first[1] < 16
    one, cost1 = fkreg.sweep_split(4_000_000, 1, H=w.H, **kw)
    assert one == [0, 16] and cost2 < 0.8 * cost1
    g_all = fkreg.geometry(H=w.H, **kw)
    g_narrow = fkreg.geometry(H=w.H[:first[1]], **kw)
    g_wide = fkreg.geometry(H=w.H[first[1]:], **kw)
    assert g_narrow["period"][0] < g_all["period"][0]
    assert g_narrow["nf"][0] < g_all["nf"][0] and g_wide["nf"][0] < g_all["nf"][0]
    # more groups allowed never raise the modelled cost
    first3, cost3 = fkreg.sweep_split(4_000_000, 3, H=w.H, **kw)
    assert cost3 <= cost2 + 1e-12
    # a single bandwidth, and the headline's diagonal bandwidth
    assert fkreg.sweep_split(4_000_000, 4, H=w.H[:1], **kw)[0] == [0, 1]
    w2 = inputs.ll2d(n=10)
    assert fkreg.sweep_split(1_000_000, 2, d=2, order=1, grid_n=w2.grid_n, lo=w2.lo, hi=w2.hi,
                             H=w2.H, n_rhs=1, max_probes=10)[0] == [0, 1]
    with pytest.raises(fkreg.FkregError):
        fkreg.sweep_split(1000, 0, H=w.H, **kw)


def test_sweep_picks_direct_sums_only_where_they_pay():
    # narrow Gaussians over few samples: direct sums; the 3-D sweep's
    # bandwidths over 4e6 samples: the NUFFT for every group
    import numpy as np
    from paper_2204_07716_gb300 import fkreg, inputs
    H = np.array([np.eye(2) * s * s for s in (0.0015, 0.003, 0.05)])
    first, _, kern = fkreg.sweep_split(200_000, 3, with_kernels=True, d=2, order=0,
                                       grid_n=(100, 100), lo=(0, 0), hi=(1, 1), H=H, n_rhs=1,
                                       max_probes=0, tol=1e-6, precision="f32")
    assert kern[0] == "gaussian_direct" and kern[-1] == "gaussian"
    w = inputs.nw3d_df(n=10)
    _, _, kern3 = fkreg.sweep_split(4_000_000, 2, with_kernels=True, d=3, order=0,
                                    grid_n=w.grid_n, lo=w.lo, hi=w.hi, H=w.H, n_rhs=1,
                                    max_probes=32, tol=1e-6, precision="f32")
    assert kern3 == ["gaussian", "gaussian"]
    # the direct path's geometry: bins on the output lattice, sized from the
    # cut radius R sigma, R^2 = 2 ln(10 / tol)
    g = fkreg.geometry(d=2, order=1, grid_n=(128, 128), lo=(0, 0), hi=(1, 1), H=H[1:2],
                       kernel="gaussian_direct", tol=1e-6)
    assert g["nf"] == [128, 128] and g["modes"] == [1, 1]
    with pytest.raises(fkreg.FkregError):
        fkreg.geometry(d=2, order=1, grid_n=(128, 128), lo=(0, 0), hi=(1, 1), H=H[1:2],
                       kernel="gaussian_direct", flags=fkreg.FKREG_WANT_BACKWARD)


def _standin_plan(n, n_rhs=1, n_bw=1, y_complex=False, d=2):
    # a Plan object without a device plan: only the argument marshalling runs
    import torch
    p = fkreg.Plan.__new__(fkreg.Plan)
    p.torch = torch
    p.device = torch.device("cpu")
    p.d, p.n_rhs, p.n_bw, p.n = d, n_rhs, n_bw, n
    p.y_complex = y_complex
    p.dtype, p.cdtype = torch.float32, torch.complex64
    return p


def test_inputs_smaller_than_the_call_reads_are_refused():
    # the C calls read [n_rhs, n] responses, [n_probes, n] probes and
    # [n_bw, n_rhs, n] at-sample estimates from device memory by size alone:
    # the binding refuses a tensor with fewer values, which the device would
    # read past its end, and accepts every shape the plan calls produce
    import torch
    p = _standin_plan(10)
    assert tuple(p._y(torch.zeros(10)).shape) == (1, 10)
    assert tuple(p._y(np.zeros((1, 10))).shape) == (1, 10)
    with pytest.raises(fkreg.FkregError, match="INVALID_ARG: y"):
        p._y(torch.zeros(9))
    p2 = _standin_plan(10, n_rhs=2, n_bw=3)
    assert tuple(p2._y(torch.zeros(2, 10)).shape) == (2, 10)
    with pytest.raises(fkreg.FkregError, match="INVALID_ARG: y"):
        p2._y(torch.zeros(10))
    assert p2._probes(None, 4) is None
    assert tuple(p2._probes(torch.zeros(4, 10), 4).shape) == (4, 10)
    assert tuple(p2._probes(torch.zeros(5, 10), 4).shape) == (5, 10)
    with pytest.raises(fkreg.FkregError, match="INVALID_ARG: probes"):
        p2._probes(torch.zeros(3, 10), 4)
    assert p2._mhat_at_x(torch.zeros(3, 2, 10), False).numel() == 60
    with pytest.raises(fkreg.FkregError, match="INVALID_ARG: mhat_at_x"):
        p2._mhat_at_x(torch.zeros(1, 2, 10), False)
    # complex responses: interleaved (re, im), twice the values
    pc = _standin_plan(10, y_complex=True)
    assert tuple(pc._y(torch.zeros(10, dtype=torch.complex64)).shape) == (1, 10, 2)
    with pytest.raises(fkreg.FkregError, match="INVALID_ARG: y"):
        pc._y(torch.zeros(10))
    assert pc._mhat_at_x(torch.zeros(1, 1, 10, dtype=torch.complex64), True).numel() == 20
    # no samples yet (or none at all): nothing is read, the outputs of a
    # plan with n = 0 (one padding value) pass
    p0 = _standin_plan(0)
    assert p0._y(torch.zeros(0)).numel() == 0
    assert p0._mhat_at_x(torch.zeros(1, 1, 1), False).numel() == 1


def test_sample_arrays_must_match_the_plan_dimension():
    import torch
    p = _standin_plan(0, d=2)
    assert p._sample_count(torch.zeros(7, 2)) == 7
    assert p._sample_count(torch.zeros(0, 2)) == 0
    for bad in (torch.zeros(7, 3), torch.zeros(7), torch.zeros(7, 2, 1)):
        with pytest.raises(fkreg.FkregError, match="INVALID_ARG"):
            p._sample_count(bad)
    p1 = _standin_plan(0, d=1)
    assert p1._sample_count(torch.zeros(7)) == 7
    assert p1._sample_count(torch.zeros(7, 1)) == 7


def test_batch_capture_refuses_inputs_the_kernels_cannot_read(monkeypatch):
    # Batch.capture hands raw pointers to the recorded kernels: every tensor
    # must be on the batch's device, in the problem's precision, contiguous
    # and large enough; the check runs before anything is recorded
    import types
    import torch
    monkeypatch.setattr(torch.cuda, "current_stream",
                        lambda *a, **k: types.SimpleNamespace(cuda_stream=0))
    b = fkreg.Batch.__new__(fkreg.Batch)
    b.torch, b.device, b.h = torch, torch.device("cpu"), None
    b.problems = [dict(d=2, grid_n=(8, 8), H=np.eye(2) * 0.01, y_complex=True, precision="f32")]
    reached = []

    class StandInLib:
        def fkreg_batch_capture(self, *a):
            reached.append(a)
            return 0

    b.L = StandInLib()
    x, y = torch.zeros(5, 2), torch.zeros(5, 2)            # y: (re, im) pairs
    b.capture([x], [y])
    b.capture([x], [torch.zeros(5, dtype=torch.complex64)])
    assert len(reached) == 2
    for xs, ys in (([torch.zeros(5, 2, dtype=torch.float64)], [y]),      # wrong precision
                   ([torch.zeros(5, 3)], [y]),                            # wrong dimension
                   ([torch.zeros(2, 5).t()], [y]),                        # not contiguous
                   ([x], [torch.zeros(5)]),                               # complex needs 2n values
                   ([x, x], [y, y])):                                     # one problem only
        with pytest.raises(fkreg.FkregError, match="INVALID_ARG"):
            b.capture(xs, ys)
    assert len(reached) == 2


def test_predict_and_interval_refuse_host_arrays():
    # both hand raw pointers to a kernel: a host tensor is refused before any
    # launch (query points on the host are copied to the grid's device)
    import torch
    g = torch.zeros(4, 4, dtype=torch.float64)
    with pytest.raises(fkreg.FkregError, match="CUDA tensor"):
        fkreg.predict(g, (4, 4), (0, 0), (1, 1), torch.zeros(3, 2))
    with pytest.raises(fkreg.FkregError, match="unknown method"):
        fkreg.predict(g, (4, 4), (0, 0), (1, 1), torch.zeros(3, 2), "nearest")
    with pytest.raises(fkreg.FkregError, match="CUDA tensor"):
        fkreg.interval(g, torch.ones(4, 4, dtype=torch.float64))


def _compositions(n, k_max):
    # every split of [0, n) into at most k_max contiguous non-empty groups
    import itertools
    for k in range(1, min(k_max, n) + 1):
        for cuts in itertools.combinations(range(1, n), k - 1):
            yield [0, *cuts, n]


SPLIT_CASES = [  # d, samples, seed, bandwidth range, grid points per axis
    (2, 200_000, 1, (0.0015, 0.3), 100),   # unsorted; three groups, one of direct sums
    (2, 1_000_000, 6, (0.002, 0.25), 128),  # two groups
    (2, 4_000_000, 2, (0.003, 0.3), 256),   # one group
    (3, 2_000_000, 3, (0.004, 0.15), 96),   # unsorted; direct sums for the narrow group
    (1, 50_000, 4, (0.0005, 0.3), 512),
]


@pytest.mark.parametrize("d,max_n,seed,srange,grid", SPLIT_CASES)
def test_sweep_split_is_the_cheapest_contiguous_split(d, max_n, seed, srange, grid):
    # the split's dynamic program against brute force over every contiguous
    # split into at most K groups, each group priced by the same entry point
    # on that sub-list alone (one group); refused groups are infeasible
    rng = np.random.default_rng(seed)
    n_bw = 6 if d < 3 else 5
    sig = np.sort(np.exp(rng.uniform(np.log(srange[0]), np.log(srange[1]), n_bw)))
    if seed % 2:
        sig = sig[rng.permutation(n_bw)]           # the caller's order, not sorted
    H = np.array([np.eye(d) * s * s for s in sig])
    kw = dict(d=d, order=1 if d < 3 else 0, grid_n=(grid,) * d, lo=(0.0,) * d, hi=(1.0,) * d,
              n_rhs=1, max_probes=4, tol=1e-6, precision="f32")
    memo = {}

    def group(a, b):
        if (a, b) not in memo:
            first, cost, kern = fkreg.sweep_split(max_n, 1, with_kernels=True, H=H[a:b], **kw)
            memo[(a, b)] = (cost, kern[0]) if cost >= 0 else (None, None)
        return memo[(a, b)]

    for K in (1, 2, 3):
        first, cost, kern = fkreg.sweep_split(max_n, K, with_kernels=True, H=H, **kw)
        best = None
        for split in _compositions(n_bw, K):
            parts = [group(a, b)[0] for a, b in zip(split, split[1:])]
            if any(p is None for p in parts):
                continue
            tot = sum(parts)
            best = tot if best is None else min(best, tot)
        assert best is not None
        assert cost == pytest.approx(best, rel=1e-12), (K, first)
        assert len(first) - 1 <= K and first[0] == 0 and first[-1] == n_bw
        chosen = [group(a, b) for a, b in zip(first, first[1:])]
        assert sum(c for c, _ in chosen) == pytest.approx(cost, rel=1e-12)
        assert kern == [k for _, k in chosen]


def test_the_split_cases_include_real_splits():
    # the brute-force cases above are not all single groups
    groups = []
    for d, max_n, seed, srange, grid in SPLIT_CASES:
        rng = np.random.default_rng(seed)
        n_bw = 6 if d < 3 else 5
        sig = np.sort(np.exp(rng.uniform(np.log(srange[0]), np.log(srange[1]), n_bw)))
        if seed % 2:
            sig = sig[rng.permutation(n_bw)]
        H = np.array([np.eye(d) * s * s for s in sig])
        first, _, kern = fkreg.sweep_split(
            max_n, 3, with_kernels=True, d=d, order=1 if d < 3 else 0, grid_n=(grid,) * d,
            lo=(0.0,) * d, hi=(1.0,) * d, H=H, n_rhs=1, max_probes=4, tol=1e-6, precision="f32")
        groups.append((len(first) - 1, kern))
    assert max(g for g, _ in groups) == 3 and any(g == 2 for g, _ in groups)
    assert any("gaussian_direct" in k for _, k in groups)


class _RecordingLib:
    # stands in for the C library: every entry point returns FKREG_OK and is recorded
    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def call(*a):
            self.calls.append(name)
            return 0
        return call


@pytest.mark.parametrize("cls", ["Plan", "Sweep"])
def test_plan_methods_marshal_the_shapes_the_calls_use(cls, monkeypatch):
    # a dry run of every plan call on host tensors with a stand-in library:
    # the marshalling (shapes, the size checks, the entry point each call
    # reaches) runs exactly as on the GPU, no kernel does
    import types
    import torch
    monkeypatch.setattr(torch.cuda, "current_stream",
                        lambda *a, **k: types.SimpleNamespace(cuda_stream=0))
    p = getattr(fkreg, cls).__new__(getattr(fkreg, cls))
    p.torch, p.device = torch, torch.device("cpu")
    p.d, p.order, p.n_rhs, p.n_bw, p.n = 2, 1, 1, 2, 0
    p.grid_n, p.M, p.ns, p.nt, p.max_probes = (8, 8), 64, 6, 3, 4
    p.y_complex, p.precision = False, "f32"
    p.dtype, p.cdtype = torch.float32, torch.complex64
    p.L, p.h = _RecordingLib(), ctypes.c_void_p(0)
    n = 50
    p.set_points(torch.rand(n, 2, dtype=torch.float64))
    assert p.n == n
    y = torch.randn(n)
    o = p.smooth(y, want=("mhat_grid", "mask", "mhat_at_x"))
    assert o["mhat_at_x"].shape == (2, 1, n)
    o = p.df(y, 4, probes=torch.randn(4, n), want=("mhat_grid", "mhat_at_x"))
    assert o["gcv"].shape == (2, 1) and o["trace"].shape == (2, 3)
    p.df(y, 4)
    s2 = p.variance(y, o["mhat_at_x"])
    assert s2.shape == (2, 1, 8, 8)
    lv = p.log_variance(y, o["mhat_at_x"])
    assert lv["v_at_x"].shape == (2, 1, n) and lv["kappa"].shape == (2, 1)
    g = p.backward(y, 4, probes=torch.randn(4, n), b=1)
    assert g["dy"].shape == (n,) and g["dx"].shape == (n, 2) and g["dlogh"].shape == (2,)
    with pytest.raises(fkreg.FkregError, match="INVALID_ARG: probes"):
        p.df(y, 4, probes=torch.randn(3, n))
    with pytest.raises(fkreg.FkregError, match="INVALID_ARG: mhat_at_x"):
        p.variance(y, o["mhat_at_x"][:1])
    if cls == "Plan":
        r = p.backward_grid(y, torch.zeros(8, 8), b=0)
        assert r["dy"].shape == (1, n)
        names = ["fkreg_set_points", "fkreg_smooth", "fkreg_df", "fkreg_df", "fkreg_variance",
                 "fkreg_log_variance", "fkreg_backward", "fkreg_backward_grid"]
    else:
        names = ["fkreg_sweep_set_points", "fkreg_sweep_smooth", "fkreg_sweep_df",
                 "fkreg_sweep_df", "fkreg_sweep_variance", "fkreg_sweep_log_variance",
                 "fkreg_sweep_backward"]
    assert p.L.calls == names
    p.h = None                                   # nothing to destroy


def test_complex_plan_marshals_interleaved_values(monkeypatch):
    # complex responses and complex locations go to the C calls as (re, im)
    # pairs; the at-sample estimates a smooth returns feed the variance pass
    import types
    import torch
    monkeypatch.setattr(torch.cuda, "current_stream",
                        lambda *a, **k: types.SimpleNamespace(cuda_stream=0))
    p = fkreg.Plan.__new__(fkreg.Plan)
    p.torch, p.device = torch, torch.device("cpu")
    p.d, p.order, p.n_rhs, p.n_bw, p.n = 2, 1, 1, 1, 0
    p.grid_n, p.M, p.ns, p.nt, p.max_probes = (8, 8), 64, 6, 3, 0
    p.y_complex, p.precision = True, "f64"
    p.dtype, p.cdtype = torch.float64, torch.complex128
    p.L, p.h = _RecordingLib(), ctypes.c_void_p(0)
    n = 30
    p.set_points(torch.rand(n, dtype=torch.float64) + 1j * torch.rand(n, dtype=torch.float64))
    assert p.n == n and tuple(p._x.shape) == (n, 2)
    y = torch.randn(n, dtype=torch.complex128)
    o = p.smooth(y, want=("mhat_grid", "mhat_at_x"))
    assert o["mhat_at_x"].dtype == torch.complex128 and o["mhat_at_x"].shape == (1, 1, n)
    s2 = p.variance(y, o["mhat_at_x"])
    assert s2.dtype == torch.float64
    with pytest.raises(fkreg.FkregError, match="INVALID_ARG: y"):
        p.smooth(y.real)                          # half the values a complex call reads
    assert p.L.calls == ["fkreg_set_points", "fkreg_smooth", "fkreg_variance"]
    p.h = None
