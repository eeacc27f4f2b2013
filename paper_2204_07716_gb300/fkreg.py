"""Thin Python binding of libfkreg.so (argument marshalling only).

Every computation of the smoother happens inside the CUDA library; this
module only builds the C structs, hands device pointers of torch tensors and
the current CUDA stream to the C ABI declared in ``include/fkreg.h``, and
raises on a non-OK status.  There is no CPU fallback: if the library is
missing the import of a plan fails loudly.

Contents: ``Plan`` (one problem: set_points, smooth, df, variance,
log_variance, backward), ``Batch`` (uneven problems in one captured graph),
``StepGraph`` (a sequence of calls captured as one graph), ``predict`` and
``interval`` (device post-processing calls), and host-side conveniences
that only orchestrate those calls or work on host scalars:
``bandwidth_list`` (candidate H lists, get_hList of Sec. 4),
``select_bandwidth`` (the dstd rule of Table 1), ``cv_fkreg`` (Sec. 4's
one-call bandwidth selection and smoothing), ``gcv`` (GCV as a
differentiable torch function through fkreg_backward), ``autotune_tile``.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Iterable, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# FKREG_CHECKED=1 in the environment loads the checked build (range checks on
# the kernels' index arithmetic, reported through fkreg_sync_status)
CHECKED = os.environ.get("FKREG_CHECKED", "") == "1"
LIB_PATH = os.path.join(HERE, "libfkreg_checked.so" if CHECKED else "libfkreg.so")

FKREG_F32, FKREG_F64 = 0, 1
FKREG_SPREAD_ES, FKREG_SPREAD_GAUSS = 0, 1
KERNELS = {"gaussian": 0, "uniform": 1, "box": 1, "epanechnikov": 2, "triangle": 3,
           "biweight": 4, "triweight": 5, "gaussian_direct": 6}
FKREG_GCV_EXACT_TRACE = 1
FKREG_WANT_BACKWARD = 2
STAGES = ["sort", "strengths", "spread", "fft_fwd", "kmul_grid", "fft_grid", "grid_solve",
          "kmul_t2", "fft_t2", "interp", "finalize", "backward"]

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "WORKSPACE", 4: "CUDA", 5: "CUFFT",
          6: "TIMEOUT", 7: "DEVICE", 8: "STATE"}

EXPORTS = ["fkreg_geometry_query", "fkreg_spread_kernel_ft", "fkreg_spread_kernel_values",
           "fkreg_plan_create",
           "fkreg_workspace_bytes", "fkreg_set_workspace", "fkreg_set_points", "fkreg_get_sort",
           "fkreg_smooth", "fkreg_df", "fkreg_backward", "fkreg_backward_grid", "fkreg_variance",
           "fkreg_log_variance", "fkreg_interval", "fkreg_predict", "fkreg_set_timing",
           "fkreg_stage_times", "fkreg_set_wait_limit", "fkreg_bin_sort_static",
           "fkreg_sync_status", "fkreg_checked_build", "fkreg_check_selftest",
           "fkreg_last_error", "fkreg_global_error", "fkreg_plan_destroy",
           "fkreg_batch_create", "fkreg_batch_workspace_bytes", "fkreg_batch_set_workspace",
           "fkreg_batch_capture", "fkreg_batch_launch", "fkreg_batch_latencies",
           "fkreg_batch_plan", "fkreg_batch_last_error", "fkreg_batch_destroy",
           "fkreg_measure_peaks",
           "fkreg_sweep_create", "fkreg_sweep_split", "fkreg_sweep_groups", "fkreg_sweep_workspace_bytes",
           "fkreg_sweep_set_workspace", "fkreg_sweep_set_points", "fkreg_sweep_smooth",
           "fkreg_sweep_df", "fkreg_sweep_variance", "fkreg_sweep_log_variance",
           "fkreg_sweep_backward", "fkreg_sweep_sync_status",
           "fkreg_sweep_set_timing", "fkreg_sweep_stage_times", "fkreg_sweep_last_error",
           "fkreg_sweep_destroy"]


class Opts(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("order", ctypes.c_int), ("kernel", ctypes.c_int),
                ("spread_kernel", ctypes.c_int), ("precision", ctypes.c_int),
                ("y_complex", ctypes.c_int), ("grid_n", ctypes.c_int64 * 3),
                ("grid_lo", ctypes.c_double * 3), ("grid_hi", ctypes.c_double * 3),
                ("n_bw", ctypes.c_int), ("H", ctypes.POINTER(ctypes.c_double)),
                ("n_rhs", ctypes.c_int), ("max_probes", ctypes.c_int), ("tol", ctypes.c_double),
                ("mask_rho", ctypes.c_double), ("tile", ctypes.c_int), ("flags", ctypes.c_int)]


class Geometry(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("delta", ctypes.c_double * 3),
                ("period", ctypes.c_double * 3), ("ldft", ctypes.c_int64 * 3),
                ("modes", ctypes.c_int64 * 3), ("nf", ctypes.c_int64 * 3), ("w", ctypes.c_int),
                ("beta", ctypes.c_double), ("tile", ctypes.c_int64 * 3),
                ("nbins", ctypes.c_int64 * 3), ("inv_h", ctypes.c_double * 3),
                ("ns", ctypes.c_int), ("nt", ctypes.c_int)]

    def as_dict(self) -> dict:
        d = self.dim
        out = {"dim": d, "w": self.w, "beta": self.beta, "ns": self.ns, "nt": self.nt}
        for k in ("delta", "period", "ldft", "modes", "nf", "tile", "nbins", "inv_h"):
            out[k] = list(getattr(self, k))[:d]
        return out


class Outputs(ctypes.Structure):
    _fields_ = [("mhat_grid", ctypes.c_void_p), ("mask", ctypes.c_void_p),
                ("moments", ctypes.c_void_p), ("mhat_at_x", ctypes.c_void_p),
                ("rss", ctypes.c_void_p), ("trace", ctypes.c_void_p), ("gcv", ctypes.c_void_p)]


_lib = None


class Peaks(ctypes.Structure):
    _fields_ = [("sm_count", ctypes.c_int), ("sm_mhz", ctypes.c_double),
                ("fp32_tflops", ctypes.c_double), ("fp32x2_tflops", ctypes.c_double),
                ("tf32_mma_tflops", ctypes.c_double), ("smem_load_gbs", ctypes.c_double * 3), ("smem_bcast16_gbs", ctypes.c_double),
                ("smem_atomic_gops", ctypes.c_double), ("gmem_atomic_gops", ctypes.c_double)]


PEAKS_SCRATCH_BYTES = 4 << 20


class FkregError(RuntimeError):
    pass


def load():
    """Load libfkreg.so (build it first with paper_2204_07716_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise FkregError(f"{LIB_PATH} is missing: run paper_2204_07716_gb300.build.build() "
                         "(there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, st = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.fkreg_geometry_query.argtypes = [ctypes.POINTER(Opts), ctypes.POINTER(Geometry)]
    L.fkreg_spread_kernel_ft.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, i64, i64,
                                         ctypes.POINTER(ctypes.c_double)]
    L.fkreg_spread_kernel_values.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_int, i64, vp, vp, vp]
    L.fkreg_plan_create.argtypes = [ctypes.POINTER(Opts), i64, ctypes.POINTER(vp)]
    L.fkreg_workspace_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    L.fkreg_set_workspace.argtypes = [vp, vp, ctypes.c_size_t, vp]
    L.fkreg_set_points.argtypes = [vp, i64, vp, vp]
    L.fkreg_get_sort.argtypes = [vp, vp, vp, ctypes.POINTER(i64), vp]
    L.fkreg_smooth.argtypes = [vp, vp, ctypes.POINTER(Outputs), vp]
    L.fkreg_df.argtypes = [vp, vp, ctypes.c_int, ctypes.c_uint64, vp, ctypes.POINTER(Outputs), vp]
    L.fkreg_variance.argtypes = [vp, vp, vp, vp, vp]
    L.fkreg_log_variance.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    L.fkreg_interval.argtypes = [ctypes.c_int, ctypes.c_int64, vp, vp, ctypes.c_double, vp, vp, vp]
    L.fkreg_predict.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp, ctypes.c_int, vp,
                                ctypes.c_int64, vp, ctypes.c_int, vp, vp]
    L.fkreg_backward.argtypes = [vp, vp, ctypes.c_int, ctypes.c_uint64, vp, ctypes.c_int, vp, vp,
                                 vp, vp, vp]
    L.fkreg_backward_grid.argtypes = [vp, vp, vp, ctypes.c_int, vp, vp, vp, vp]
    L.fkreg_set_timing.argtypes = [vp, ctypes.c_int]
    L.fkreg_set_wait_limit.argtypes = [vp, i64]
    L.fkreg_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64),
                                    ctypes.POINTER(i64)]
    L.fkreg_bin_sort_static.argtypes = [ctypes.POINTER(Geometry), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double), ctypes.c_int, i64, vp, vp,
                                        vp, vp, vp]
    L.fkreg_sync_status.argtypes = [vp, vp]
    L.fkreg_last_error.argtypes = [vp]
    L.fkreg_last_error.restype = ctypes.c_char_p
    L.fkreg_global_error.argtypes = []
    L.fkreg_global_error.restype = ctypes.c_char_p
    L.fkreg_plan_destroy.argtypes = [vp]
    L.fkreg_plan_destroy.restype = None
    L.fkreg_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(Opts), ctypes.POINTER(i64),
                                     ctypes.POINTER(vp)]
    L.fkreg_batch_workspace_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    L.fkreg_batch_set_workspace.argtypes = [vp, vp, ctypes.c_size_t, vp]
    L.fkreg_batch_capture.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(vp),
                                      ctypes.POINTER(vp), ctypes.POINTER(Outputs),
                                      ctypes.POINTER(vp), vp]
    L.fkreg_batch_launch.argtypes = [vp, vp]
    L.fkreg_batch_latencies.argtypes = [vp, ctypes.POINTER(ctypes.c_double), vp]
    L.fkreg_batch_plan.argtypes = [vp, ctypes.c_int]
    L.fkreg_batch_plan.restype = vp
    L.fkreg_batch_last_error.argtypes = [vp]
    L.fkreg_batch_last_error.restype = ctypes.c_char_p
    L.fkreg_batch_destroy.argtypes = [vp]
    L.fkreg_batch_destroy.restype = None
    L.fkreg_measure_peaks.argtypes = [ctypes.POINTER(Peaks), vp, ctypes.c_size_t, vp]
    L.fkreg_sweep_create.argtypes = [ctypes.POINTER(Opts), i64, ctypes.c_int, ctypes.POINTER(vp)]
    L.fkreg_checked_build.argtypes = []
    L.fkreg_check_selftest.argtypes = [vp, vp]
    L.fkreg_sweep_split.argtypes = [ctypes.POINTER(Opts), i64, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    L.fkreg_sweep_groups.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(Geometry)]
    L.fkreg_sweep_workspace_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    L.fkreg_sweep_set_workspace.argtypes = [vp, vp, ctypes.c_size_t, vp]
    L.fkreg_sweep_set_points.argtypes = [vp, i64, vp, vp]
    L.fkreg_sweep_smooth.argtypes = [vp, vp, ctypes.POINTER(Outputs), vp]
    L.fkreg_sweep_df.argtypes = [vp, vp, ctypes.c_int, ctypes.c_uint64, vp,
                                 ctypes.POINTER(Outputs), vp]
    L.fkreg_sweep_variance.argtypes = [vp, vp, vp, vp, vp]
    L.fkreg_sweep_log_variance.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    L.fkreg_sweep_backward.argtypes = [vp, vp, ctypes.c_int, ctypes.c_uint64, vp, ctypes.c_int,
                                       vp, vp, vp, vp, vp]
    L.fkreg_sweep_sync_status.argtypes = [vp, vp]
    L.fkreg_sweep_set_timing.argtypes = [vp, ctypes.c_int]
    L.fkreg_sweep_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_int64),
                                          ctypes.POINTER(ctypes.c_int64)]
    L.fkreg_sweep_last_error.argtypes = [vp]
    L.fkreg_sweep_last_error.restype = ctypes.c_char_p
    L.fkreg_sweep_destroy.argtypes = [vp]
    L.fkreg_sweep_destroy.restype = None
    no_status = ("fkreg_last_error", "fkreg_global_error", "fkreg_plan_destroy", "fkreg_batch_plan",
                 "fkreg_batch_last_error", "fkreg_batch_destroy", "fkreg_sweep_last_error",
                 "fkreg_sweep_destroy")
    for name in EXPORTS:
        if name not in no_status:
            getattr(L, name).restype = st
    _lib = L
    return L


def make_opts(d: int, order: int, grid_n: Sequence[int], lo: Sequence[float],
              hi: Sequence[float], H: np.ndarray, n_rhs: int = 1, max_probes: int = 0,
              tol: float = 1e-6, precision: str = "f32", y_complex: bool = False,
              spread_kernel: str = "es", mask_rho: float = 0.0, tile: int = 0,
              flags: int = 0, kernel: str = "gaussian"):
    """Build an Opts struct; returns (opts, keepalive) -- keep both alive."""
    if kernel not in KERNELS:
        raise FkregError(f"unknown kernel {kernel!r} (one of {sorted(KERNELS)})")
    if spread_kernel not in ("es", "gauss"):
        raise FkregError(f"unknown spread_kernel {spread_kernel!r} ('es' or 'gauss')")
    if precision not in ("f32", "f64"):
        raise FkregError(f"unknown precision {precision!r} ('f32' or 'f64')")
    H = np.ascontiguousarray(np.asarray(H, dtype=np.float64).reshape(-1, d, d))
    o = Opts()
    o.dim, o.order, o.kernel = d, order, KERNELS[kernel]
    o.spread_kernel = FKREG_SPREAD_ES if spread_kernel == "es" else FKREG_SPREAD_GAUSS
    o.precision = FKREG_F32 if precision == "f32" else FKREG_F64
    o.y_complex = int(bool(y_complex))
    for j in range(3):
        o.grid_n[j] = int(grid_n[j]) if j < d else 1
        o.grid_lo[j] = float(lo[j]) if j < d else 0.0
        o.grid_hi[j] = float(hi[j]) if j < d else 1.0
    o.n_bw = H.shape[0]
    o.H = H.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    o.n_rhs, o.max_probes, o.tol = n_rhs, max_probes, tol
    o.mask_rho, o.tile, o.flags = mask_rho, tile, flags
    return o, H


def geometry(**kw) -> dict:
    """Planner geometry (host only, no GPU needed)."""
    L = load()
    o, keep = make_opts(**kw)
    g = Geometry()
    st = L.fkreg_geometry_query(ctypes.byref(o), ctypes.byref(g))
    if st != 0:
        raise FkregError(f"{STATUS.get(st, st)}: {L.fkreg_global_error().decode()}")
    return g.as_dict()


def spread_kernel_ft(kind: str, w: int, beta: float, nf: int, nk: int) -> np.ndarray:
    L = load()
    out = np.zeros(nk)
    st = L.fkreg_spread_kernel_ft(FKREG_SPREAD_ES if kind == "es" else FKREG_SPREAD_GAUSS, w,
                                  beta, nf, nk, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if st != 0:
        raise FkregError(L.fkreg_global_error().decode())
    return out


KERNEL_NAMES = {0: "gaussian", 1: "uniform", 2: "epanechnikov", 3: "triangle", 4: "biweight",
                5: "triweight", 6: "gaussian_direct"}


def sweep_split(max_n: int, max_groups: int = 2, with_kernels: bool = False, **kw):
    """Host-only: the split of the bandwidth list a Sweep would use
    (fkreg_sweep_split): (first bandwidth of each group + [n_bw], modelled
    seconds), and with ``with_kernels`` each group's kernel name after them.
    Keyword arguments as for make_opts."""
    L = load()
    o, keep = make_opts(**kw)
    ng = ctypes.c_int()
    first = (ctypes.c_int * (o.n_bw + 1))()
    kern = (ctypes.c_int * o.n_bw)()
    cost = ctypes.c_double()
    st = L.fkreg_sweep_split(ctypes.byref(o), int(max_n), int(max_groups), ctypes.byref(ng),
                             first, kern, ctypes.byref(cost))
    if st != 0:
        raise FkregError(f"fkreg_sweep_split: {STATUS.get(st, st)}")
    out = (list(first[: ng.value + 1]), float(cost.value))
    if with_kernels:
        out = out + ([KERNEL_NAMES[k] for k in kern[: ng.value]],)
    return out


def spread_kernel_values(kind: str, w: int, beta: float, z):
    """phi(z) on the device (fkreg_spread_kernel_values) for a CUDA tensor z
    of float32 or float64 offsets, in z's precision."""
    import torch
    L = load()
    if not (z.is_cuda and z.is_contiguous() and z.dtype in (torch.float32, torch.float64)):
        raise FkregError("z must be a contiguous float32 or float64 CUDA tensor")
    out = torch.empty_like(z)
    prec = FKREG_F32 if z.dtype == torch.float32 else FKREG_F64
    st = L.fkreg_spread_kernel_values(FKREG_SPREAD_ES if kind == "es" else FKREG_SPREAD_GAUSS, w,
                                      beta, prec, z.numel(), z.data_ptr(), out.data_ptr(),
                                      torch.cuda.current_stream(z.device).cuda_stream)
    if st != 0:
        raise FkregError(f"fkreg_spread_kernel_values: {STATUS.get(st, st)}")
    return out


def measure_peaks(device=None) -> dict:
    """SM-side peaks of the GPU (fkreg_measure_peaks): SM count and clock,
    FP32 FMA TFLOP/s (scalar, packed), TF32 mma.sync TFLOP/s, shared-memory
    load GB/s for 4/8/16-byte
    lanes and a 16-byte broadcast, shared and global atomic Gop/s, and the
    shared-memory bytes per clock per SM that the 16-byte rate implies."""
    import torch
    L = load()
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    scratch = torch.empty(PEAKS_SCRATCH_BYTES, dtype=torch.uint8, device=dev)
    out = Peaks()
    with torch.cuda.device(dev):
        st = L.fkreg_measure_peaks(ctypes.byref(out), ctypes.c_void_p(scratch.data_ptr()),
                                   PEAKS_SCRATCH_BYTES,
                                   ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
    if st != 0:
        raise FkregError(f"fkreg_measure_peaks failed ({STATUS.get(st, st)})")
    r = {"sm_count": out.sm_count, "sm_mhz": out.sm_mhz, "fp32_tflops": out.fp32_tflops,
         "fp32x2_tflops": out.fp32x2_tflops, "tf32_mma_tflops": out.tf32_mma_tflops,
         "smem_load_gbs": list(out.smem_load_gbs),
         "smem_bcast16_gbs": out.smem_bcast16_gbs, "smem_atomic_gops": out.smem_atomic_gops,
         "gmem_atomic_gops": out.gmem_atomic_gops}
    clk = out.sm_count * out.sm_mhz * 1e6
    r["smem_bytes_per_clk_sm"] = [v * 1e9 / clk for v in out.smem_load_gbs] if clk > 0 else None
    return r


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


class Plan:
    """One smoothing problem on one GPU.  Owns a torch workspace tensor.

    The methods mirror the C calls: ``set_points`` (bin + stable sort),
    ``smooth``, ``df`` (Monte-Carlo DF + GCV), ``variance`` (eq. 23).
    """

    # C entry points that a Sweep routes through its own (same arguments)
    _fn_backward = "fkreg_backward"
    _fn_log_variance = "fkreg_log_variance"

    def __init__(self, d: int, order: int, grid_n, lo, hi, H, max_n: int, n_rhs: int = 1,
                 max_probes: int = 0, tol: float = 1e-6, precision: str = "f32",
                 y_complex: bool = False, spread_kernel: str = "es", mask_rho: float = 0.0,
                 tile: int = 0, flags: int = 0, device=None, kernel: str = "gaussian"):
        import torch
        self.torch = torch
        self.L = load()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.d, self.order, self.n_rhs = d, order, n_rhs
        self.grid_n = tuple(int(v) for v in grid_n)
        self.M = int(np.prod(self.grid_n))
        self.max_probes = max_probes
        self.precision = precision
        self.y_complex = bool(y_complex)
        self.dtype = torch.float32 if precision == "f32" else torch.float64
        self.cdtype = torch.complex64 if precision == "f32" else torch.complex128
        self._opts, self._keep = make_opts(d, order, grid_n, lo, hi, H, n_rhs, max_probes, tol,
                                           precision, y_complex, spread_kernel, mask_rho, tile,
                                           flags, kernel)
        self.n_bw = self._opts.n_bw
        g = Geometry()
        self._check_global(self.L.fkreg_geometry_query(ctypes.byref(self._opts), ctypes.byref(g)))
        self.geom = g.as_dict()
        self.ns, self.nt = g.ns, g.nt
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            self._check_global(self.L.fkreg_plan_create(ctypes.byref(self._opts), int(max_n),
                                                        ctypes.byref(h)))
        self.h = h
        nbytes = ctypes.c_size_t()
        self._check(self.L.fkreg_workspace_bytes(self.h, ctypes.byref(nbytes)))
        self.ws_bytes = int(nbytes.value)
        self._ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
        base = self._ws.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self._check(self.L.fkreg_set_workspace(self.h, ctypes.c_void_p(self._ws_ptr),
                                               self.ws_bytes, self._stream()))
        self.n = 0

    # -- helpers -----------------------------------------------------------
    def _stream(self):
        return ctypes.c_void_p(self.torch.cuda.current_stream(self.device).cuda_stream)

    def _check_global(self, st):
        if st != 0:
            raise FkregError(f"{STATUS.get(st, st)}: {self.L.fkreg_global_error().decode()}")

    def _check(self, st):
        if st != 0:
            raise FkregError(f"{STATUS.get(st, st)}: {self.L.fkreg_last_error(self.h).decode()}")

    def _as_dev(self, a, complex_ok=False):
        t = self.torch
        if not isinstance(a, t.Tensor):
            a = t.as_tensor(np.asarray(a))
        if a.is_complex():
            if not complex_ok:
                raise FkregError("complex input where real expected")
            a = a.to(self.cdtype)
            a = t.view_as_real(a)
        else:
            a = a.to(self.dtype)
        return a.to(self.device).contiguous()

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.L.fkreg_plan_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- calls -------------------------------------------------------------
    def set_points(self, x):
        """Sample locations [n, d].  A complex vector z on a 2-D plan is the
        set of points (Re z, Im z): the complex-location regression of
        Sec. 4.4 smooths over the complex plane as over R^2."""
        t = self.torch
        cplx = x.is_complex() if isinstance(x, t.Tensor) else np.iscomplexobj(x)
        if cplx:
            if self.d != 2:
                raise FkregError("complex locations need a 2-D plan")
            x = self._as_dev(x, complex_ok=True)
            if x.dim() != 2 or x.shape[1] != 2:
                raise FkregError("complex locations are a vector of n points")
        else:
            x = self._as_dev(x)
        n = self._sample_count(x)
        self._x = x
        self._check(self.L.fkreg_set_points(self.h, n, ctypes.c_void_p(x.data_ptr()), self._stream()))
        self.n = n

    def _sample_count(self, x) -> int:
        """n of samples x [n, d] (or [n] when d = 1); the C call reads n * d values."""
        n = int(x.shape[0]) if x.dim() > 0 else 0
        if (x.dim() == 2 and int(x.shape[1]) != self.d) or x.dim() > 2:
            raise FkregError(f"INVALID_ARG: samples of shape {tuple(x.shape)} for a {self.d}-D plan")
        self._need(x, n * self.d, f"x ([n, {self.d}] samples)")
        return n

    def sync(self):
        self._check(self.L.fkreg_sync_status(self.h, self._stream()))

    def check_selftest(self):
        """One deliberately out-of-bounds checked access (fkreg_check_selftest);
        in the checked build the next sync raises with site 15, index 20."""
        self._check(self.L.fkreg_check_selftest(self.h, self._stream()))

    def set_wait_limit(self, polls: int = -1):
        """Polls of a staged-window wait before a call gives up with a timeout
        (fkreg_set_wait_limit; < 0 restores the default)."""
        self._check(self.L.fkreg_set_wait_limit(self.h, int(polls)))

    def set_timing(self, enable: bool = True):
        self._check(self.L.fkreg_set_timing(self.h, int(bool(enable))))

    def stage_times(self):
        """(ms per stage, calls per stage, own kernel launches) since the last query."""
        n = len(STAGES)
        ms = (ctypes.c_double * n)()
        calls = (ctypes.c_int64 * n)()
        kl = ctypes.c_int64()
        self._check(self.L.fkreg_stage_times(self.h, ms, calls, ctypes.byref(kl)))
        return ({STAGES[i]: ms[i] for i in range(n)}, {STAGES[i]: calls[i] for i in range(n)},
                int(kl.value))

    def get_sort(self):
        t = self.torch
        nb = ctypes.c_int64()
        self.L.fkreg_get_sort(self.h, None, None, ctypes.byref(nb), self._stream())
        perm = t.empty(max(self.n, 1), dtype=t.int32, device=self.device)
        bstart = t.empty(int(nb.value) + 1, dtype=t.int32, device=self.device)
        self._check(self.L.fkreg_get_sort(self.h, ctypes.c_void_p(perm.data_ptr()),
                                          ctypes.c_void_p(bstart.data_ptr()), ctypes.byref(nb),
                                          self._stream()))
        return perm[: self.n], bstart

    def _outputs(self, want: Iterable[str], df: bool) -> Dict[str, object]:
        t = self.torch
        want = set(want)
        o = {}
        cplx = self.y_complex
        M, nb, R, n = self.M, self.n_bw, self.n_rhs, self.n
        fdt = self.cdtype if cplx else self.dtype
        if "mhat_grid" in want:
            o["mhat_grid"] = t.empty((nb, R) + self.grid_n, dtype=fdt, device=self.device)
        if "mask" in want:
            o["mask"] = t.empty((nb,) + self.grid_n, dtype=t.uint8, device=self.device)
        if "moments" in want:
            per = self.ns + R * self.nt * (2 if cplx else 1)
            o["moments"] = t.empty((nb, per) + self.grid_n, dtype=self.dtype, device=self.device)
        if "mhat_at_x" in want:
            o["mhat_at_x"] = t.empty((nb, R, max(n, 1)), dtype=fdt, device=self.device)
        if "rss" in want or df:
            o["rss"] = t.empty((nb, R), dtype=t.float64, device=self.device)
        if df:
            o["trace"] = t.empty((nb, 3), dtype=t.float64, device=self.device)
            o["gcv"] = t.empty((nb, R), dtype=t.float64, device=self.device)
        return o

    def _struct(self, o) -> Outputs:
        s = Outputs()
        for k in ("mhat_grid", "mask", "moments", "mhat_at_x", "rss", "trace", "gcv"):
            setattr(s, k, o[k].data_ptr() if k in o else None)
        return s

    def _need(self, a, count: int, what: str):
        """The C call reads ``count`` values of ``a``: refuse a smaller tensor,
        which the device would read past its end."""
        if a.numel() < count:
            raise FkregError(f"INVALID_ARG: {what} holds {a.numel()} values where the call "
                             f"reads {count}")

    def _y(self, y):
        y = self._as_dev(y, complex_ok=self.y_complex)
        if self.y_complex and y.dim() == 2:      # [n, 2] from a 1-D complex vector
            y = y.unsqueeze(0)
        if not self.y_complex and y.dim() == 1:
            y = y.unsqueeze(0)
        self._need(y, self.n_rhs * self.n * (2 if self.y_complex else 1),
                   "y ([n_rhs, n] responses)")
        return y.contiguous()

    def _probes(self, probes, n_probes: int):
        if probes is None:
            return None
        pr = self._as_dev(probes)
        self._need(pr, max(int(n_probes), 0) * self.n, "probes ([n_probes, n])")
        return pr

    def _mhat_at_x(self, mhat_at_x, complex_ok: bool):
        mh = self._as_dev(mhat_at_x, complex_ok=complex_ok)
        self._need(mh, self.n_bw * self.n_rhs * self.n * (2 if self.y_complex else 1),
                   "mhat_at_x ([n_bw, n_rhs, n])")
        return mh

    def smooth(self, y, want=("mhat_grid", "mask")) -> Dict[str, object]:
        y = self._y(y)
        o = self._outputs(want, df=False)
        s = self._struct(o)
        self._check(self.L.fkreg_smooth(self.h, ctypes.c_void_p(y.data_ptr()), ctypes.byref(s),
                                        self._stream()))
        self._y_keep = y
        return o

    def df(self, y, n_probes: int, seed: int = 0, probes=None,
           want=("mhat_grid", "mask")) -> Dict[str, object]:
        y = self._y(y)
        pr = self._probes(probes, n_probes)
        o = self._outputs(want, df=True)
        s = self._struct(o)
        self._check(self.L.fkreg_df(self.h, ctypes.c_void_p(y.data_ptr()), int(n_probes),
                                    ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF),
                                    None if pr is None else ctypes.c_void_p(pr.data_ptr()),
                                    ctypes.byref(s), self._stream()))
        self._y_keep = (y, pr)
        return o

    def backward(self, y, n_probes: int, seed: int = 0, probes=None, b: int = 0,
                 want=("dlogh", "dy", "dx")) -> Dict[str, object]:
        """GCV of bandwidth b and its gradient (fkreg_backward)."""
        t = self.torch
        y = self._y(y)
        pr = self._probes(probes, n_probes)
        n = max(self.n, 1)
        out = {"gcv": t.empty(1, dtype=t.float64, device=self.device)}
        if "dlogh" in want:
            out["dlogh"] = t.empty(self.d, dtype=t.float64, device=self.device)
        if "dy" in want:
            out["dy"] = t.empty(n, dtype=self.dtype, device=self.device)
        if "dx" in want:
            out["dx"] = t.empty((n, self.d), dtype=self.dtype, device=self.device)
        ptr = lambda k: ctypes.c_void_p(out[k].data_ptr()) if k in out else None
        self._check(getattr(self.L, self._fn_backward)(self.h, ctypes.c_void_p(y.data_ptr()), int(n_probes),
                                          ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF),
                                          None if pr is None else ctypes.c_void_p(pr.data_ptr()),
                                          int(b), ptr("gcv"), ptr("dlogh"), ptr("dy"), ptr("dx"),
                                          self._stream()))
        self._y_keep = (y, pr)
        return out

    def backward_grid(self, y, grad_mhat, b: int = 0, want=("dlogh", "dy", "dx")) -> Dict[str, object]:
        """Gradients of L = sum grad_mhat * mhat_grid (bandwidth b) with respect to
        log sigma [d], y [n_rhs, n] and x [n, d] (fkreg_backward_grid)."""
        t = self.torch
        y = self._y(y)
        gm = self._as_dev(grad_mhat).reshape(self.n_rhs, self.M).contiguous()
        n = max(self.n, 1)
        out = {}
        if "dlogh" in want:
            out["dlogh"] = t.empty(self.d, dtype=t.float64, device=self.device)
        if "dy" in want:
            out["dy"] = t.empty((self.n_rhs, n), dtype=self.dtype, device=self.device)
        if "dx" in want:
            out["dx"] = t.empty((n, self.d), dtype=self.dtype, device=self.device)
        ptr = lambda k: ctypes.c_void_p(out[k].data_ptr()) if k in out else None
        self._check(self.L.fkreg_backward_grid(self.h, ctypes.c_void_p(y.data_ptr()),
                                               ctypes.c_void_p(gm.data_ptr()), int(b),
                                               ptr("dlogh"), ptr("dy"), ptr("dx"), self._stream()))
        self._y_keep = (y, gm)
        return out

    def variance(self, y, mhat_at_x):
        t = self.torch
        y = self._y(y)
        mh = self._mhat_at_x(mhat_at_x, complex_ok=self.y_complex)
        out = t.empty((self.n_bw, self.n_rhs) + self.grid_n, dtype=self.dtype, device=self.device)
        self._check(self.L.fkreg_variance(self.h, ctypes.c_void_p(y.data_ptr()),
                                          ctypes.c_void_p(mh.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), self._stream()))
        self._y_keep = (y, mh)
        return out

    def log_variance(self, y, mhat_at_x, want_sigma2=True):
        """Log-variance estimator (eqs. 24-26): v on the grid and at the samples,
        kappa per bandwidth and response, and sigma^2 = exp(v) / kappa on the grid."""
        t = self.torch
        y = self._y(y)
        mh = self._mhat_at_x(mhat_at_x, complex_ok=False)
        v_grid = t.empty((self.n_bw, self.n_rhs) + self.grid_n, dtype=self.dtype, device=self.device)
        v_x = t.empty((self.n_bw, self.n_rhs, self.n), dtype=self.dtype, device=self.device)
        kappa = t.empty((self.n_bw, self.n_rhs), dtype=t.float64, device=self.device)
        s2 = (t.empty((self.n_bw, self.n_rhs) + self.grid_n, dtype=self.dtype, device=self.device)
              if want_sigma2 else None)
        self._check(getattr(self.L, self._fn_log_variance)(
            self.h, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(mh.data_ptr()),
            ctypes.c_void_p(v_grid.data_ptr()), ctypes.c_void_p(v_x.data_ptr()),
            ctypes.c_void_p(kappa.data_ptr()),
            ctypes.c_void_p(s2.data_ptr() if s2 is not None else 0), self._stream()))
        self._y_keep = (y, mh)
        out = {"v_grid": v_grid, "v_at_x": v_x, "kappa": kappa}
        if s2 is not None:
            out["sigma2"] = s2
        return out


def bandwidth_list(n, ranges, spacing: str = "log") -> np.ndarray:
    """Candidate bandwidths (Sec. 4, get_hList) as the H matrices a plan takes.

    ``n`` is the number of candidates per axis (an int, or one per axis),
    ``ranges`` the (lo, hi) standard-deviation range per axis, ``spacing``
    "log" (lo to hi evenly in log10, both ends included) or "lin".  One axis
    gives sigma values; several axes give every combination (axis 0 varies
    slowest), each as H = diag(sigma^2).  Returns [n_bw, d, d] float64.
    """
    rng = np.asarray(ranges, dtype=np.float64).reshape(-1, 2)
    d = rng.shape[0]
    counts = [int(n)] * d if np.ndim(n) == 0 else [int(v) for v in n]
    if len(counts) != d or min(counts) < 1 or np.any(rng <= 0) or np.any(rng[:, 1] < rng[:, 0]):
        raise FkregError("bandwidth_list: one count >= 1 and one 0 < lo <= hi range per axis")
    axes = []
    for (lo, hi), k in zip(rng, counts):
        if spacing == "log":
            e = np.linspace(np.log10(lo), np.log10(hi), k) if k > 1 else np.array([np.log10(lo)])
            axes.append(np.power(10.0, e))
        elif spacing == "lin":
            axes.append(np.linspace(lo, hi, k) if k > 1 else np.array([lo]))
        else:
            raise FkregError(f"bandwidth_list: unknown spacing {spacing!r}")
    mesh = np.meshgrid(*axes, indexing="ij")
    sig = np.stack([m.reshape(-1) for m in mesh], axis=1)          # [n_bw, d]
    H = np.zeros((sig.shape[0], d, d))
    for j in range(d):
        H[:, j, j] = sig[:, j] ** 2
    return H


def select_bandwidth(gcv, dstd: float = 0.0) -> int:
    """Index of the chosen candidate (Table 1's dstd rule, with the GCV values
    of a candidate list in increasing bandwidth order): the last candidate
    whose GCV is at most min GCV + dstd * std(GCV); dstd = 0 is the argmin,
    ties going to the later candidate.  NaN values are ignored."""
    g = np.asarray(gcv, dtype=np.float64).reshape(-1)
    ok = np.isfinite(g)
    if not ok.any():
        raise FkregError("select_bandwidth: no finite GCV value")
    lim = np.min(g[ok]) + (dstd * float(np.std(g[ok])) if dstd else 0.0)
    return int(np.nonzero(ok & (g <= lim))[0].max())


def cv_fkreg(x, y, hlist, grid_n, lo=None, hi=None, order: int = 1, n_probes: int = 10,
             dstd: float = 0.0, seed: int = 0, precision: str = "f32", tol=None,
             kernel: str = "gaussian", variance: bool = False, standardize: bool = False,
             device=None) -> Dict[str, object]:
    """Bandwidth selection and smoothing in one call (Sec. 4's cv_fkreg).

    x: [n, d] (or [n] for d = 1) sample locations; y: [n] or [R, n] responses
    (complex for complex responses); hlist: [n_bw, d, d] candidate H (see
    ``bandwidth_list``); grid_n: grid points per axis; lo/hi: the grid's
    box, by default the samples' extent.  One plan holds every candidate:
    the samples are sorted once and ``df`` returns every candidate's GCV
    (eq. 22, Girard probes drawn on the device from ``seed``).  The
    candidate is chosen on the first response's GCV by ``select_bandwidth``
    with ``dstd``.  Returns a dict: "index", "H" [d, d], "gcv" [n_bw],
    "trace" [n_bw, 3] (Girard, Hutchinson, exact), "mhat_grid" [R, *grid],
    "mask" [*grid], "mhat_at_x" [R, n], and with ``variance`` "sigma2"
    [R, *grid] (eq. 23) of the chosen candidate; "plan" is the plan.
    With ``standardize`` (the toolbox's convention, Sec. 4) every axis of x,
    lo and hi is divided by the samples' standard deviation (N - 1
    normalisation) and hlist is read on that scale; "H" is then the chosen
    candidate on the standardised scale and "H_original" = S H S with
    S = diag(std) on the samples' own scale.
    """
    import torch
    xt = torch.as_tensor(x)
    if xt.is_complex():          # complex locations: the points (Re z, Im z)
        xt = torch.view_as_real(xt.reshape(-1))
    if xt.dim() == 1:
        xt = xt.reshape(-1, 1)
    n, d = int(xt.shape[0]), int(xt.shape[1])
    xh = xt.detach().to("cpu", torch.float64).numpy()
    sd = np.ones(d)
    if standardize:
        # divide in FP64, then round to x's own type; the default box is the
        # extent of those rounded values and a given box is divided likewise
        # and widened to hold them, so no sample falls outside the box that
        # the device compares against in its own precision
        sd = xh.std(axis=0, ddof=1) if n > 1 else np.ones(d)
        sd = np.where(sd > 0, sd, 1.0)
        xs = torch.as_tensor(xh / sd).to(xt.dtype)
        xh = xs.numpy().astype(np.float64)
        xt = xs.to(xt.device)
        if lo is not None:
            lo = np.minimum(np.atleast_1d(np.asarray(lo, dtype=np.float64)) / sd, xh.min(axis=0))
        if hi is not None:
            hi = np.maximum(np.atleast_1d(np.asarray(hi, dtype=np.float64)) / sd, xh.max(axis=0))
    lo = [float(v) for v in (xh.min(axis=0) if lo is None else np.atleast_1d(lo))]
    hi = [float(v) for v in (xh.max(axis=0) if hi is None else np.atleast_1d(hi))]
    hi = [h if h > l else l + 1.0 for l, h in zip(lo, hi)]
    H = np.asarray(hlist, dtype=np.float64).reshape(-1, d, d)
    yt = torch.as_tensor(y)
    if yt.dim() == 1:
        yt = yt.reshape(1, -1)
    R = int(yt.shape[0])
    cplx = bool(yt.is_complex())
    if tol is None:
        tol = 1e-6 if precision == "f32" else 1e-12
    grid_n = [int(v) for v in np.atleast_1d(grid_n)]
    if len(grid_n) == 1 and d > 1:
        grid_n = grid_n * d
    plan = Plan(d, order, grid_n, lo, hi, H, max_n=max(n, 1), n_rhs=R, max_probes=n_probes,
                tol=tol, precision=precision, y_complex=cplx, device=device, kernel=kernel)
    plan.set_points(xt)
    out = plan.df(yt, n_probes, seed=seed, want=("mhat_grid", "mask", "mhat_at_x"))
    gcv = out["gcv"][:, 0].detach().cpu().numpy()
    k = select_bandwidth(gcv, dstd)
    res = {"index": k, "H": H[k], "H_original": np.diag(sd) @ H[k] @ np.diag(sd), "gcv": gcv,
           "trace": out["trace"].detach().cpu().numpy(),
           "mhat_grid": out["mhat_grid"][k], "mask": out["mask"][k],
           "mhat_at_x": out["mhat_at_x"][k], "plan": plan}
    if variance:
        res["sigma2"] = plan.variance(yt, out["mhat_at_x"])[k]
    plan.sync()
    return res


class _PlanCache:
    """The plan of the last differentiable call, reused while its options (the
    bandwidth included: a plan's H is fixed) and sample count stay the same."""

    def __init__(self):
        self.key, self.plan = None, None

    def get(self, key, make):
        if self.key != key:
            self.plan, self.key = make(), key
        return self.plan


_GCV_PLANS = _PlanCache()
_GRID_PLANS = _PlanCache()


def gcv(x, y, log_sigma, grid_n, lo, hi, order: int = 1, n_probes: int = 10, seed: int = 0,
        precision: str = "f32", tol=None, device=None):
    """GCV (eq. 22) of one diagonal bandwidth H = diag(exp(2 log_sigma)) as a
    differentiable torch function of the samples x [n, d], the responses
    y [n] and log_sigma [d]: ``fkreg_backward`` computes the value and the
    three gradients in one call (Monte-Carlo trace of Sec. 2.1 with probes
    drawn from ``seed``, held fixed), and autograd chains them.  A plan is
    built for each new bandwidth (a plan's H is fixed) and reused while the
    bandwidth and the problem's shape stay the same.
    """
    import torch

    class _GCV(torch.autograd.Function):
        @staticmethod
        def forward(ctx, xx, yy, ls):
            d = int(xx.shape[1])
            sig = torch.exp(ls.detach().to("cpu", torch.float64)).numpy()
            H = np.diag(sig * sig).reshape(1, d, d)
            t = tol if tol is not None else (1e-6 if precision == "f32" else 1e-12)
            n = max(int(xx.shape[0]), 1)
            key = (d, order, tuple(grid_n), tuple(lo), tuple(hi), tuple(sig.tolist()), n,
                   n_probes, precision, t, str(device))
            plan = _GCV_PLANS.get(key, lambda: Plan(
                d, order, grid_n, lo, hi, H, max_n=n, n_rhs=1, max_probes=n_probes, tol=t,
                precision=precision, flags=FKREG_WANT_BACKWARD, device=device))
            plan.set_points(xx.detach())
            out = plan.backward(yy.detach(), n_probes, seed=seed, b=0)
            plan.sync()
            ctx.save_for_backward(out["dx"].to(xx.device, xx.dtype),
                                  out["dy"].to(yy.device, yy.dtype),
                                  out["dlogh"].to(ls.device, ls.dtype))
            return out["gcv"][0].to(ls.device, ls.dtype)

        @staticmethod
        def backward(ctx, g):
            dx, dy, dl = ctx.saved_tensors
            return g * dx, g * dy, g * dl

    xt = torch.as_tensor(x)
    if xt.dim() == 1:
        xt = xt.reshape(-1, 1)
    return _GCV.apply(xt, torch.as_tensor(y).reshape(-1), torch.as_tensor(log_sigma).reshape(-1))


def smooth_grid(x, y, log_sigma, grid_n, lo, hi, order: int = 1, precision: str = "f64",
                tol=None, mask_rho: float = 0.0, device=None):
    """The grid estimate of eq. 11 as a differentiable torch function of the
    samples x [n, d], the responses y ([n] or [R, n]) and log_sigma [d]
    (H = diag(exp(2 log_sigma))): returns mhat [R, *grid_n] (NaN where masked).
    The backward is ``fkreg_backward_grid``: the adjoints of the per-grid-point
    solves, the adjoint of the inverse grid transform and a type-2 evaluation
    at the samples, and a spectral inner product for log sigma; masked points
    and non-finite incoming gradients contribute nothing.  A plan is built for
    each new bandwidth and reused while it and the problem's shape stay the
    same.
    """
    import torch

    class _Smooth(torch.autograd.Function):
        @staticmethod
        def forward(ctx, xx, yy, ls):
            d = int(xx.shape[1])
            R = int(yy.shape[0])
            sig = torch.exp(ls.detach().to("cpu", torch.float64)).numpy()
            H = np.diag(sig * sig).reshape(1, d, d)
            t = tol if tol is not None else (1e-6 if precision == "f32" else 1e-12)
            n = max(int(xx.shape[0]), 1)
            key = (d, order, tuple(grid_n), tuple(lo), tuple(hi), tuple(sig.tolist()), n, R,
                   precision, t, mask_rho, str(device))
            plan = _GRID_PLANS.get(key, lambda: Plan(
                d, order, grid_n, lo, hi, H, max_n=n, n_rhs=R, tol=t, precision=precision,
                mask_rho=mask_rho, flags=FKREG_WANT_BACKWARD, device=device))
            plan.set_points(xx.detach())
            out = plan.smooth(yy.detach(), want=("mhat_grid",))
            plan.sync()
            ctx.plan = plan
            ctx.save_for_backward(xx, yy, ls)
            return out["mhat_grid"][0].to(yy.device, yy.dtype)

        @staticmethod
        def backward(ctx, g):
            xx, yy, ls = ctx.saved_tensors
            plan = ctx.plan
            plan.set_points(xx.detach())
            r = plan.backward_grid(yy.detach(), torch.nan_to_num(g.detach(), nan=0.0), b=0)
            plan.sync()
            return (r["dx"][: xx.shape[0]].to(xx.device, xx.dtype).reshape(xx.shape),
                    r["dy"][:, : yy.shape[1]].to(yy.device, yy.dtype).reshape(yy.shape),
                    r["dlogh"].to(ls.device, ls.dtype))

    xt = torch.as_tensor(x)
    if xt.dim() == 1:
        xt = xt.reshape(-1, 1)
    yt = torch.as_tensor(y)
    if yt.dim() == 1:
        yt = yt.reshape(1, -1)
    return _Smooth.apply(xt, yt, torch.as_tensor(log_sigma).reshape(-1))


def interval(mhat, var, alpha: float = 0.05):
    """Pointwise interval of eq. 28 on device tensors of one dtype (float32 or
    float64): returns (lower, upper) = mhat -/+ z_(1-alpha/2) sqrt(var)."""
    import torch
    L = load()
    if not (mhat.is_cuda and mhat.dtype in (torch.float32, torch.float64)):
        raise FkregError("interval: mhat must be a float32 or float64 CUDA tensor")
    m = mhat.contiguous()
    v = torch.as_tensor(var).to(device=m.device, dtype=m.dtype).contiguous()
    if v.shape != m.shape:
        v = v.expand(m.shape).contiguous()
    lo, hi = torch.empty_like(m), torch.empty_like(m)
    prec = FKREG_F32 if m.dtype == torch.float32 else FKREG_F64
    st = L.fkreg_interval(prec, m.numel(), ctypes.c_void_p(m.data_ptr()),
                          ctypes.c_void_p(v.data_ptr()), float(alpha),
                          ctypes.c_void_p(lo.data_ptr()), ctypes.c_void_p(hi.data_ptr()),
                          ctypes.c_void_p(torch.cuda.current_stream(m.device).cuda_stream))
    if st != 0:
        raise FkregError(f"fkreg_interval: {STATUS.get(st, st)}")
    return lo, hi


def predict(grid, grid_n, lo, hi, xq, method: str = "linear"):
    """Values of grid estimates at new points (device tensors).

    grid: [..., M_1..M_d] float32 or float64 on the GPU (leading dims
    flattened into count); xq: [nq, d] points, taken to the grid's device and
    dtype.  method "linear" or "cubic".  Returns [..., nq].
    """
    import torch
    L = load()
    if method not in ("linear", "cubic"):
        raise FkregError(f"predict: unknown method {method!r} ('linear' or 'cubic')")
    d = len(grid_n)
    if xq.is_complex():  # complex new points on a 2-D grid: (Re z, Im z)
        if d != 2:
            raise FkregError("complex points need a 2-D grid")
        xq = torch.view_as_real(xq.reshape(-1))
    if not (grid.is_cuda and grid.dtype in (torch.float32, torch.float64)):
        raise FkregError("predict: grid must be a float32 or float64 CUDA tensor")
    lead = grid.shape[: grid.dim() - d]
    g = grid.reshape(-1, *grid_n).contiguous()
    # the points go to the grid's device: the kernel reads both by pointer
    x = xq.to(device=g.device, dtype=g.dtype).reshape(-1, d).contiguous()
    out = torch.empty((g.shape[0], x.shape[0]), dtype=g.dtype, device=g.device)
    gn = (ctypes.c_int64 * d)(*[int(v) for v in grid_n])
    glo = (ctypes.c_double * d)(*[float(v) for v in lo])
    ghi = (ctypes.c_double * d)(*[float(v) for v in hi])
    prec = FKREG_F32 if g.dtype == torch.float32 else FKREG_F64
    st = L.fkreg_predict(prec, d, gn, glo, ghi, g.shape[0], ctypes.c_void_p(g.data_ptr()),
                         x.shape[0], ctypes.c_void_p(x.data_ptr()),
                         0 if method == "linear" else 1, ctypes.c_void_p(out.data_ptr()),
                         ctypes.c_void_p(torch.cuda.current_stream(g.device).cuda_stream))
    if st != 0:
        raise FkregError(f"fkreg_predict: {STATUS.get(st, st)}")
    return out.reshape(*lead, x.shape[0])


class StepGraph:
    """A sequence of plan calls captured once as a CUDA graph.

    ``fn()`` issues the calls on the current stream and returns their
    outputs.  It runs ``warmup`` times on a side stream, then once under
    capture; ``replay()`` re-issues every kernel, copy and FFT of the
    sequence with one launch, reading the same input buffers (copy new data
    into them before a replay) and writing the tensors ``fn`` returned at
    capture (``outputs``).  Stage timing must be off during capture.  Seeds
    given to the captured calls are fixed at capture.
    """

    def __init__(self, fn, warmup: int = 2):
        import torch
        self.torch = torch
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(warmup):
                fn()
        torch.cuda.current_stream().wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.outputs = fn()

    def replay(self):
        self.graph.replay()


class Sweep(Plan):
    """A bandwidth sweep with one Fourier period per group of bandwidths
    (fkreg_sweep_*): the bandwidth list split into contiguous groups, one
    plan per group, run one after another.  ``max_groups=1`` is one plan.
    Methods and output layouts as for Plan (set_points, smooth, df,
    variance); ``groups`` gives the split."""

    def __init__(self, d: int, order: int, grid_n, lo, hi, H, max_n: int, n_rhs: int = 1,
                 max_probes: int = 0, tol: float = 1e-6, precision: str = "f32",
                 y_complex: bool = False, spread_kernel: str = "es", mask_rho: float = 0.0,
                 tile: int = 0, flags: int = 0, device=None, max_groups: int = 2):
        import torch
        self.torch = torch
        self.L = load()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.d, self.order, self.n_rhs = d, order, n_rhs
        self.grid_n = tuple(int(v) for v in grid_n)
        self.M = int(np.prod(self.grid_n))
        self.max_probes = max_probes
        self.precision = precision
        self.y_complex = bool(y_complex)
        self.dtype = torch.float32 if precision == "f32" else torch.float64
        self.cdtype = torch.complex64 if precision == "f32" else torch.complex128
        self._opts, self._keep = make_opts(d, order, grid_n, lo, hi, H, n_rhs, max_probes, tol,
                                           precision, y_complex, spread_kernel, mask_rho, tile,
                                           flags, "gaussian")
        self.n_bw = self._opts.n_bw
        g = Geometry()
        self._check_global(self.L.fkreg_geometry_query(ctypes.byref(self._opts), ctypes.byref(g)))
        self.geom = g.as_dict()
        self.ns, self.nt = g.ns, g.nt
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            self._check_global(self.L.fkreg_sweep_create(ctypes.byref(self._opts), int(max_n),
                                                         int(max_groups), ctypes.byref(h)))
        self.h = h
        nbytes = ctypes.c_size_t()
        self._check(self.L.fkreg_sweep_workspace_bytes(self.h, ctypes.byref(nbytes)))
        self.ws_bytes = int(nbytes.value)
        self._ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
        self._ws_ptr = (self._ws.data_ptr() + 255) // 256 * 256
        self._check(self.L.fkreg_sweep_set_workspace(self.h, ctypes.c_void_p(self._ws_ptr),
                                                     self.ws_bytes, self._stream()))
        self.n = 0

    def _check(self, st):
        if st != 0:
            raise FkregError(f"{STATUS.get(st, st)}: {self.L.fkreg_sweep_last_error(self.h).decode()}")

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.L.fkreg_sweep_destroy(self.h)
            self.h = ctypes.c_void_p()

    def groups(self, with_kernels: bool = False):
        """(first bandwidth of each group + [n_bw], geometry dict per group),
        and with ``with_kernels`` each group's kernel name after them."""
        ng = ctypes.c_int()
        self._check(self.L.fkreg_sweep_groups(self.h, ctypes.byref(ng), None, None, None))
        first = (ctypes.c_int * (ng.value + 1))()
        kern = (ctypes.c_int * ng.value)()
        geoms = (Geometry * ng.value)()
        self._check(self.L.fkreg_sweep_groups(self.h, ctypes.byref(ng), first, kern, geoms))
        out = (list(first), [gg.as_dict() for gg in geoms])
        if with_kernels:
            out = out + ([KERNEL_NAMES[k] for k in kern],)
        return out

    def set_points(self, x):
        x = self._as_dev(x)
        n = self._sample_count(x)
        self._x = x
        self._check(self.L.fkreg_sweep_set_points(self.h, n, ctypes.c_void_p(x.data_ptr()),
                                                  self._stream()))
        self.n = n

    def sync(self):
        self._check(self.L.fkreg_sweep_sync_status(self.h, self._stream()))

    def set_timing(self, enable: bool = True):
        self._check(self.L.fkreg_sweep_set_timing(self.h, int(bool(enable))))

    def stage_times(self):
        n = len(STAGES)
        ms = (ctypes.c_double * n)()
        calls = (ctypes.c_int64 * n)()
        kl = ctypes.c_int64()
        self._check(self.L.fkreg_sweep_stage_times(self.h, ms, calls, ctypes.byref(kl)))
        return ({STAGES[i]: ms[i] for i in range(n)}, {STAGES[i]: calls[i] for i in range(n)},
                int(kl.value))

    def smooth(self, y, want=("mhat_grid", "mask")) -> Dict[str, object]:
        y = self._y(y)
        o = self._outputs(want, df=False)
        s = self._struct(o)
        self._check(self.L.fkreg_sweep_smooth(self.h, ctypes.c_void_p(y.data_ptr()),
                                              ctypes.byref(s), self._stream()))
        self._y_keep = y
        return o

    def df(self, y, n_probes: int, seed: int = 0, probes=None,
           want=("mhat_grid", "mask")) -> Dict[str, object]:
        y = self._y(y)
        pr = self._probes(probes, n_probes)
        o = self._outputs(want, df=True)
        s = self._struct(o)
        self._check(self.L.fkreg_sweep_df(self.h, ctypes.c_void_p(y.data_ptr()), int(n_probes),
                                          ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF),
                                          None if pr is None else ctypes.c_void_p(pr.data_ptr()),
                                          ctypes.byref(s), self._stream()))
        self._y_keep = (y, pr)
        return o

    def variance(self, y, mhat_at_x):
        t = self.torch
        y = self._y(y)
        mh = self._mhat_at_x(mhat_at_x, complex_ok=self.y_complex)
        out = t.empty((self.n_bw, self.n_rhs) + self.grid_n, dtype=self.dtype, device=self.device)
        self._check(self.L.fkreg_sweep_variance(self.h, ctypes.c_void_p(y.data_ptr()),
                                                ctypes.c_void_p(mh.data_ptr()),
                                                ctypes.c_void_p(out.data_ptr()), self._stream()))
        self._y_keep = (y, mh)
        return out

    _fn_backward = "fkreg_sweep_backward"
    _fn_log_variance = "fkreg_sweep_log_variance"

    def _unsupported(self, *a, **k):
        raise FkregError("UNSUPPORTED: a sweep offers set_points, smooth, df, variance, "
                         "log_variance and backward")

    backward_grid = get_sort = set_wait_limit = _unsupported


class Batch:
    """Independent problems replayed as one captured CUDA graph.

    ``problems`` is a list of dicts with the keyword arguments of
    :func:`make_opts` plus ``max_n``.  ``capture`` records, per problem, the
    bin sort, the smoothing (grid estimate + values at the samples) and the
    conditional-variance pass; ``launch`` replays it; ``latencies`` returns
    each problem's completion time (ms) after the start of the last launch.
    """

    def __init__(self, problems, device=None):
        import torch
        self.torch = torch
        self.L = load()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.problems = [dict(p) for p in problems]
        n = len(problems)
        self._opts = (Opts * n)()
        self._keep = []
        maxn = (ctypes.c_int64 * n)()
        for i, p in enumerate(problems):
            kw = {k: v for k, v in p.items() if k != "max_n"}
            o, keep = make_opts(**kw)
            self._opts[i] = o
            self._keep.append(keep)
            maxn[i] = int(p["max_n"])
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = self.L.fkreg_batch_create(n, self._opts, maxn, ctypes.byref(h))
        if st != 0:
            raise FkregError(f"{STATUS.get(st, st)}: {self.L.fkreg_global_error().decode()}")
        self.h = h
        nb = ctypes.c_size_t()
        self.L.fkreg_batch_workspace_bytes(self.h, ctypes.byref(nb))
        self._ws = torch.empty(int(nb.value) + 256, dtype=torch.uint8, device=self.device)
        self._ws_ptr = (self._ws.data_ptr() + 255) // 256 * 256
        self._check(self.L.fkreg_batch_set_workspace(
            self.h, ctypes.c_void_p(self._ws_ptr), int(nb.value),
            ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)))

    def _check(self, st):
        if st != 0:
            raise FkregError(f"{STATUS.get(st, st)}: {self.L.fkreg_batch_last_error(self.h).decode()}")

    def capture(self, xs, ys, variance=True):
        """Record the batch; xs, ys are device tensors per problem (kept alive)."""
        t = self.torch
        n = len(self.problems)
        xs, ys = list(xs), list(ys)
        if len(xs) != n or len(ys) != n:
            raise FkregError(f"INVALID_ARG: {n} problems, {len(xs)} sample and {len(ys)} "
                             "response tensors")
        self._inputs = (xs, ys)
        outs = []
        arr_out = (Outputs * n)()
        nn = (ctypes.c_int64 * n)()
        px = (ctypes.c_void_p * n)()
        py = (ctypes.c_void_p * n)()
        ps2 = (ctypes.c_void_p * n)()
        for i, p in enumerate(self.problems):
            d = p["d"]
            cplx = bool(p.get("y_complex", False))
            prec = p.get("precision", "f32")
            dt = t.float32 if prec == "f32" else t.float64
            cdt = t.complex64 if prec == "f32" else t.complex128
            grid = tuple(int(v) for v in p["grid_n"])
            nbw = np.asarray(p["H"]).reshape(-1, d, d).shape[0]
            x = xs[i]
            ni = int(x.shape[0])
            # the recorded kernels read these pointers by size alone: each
            # tensor must live on the batch's device, in the problem's
            # precision, contiguous and at least as large as the call reads
            for name, a, count in (("x", x, ni * d), ("y", ys[i], ni * (2 if cplx else 1))):
                real = t.view_as_real(a) if a.is_complex() else a
                other = (a.device.type != self.device.type or (
                    self.device.index is not None and a.device.index != self.device.index))
                if (other or real.dtype != dt or not a.is_contiguous()
                        or real.numel() < count or (name == "x" and x.dim() == 2
                                                    and int(x.shape[1]) != d)):
                    raise FkregError(f"INVALID_ARG: problem {i}: {name} must be a contiguous "
                                     f"{dt} tensor on {self.device} with at least {count} "
                                     f"values (got {tuple(a.shape)} {a.dtype} on {a.device})")
            o = {"mhat_grid": t.empty((nbw, 1) + grid, dtype=cdt if cplx else dt, device=self.device),
                 "mask": t.empty((nbw,) + grid, dtype=t.uint8, device=self.device),
                 "mhat_at_x": t.empty((nbw, 1, max(ni, 1)), dtype=cdt if cplx else dt,
                                      device=self.device)}
            if variance:
                o["sigma2"] = t.empty((nbw, 1) + grid, dtype=dt, device=self.device)
            outs.append(o)
            s = Outputs()
            s.mhat_grid = o["mhat_grid"].data_ptr()
            s.mask = o["mask"].data_ptr()
            s.mhat_at_x = o["mhat_at_x"].data_ptr()
            arr_out[i] = s
            nn[i] = ni
            px[i] = x.data_ptr()
            py[i] = ys[i].data_ptr()
            ps2[i] = o["sigma2"].data_ptr() if variance else None
        self.outs = outs
        self._check(self.L.fkreg_batch_capture(
            self.h, nn, px, py, arr_out, ps2,
            ctypes.c_void_p(t.cuda.current_stream(self.device).cuda_stream)))
        return outs

    def launch(self):
        self._check(self.L.fkreg_batch_launch(
            self.h, ctypes.c_void_p(self.torch.cuda.current_stream(self.device).cuda_stream)))

    def latencies(self) -> np.ndarray:
        n = len(self.problems)
        ms = (ctypes.c_double * n)()
        self._check(self.L.fkreg_batch_latencies(
            self.h, ms, ctypes.c_void_p(self.torch.cuda.current_stream(self.device).cuda_stream)))
        return np.array(ms[:])

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.L.fkreg_batch_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune_tile(problem: dict, x, y, candidates=None, reps: int = 3) -> int:
    """Pick the spreading tile for one problem by timing fkreg_set_points +
    fkreg_smooth (grid estimate and values at the samples) for each candidate
    tile with CUDA events; returns the fastest.  ``problem`` holds the keyword
    arguments of :class:`Plan` (including ``max_n``)."""
    import torch
    d = problem["d"]
    if candidates is None:
        candidates = {1: (512, 1024, 2048, 4096), 2: (8, 16, 32), 3: (4, 8, 16)}[d]
    best, best_t = None, None
    for tile in candidates:
        kw = dict(problem)
        kw["tile"] = tile
        try:
            p = Plan(**kw)
        except FkregError:
            continue
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(1):
            p.set_points(x)
            p.smooth(y, want=("mhat_grid", "mhat_at_x"))
        ev0.record()
        for _ in range(reps):
            p.set_points(x)
            p.smooth(y, want=("mhat_grid", "mhat_at_x"))
        ev1.record()
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1) / reps
        p.close()
        if best_t is None or ms < best_t:
            best, best_t = tile, ms
    return int(best) if best is not None else 0
