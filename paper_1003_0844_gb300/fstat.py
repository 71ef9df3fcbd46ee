"""Python binding of the C ABI in include/fstat.h (argument marshalling only).

Every computation runs in the CUDA library libfstat.so built in-tree by
``paper_1003_0844_gb300.build``; nothing here computes on the CPU.  Device
arrays are torch tensors; the current torch CUDA stream is passed to the
library unless a stream is given.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import weakref

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfstat.so")

FS_OK = 0
STATUS = {0: "FS_OK", 1: "FS_ERR_ARG", 2: "FS_ERR_SHAPE", 3: "FS_ERR_CAPACITY", 4: "FS_ERR_NONFINITE",
          5: "FS_ERR_CUDA", 6: "FS_ERR_TIMEOUT", 7: "FS_ERR_UNSUPPORTED", 8: "FS_ERR_NOMEM", 9: "FS_ERR_SCRATCH",
          10: "FS_ERR_CORRUPT"}
PREC = {"f32": 0, "f64": 1}
INTERP = {"spline": 0, "nearest": 1}
EXPORTS = ["fs_create", "fs_destroy", "fs_prepare_segment", "fs_prepare_segment_eph", "fs_seg_destroy", "fs_seg_load", "fs_search",
           "fs_sync_status", "fs_strerror", "fs_seg_upsampled", "fs_demodulate", "fs_inject", "fs_set_profiling",
           "fs_get_stats", "fs_search_noalloc", "fs_search_batch", "fs_set_tuning", "fs_get_tuning", "fs_autotune",
           "fs_fstat_points", "fs_refine", "fs_points_from_candidates", "fs_amplitudes", "fs_false_alarm_cell",
           "fs_fstat_resampled", "fs_fstat_resampled_grad", "fs_refine_resampled",
           "fs_false_alarm", "fs_threshold", "fs_cell_count", "fs_linear_model_fisher", "fs_lattice",
           "fs_lattice_nodes", "fs_lattice_templates", "fs_search_lattice", "fs_search_lattice_noalloc",
           "fs_search_lattice_batch", "fs_selftest_wait"]
PROF_KINDS = ("prepare", "demodulate", "pass1", "pass2", "other")


class FstatError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__("%s failed: %s (%d)" % (what, STATUS.get(status, "?"), status))
        self.status = status


class _Detector(ctypes.Structure):
    _fields_ = [("lat", ctypes.c_double), ("lon", ctypes.c_double), ("gamma", ctypes.c_double),
                ("eps", ctypes.c_double), ("lambda_e0", ctypes.c_double), ("theta_g0", ctypes.c_double)]


class _SegDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nfft", ctypes.c_int64), ("dt", ctypes.c_double), ("fl", ctypes.c_double),
                ("S0", ctypes.c_double), ("precision", ctypes.c_int32), ("interp", ctypes.c_int32),
                ("x_dtype", ctypes.c_int32), ("options", ctypes.c_int32), ("t0", ctypes.c_double)]


class _Tuning(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_int32), ("queue_round", ctypes.c_int32), ("queue_lag", ctypes.c_int32),
                ("group_skies", ctypes.c_int32), ("ms_per_template", ctypes.c_float), ("reserved", ctypes.c_int32)]


class _Stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("ms", ctypes.c_double * 5), ("count", ctypes.c_int64 * 5),
                ("workspace_bytes", ctypes.c_int64)]


class _Injection(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("f0", "f1", "alpha", "delta", "psi", "cos_iota", "phi0", "snr")]


_lib = None


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load libfstat.so (built by paper_1003_0844_gb300.build, or the file named by
    the FSTAT_LIB environment variable); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("FSTAT_LIB") or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libfstat.so is not built (%s); run paper_1003_0844_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    vp, i32, i64, f32, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double
    lib.fs_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_Detector), i32]
    lib.fs_destroy.argtypes = [vp]
    lib.fs_destroy.restype = None
    lib.fs_prepare_segment.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(_SegDesc), vp, vp]
    lib.fs_prepare_segment_eph.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(_SegDesc), vp, vp, vp, vp]
    lib.fs_seg_destroy.argtypes = [vp]
    lib.fs_seg_destroy.restype = None
    lib.fs_seg_load.argtypes = [vp, vp, vp]
    lib.fs_set_profiling.argtypes = [vp, i32]
    lib.fs_get_stats.argtypes = [vp, ctypes.POINTER(_Stats), i32]
    lib.fs_search.argtypes = [vp, vp, vp, vp, i32, vp, i32, f32, vp, i64, vp, i64, vp, vp]
    lib.fs_search_noalloc.argtypes = [vp, vp, vp, vp, i32, vp, i32, f32, vp, i64, vp, i64, vp, vp]
    lib.fs_sync_status.argtypes = [vp, vp]
    lib.fs_strerror.argtypes = [ctypes.c_int]
    lib.fs_strerror.restype = ctypes.c_char_p
    lib.fs_seg_upsampled.argtypes = [vp, vp, vp]
    lib.fs_demodulate.argtypes = [vp, vp, f64, f64, vp, vp, vp, vp, vp]
    lib.fs_inject.argtypes = [vp, vp, i64, f64, f64, f64, f64, ctypes.POINTER(_Injection), i32, vp]
    lib.fs_search_batch.argtypes = [vp, ctypes.POINTER(vp), i32, vp, vp, i32, vp, i32, f32, vp, i64, vp, vp]
    pv, pi = ctypes.POINTER(vp), ctypes.POINTER(i32)
    lib.fs_search_lattice_batch.argtypes = [vp, pv, i32, pv, pv, pi, pv, pv, pi, f32, vp, i64, vp, vp]
    lib.fs_set_tuning.argtypes = [vp, i64, ctypes.POINTER(_Tuning)]
    lib.fs_get_tuning.argtypes = [vp, i64, ctypes.POINTER(_Tuning)]
    lib.fs_autotune.argtypes = [vp, vp, vp, vp, i32, vp, i32, i32, ctypes.POINTER(_Tuning), vp]
    lib.fs_fstat_points.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp, vp]
    lib.fs_refine.argtypes = [vp, vp, vp, i32, i32, vp, vp]
    lib.fs_fstat_resampled.argtypes = [vp, vp, vp, i32, vp, vp]
    lib.fs_fstat_resampled_grad.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp]
    lib.fs_refine_resampled.argtypes = [vp, vp, vp, i32, i32, vp, vp]
    lib.fs_points_from_candidates.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp, vp]
    lib.fs_amplitudes.argtypes = [vp, vp, vp, i32, vp, vp]
    lib.fs_false_alarm_cell.argtypes = [f64]
    lib.fs_false_alarm_cell.restype = f64
    lib.fs_false_alarm.argtypes = [f64, f64, ctypes.POINTER(f64), ctypes.POINTER(f64)]
    lib.fs_threshold.argtypes = [f64, f64, ctypes.POINTER(f64)]
    lib.fs_cell_count.argtypes = [i32, ctypes.POINTER(f64), f64, ctypes.POINTER(f64)]
    lib.fs_linear_model_fisher.argtypes = [ctypes.POINTER(_Detector), i64, f64, f64, ctypes.POINTER(f64)]
    lib.fs_lattice.argtypes = [i32, ctypes.POINTER(f64), f64, f64, i32, ctypes.POINTER(f64), ctypes.POINTER(f64)]
    lib.fs_lattice_nodes.argtypes = [ctypes.POINTER(f64), ctypes.POINTER(_Detector), f64, f64, f64, f64, f64, vp,
                                     i64, ctypes.POINTER(i64)]
    lib.fs_lattice_templates.argtypes = [ctypes.POINTER(f64), ctypes.POINTER(_Detector), f64, i64, f64, f64, f64,
                                         vp, vp, vp, vp, vp, i64, i32, ctypes.POINTER(i64), ctypes.POINTER(i32)]
    lib.fs_search_lattice.argtypes = [vp, vp, vp, vp, i32, vp, vp, i32, f32, vp, i64, vp, i64, vp, vp]
    lib.fs_search_lattice_noalloc.argtypes = [vp, vp, vp, vp, i32, vp, vp, i32, f32, vp, i64, vp, i64, vp, vp]
    lib.fs_selftest_wait.argtypes = [vp, vp]
    for name in ("fs_create", "fs_prepare_segment", "fs_prepare_segment_eph", "fs_seg_load", "fs_search", "fs_search_noalloc", "fs_sync_status",
                 "fs_seg_upsampled", "fs_demodulate", "fs_inject", "fs_set_profiling", "fs_get_stats",
                 "fs_search_batch", "fs_set_tuning", "fs_get_tuning", "fs_autotune", "fs_fstat_points", "fs_refine",
                 "fs_points_from_candidates", "fs_amplitudes", "fs_false_alarm", "fs_threshold", "fs_cell_count",
                 "fs_linear_model_fisher", "fs_lattice", "fs_lattice_nodes", "fs_lattice_templates",
                 "fs_search_lattice", "fs_search_lattice_noalloc", "fs_search_lattice_batch",
                 "fs_selftest_wait", "fs_fstat_resampled", "fs_fstat_resampled_grad", "fs_refine_resampled"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int, what: str):
    if status != FS_OK:
        raise FstatError(status, what)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def _need_cuda(t: torch.Tensor, name: str, dtype=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise ValueError("%s must be %s" % (name, dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)


class Context:
    """A library context on one CUDA device for one detector (fs_create)."""

    def __init__(self, det, device: int = 0):
        self.lib = load_library()
        d = _Detector(det.lat, det.lon, det.gamma, det.eps, det.lambda_e0, det.theta_g0)
        h = ctypes.c_void_p()
        _check(self.lib.fs_create(ctypes.byref(h), ctypes.byref(d), int(device)), "fs_create")
        self.handle = h
        self.device = device
        self._segments = weakref.WeakSet()

    def close(self):
        """Release the context; fs_destroy also releases its segments still alive."""
        if self.handle:
            for sg in list(self._segments):
                sg.handle = None
            self.lib.fs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync_status(self, stream=None) -> int:
        return self.lib.fs_sync_status(self.handle, _stream(stream))

    def selftest_wait(self, stream=None):
        """fs_selftest_wait: one bounded wait that runs out (status via sync_status)."""
        _check(self.lib.fs_selftest_wait(self.handle, _stream(stream)), "fs_selftest_wait")

    def check(self, stream=None):
        _check(self.sync_status(stream), "device status")

    def set_profiling(self, on: bool):
        _check(self.lib.fs_set_profiling(self.handle, 1 if on else 0), "fs_set_profiling")

    def stats(self, reset: bool = True) -> dict:
        """Launch count, the bytes held by the context's workspaces and, with
        profiling on, summed event time / launches per kind."""
        st = _Stats()
        _check(self.lib.fs_get_stats(self.handle, ctypes.byref(st), 1 if reset else 0), "fs_get_stats")
        return {"launches": st.launches, "workspace_bytes": st.workspace_bytes,
                "ms": {k: st.ms[i] for i, k in enumerate(PROF_KINDS)},
                "count": {k: st.count[i] for i, k in enumerate(PROF_KINDS)}}

    def set_tuning(self, nfft: int, n1: int = 0, queue_round: int = 0, queue_lag: int = 0, group_skies: int = 0):
        """Launch configuration for transforms of length nfft (fs_set_tuning)."""
        t = _Tuning(int(n1), int(queue_round), int(queue_lag), int(group_skies), 0.0, 0)
        _check(self.lib.fs_set_tuning(self.handle, int(nfft), ctypes.byref(t)), "fs_set_tuning")

    def clear_tuning(self, nfft: int):
        _check(self.lib.fs_set_tuning(self.handle, int(nfft), None), "fs_set_tuning")

    def get_tuning(self, nfft: int) -> dict | None:
        t = _Tuning()
        st = self.lib.fs_get_tuning(self.handle, int(nfft), ctypes.byref(t))
        if st == 7:
            return None
        _check(st, "fs_get_tuning")
        return _tuning_dict(t)

    def autotune(self, seg: "Segment", alpha: torch.Tensor, delta: torch.Tensor, f1: torch.Tensor, reps: int = 3,
                 stream=None) -> dict:
        """Time the candidate configurations on this grid and keep the fastest (fs_autotune)."""
        for t, nm in ((alpha, "alpha"), (delta, "delta"), (f1, "f1")):
            _need_cuda(t, nm, torch.float64)
        out = _Tuning()
        _check(self.lib.fs_autotune(self.handle, seg.handle, _ptr(alpha), _ptr(delta), alpha.numel(), _ptr(f1),
                                    f1.numel(), int(reps), ctypes.byref(out), _stream(stream)), "fs_autotune")
        return _tuning_dict(out)


def _tuning_dict(t) -> dict:
    return {"n1": t.n1, "queue_round": t.queue_round, "queue_lag": t.queue_lag, "group_skies": t.group_skies,
            "ms_per_template": t.ms_per_template}


class Segment:
    """One prepared data segment (fs_prepare_segment): tables, x2 upsampling, spline.

    eph: None for the analytic Earth, else (r, v), device float64 tensors of shape
    (3, n): the detector's SSB position r_d(t_m)/c [light-seconds] and velocity
    v_d(t_m)/c at t_m = m dt, ecliptic axes (fs_prepare_segment_eph)."""

    def __init__(self, ctx: Context, x: torch.Tensor, dt: float, nfft: int, fl: float, S0: float,
                 precision: str = "f32", interp: str = "spline", t0: float = 0.0, interbin: bool = False,
                 eph=None, stream=None):
        _need_cuda(x, "x")
        if x.dtype not in (torch.float32, torch.float64):
            raise ValueError("x must be float32 or float64")
        self.ctx = ctx
        self.n = x.numel()
        self.nfft = int(nfft)
        self.dt, self.fl, self.S0 = float(dt), float(fl), float(S0)
        self.precision = precision
        self.t0 = float(t0)
        self.interbin = bool(interbin)
        d = _SegDesc(self.n, self.nfft, self.dt, self.fl, self.S0, PREC[precision], INTERP[interp],
                     0 if x.dtype == torch.float32 else 1, 1 if interbin else 0, self.t0)
        h = ctypes.c_void_p()
        if eph is None:
            _check(ctx.lib.fs_prepare_segment(ctx.handle, ctypes.byref(h), ctypes.byref(d), _ptr(x),
                                              _stream(stream)), "fs_prepare_segment")
        else:
            r, v = eph
            for t, nm in ((r, "r"), (v, "v")):
                _need_cuda(t, nm, torch.float64)
                if tuple(t.shape) != (3, self.n) or not t.is_contiguous():
                    raise ValueError("%s must be a contiguous (3, %d) tensor" % (nm, self.n))
            _check(ctx.lib.fs_prepare_segment_eph(ctx.handle, ctypes.byref(h), ctypes.byref(d), _ptr(x), _ptr(r),
                                                  _ptr(v), _stream(stream)), "fs_prepare_segment_eph")
        self.eph = eph is not None
        self.handle = h
        ctx._segments.add(self)

    def close(self):
        # a segment whose context is gone was released with it (fs_destroy)
        if self.handle and self.ctx.handle:
            self.ctx.lib.fs_seg_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, x: torch.Tensor, stream=None):
        """Re-run the preparation on new data of the same shape (fs_seg_load, no allocation)."""
        _need_cuda(x, "x")
        if x.numel() != self.n:
            raise ValueError("x has %d samples, the segment %d" % (x.numel(), self.n))
        _check(self.ctx.lib.fs_seg_load(self.handle, _ptr(x), _stream(stream)), "fs_seg_load")

    def upsampled(self, stream=None) -> torch.Tensor:
        out = torch.empty(2 * self.n, dtype=torch.float64, device="cuda")
        _check(self.ctx.lib.fs_seg_upsampled(self.handle, _ptr(out), _stream(stream)), "fs_seg_upsampled")
        return out


@dataclasses.dataclass
class SearchResult:
    F: torch.Tensor | None         # [nsky*nspin, nbins] or None
    cand: torch.Tensor             # int32 [cap, 4]: sky, spin, bin, F bits
    n_cand: torch.Tensor           # int64 [1] on the device

    def candidates(self):
        """(sky, spin, bin, F) numpy arrays of the stored candidates (synchronises)."""
        n = int(self.n_cand.item())
        n = min(n, self.cand.shape[0])
        c = self.cand[:n].cpu()
        F = c[:, 3].view(torch.float32).numpy().copy()
        u = c[:, :3].numpy().astype("int64")
        return u[:, 0], u[:, 1], u[:, 2], F


def search(ctx: Context, seg: Segment, alpha: torch.Tensor, delta: torch.Tensor, f1: torch.Tensor,
           F_thr: float, write_F: bool = True, nbins: int | None = None, cand_cap: int = 1 << 16,
           F_out: torch.Tensor | None = None, cand: torch.Tensor | None = None,
           n_cand: torch.Tensor | None = None, stream=None) -> SearchResult:
    """fs_search over len(alpha) x len(f1) templates; returns device tensors."""
    for t, nm in ((alpha, "alpha"), (delta, "delta"), (f1, "f1")):
        _need_cuda(t, nm, torch.float64)
    nsky, nspin = alpha.numel(), f1.numel()
    if delta.numel() != nsky:
        raise ValueError("alpha and delta differ in length")
    nb = (seg.nfft if seg.interbin else seg.nfft // 2) if nbins is None else int(nbins)
    fdt = torch.float32 if seg.precision == "f32" else torch.float64
    if write_F and F_out is None:
        F_out = torch.empty((nsky * nspin, nb), dtype=fdt, device="cuda")
    if not write_F:
        F_out = None
    if cand is None:
        cand = torch.empty((max(cand_cap, 1), 4), dtype=torch.int32, device="cuda")
    if n_cand is None:
        n_cand = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = ctx.lib.fs_search(ctx.handle, seg.handle, _ptr(alpha), _ptr(delta), nsky, _ptr(f1), nspin,
                           float(F_thr), _ptr(F_out) if F_out is not None else None, nb, _ptr(cand),
                           int(cand.shape[0]) if cand_cap > 0 else 0, _ptr(n_cand), _stream(stream))
    _check(st, "fs_search")
    return SearchResult(F_out, cand, n_cand)


@dataclasses.dataclass
class BatchResult:
    cand: torch.Tensor             # int32 [nseg, cap, 4]: sky, spin, bin, F bits per segment
    n_cand: torch.Tensor           # int64 [nseg] on the device

    def candidates(self, s: int):
        """(sky, spin, bin, F) numpy arrays of segment s's stored candidates (synchronises)."""
        n = min(int(self.n_cand[s].item()), self.cand.shape[1])
        c = self.cand[s, :n].cpu()
        F = c[:, 3].view(torch.float32).numpy().copy()
        u = c[:, :3].numpy().astype("int64")
        return u[:, 0], u[:, 1], u[:, 2], F


def search_batch(ctx: Context, segs, alpha: torch.Tensor, delta: torch.Tensor, f1: torch.Tensor, F_thr: float,
                 cand_cap: int = 1 << 14, cand: torch.Tensor | None = None, n_cand: torch.Tensor | None = None,
                 stream=None) -> BatchResult:
    """fs_search_batch: the same grid over every segment of `segs`, candidates only."""
    for t, nm in ((alpha, "alpha"), (delta, "delta"), (f1, "f1")):
        _need_cuda(t, nm, torch.float64)
    nsky, nspin, nseg = alpha.numel(), f1.numel(), len(segs)
    if delta.numel() != nsky:
        raise ValueError("alpha and delta differ in length")
    if cand is None:
        cand = torch.empty((nseg, max(cand_cap, 1), 4), dtype=torch.int32, device="cuda")
    if n_cand is None:
        n_cand = torch.zeros(nseg, dtype=torch.int64, device="cuda")
    handles = (ctypes.c_void_p * nseg)(*[sg.handle.value for sg in segs])
    st = ctx.lib.fs_search_batch(ctx.handle, handles, nseg, _ptr(alpha), _ptr(delta), nsky, _ptr(f1), nspin,
                                 float(F_thr), _ptr(cand), int(cand.shape[1]) if cand_cap > 0 else 0, _ptr(n_cand),
                                 _stream(stream))
    _check(st, "fs_search_batch")
    return BatchResult(cand, n_cand)


def search_lattice_batch(ctx: Context, segs, templates, F_thr: float, cand_cap: int = 1 << 14,
                         cand: torch.Tensor | None = None, n_cand: torch.Tensor | None = None,
                         stream=None) -> BatchResult:
    """fs_search_lattice_batch: segment s searches its own lattice templates[s] =
    (alpha, delta, f1, offset), device float64 tensors with alpha, delta [nsky] and
    f1, offset [nsky, nspin] (as for search_lattice); candidates only."""
    nseg = len(segs)
    if len(templates) != nseg:
        raise ValueError("one template set per segment expected")
    for a, d, f, o in templates:
        for t, nm in ((a, "alpha"), (d, "delta"), (f, "f1"), (o, "offset")):
            _need_cuda(t, nm, torch.float64)
        if d.numel() != a.numel() or f.dim() != 2 or f.shape[0] != a.numel() or tuple(o.shape) != tuple(f.shape):
            raise ValueError("alpha, delta [nsky] and f1, offset [nsky, nspin] expected")
    if cand is None:
        cand = torch.empty((nseg, max(cand_cap, 1), 4), dtype=torch.int32, device="cuda")
    if n_cand is None:
        n_cand = torch.zeros(nseg, dtype=torch.int64, device="cuda")
    P, I = ctypes.c_void_p * nseg, ctypes.c_int32 * nseg
    handles = P(*[sg.handle.value for sg in segs])
    ptrs = [P(*[t[k].data_ptr() for t in templates]) for k in range(4)]
    nsky = I(*[t[0].numel() for t in templates])
    nspin = I(*[t[2].shape[1] for t in templates])
    st = ctx.lib.fs_search_lattice_batch(ctx.handle, handles, nseg, ptrs[0], ptrs[1], nsky, ptrs[2], ptrs[3], nspin,
                                         float(F_thr), _ptr(cand), int(cand.shape[1]) if cand_cap > 0 else 0,
                                         _ptr(n_cand), _stream(stream))
    _check(st, "fs_search_lattice_batch")
    return BatchResult(cand, n_cand)


# ---- fine search: points are float64 CUDA tensors [npt, 4] = (f0, f1, alpha, delta)

def fstat_points(ctx: Context, seg: Segment, pts: torch.Tensor, grad: bool = True, metric: bool = False,
                 hess: bool = False, stream=None):
    """Exact F at continuous points (fs_fstat_points): (F [npt], dF [npt, 4] or None,
    reduced Fisher matrix upper triangles [npt, 10] or None) and, with hess=True, a
    fourth value: the Hessian upper triangles [npt, 10]."""
    _need_cuda(pts, "pts", torch.float64)
    if pts.dim() != 2 or pts.shape[1] != 4:
        raise ValueError("pts must have shape [npt, 4]")
    npt = pts.shape[0]
    F = torch.empty(npt, dtype=torch.float64, device=pts.device)
    g = torch.empty((npt, 4), dtype=torch.float64, device=pts.device) if grad else None
    m = torch.empty((npt, 10), dtype=torch.float64, device=pts.device) if metric else None
    h = torch.empty((npt, 10), dtype=torch.float64, device=pts.device) if hess else None
    _check(ctx.lib.fs_fstat_points(ctx.handle, seg.handle, _ptr(pts), npt, _ptr(F), _ptr(g) if grad else None,
                                   _ptr(h) if hess else None, _ptr(m) if metric else None, _stream(stream)),
           "fs_fstat_points")
    return (F, g, m, h) if hess else (F, g, m)


class FstatAt(torch.autograd.Function):
    """F(pts) as a differentiable function of the points: forward and backward both
    come from one fs_fstat_points call (the gradient is kept for the backward)."""

    @staticmethod
    def forward(fctx, pts, ctx, seg):
        F, g, _ = fstat_points(ctx, seg, pts.detach().contiguous(), grad=True)
        fctx.save_for_backward(g)
        return F

    @staticmethod
    def backward(fctx, gF):
        (g,) = fctx.saved_tensors
        return gF[:, None] * g, None, None


def fstat_at(ctx: Context, seg: Segment, pts: torch.Tensor) -> torch.Tensor:
    """Differentiable exact F at the points (see FstatAt)."""
    return FstatAt.apply(pts, ctx, seg)


def fstat_resampled(ctx: Context, seg: Segment, pts: torch.Tensor, stream=None) -> torch.Tensor:
    """The coarse search's F at continuous points (fs_fstat_resampled): F [npt]."""
    _need_cuda(pts, "pts", torch.float64)
    if pts.dim() != 2 or pts.shape[1] != 4:
        raise ValueError("pts must have shape [npt, 4]")
    pts = pts.contiguous()
    F = torch.empty(pts.shape[0], dtype=torch.float64, device=pts.device)
    _check(ctx.lib.fs_fstat_resampled(ctx.handle, seg.handle, _ptr(pts), pts.shape[0], _ptr(F), _stream(stream)),
           "fs_fstat_resampled")
    return F


def fstat_resampled_grad(ctx: Context, seg: Segment, pts: torch.Tensor, gF: torch.Tensor = None, stream=None):
    """The backward call (fs_fstat_resampled_grad): (F [npt], gF dF/dpts [npt, 4]);
    gF None for ones."""
    _need_cuda(pts, "pts", torch.float64)
    if pts.dim() != 2 or pts.shape[1] != 4:
        raise ValueError("pts must have shape [npt, 4]")
    pts = pts.contiguous()
    npt = pts.shape[0]
    if gF is not None:
        _need_cuda(gF, "gF", torch.float64)
        if gF.shape != (npt,):
            raise ValueError("gF must have shape [npt]")
        gF = gF.contiguous()
    F = torch.empty(npt, dtype=torch.float64, device=pts.device)
    g = torch.empty((npt, 4), dtype=torch.float64, device=pts.device)
    _check(ctx.lib.fs_fstat_resampled_grad(ctx.handle, seg.handle, _ptr(pts), npt, _ptr(gF) if gF is not None else None,
                                           _ptr(F), _ptr(g), _stream(stream)), "fs_fstat_resampled_grad")
    return F, g


class FstatResampled(torch.autograd.Function):
    """The coarse search's F at the points as a differentiable function: the forward
    call keeps only the points; the backward call recomputes the resampled series
    and returns gF dF/dpts (the adjoint kernel)."""

    @staticmethod
    def forward(fctx, pts, ctx, seg):
        pts = pts.detach().contiguous()
        fctx.save_for_backward(pts)
        fctx.handles = (ctx, seg)
        return fstat_resampled(ctx, seg, pts)

    @staticmethod
    def backward(fctx, gF):
        (pts,) = fctx.saved_tensors
        ctx, seg = fctx.handles
        _, g = fstat_resampled_grad(ctx, seg, pts, gF.detach().to(torch.float64).contiguous())
        return g, None, None


def fstat_resampled_at(ctx: Context, seg: Segment, pts: torch.Tensor) -> torch.Tensor:
    """Differentiable coarse-search F at the points (see FstatResampled)."""
    return FstatResampled.apply(pts, ctx, seg)


def refine_resampled(ctx: Context, seg: Segment, pts: torch.Tensor, nsteps: int = 20, stream=None):
    """Gradient ascent of the coarse search's F from each point (fs_refine_resampled):
    returns (refined points, F)."""
    _need_cuda(pts, "pts", torch.float64)
    out = pts.clone().contiguous()
    F = torch.empty(out.shape[0], dtype=torch.float64, device=out.device)
    _check(ctx.lib.fs_refine_resampled(ctx.handle, seg.handle, _ptr(out), out.shape[0], int(nsteps), _ptr(F),
                                       _stream(stream)), "fs_refine_resampled")
    return out, F


def refine(ctx: Context, seg: Segment, pts: torch.Tensor, nsteps: int = 20, stream=None):
    """Fine search from each point (fs_refine): returns (refined points, F)."""
    _need_cuda(pts, "pts", torch.float64)
    out = pts.clone().contiguous()
    F = torch.empty(out.shape[0], dtype=torch.float64, device=out.device)
    _check(ctx.lib.fs_refine(ctx.handle, seg.handle, _ptr(out), out.shape[0], int(nsteps), _ptr(F),
                             _stream(stream)), "fs_refine")
    return out, F


def points_from_candidates(ctx: Context, seg: Segment, cand: torch.Tensor, n: int, alpha: torch.Tensor,
                           delta: torch.Tensor, f1: torch.Tensor, stream=None) -> torch.Tensor:
    """Starting points of the fine search from the first n candidates (int32 [>=n, 4])."""
    pts = torch.empty((n, 4), dtype=torch.float64, device=cand.device)
    _check(ctx.lib.fs_points_from_candidates(ctx.handle, seg.handle, _ptr(cand), int(n), _ptr(alpha), _ptr(delta),
                                             _ptr(f1), _ptr(pts), _stream(stream)), "fs_points_from_candidates")
    return pts


def amplitudes(ctx: Context, seg: Segment, pts: torch.Tensor, stream=None) -> torch.Tensor:
    """ML amplitude estimators A1..A4 at the points (fs_amplitudes): float64 [npt, 4]."""
    _need_cuda(pts, "pts", torch.float64)
    amp = torch.empty((pts.shape[0], 4), dtype=torch.float64, device=pts.device)
    _check(ctx.lib.fs_amplitudes(ctx.handle, seg.handle, _ptr(pts), pts.shape[0], _ptr(amp), _stream(stream)),
           "fs_amplitudes")
    return amp


def false_alarm(F0: float, n_cells: float):
    """(alpha, expected false alarms) of threshold F0 over n_cells cells (fs_false_alarm)."""
    lib = load_library()
    a, nf = ctypes.c_double(), ctypes.c_double()
    _check(lib.fs_false_alarm(float(F0), float(n_cells), ctypes.byref(a), ctypes.byref(nf)), "fs_false_alarm")
    return a.value, nf.value


def threshold(alpha: float, n_cells: float) -> float:
    """Threshold F0 of false-alarm probability alpha over n_cells cells (fs_threshold)."""
    lib = load_library()
    F0 = ctypes.c_double()
    _check(lib.fs_threshold(float(alpha), float(n_cells), ctypes.byref(F0)), "fs_threshold")
    return F0.value


def cell_count(G, v_total: float) -> float:
    """Number of cells of volume v_total for the reduced Fisher matrix G (fs_cell_count)."""
    import numpy as np
    g = np.ascontiguousarray(np.asarray(G, dtype=np.float64))
    lib = load_library()
    n = ctypes.c_double()
    _check(lib.fs_cell_count(int(g.shape[0]), g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(v_total),
                             ctypes.byref(n)), "fs_cell_count")
    return n.value


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def linear_model_fisher(det, n: int, dt: float, t0: float = 0.0):
    """Reduced Fisher matrix of the linear phase model (fs_linear_model_fisher), 4 x 4."""
    import numpy as np
    lib = load_library()
    d = _Detector(det.lat, det.lon, det.gamma, det.eps, det.lambda_e0, det.theta_g0)
    G = np.empty(16)
    _check(lib.fs_linear_model_fisher(ctypes.byref(d), int(n), float(dt), float(t0), _dptr(G)),
           "fs_linear_model_fisher")
    return G.reshape(4, 4)


def lattice(G, C0: float, dp0: float, constraint2: bool = True):
    """Constrained lattice covering (fs_lattice): (basis rows, thickness)."""
    import numpy as np
    lib = load_library()
    g = np.ascontiguousarray(np.asarray(G, dtype=np.float64))
    dim = g.shape[0]
    B = np.empty(dim * dim)
    th = ctypes.c_double()
    _check(lib.fs_lattice(dim, _dptr(g), float(C0), float(dp0), 1 if constraint2 else 0, _dptr(B), ctypes.byref(th)),
           "fs_lattice")
    return B.reshape(dim, dim), th.value


def lattice_nodes(basis, det, fl: float, f0_range, f1_range, cap: int = 1 << 20):
    """Template points (f0, f1, alpha, delta) of the lattice in a band (fs_lattice_nodes)."""
    import numpy as np
    lib = load_library()
    b = np.ascontiguousarray(np.asarray(basis, dtype=np.float64))
    d = _Detector(det.lat, det.lon, det.gamma, det.eps, det.lambda_e0, det.theta_g0)
    pts = np.empty((cap, 4))
    cnt = ctypes.c_int64()
    st = lib.fs_lattice_nodes(_dptr(b), ctypes.byref(d), float(fl), float(f0_range[0]), float(f0_range[1]),
                              float(f1_range[0]), float(f1_range[1]), pts.ctypes.data_as(ctypes.c_void_p), int(cap),
                              ctypes.byref(cnt))
    _check(st, "fs_lattice_nodes")
    return pts[:cnt.value].copy()


def lattice_templates(basis, det, fl: float, nfft: int, dt: float, f1_range, box=None):
    """Templates of the FFT search of the lattice (fs_lattice_templates): numpy arrays
    alpha [nsky], delta [nsky], f1 [nsky, nspin], bin offset [nsky, nspin]."""
    import numpy as np
    lib = load_library()
    b = np.ascontiguousarray(np.asarray(basis, dtype=np.float64))
    d = _Detector(det.lat, det.lon, det.gamma, det.eps, det.lambda_e0, det.theta_g0)
    bx = None if box is None else np.ascontiguousarray(np.asarray(box, dtype=np.float64))
    ns, nm = ctypes.c_int64(), ctypes.c_int32()
    args = (_dptr(b), ctypes.byref(d), float(fl), int(nfft), float(dt), float(f1_range[0]), float(f1_range[1]),
            bx.ctypes.data_as(ctypes.c_void_p) if bx is not None else None)
    _check(lib.fs_lattice_templates(*args, None, None, None, None, 0, 0, ctypes.byref(ns), ctypes.byref(nm)),
           "fs_lattice_templates")
    a, de = np.empty(ns.value), np.empty(ns.value)
    f1, off = np.empty((ns.value, nm.value)), np.empty((ns.value, nm.value))
    vpp = lambda x: x.ctypes.data_as(ctypes.c_void_p)
    _check(lib.fs_lattice_templates(*args, vpp(a), vpp(de), vpp(f1), vpp(off), ns.value, nm.value, ctypes.byref(ns),
                                    ctypes.byref(nm)), "fs_lattice_templates")
    return a, de, f1, off


def search_lattice(ctx: Context, seg: Segment, alpha: torch.Tensor, delta: torch.Tensor, f1: torch.Tensor,
                   offset: torch.Tensor, F_thr: float, write_F: bool = True, cand_cap: int = 1 << 16,
                   F_out: torch.Tensor | None = None, cand: torch.Tensor | None = None,
                   n_cand: torch.Tensor | None = None, stream=None) -> SearchResult:
    """fs_search_lattice: sky s and row m have spindown f1[s, m] and F at the bins
    k + offset[s, m] (device float64 [nsky, nspin] each); returns device tensors
    (F_out, cand, n_cand are allocated unless given, as for search)."""
    for t, nm in ((alpha, "alpha"), (delta, "delta"), (f1, "f1"), (offset, "offset")):
        _need_cuda(t, nm, torch.float64)
    nsky = alpha.numel()
    if delta.numel() != nsky or f1.dim() != 2 or f1.shape[0] != nsky or tuple(offset.shape) != tuple(f1.shape):
        raise ValueError("alpha, delta [nsky] and f1, offset [nsky, nspin] expected")
    nspin = f1.shape[1]
    nb = seg.nfft // 2
    if write_F and F_out is None:
        fdt = torch.float32 if seg.precision == "f32" else torch.float64
        F_out = torch.empty((nsky * nspin, nb), dtype=fdt, device="cuda")
    if not write_F:
        F_out = None
    if cand is None:
        cand = torch.empty((max(cand_cap, 1), 4), dtype=torch.int32, device="cuda")
    if n_cand is None:
        n_cand = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = ctx.lib.fs_search_lattice(ctx.handle, seg.handle, _ptr(alpha), _ptr(delta), nsky, _ptr(f1), _ptr(offset),
                                   nspin, float(F_thr), _ptr(F_out) if F_out is not None else None, nb, _ptr(cand),
                                   int(cand.shape[0]) if cand_cap > 0 else 0, _ptr(n_cand), _stream(stream))
    _check(st, "fs_search_lattice")
    return SearchResult(F_out, cand, n_cand)


def demodulate(ctx: Context, seg: Segment, alpha: float, delta: float, stream=None):
    """Per-sky resampled, demodulated series (fs_demodulate) as device tensors:
    (y^a complex128 [n], y^b complex128 [n], t_src float64 [n], (<a^2>, <b^2>))."""
    n = seg.n
    ya = torch.empty(2 * n, dtype=torch.float64, device="cuda")
    yb = torch.empty(2 * n, dtype=torch.float64, device="cuda")
    ts = torch.empty(n, dtype=torch.float64, device="cuda")
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    _check(ctx.lib.fs_demodulate(ctx.handle, seg.handle, float(alpha), float(delta), _ptr(ya), _ptr(yb), _ptr(ts),
                                 _ptr(ab), _stream(stream)), "fs_demodulate")
    return torch.view_as_complex(ya.view(n, 2)), torch.view_as_complex(yb.view(n, 2)), ts, ab


def inject(ctx: Context, x: torch.Tensor, dt: float, fl: float, sigma: float, injections, t0: float = 0.0,
           stream=None):
    """Add simulated signals (fs_inject) to the float64 CUDA tensor x in place; t0 is the
    epoch of the first sample (as for a Segment)."""
    _need_cuda(x, "x", torch.float64)
    arr = (_Injection * max(len(injections), 1))()
    for i, j in enumerate(injections):
        arr[i] = _Injection(j.f0, j.f1, j.alpha, j.delta, j.psi, j.cos_iota, j.phi0, j.snr)
    _check(ctx.lib.fs_inject(ctx.handle, _ptr(x), x.numel(), float(dt), float(fl), float(sigma), float(t0), arr,
                             len(injections), _stream(stream)), "fs_inject")
    return x
