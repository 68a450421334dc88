"""Python binding of libkfscan (include/kfscan.h): temporally parallel Kalman
filtering and smoothing as all-prefix-sums (arXiv 2511.10363) on GB300.

Argument marshalling only: every step of the computation runs in the CUDA
library.  PyTorch supplies device memory and streams.  The binding refuses
to run if the compiled library is missing; there is no CPU fallback.

Function names match the C ABI:
    kf_filter, kf_rts_smooth, kf_two_filter_smooth,
    kf_tv_filter, kf_tv_rts_smooth, kf_tv_two_filter_smooth (time-varying models),
    kf_workspace_size, kf_sync_status, kf_set_option, kf_get_option,
    kf_status_string, kf_version.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
# KFSCAN_LIB selects another build of the library (the bounds-checked one)
LIB_PATH = os.environ.get("KFSCAN_LIB") or _build.LIB

# enums of kfscan.h
SCANS = {"auto": 0, "dlb": 1, "decoupled_lookback": 1, "hillis_steele": 2, "hs": 2,
         "blelloch": 3, "ladner_fischer": 4, "lafi": 4, "sengupta": 5}
PRECISIONS = {"fp64": 0, "fp32": 1, "fp32_fp64solve": 2, "mixed": 2}
OPS = {"filter": 0, "rts": 1, "two_filter": 2, "tf": 2}
STATUS = {0: "KF_OK", 1: "KF_ERR_ARG", 2: "KF_ERR_NOT_PD", 3: "KF_ERR_CUDA", 4: "KF_ERR_OOM",
          5: "KF_ERR_TIMEOUT", 6: "KF_ERR_BUDGET", 7: "KF_ERR_BUSY", 8: "KF_ERR_CAPACITY",
          9: "KF_ERR_CANCELLED", 10: "KF_ERR_BOUNDS"}
OPTIONS = {"wait_timeout_ns": 0, "test_skip_tile": 1, "positions_per_thread": 2, "threads": 3, "general_solve": 4,
           "lookback_warps": 5, "sengupta_n": 6, "filter_kernel": 7,
           "rts_kernel": 8, "covariance_tables": 9, "call_graphs": 10}

_lib = None


class KfError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = int(status)
        super().__init__("%s%s (%d: %s)" % (where + ": " if where else "", STATUS.get(self.status, "?"),
                                             self.status, kf_status_string(self.status)))


class _Model(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int)] + [
        (k, ctypes.POINTER(ctypes.c_double)) for k in ("F", "Q", "H", "R", "m0", "P0")]


class _TvModel(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int)] + [
        (k, ctypes.c_void_p) for k in ("F", "Q", "u", "H", "R", "d")] + [
        (k, ctypes.POINTER(ctypes.c_double)) for k in ("m0", "P0")]


def lib():
    """The loaded library.  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libkfscan.so is not built: run paper_2511_10363_gb300.build.build() "
                               "(or __graft_entry__.build()) first")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        MP = ctypes.POINTER(_Model)
        L.kf_filter.argtypes = [MP, i64, vp, i, i, vp, vp, vp, vp, vp]
        L.kf_rts_smooth.argtypes = [MP, i64, vp, i, i, vp, vp, vp, vp, vp, vp, vp]
        L.kf_two_filter_smooth.argtypes = [MP, i64, vp, i, i, vp, vp, vp, vp, vp, vp, vp]
        for f in ("kf_filter", "kf_rts_smooth", "kf_two_filter_smooth", "kf_sync_status", "kf_set_option"):
            getattr(L, f).restype = ctypes.c_int
        L.kf_sync_status.argtypes = [vp]
        L.kf_set_option.argtypes = [i, i64]
        L.kf_get_option.argtypes = [i]
        L.kf_get_option.restype = i64
        L.kf_workspace_size.argtypes = [i, i, i, i64, i, i]
        L.kf_workspace_size.restype = ctypes.c_size_t
        L.kf_status_string.argtypes = [i]
        L.kf_status_string.restype = ctypes.c_char_p
        L.kf_version.restype = ctypes.c_char_p
        for f in ("kf_timing_enable", "kf_timing_reset", "kf_timing_read", "kf_measure_fma_peak"):
            getattr(L, f).restype = ctypes.c_int
        L.kf_timing_enable.argtypes = [i]
        L.kf_timing_read.argtypes = [i, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]
        L.kf_measure_fma_peak.argtypes = [i, ctypes.POINTER(ctypes.c_double)]
        L.kf_trace_phases.argtypes = [i, vp, i]
        L.kf_autotune.argtypes = [i, MP, i64, vp, i, vp, vp, i, vp, vp]
        IP = ctypes.POINTER(ctypes.c_int)
        L.kf_tuning_get.argtypes = [i, i, i, i, i64, IP, IP, IP, IP, ctypes.POINTER(ctypes.c_double)]
        L.kf_tuning_save.argtypes = [ctypes.c_char_p]
        L.kf_tuning_load.argtypes = [ctypes.c_char_p]
        L.kf_autotune_batch.argtypes = [i, MP, i, vp, i, vp, vp, i, vp, vp, i, vp, vp]
        L.kf_batch_tuning_get.argtypes = [i, i, i, i, i64, IP, IP, ctypes.POINTER(ctypes.c_double)]
        L.kf_last_launch_config.argtypes = [IP, IP, IP, IP]
        DP = ctypes.POINTER(ctypes.c_double)
        L.kf_covariance_tables.argtypes = [MP, IP, IP, DP, DP, DP, DP]
        L.kf_covariance_tables.restype = ctypes.c_int
        L.kf_call_graph_stats.argtypes = [ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.kf_call_graph_stats.restype = ctypes.c_int
        L.kf_bounds_checked.argtypes = []
        L.kf_bounds_checked.restype = ctypes.c_int
        for f in ("kf_autotune", "kf_tuning_get", "kf_tuning_save", "kf_tuning_load", "kf_tuning_clear",
                  "kf_autotune_batch", "kf_batch_tuning_get", "kf_last_launch_config"):
            getattr(L, f).restype = ctypes.c_int
        L.kf_rts_smooth_noalloc.argtypes = [MP, i64, vp, i, vp, vp, vp, vp, vp]
        L.kf_batch_smooth.argtypes = [i, MP, i, vp, i, vp, vp, i, vp, vp, vp, vp, vp]
        L.kf_batch_rts_smooth.argtypes = [MP, i, vp, i, vp, vp, i, vp, vp, vp, vp, vp]
        L.kf_batch_rts_smooth.restype = ctypes.c_int
        L.kf_stream_status.argtypes = [vp]
        L.kf_stream_status.restype = ctypes.c_int
        L.kf_batch_smooth.restype = ctypes.c_int
        L.kf_batch_graph_create.argtypes = [i, MP, i, vp, i, vp, vp, i, vp, vp, vp, ctypes.POINTER(vp)]
        L.kf_batch_graph_launch.argtypes = [vp, vp]
        L.kf_batch_graph_destroy.argtypes = [vp]
        for f in ("kf_batch_graph_create", "kf_batch_graph_launch", "kf_batch_graph_destroy"):
            getattr(L, f).restype = ctypes.c_int
        L.kf_batch_workspace_size.argtypes = [i, i, i, i64, i, i, i, i]
        L.kf_batch_workspace_size.restype = ctypes.c_size_t
        L.kf_server_create.argtypes = [ctypes.c_size_t, i, i64, ctypes.POINTER(vp)]
        L.kf_server_submit.argtypes = [vp, i, MP, i64, vp, i, vp, vp, vp, ctypes.POINTER(i64)]
        L.kf_server_poll.argtypes = [vp, i64, ctypes.POINTER(i), ctypes.POINTER(ctypes.c_double)]
        L.kf_server_wait.argtypes = [vp, i64, ctypes.c_double]
        L.kf_server_release.argtypes = [vp, i64]
        L.kf_server_destroy.argtypes = [vp]
        L.kf_server_cancel.argtypes = [vp, i64]
        for f in ("kf_server_create", "kf_server_submit", "kf_server_poll", "kf_server_wait", "kf_server_release",
                  "kf_server_destroy", "kf_server_cancel"):
            getattr(L, f).restype = ctypes.c_int
        L.kf_rts_smooth_noalloc.restype = ctypes.c_int
        L.kf_trace_phases.restype = ctypes.c_int
        TP = ctypes.POINTER(_TvModel)
        L.kf_tv_filter.argtypes = [TP, i64, vp, i, i, vp, vp, vp, vp, vp]
        L.kf_tv_rts_smooth.argtypes = [TP, i64, vp, i, i, vp, vp, vp, vp, vp, vp, vp]
        L.kf_tv_two_filter_smooth.argtypes = [TP, i64, vp, i, i, vp, vp, vp, vp, vp, vp, vp]
        for f in ("kf_tv_filter", "kf_tv_rts_smooth", "kf_tv_two_filter_smooth"):
            getattr(L, f).restype = ctypes.c_int
        L.kf_count_step_flops.argtypes = [i, i, ctypes.POINTER(ctypes.c_int64)]
        L.kf_count_step_flops.restype = ctypes.c_int
        _lib = L
    return _lib


def kf_status_string(status: int) -> str:
    return lib().kf_status_string(int(status)).decode()


def kf_version() -> str:
    return lib().kf_version().decode()


class Model:
    """Host FP64 copy of (F, Q, H, R, m0, P0) laid out for kf_model_t."""

    def __init__(self, model):
        self.arrays = {k: np.ascontiguousarray(np.asarray(model[k], dtype=np.float64))
                       for k in ("F", "Q", "H", "R", "m0", "P0")}
        self.nx = int(self.arrays["F"].shape[0])
        self.ny = int(self.arrays["H"].shape[0])
        D = ctypes.POINTER(ctypes.c_double)
        self.c = _Model(self.nx, self.ny, *[self.arrays[k].ctypes.data_as(D)
                                             for k in ("F", "Q", "H", "R", "m0", "P0")])


def _as_model(model):
    return model if isinstance(model, Model) else Model(model)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def dtype_of(precision):
    import torch
    return torch.float64 if PRECISIONS[precision] == 0 else torch.float32


def _check(rc, where):
    if rc != 0:
        raise KfError(rc, where)


def _prep(model, y, precision):
    import torch
    m = _as_model(model)
    if not (isinstance(y, torch.Tensor) and y.is_cuda):
        raise TypeError("y must be a CUDA tensor")
    dt = dtype_of(precision)
    if y.dtype != dt or not y.is_contiguous() or y.dim() != 2 or y.shape[1] != m.ny:
        raise ValueError("y must be contiguous [T, ny] of dtype %s" % dt)
    return m, dt


def kf_workspace_size(op, nx, ny, total_steps, precision="fp32", scan="dlb"):
    return int(lib().kf_workspace_size(OPS[op], nx, ny, int(total_steps), PRECISIONS[precision], SCANS[scan]))


def kf_filter(model, y, precision="fp32", scan="dlb", m_out=None, P_out=None, loglik=False,
              workspace=None, stream=None, want_cov=True):
    """Alg. pkf.  Returns (m [T,nx], P [T,nx,nx] or None, loglik tensor [1] or None)."""
    import torch
    m, dt = _prep(model, y, precision)
    T = y.shape[0]
    dev = y.device
    if m_out is None:
        m_out = torch.empty((T, m.nx), dtype=dt, device=dev)
    if P_out is None and want_cov:
        P_out = torch.empty((T, m.nx, m.nx), dtype=dt, device=dev)
    ll = torch.empty(1, dtype=torch.float64, device=dev) if loglik else None
    rc = lib().kf_filter(ctypes.byref(m.c), T, _ptr(y), PRECISIONS[precision], SCANS[scan], _ptr(m_out),
                         _ptr(P_out), _ptr(ll), _ptr(workspace), _stream(stream))
    _check(rc, "kf_filter")
    return m_out, P_out, ll


def _smooth(fn, name, model, y, precision, scan, ms_out, Ps_out, mf_out, Pf_out, loglik, workspace, stream):
    import torch
    m, dt = _prep(model, y, precision)
    T = y.shape[0]
    dev = y.device
    if ms_out is None:
        ms_out = torch.empty((T, m.nx), dtype=dt, device=dev)
    if Ps_out is None:
        Ps_out = torch.empty((T, m.nx, m.nx), dtype=dt, device=dev)
    if isinstance(loglik, torch.Tensor):   # a caller's CUDA float64 [1] buffer
        ll = loglik
    else:
        ll = torch.empty(1, dtype=torch.float64, device=dev) if loglik else None
    rc = fn(ctypes.byref(m.c), T, _ptr(y), PRECISIONS[precision], SCANS[scan], _ptr(ms_out), _ptr(Ps_out),
            _ptr(mf_out), _ptr(Pf_out), _ptr(ll), _ptr(workspace), _stream(stream))
    _check(rc, name)
    return ms_out, Ps_out, ll


def kf_rts_smooth(model, y, precision="fp32", scan="dlb", ms_out=None, Ps_out=None, mf_out=None, Pf_out=None,
                  loglik=False, workspace=None, stream=None):
    """Alg. prts (with its filter pass).  Returns (ms, Ps, loglik or None)."""
    return _smooth(lib().kf_rts_smooth, "kf_rts_smooth", model, y, precision, scan, ms_out, Ps_out, mf_out,
                   Pf_out, loglik, workspace, stream)


def kf_two_filter_smooth(model, y, precision="fp32", scan="dlb", ms_out=None, Ps_out=None, mf_out=None,
                         Pf_out=None, loglik=False, workspace=None, stream=None):
    """Alg. ptf (with its filter pass).  Returns (ms, Ps, loglik or None)."""
    return _smooth(lib().kf_two_filter_smooth, "kf_two_filter_smooth", model, y, precision, scan, ms_out,
                   Ps_out, mf_out, Pf_out, loglik, workspace, stream)


class TvModel:
    """A time-varying model laid out for kf_tv_model_t: the per-step arrays
    F [T,nx,nx], Q [T,nx,nx], u [T,nx] or None, H [T,ny,nx], R [T,ny,ny],
    d [T,ny] or None as contiguous CUDA tensors of the working dtype (record
    t is time t + 1: F[t] = F_{k-1}, H[t] = H_k), and the host FP64 prior
    m0, P0.  Arrays given as numpy or host tensors are copied to ``device``."""

    def __init__(self, model, precision="fp32", device="cuda"):
        import torch
        dt = dtype_of(precision)
        self.precision = precision
        self.t = {}
        for k in ("F", "Q", "u", "H", "R", "d"):
            v = model.get(k) if hasattr(model, "get") else model[k]
            if v is None:
                self.t[k] = None
                continue
            if not isinstance(v, torch.Tensor):
                v = torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64))
            self.t[k] = v.to(device=device, dtype=dt).contiguous()
        self.m0 = np.ascontiguousarray(np.asarray(model["m0"], dtype=np.float64))
        self.P0 = np.ascontiguousarray(np.asarray(model["P0"], dtype=np.float64))
        F, H = self.t["F"], self.t["H"]
        self.T, self.nx, self.ny = int(F.shape[0]), int(F.shape[1]), int(H.shape[1])
        shapes = {"F": (self.T, self.nx, self.nx), "Q": (self.T, self.nx, self.nx), "u": (self.T, self.nx),
                  "H": (self.T, self.ny, self.nx), "R": (self.T, self.ny, self.ny), "d": (self.T, self.ny)}
        for k, shp in shapes.items():
            if self.t[k] is not None and tuple(self.t[k].shape) != shp:
                raise ValueError("time-varying model: %s must have shape %s" % (k, shp))
        D = ctypes.POINTER(ctypes.c_double)
        self.c = _TvModel(self.nx, self.ny, *[_ptr(self.t[k]) for k in ("F", "Q", "u", "H", "R", "d")],
                          self.m0.ctypes.data_as(D), self.P0.ctypes.data_as(D))


def _tv_prep(model, y, precision):
    import torch
    m = model if isinstance(model, TvModel) else TvModel(model, precision, y.device)
    if m.precision != precision and dtype_of(m.precision) != dtype_of(precision):
        raise ValueError("the model arrays are %s; the call asks for %s" % (m.precision, precision))
    if not (isinstance(y, torch.Tensor) and y.is_cuda):
        raise TypeError("y must be a CUDA tensor")
    dt = dtype_of(precision)
    if y.dtype != dt or not y.is_contiguous() or y.dim() != 2 or y.shape[1] != m.ny or y.shape[0] > m.T:
        raise ValueError("y must be contiguous [T, ny] of dtype %s with T <= the model's steps" % dt)
    return m, dt


def kf_tv_filter(model, y, precision="fp32", scan="dlb", m_out=None, P_out=None, loglik=False, workspace=None,
                 stream=None, want_cov=True):
    """Alg. pkf on a time-varying model (TvModel or dict of per-step arrays).
    Returns (m [T,nx], P [T,nx,nx] or None, loglik tensor [1] or None)."""
    import torch
    m, dt = _tv_prep(model, y, precision)
    T = y.shape[0]
    dev = y.device
    if m_out is None:
        m_out = torch.empty((T, m.nx), dtype=dt, device=dev)
    if P_out is None and want_cov:
        P_out = torch.empty((T, m.nx, m.nx), dtype=dt, device=dev)
    ll = torch.empty(1, dtype=torch.float64, device=dev) if loglik else None
    rc = lib().kf_tv_filter(ctypes.byref(m.c), T, _ptr(y), PRECISIONS[precision], SCANS[scan], _ptr(m_out),
                            _ptr(P_out), _ptr(ll), _ptr(workspace), _stream(stream))
    _check(rc, "kf_tv_filter")
    return m_out, P_out, ll


def _tv_smooth(fn, name, model, y, precision, scan, ms_out, Ps_out, mf_out, Pf_out, loglik, workspace, stream):
    import torch
    m, dt = _tv_prep(model, y, precision)
    T = y.shape[0]
    dev = y.device
    if ms_out is None:
        ms_out = torch.empty((T, m.nx), dtype=dt, device=dev)
    if Ps_out is None:
        Ps_out = torch.empty((T, m.nx, m.nx), dtype=dt, device=dev)
    if isinstance(loglik, torch.Tensor):   # a caller's CUDA float64 [1] buffer
        ll = loglik
    else:
        ll = torch.empty(1, dtype=torch.float64, device=dev) if loglik else None
    rc = fn(ctypes.byref(m.c), T, _ptr(y), PRECISIONS[precision], SCANS[scan], _ptr(ms_out), _ptr(Ps_out),
            _ptr(mf_out), _ptr(Pf_out), _ptr(ll), _ptr(workspace), _stream(stream))
    _check(rc, name)
    return ms_out, Ps_out, ll


def kf_tv_rts_smooth(model, y, precision="fp32", scan="dlb", ms_out=None, Ps_out=None, mf_out=None, Pf_out=None,
                     loglik=False, workspace=None, stream=None):
    """Alg. prts on a time-varying model.  Returns (ms, Ps, loglik or None)."""
    return _tv_smooth(lib().kf_tv_rts_smooth, "kf_tv_rts_smooth", model, y, precision, scan, ms_out, Ps_out,
                      mf_out, Pf_out, loglik, workspace, stream)


def kf_tv_two_filter_smooth(model, y, precision="fp32", scan="dlb", ms_out=None, Ps_out=None, mf_out=None,
                            Pf_out=None, loglik=False, workspace=None, stream=None):
    """Alg. ptf on a time-varying model.  Returns (ms, Ps, loglik or None)."""
    return _tv_smooth(lib().kf_tv_two_filter_smooth, "kf_tv_two_filter_smooth", model, y, precision, scan, ms_out,
                      Ps_out, mf_out, Pf_out, loglik, workspace, stream)


def kf_sync_status(stream=None):
    """Wait for the stream; return the kernels' status (0 = OK) and clear it."""
    return int(lib().kf_sync_status(_stream(stream)))


def kf_stream_status(stream=None):
    """The same as kf_sync_status."""
    return int(lib().kf_stream_status(_stream(stream)))


def kf_set_option(name, value):
    _check(lib().kf_set_option(OPTIONS[name], int(value)), "kf_set_option")


def kf_get_option(name):
    return int(lib().kf_get_option(OPTIONS[name]))


def kf_timing_enable(on=True):
    _check(lib().kf_timing_enable(1 if on else 0), "kf_timing_enable")


def kf_timing_reset():
    _check(lib().kf_timing_reset(), "kf_timing_reset")


def timing_read(kind):
    """(kernel launches, total ms) of one kf_kernel_t kind since the last reset."""
    n = ctypes.c_int64(0)
    ms = ctypes.c_double(0)
    _check(lib().kf_timing_read(int(kind), ctypes.byref(n), ctypes.byref(ms)), "kf_timing_read")
    return int(n.value), float(ms.value)


def measure_fma_peak(fp64=False):
    """Measured FMA throughput of the current device in FLOP/s."""
    v = ctypes.c_double(0)
    _check(lib().kf_measure_fma_peak(1 if fp64 else 0, ctypes.byref(v)), "kf_measure_fma_peak")
    return float(v.value)


def rts_smooth_host(model, y_host, precision, scan, ms_host, Ps_host, ll_host=None, workspace=None, op="rts",
                    y_dev=None, ms_dev=None, Ps_dev=None, ll_dev=None, stream=None):
    """Smooth a sequence held in (pinned) host memory: copy y to the device,
    run kf_rts_smooth (or kf_two_filter_smooth with op="tf"), and copy the
    smoothed means, covariances and log-likelihood back, all enqueued on one
    stream.  Device staging buffers may be passed in to avoid allocation."""
    import torch
    T = y_host.shape[0]
    m = _as_model(model)
    dt = dtype_of(precision)
    if y_dev is None:
        y_dev = torch.empty(y_host.shape, dtype=dt, device="cuda")
    if ms_dev is None:
        ms_dev = torch.empty((T, m.nx), dtype=dt, device="cuda")
    if Ps_dev is None:
        Ps_dev = torch.empty((T, m.nx, m.nx), dtype=dt, device="cuda")
    if ll_host is not None and ll_dev is None:
        ll_dev = torch.empty(1, dtype=torch.float64, device="cuda")
    y_dev.copy_(y_host, non_blocking=True)
    fn = lib().kf_rts_smooth if op == "rts" else lib().kf_two_filter_smooth
    rc = fn(ctypes.byref(m.c), T, _ptr(y_dev), PRECISIONS[precision], SCANS[scan], _ptr(ms_dev), _ptr(Ps_dev),
            None, None, _ptr(ll_dev) if ll_host is not None else None, _ptr(workspace), _stream(stream))
    _check(rc, "kf_rts_smooth")
    ms_host.copy_(ms_dev, non_blocking=True)
    Ps_host.copy_(Ps_dev, non_blocking=True)
    if ll_host is not None:
        ll_host.copy_(ll_dev, non_blocking=True)
    return ms_host, Ps_host, ll_host


def kf_trace_phases(kind, buf=None):
    """Set (or clear, buf=None) the phase-trace device buffer (int64 tensor
    of 16 * capacity entries) of a look-back scan kind."""
    cap = 0 if buf is None else buf.numel() // 16
    _check(lib().kf_trace_phases(int(kind), _ptr(buf), cap), "kf_trace_phases")


NOALLOC_SCRATCH_BYTES = 16 << 20


def kf_rts_smooth_noalloc(model, y, precision, ms_out, Ps_out, loglik=None, status_out=None, stream=None):
    """RTS smoother that allocates no device memory (kfscan.h): its scratch
    is a fixed device array inside the library, so every output buffer must
    be passed in.  loglik: CUDA float64 tensor [1] or None; status_out: CUDA
    int32 tensor [1] or None (receives a kernel's bounded-wait status)."""
    m, _ = _prep(model, y, precision)
    rc = lib().kf_rts_smooth_noalloc(ctypes.byref(m.c), y.shape[0], _ptr(y), PRECISIONS[precision], _ptr(ms_out),
                                     _ptr(Ps_out), _ptr(loglik), _ptr(status_out), _stream(stream))
    _check(rc, "kf_rts_smooth_noalloc")
    return ms_out, Ps_out


def kf_batch_workspace_size(op, nx, ny, total_steps, nseq, nmodels, precision="fp32", loglik=True):
    return int(lib().kf_batch_workspace_size(OPS[op], nx, ny, int(total_steps), int(nseq), int(nmodels),
                                             PRECISIONS[precision], 1 if loglik else 0))


def _batch_args(models, offsets, y, precision, model_of, m_out, P_out, loglik):
    import torch
    if isinstance(models, (list, tuple)):
        ms = [_as_model(m) for m in models]
    else:
        ms = [_as_model(models)]
    arr = (_Model * len(ms))(*[m.c for m in ms])
    offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    nseq = len(offs) - 1
    mof = None if model_of is None else np.ascontiguousarray(np.asarray(model_of, dtype=np.int32))
    dt = dtype_of(precision)
    total = int(offs[-1])
    if not (isinstance(y, torch.Tensor) and y.is_cuda and y.dtype == dt and y.is_contiguous()
            and y.shape == (total, ms[0].ny)):
        raise ValueError("y must be a contiguous CUDA tensor [total, ny] of dtype %s" % dt)
    nx = ms[0].nx
    if m_out is None:
        m_out = torch.empty((total, nx), dtype=dt, device=y.device)
    if P_out is None:
        P_out = torch.empty((total, nx, nx), dtype=dt, device=y.device)
    ll = torch.empty(nseq, dtype=torch.float64, device=y.device) if loglik else None
    return ms, arr, offs, nseq, mof, m_out, P_out, ll


def kf_batch_smooth(op, models, offsets, y, precision="fp32", model_of=None, m_out=None, P_out=None, loglik=False,
                    workspace=None, stream=None):
    """Batch of sequences concatenated in y [total, ny] (segmented scan).
    models: one model dict (or Model) or a list; offsets: int64 array
    [nseq + 1]; model_of: int32 array [nseq] or None.  Returns (m, P, ll)."""
    ms, arr, offs, nseq, mof, m_out, P_out, ll = _batch_args(models, offsets, y, precision, model_of, m_out, P_out,
                                                             loglik)
    rc = lib().kf_batch_smooth(OPS[op], arr, len(ms), None if mof is None else mof.ctypes.data_as(ctypes.c_void_p),
                               nseq, offs.ctypes.data_as(ctypes.c_void_p), _ptr(y), PRECISIONS[precision],
                               _ptr(m_out), _ptr(P_out), _ptr(ll), _ptr(workspace), _stream(stream))
    _check(rc, "kf_batch_smooth")
    return m_out, P_out, ll


def kf_batch_rts_smooth(models, offsets, y, precision="fp32", model_of=None, ms_out=None, Ps_out=None, loglik=False,
                        workspace=None, stream=None):
    """kf_batch_smooth with the RTS smoother.  Returns (ms, Ps, ll)."""
    ms, arr, offs, nseq, mof, ms_out, Ps_out, ll = _batch_args(models, offsets, y, precision, model_of, ms_out,
                                                               Ps_out, loglik)
    rc = lib().kf_batch_rts_smooth(arr, len(ms), None if mof is None else mof.ctypes.data_as(ctypes.c_void_p), nseq,
                                   offs.ctypes.data_as(ctypes.c_void_p), _ptr(y), PRECISIONS[precision],
                                   _ptr(ms_out), _ptr(Ps_out), _ptr(ll), _ptr(workspace), _stream(stream))
    _check(rc, "kf_batch_rts_smooth")
    return ms_out, Ps_out, ll


class BatchGraph:
    """kf_batch_graph_* of kfscan.h: one batched call captured in a CUDA graph
    on fixed device buffers.  Construction runs the call once (filling
    m_out, P_out, ll); launch() replays it on the current contents of y."""

    def __init__(self, op, models, offsets, y, precision="fp32", model_of=None, loglik=False):
        import torch
        ms = [_as_model(m) for m in models] if isinstance(models, (list, tuple)) else [_as_model(models)]
        self._keep = ms
        arr = (_Model * len(ms))(*[m.c for m in ms])
        offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        nseq = len(offs) - 1
        mof = None if model_of is None else np.ascontiguousarray(np.asarray(model_of, dtype=np.int32))
        dt = dtype_of(precision)
        total = int(offs[-1])
        if not (isinstance(y, torch.Tensor) and y.is_cuda and y.dtype == dt and y.is_contiguous()
                and y.shape == (total, ms[0].ny)):
            raise ValueError("y must be a contiguous CUDA tensor [total, ny] of dtype %s" % dt)
        nx = ms[0].nx
        self.y = y
        self.m = torch.empty((total, nx), dtype=dt, device=y.device)
        self.P = torch.empty((total, nx, nx), dtype=dt, device=y.device)
        self.ll = torch.empty(nseq, dtype=torch.float64, device=y.device) if loglik else None
        self.h = ctypes.c_void_p()
        _check(lib().kf_batch_graph_create(OPS[op], arr, len(ms),
                                           None if mof is None else mof.ctypes.data_as(ctypes.c_void_p), nseq,
                                           offs.ctypes.data_as(ctypes.c_void_p), _ptr(y), PRECISIONS[precision],
                                           _ptr(self.m), _ptr(self.P), _ptr(self.ll), ctypes.byref(self.h)),
               "kf_batch_graph_create")

    def launch(self, stream=None):
        _check(lib().kf_batch_graph_launch(self.h, _stream(stream)), "kf_batch_graph_launch")
        return self.m, self.P, self.ll

    def close(self):
        if self.h:
            lib().kf_batch_graph_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server (kf_server_* of kfscan.h).  Jobs take host
    torch tensors (page-locked for overlap) and write results into host
    tensors, which the caller keeps alive until the job is done."""

    def __init__(self, budget_bytes=8 << 30, max_inflight=4, max_batch_steps=1 << 24):
        self.h = ctypes.c_void_p()
        _check(lib().kf_server_create(int(budget_bytes), int(max_inflight), int(max_batch_steps),
                                      ctypes.byref(self.h)), "kf_server_create")
        self._keep = {}

    def submit(self, op, model, y_host, precision, m_host=None, P_host=None, ll_host=None):
        m = _as_model(model)
        jid = ctypes.c_int64(0)
        rc = lib().kf_server_submit(self.h, OPS[op], ctypes.byref(m.c), int(y_host.shape[0]), _ptr(y_host),
                                    PRECISIONS[precision], _ptr(m_host), _ptr(P_host), _ptr(ll_host),
                                    ctypes.byref(jid))
        _check(rc, "kf_server_submit")
        self._keep[jid.value] = (m, y_host, m_host, P_host, ll_host)
        return jid.value

    def poll(self, jid):
        done = ctypes.c_int(0)
        info = (ctypes.c_double * 4)()
        rc = lib().kf_server_poll(self.h, int(jid), ctypes.byref(done), info)
        if done.value:
            _check(rc, "kf_server_poll")
        return bool(done.value), tuple(info)

    def wait(self, jid, timeout_s=60.0):
        _check(lib().kf_server_wait(self.h, int(jid), float(timeout_s)), "kf_server_wait")

    def cancel(self, jid):
        """Take a queued job out of the queue (True), or False when it has
        started or finished already (kf_server_cancel)."""
        rc = lib().kf_server_cancel(self.h, int(jid))
        if rc == 7:   # KF_ERR_BUSY
            return False
        _check(rc, "kf_server_cancel")
        return True

    def release(self, jid):
        _check(lib().kf_server_release(self.h, int(jid)), "kf_server_release")
        self._keep.pop(jid, None)

    def close(self):
        if self.h:
            _check(lib().kf_server_destroy(self.h), "kf_server_destroy")
            self.h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


SCAN_NAMES = {1: "dlb", 2: "hillis_steele", 3: "blelloch", 4: "ladner_fischer", 5: "sengupta"}


def kf_autotune(op, model, y, precision="fp32", reps=5, workspace=None, stream=None):
    """Time the candidate configurations of one call on these inputs and
    record the fastest (see kfscan.h).  Returns the recorded entry."""
    import torch
    m, dt = _prep(model, y, precision)
    T = y.shape[0]
    mo = torch.empty((T, m.nx), dtype=dt, device=y.device)
    Po = torch.empty((T, m.nx, m.nx), dtype=dt, device=y.device)
    _check(lib().kf_autotune(OPS[op], ctypes.byref(m.c), T, _ptr(y), PRECISIONS[precision], _ptr(mo), _ptr(Po),
                             int(reps), _ptr(workspace), _stream(stream)), "kf_autotune")
    return kf_tuning_get(op, m.nx, m.ny, precision, T)


def kf_tuning_get(op, nx, ny, precision, T):
    v = [ctypes.c_int(0) for _ in range(4)]
    ms = ctypes.c_double(0)
    rc = lib().kf_tuning_get(OPS[op], nx, ny, PRECISIONS[precision], int(T), *[ctypes.byref(x) for x in v],
                             ctypes.byref(ms))
    if rc != 0:
        return None
    return {"scan": SCAN_NAMES[v[0].value], "threads": v[1].value, "lookback_warps": v[2].value,
            "steps_per_thread": v[3].value, "ms": ms.value}


def kf_autotune_batch(op, models, offsets, y, precision="fp32", model_of=None, reps=5, workspace=None,
                      stream=None):
    """Time kf_batch_smooth's candidate configurations on this batch and
    record the fastest (see kfscan.h).  Returns the recorded entry."""
    ms, arr, offs, nseq, mof, m_out, P_out, _ = _batch_args(models, offsets, y, precision, model_of, None, None,
                                                            False)
    rc = lib().kf_autotune_batch(OPS[op], arr, len(ms), None if mof is None else mof.ctypes.data_as(ctypes.c_void_p),
                                 nseq, offs.ctypes.data_as(ctypes.c_void_p), _ptr(y), PRECISIONS[precision],
                                 _ptr(m_out), _ptr(P_out), int(reps), _ptr(workspace), _stream(stream))
    _check(rc, "kf_autotune_batch")
    return kf_batch_tuning_get(op, ms[0].nx, ms[0].ny, precision, int(offs[-1]))


def kf_batch_tuning_get(op, nx, ny, precision, total_steps):
    v = [ctypes.c_int(0) for _ in range(2)]
    t = ctypes.c_double(0)
    rc = lib().kf_batch_tuning_get(OPS[op], nx, ny, PRECISIONS[precision], int(total_steps),
                                   *[ctypes.byref(x) for x in v], ctypes.byref(t))
    if rc != 0:
        return None
    return {"lookback_warps": v[0].value, "steps_per_thread": v[1].value, "ms": t.value}


def kf_covariance_tables(model):
    """The covariance tables of a time-invariant model (see kfscan.h): a dict
    of k0, kb and the settled P_inf, K_inf, E_inf, Ps_inf, or None when the
    tables do not apply.  Host only."""
    import numpy as np
    m = _as_model(model)
    n, ny = m.nx, m.ny
    k0, kb = ctypes.c_int(0), ctypes.c_int(0)
    out = {k: np.zeros(s) for k, s in (("P_inf", (n, n)), ("K_inf", (n, ny)), ("E_inf", (n, n)),
                                        ("Ps_inf", (n, n)))}
    ptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    rc = lib().kf_covariance_tables(ctypes.byref(m.c), ctypes.byref(k0), ctypes.byref(kb), ptr(out["P_inf"]),
                                    ptr(out["K_inf"]), ptr(out["E_inf"]), ptr(out["Ps_inf"]))
    if rc != 0:
        return None
    out["k0"], out["kb"] = k0.value, kb.value
    return out


def kf_call_graph_stats():
    """Call graphs captured and replayed since the library was loaded."""
    c, r = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib().kf_call_graph_stats(ctypes.byref(c), ctypes.byref(r)), "kf_call_graph_stats")
    return {"captured": c.value, "replayed": r.value}


def kf_bounds_checked():
    """True when the loaded library is the bounds-checked build."""
    return bool(lib().kf_bounds_checked())


def kf_last_launch_config():
    """The calling thread's last launch request (see kfscan.h): a dict of
    scan, threads, lookback_warps and steps_per_thread (0 = library's choice)."""
    v = [ctypes.c_int(0) for _ in range(4)]
    _check(lib().kf_last_launch_config(*[ctypes.byref(x) for x in v]), "kf_last_launch_config")
    return {"scan": v[0].value, "threads": v[1].value, "lookback_warps": v[2].value,
            "steps_per_thread": v[3].value}


def kf_tuning_save(path):
    _check(lib().kf_tuning_save(str(path).encode()), "kf_tuning_save")


def kf_tuning_load(path):
    _check(lib().kf_tuning_load(str(path).encode()), "kf_tuning_load")


def kf_tuning_clear():
    _check(lib().kf_tuning_clear(), "kf_tuning_clear")


STEP_KINDS = {"filter_fold": 0, "filter_carry": 1, "filter_carry_loglik": 2, "rts_fold": 3, "rts_carry": 4}


def kf_count_step_flops(nx, step):
    """Flops of one time step of a kernel phase, counted from the kernels'
    own step code (kfscan.h): dict with total, add, mul, rcp, sqrt, log."""
    c = (ctypes.c_int64 * 6)()
    _check(lib().kf_count_step_flops(int(nx), STEP_KINDS.get(step, step), c), "kf_count_step_flops")
    return dict(zip(("total", "add", "mul", "rcp", "sqrt", "log"), [int(v) for v in c]))
