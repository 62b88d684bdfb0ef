"""Thin Python binding of libncf's C ABI (include/ncf.h).

Argument marshalling only: every step of the computation runs in libncf's
CUDA kernels.  PyTorch supplies device memory for inputs and outputs and the
current CUDA stream.  If libncf.so is missing the first call raises; there is
no fallback implementation.

    ncf.corr(t, x, lags, kernel="gaussian", h=1.0)                # ACF
    ncf.corr(t, x, lags, kernel="rectangle", h=0.5, s=s, y=y)     # CCF
    ncf.corr_batch(offs, t, x, lags, ...)                         # B series, CSR

Names follow the paper's calling convention fn(lags, t, x, [s, y], h) -> (c, b)
(Sec. 2.6, "Unified API"), with keyword arguments in place of positional ones.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libncf.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "ncf.h")

KERNELS = {"gaussian": 0, "rectangle": 1, "hanning": 2}
PATHS = {"auto": 0, "spectral": 1, "windowed": 2}
PRECISIONS = {"fp64": 0, "fp32": 1}
NORMS = {"none": 0, "lag0": 1}


class ncf_options(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("path", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("norm", ctypes.c_int32), ("h", ctypes.c_double), ("trunc_R", ctypes.c_double),
                ("tol", ctypes.c_double)]


class ncf_series_summary(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("mean", ctypes.c_double), ("m2", ctypes.c_double),
                ("t_first", ctypes.c_double), ("t_last", ctypes.c_double), ("flags", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class ncf_pooled_stats(ctypes.Structure):
    _fields_ = [("mean_x", ctypes.c_double), ("std_x", ctypes.c_double), ("mean_y", ctypes.c_double),
                ("std_y", ctypes.c_double), ("n_x", ctypes.c_int64), ("n_y", ctypes.c_int64)]


class ncf_plan_info(ctypes.Structure):
    _fields_ = [("period", ctypes.c_double), ("modes", ctypes.c_int64), ("grid", ctypes.c_int64),
                ("width", ctypes.c_int64), ("B", ctypes.c_int64), ("K", ctypes.c_int64),
                ("buckets", ctypes.c_int64)]


class ncf_tuning(ctypes.Structure):
    _fields_ = [("rect_variant", ctypes.c_int32), ("fft_variant", ctypes.c_int32),
                ("contract_variant", ctypes.c_int32), ("spread_variant", ctypes.c_int32)]


class NcfError(RuntimeError):
    def __init__(self, status: int, name: str, message: str):
        super().__init__(f"{name}: {message}")
        self.status = status
        self.name = name


_lib = None
_lock = threading.Lock()


def lib():
    """Load libncf.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -m paper_2609_03866_b300.build`")
            L = ctypes.CDLL(LIB_PATH)
            vp, dp, i64p = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p
            L.ncf_options_default.argtypes = [ctypes.POINTER(ncf_options)]
            L.ncf_options_default.restype = None
            L.ncf_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]
            L.ncf_create.restype = ctypes.c_int
            L.ncf_destroy.argtypes = [vp]
            L.ncf_destroy.restype = None
            L.ncf_last_error.argtypes = [vp]
            L.ncf_last_error.restype = ctypes.c_char_p
            L.ncf_status_string.argtypes = [ctypes.c_int]
            L.ncf_status_string.restype = ctypes.c_char_p
            L.ncf_launch_count.argtypes = [vp]
            L.ncf_launch_count.restype = ctypes.c_uint64
            L.ncf_device_bytes.argtypes = [vp]
            L.ncf_device_bytes.restype = ctypes.c_size_t
            L.ncf_last_plan.argtypes = [vp, ctypes.POINTER(ncf_plan_info)]
            L.ncf_last_plan.restype = ctypes.c_int
            L.ncf_last_tuning.argtypes = [vp, ctypes.POINTER(ncf_tuning)]
            L.ncf_last_tuning.restype = ctypes.c_int
            L.ncf_profile_enable.argtypes = [vp, ctypes.c_int]
            L.ncf_profile_enable.restype = ctypes.c_int
            L.ncf_profile_report.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
            L.ncf_profile_report.restype = ctypes.c_int64
            L.ncf_profile_reset.argtypes = [vp]
            L.ncf_profile_reset.restype = None
            L.ncf_corr.argtypes = [vp, dp, dp, ctypes.c_int64, dp, dp, ctypes.c_int64, dp, ctypes.c_int64,
                                   ctypes.POINTER(ncf_options), dp, dp, i64p, vp]
            L.ncf_corr.restype = ctypes.c_int
            L.ncf_plan_create.argtypes = [vp, i64p, dp, dp, i64p, dp, dp, ctypes.c_int64, dp, ctypes.c_int64,
                                          ctypes.POINTER(ncf_options), vp, ctypes.POINTER(ctypes.c_void_p)]
            L.ncf_plan_create.restype = ctypes.c_int
            L.ncf_plan_execute.argtypes = [vp, dp, dp, dp, dp, dp, dp, i64p, vp]
            L.ncf_plan_execute.restype = ctypes.c_int
            L.ncf_plan_status.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int32)]
            L.ncf_plan_status.restype = ctypes.c_int
            L.ncf_plan_device_bytes.argtypes = [vp]
            L.ncf_plan_device_bytes.restype = ctypes.c_size_t
            L.ncf_plan_destroy.argtypes = [vp]
            L.ncf_plan_destroy.restype = None
            L.ncf_workspace_bytes.argtypes = [vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                              ctypes.c_double, ctypes.c_double, ctypes.POINTER(ncf_options),
                                              ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]
            L.ncf_workspace_bytes.restype = ctypes.c_int
            for name in ("ncf_corr_batch", "ncf_corr_batch_host"):
                fn = getattr(L, name)
                fn.argtypes = [vp, i64p, dp, dp, i64p, dp, dp, ctypes.c_int64, dp, ctypes.c_int64,
                               ctypes.POINTER(ncf_options), dp, dp, i64p, vp]
                fn.restype = ctypes.c_int
            _lib = L
    return _lib


def declared_symbols():
    """Names of the functions include/ncf.h declares with NCF_API."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"NCF_API\s+[\w\s\*]*?\b(ncf_\w+)\s*\(", txt)))


def status_name(code: int) -> str:
    return lib().ncf_status_string(code).decode()


def make_options(kernel="gaussian", h=1.0, path="auto", precision="fp64", norm="none",
                 trunc_R=0.0, tol=0.0) -> ncf_options:
    o = ncf_options()
    lib().ncf_options_default(ctypes.byref(o))
    o.kernel = KERNELS[kernel]
    o.path = PATHS[path]
    o.precision = PRECISIONS[precision]
    o.norm = NORMS[norm]
    o.h = float(h)
    o.trunc_R = float(trunc_R)
    o.tol = float(tol)
    return o


def workspace_bytes(n_x, B, K, span, max_abs_lag, n_y=0, kernel="gaussian", h=1.0, path="auto",
                    precision="fp64", norm="none", trunc_R=0.0, tol=0.0, ctx: "Context | None" = None):
    """Device (and pinned host) bytes an evaluation of these sizes needs, before any
    allocation (ncf_workspace_bytes; host arithmetic only, no GPU needed).
    Returns (device_bytes, pinned_bytes)."""
    o = make_options(kernel, h, path, precision, norm, trunc_R, tol)
    d, p = ctypes.c_size_t(), ctypes.c_size_t()
    h_ctx = ctx.handle if ctx is not None else None
    rc = lib().ncf_workspace_bytes(h_ctx, int(n_x), int(n_y), int(B), int(K), float(span), float(max_abs_lag),
                                   ctypes.byref(o), ctypes.byref(d), ctypes.byref(p))
    if rc != 0:
        msg = lib().ncf_last_error(h_ctx).decode() if ctx is not None else ""
        raise NcfError(rc, status_name(rc), msg or "ncf_workspace_bytes refused the sizes or options")
    return int(d.value), int(p.value)


class Context:
    """Owns an ncf_ctx (workspace, staging buffers) bound to one CUDA device."""

    def __init__(self, device: int = 0):
        self._h = ctypes.c_void_p()
        L = lib()
        rc = L.ncf_create(ctypes.byref(self._h), int(device))
        if rc != 0:
            raise NcfError(rc, status_name(rc), f"ncf_create(device={device}) failed")
        self.device = device

    @property
    def handle(self):
        return self._h

    def check(self, rc: int):
        if rc != 0:
            raise NcfError(rc, status_name(rc), lib().ncf_last_error(self._h).decode())

    @property
    def launches(self) -> int:
        return int(lib().ncf_launch_count(self._h))

    @property
    def device_bytes(self) -> int:
        """High-water mark of the context's device workspaces (bytes)."""
        return int(lib().ncf_device_bytes(self._h))

    def last_plan(self) -> dict:
        """Geometry of the most recent spectral call (period, modes, grid, width, B, K)."""
        info = ncf_plan_info()
        self.check(lib().ncf_last_plan(self._h, ctypes.byref(info)))
        return {f: getattr(info, f) for f, _ in ncf_plan_info._fields_}

    def last_tuning(self) -> dict:
        """The autotuner's latest choices (ncf_last_tuning): rect_variant,
        fft_variant, contract_variant, spread_variant; -1 where none was made yet."""
        info = ncf_tuning()
        self.check(lib().ncf_last_tuning(self._h, ctypes.byref(info)))
        return {f: getattr(info, f) for f, _ in ncf_tuning._fields_}

    def profile(self, on: bool = True):
        """Bracket every kernel launch of this context with CUDA events."""
        self.check(lib().ncf_profile_enable(self._h, int(on)))

    def profile_report(self) -> dict:
        """{kernel name: (launches, total ms)} accumulated since the last reset
        (synchronises on the recorded events)."""
        n = lib().ncf_profile_report(self._h, None, 0)
        buf = ctypes.create_string_buffer(int(n) + 1)
        lib().ncf_profile_report(self._h, buf, len(buf))
        out = {}
        for line in buf.value.decode().splitlines():
            name, cnt, ms = line.split()
            out[name] = (int(cnt), float(ms))
        return out

    def profile_reset(self):
        lib().ncf_profile_reset(self._h)

    def close(self):
        if self._h:
            lib().ncf_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default_ctx = {}


def default_context(device: int = 0) -> Context:
    ctx = _default_ctx.get(device)
    if ctx is None:
        ctx = _default_ctx[device] = Context(device)
    return ctx


def _dev(a, device):
    import torch
    if not isinstance(a, torch.Tensor):
        a = torch.as_tensor(np.asarray(a, dtype=np.float64))
    return a.to(device=device, dtype=torch.float64).contiguous()


def _ptr(a):
    return ctypes.c_void_p(a.data_ptr()) if a is not None else ctypes.c_void_p(0)


def _stream_handle(stream, device):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(stream.cuda_stream)


_OUT_DTYPES = (("c", "float64"), ("b", "float64"), ("count", "int64"))


def _check_out(out, shape, device):
    """Caller-supplied result buffers: out["c"] required, "b" and "count" optional;
    each contiguous, of its dtype, on `device` and of `shape`."""
    import torch
    if out.get("c") is None:
        raise ValueError('out["c"] is required')
    for key, dt in _OUT_DTYPES:
        v = out.get(key)
        if v is None:
            continue
        if not isinstance(v, torch.Tensor) or v.dtype != getattr(torch, dt) or v.device != torch.device(device) \
                or tuple(v.shape) != tuple(shape) or not v.is_contiguous():
            raise ValueError(f'out["{key}"] must be a contiguous {dt} tensor of shape {tuple(shape)} on {device}')


def _check_device_input(name, a, n, device):
    """Plan inputs are used as they are: contiguous float64 tensors on the plan's
    device with the element count the plan was built for."""
    import torch
    if not isinstance(a, torch.Tensor) or a.dtype != torch.float64 or a.device != torch.device(device) \
            or not a.is_contiguous() or a.numel() != n:
        raise ValueError(f"{name} must be a contiguous float64 tensor of {n} elements on {device}")


def corr(t, x, lags, kernel="gaussian", h=1.0, s=None, y=None, path="auto", precision="fp64",
         norm="none", trunc_R=0.0, tol=0.0, ctx: Context | None = None, stream=None):
    """One ACF (s, y omitted) or CCF on the GPU.  Returns dict(c, b, count)
    of device tensors in the order of `lags`."""
    import torch
    ctx = ctx or default_context()
    dev = torch.device("cuda", ctx.device)
    t, x, lags = _dev(t, dev), _dev(x, dev), _dev(lags, dev)
    acf = s is None
    if not acf:
        s, y = _dev(s, dev), _dev(y, dev)
    K = lags.numel()
    c = torch.empty(K, dtype=torch.float64, device=dev)
    b = torch.empty(K, dtype=torch.float64, device=dev)
    cnt = torch.empty(K, dtype=torch.int64, device=dev)
    o = make_options(kernel, h, path, precision, norm, trunc_R, tol)
    rc = lib().ncf_corr(ctx.handle, _ptr(t), _ptr(x), t.numel(), _ptr(None if acf else s),
                        _ptr(None if acf else y), 0 if acf else s.numel(), _ptr(lags), K,
                        ctypes.byref(o), _ptr(c), _ptr(b), _ptr(cnt), _stream_handle(stream, dev))
    ctx.check(rc)
    return {"c": c, "b": b, "count": cnt}


def series_stats(t, x, ctx: Context | None = None, stream=None) -> dict:
    """Statistics pass of one series on the GPU (ncf_series_stats): n, mean, m2 =
    sum (x - mean)^2, first and last time, validation flags."""
    import torch
    L = lib()
    if not getattr(L, "_stats_types", False):
        vp = ctypes.c_void_p
        L.ncf_series_stats.argtypes = [vp, vp, vp, ctypes.c_int64, ctypes.POINTER(ncf_series_summary), vp]
        L.ncf_series_stats.restype = ctypes.c_int
        L._stats_types = True
    ctx = ctx or default_context()
    dev = torch.device("cuda", ctx.device)
    t, x = _dev(t, dev), _dev(x, dev)
    out = ncf_series_summary()
    ctx.check(L.ncf_series_stats(ctx.handle, _ptr(t), _ptr(x), t.numel(), ctypes.byref(out),
                                 _stream_handle(stream, dev)))
    return {f: getattr(out, f) for f, _ in ncf_series_summary._fields_ if f != "pad"}


def corr_pooled(t, x, lags, pooled, kernel="gaussian", h=1.0, s=None, y=None, path="auto", precision="fp64",
                trunc_R=0.0, tol=0.0, ctx: Context | None = None, stream=None):
    """ncf_corr with the standardisation of a whole series pooled over its shards
    (ncf_corr_pooled).  `pooled`: dict(mean_x, std_x, n_x[, mean_y, std_y, n_y]).
    Returns dict(c, b, count) of device tensors in the order of `lags`."""
    import torch
    L = lib()
    if not getattr(L, "_pooled_types", False):
        vp = ctypes.c_void_p
        L.ncf_corr_pooled.argtypes = [vp, vp, vp, ctypes.c_int64, vp, vp, ctypes.c_int64, vp, ctypes.c_int64,
                                      ctypes.POINTER(ncf_options), ctypes.POINTER(ncf_pooled_stats), vp, vp, vp,
                                      vp]
        L.ncf_corr_pooled.restype = ctypes.c_int
        L._pooled_types = True
    ctx = ctx or default_context()
    dev = torch.device("cuda", ctx.device)
    t, x, lags = _dev(t, dev), _dev(x, dev), _dev(lags, dev)
    acf = s is None
    if not acf:
        s, y = _dev(s, dev), _dev(y, dev)
    K = lags.numel()
    c = torch.empty(K, dtype=torch.float64, device=dev)
    b = torch.empty(K, dtype=torch.float64, device=dev)
    cnt = torch.empty(K, dtype=torch.int64, device=dev)
    o = make_options(kernel, h, path, precision, "none", trunc_R, tol)
    ps = ncf_pooled_stats(float(pooled["mean_x"]), float(pooled["std_x"]), float(pooled.get("mean_y", 0.0)),
                          float(pooled.get("std_y", 1.0)), int(pooled["n_x"]), int(pooled.get("n_y", 0)))
    rc = L.ncf_corr_pooled(ctx.handle, _ptr(t), _ptr(x), t.numel(), _ptr(None if acf else s),
                           _ptr(None if acf else y), 0 if acf else s.numel(), _ptr(lags), K, ctypes.byref(o),
                           ctypes.byref(ps), _ptr(c), _ptr(b), _ptr(cnt), _stream_handle(stream, dev))
    ctx.check(rc)
    return {"c": c, "b": b, "count": cnt}


def corr_paper(t, x, lags, kernel="gaussian", h=1.0, s=None, y=None, N1=0, ctx: Context | None = None,
               stream=None):
    """The paper's own NUFFT estimator with the smoothing step (ncf_corr_paper,
    Algorithms 1-4): ACF (s, y omitted) or CCF.  N1 = 0 takes the default grid
    size round(32 n_max L / span).  Returns dict(c, b) of device tensors in the
    order of `lags` (b: the pair counts, clamped below at 1e-16)."""
    import torch
    L = lib()
    if not getattr(L, "_paper_types", False):
        vp = ctypes.c_void_p
        L.ncf_corr_paper.argtypes = [vp, vp, vp, ctypes.c_int64, vp, vp, ctypes.c_int64, vp, ctypes.c_int64,
                                     ctypes.c_int, ctypes.c_double, ctypes.c_int64, vp, vp, vp]
        L.ncf_corr_paper.restype = ctypes.c_int
        L._paper_types = True
    ctx = ctx or default_context()
    dev = torch.device("cuda", ctx.device)
    t, x, lags = _dev(t, dev), _dev(x, dev), _dev(lags, dev)
    acf = s is None
    if not acf:
        s, y = _dev(s, dev), _dev(y, dev)
    K = lags.numel()
    c = torch.empty(K, dtype=torch.float64, device=dev)
    b = torch.empty(K, dtype=torch.float64, device=dev)
    rc = L.ncf_corr_paper(ctx.handle, _ptr(t), _ptr(x), t.numel(), _ptr(None if acf else s),
                          _ptr(None if acf else y), 0 if acf else s.numel(), _ptr(lags), K, KERNELS[kernel],
                          float(h), int(N1), _ptr(c), _ptr(b), _stream_handle(stream, dev))
    ctx.check(rc)
    return {"c": c, "b": b}


def selftest_bounded_wait(ctx: Context | None = None, stream=None) -> int:
    """Runs the bounded-wait self-test (ncf_selftest_bounded_wait) and returns the
    device status word it produced (bit 1: the wait gave up as designed)."""
    import torch
    L = lib()
    L.ncf_selftest_bounded_wait.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]
    L.ncf_selftest_bounded_wait.restype = ctypes.c_int
    ctx = ctx or default_context()
    flags = ctypes.c_int32()
    rc = L.ncf_selftest_bounded_wait(ctx.handle, _stream_handle(stream, torch.device("cuda", ctx.device)),
                                     ctypes.byref(flags))
    ctx.check(rc)
    return flags.value


def corr_regular(m, x, dt, lags, kernel="gaussian", h=1.0, m_y=None, y=None, norm="none",
                 ctx: Context | None = None, stream=None):
    """Classic-FFT estimator for regularly sampled data (ncf_corr_regular): times
    m * dt with integer lattice indices m (non-decreasing).  Returns dict(c, b,
    count) of device tensors in the order of `lags`."""
    import torch
    L = lib()
    if not getattr(L, "_reg_types", False):
        vp = ctypes.c_void_p
        L.ncf_corr_regular.argtypes = [vp, vp, vp, ctypes.c_int64, vp, vp, ctypes.c_int64, ctypes.c_double, vp,
                                       ctypes.c_int64, ctypes.POINTER(ncf_options), vp, vp, vp, vp]
        L.ncf_corr_regular.restype = ctypes.c_int
        L._reg_types = True
    ctx = ctx or default_context()
    dev = torch.device("cuda", ctx.device)
    mi = torch.as_tensor(np.ascontiguousarray(m, dtype=np.int64) if not hasattr(m, "device") else m)
    mi = mi.to(device=dev, dtype=torch.int64).contiguous()
    x, lags = _dev(x, dev), _dev(lags, dev)
    ccf = y is not None
    if ccf:
        my = torch.as_tensor(np.ascontiguousarray(m_y, dtype=np.int64) if not hasattr(m_y, "device") else m_y)
        my = my.to(device=dev, dtype=torch.int64).contiguous()
        y = _dev(y, dev)
    K = lags.numel()
    out = {"c": torch.empty(K, dtype=torch.float64, device=dev), "b": torch.empty(K, dtype=torch.float64, device=dev),
           "count": torch.empty(K, dtype=torch.int64, device=dev)}
    o = make_options(kernel, h, "auto", "fp64", norm, 0.0, 0.0)
    rc = L.ncf_corr_regular(ctx.handle, _ptr(mi), _ptr(x), mi.numel(), _ptr(my if ccf else None),
                            _ptr(y if ccf else None), my.numel() if ccf else 0, float(dt), _ptr(lags), K,
                            ctypes.byref(o), _ptr(out["c"]), _ptr(out["b"]), _ptr(out["count"]),
                            _stream_handle(stream, dev))
    ctx.check(rc)
    return out


def corr_bootstrap(t, x, lags, n_boot, seed=0, kernel="gaussian", h=1.0, s=None, y=None, path="auto",
                   precision="fp64", norm="none", trunc_R=0.0, tol=0.0, ctx: Context | None = None, stream=None):
    """n_boot bootstrap replicates of one ACF (s, y omitted) or CCF, resampled on the
    GPU (ncf_corr_bootstrap).  Returns dict(c, b, count) of device tensors [n_boot, K]."""
    import torch
    L = lib()
    if not getattr(L, "_boot_types", False):
        vp = ctypes.c_void_p
        L.ncf_corr_bootstrap.argtypes = [vp, vp, vp, ctypes.c_int64, vp, vp, ctypes.c_int64, vp, ctypes.c_int64,
                                         ctypes.POINTER(ncf_options), ctypes.c_int64, ctypes.c_uint64, vp, vp, vp,
                                         vp]
        L.ncf_corr_bootstrap.restype = ctypes.c_int
        L._boot_types = True
    ctx = ctx or default_context()
    dev = torch.device("cuda", ctx.device)
    t, x, lags = _dev(t, dev), _dev(x, dev), _dev(lags, dev)
    acf = s is None
    if not acf:
        s, y = _dev(s, dev), _dev(y, dev)
    K = lags.numel()
    rows = max(int(n_boot), 0)  # the library rejects n_boot < 1 itself
    out = {"c": torch.empty(rows, K, dtype=torch.float64, device=dev),
           "b": torch.empty(rows, K, dtype=torch.float64, device=dev),
           "count": torch.empty(rows, K, dtype=torch.int64, device=dev)}
    o = make_options(kernel, h, path, precision, norm, trunc_R, tol)
    rc = L.ncf_corr_bootstrap(ctx.handle, _ptr(t), _ptr(x), t.numel(), _ptr(None if acf else s),
                              _ptr(None if acf else y), 0 if acf else s.numel(), _ptr(lags), K, ctypes.byref(o),
                              int(n_boot), int(seed) & ((1 << 64) - 1), _ptr(out["c"]), _ptr(out["b"]),
                              _ptr(out["count"]), _stream_handle(stream, dev))
    ctx.check(rc)
    return out


def _host_offs(offs):
    o = np.ascontiguousarray(np.asarray(offs.cpu() if hasattr(offs, "cpu") else offs, dtype=np.int64))
    return o, ctypes.c_void_p(o.ctypes.data)


def corr_batch(offs, t, x, lags, kernel="gaussian", h=1.0, offs_y=None, s=None, y=None, path="auto",
               precision="fp64", norm="none", trunc_R=0.0, tol=0.0, ctx: Context | None = None,
               stream=None, out=None):
    """B series packed CSR (host int64 offsets [B+1]) on one shared lag grid.
    Returns dict(c, b, count) of device tensors of shape [B, K]."""
    import torch
    ctx = ctx or default_context()
    dev = torch.device("cuda", ctx.device)
    t, x, lags = _dev(t, dev), _dev(x, dev), _dev(lags, dev)
    ox, pox = _host_offs(offs)
    B = ox.size - 1
    acf = s is None
    oy, poy = (None, ctypes.c_void_p(0)) if acf else _host_offs(offs_y)
    if not acf:
        s, y = _dev(s, dev), _dev(y, dev)
    K = lags.numel()
    if out is None:
        out = {"c": torch.empty(B, K, dtype=torch.float64, device=dev),
               "b": torch.empty(B, K, dtype=torch.float64, device=dev),
               "count": torch.empty(B, K, dtype=torch.int64, device=dev)}
    else:
        _check_out(out, (B, K), dev)
    o = make_options(kernel, h, path, precision, norm, trunc_R, tol)
    rc = lib().ncf_corr_batch(ctx.handle, pox, _ptr(t), _ptr(x), poy, _ptr(None if acf else s),
                              _ptr(None if acf else y), B, _ptr(lags), K, ctypes.byref(o),
                              _ptr(out["c"]), _ptr(out.get("b")), _ptr(out.get("count")),
                              _stream_handle(stream, dev))
    ctx.check(rc)
    return out


def _host_array(a):
    """A host float64 array for the host-buffer calls: numpy input is converted,
    a contiguous float64 CPU tensor (pinned or not) is used as it is."""
    import torch
    if a is None:
        return None
    if isinstance(a, torch.Tensor):
        if a.device.type != "cpu":
            raise ValueError("the host-buffer calls take host arrays; use corr_batch for device tensors")
        return a.to(torch.float64).contiguous()  # no copy for a contiguous float64 (pinned) tensor
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))


def corr_batch_host(offs, t, x, lags, kernel="gaussian", h=1.0, offs_y=None, s=None, y=None,
                    path="auto", precision="fp64", norm="none", trunc_R=0.0, tol=0.0,
                    ctx: Context | None = None, stream=None, out=None):
    """corr_batch on host arrays (numpy or pinned CPU tensors): the library
    copies inputs in and results out and synchronises before returning."""
    import torch
    host = _host_array
    ox, pox = _host_offs(offs)
    B = ox.size - 1
    acf = s is None
    oy, poy = (None, ctypes.c_void_p(0)) if acf else _host_offs(offs_y)
    t, x, lags, s, y = host(t), host(x), host(lags), host(s), host(y)
    K = lags.numel()
    if out is None:
        out = {"c": torch.empty(B, K, dtype=torch.float64), "b": torch.empty(B, K, dtype=torch.float64),
               "count": torch.empty(B, K, dtype=torch.int64)}
    else:
        _check_out(out, (B, K), "cpu")
    ctx = ctx or default_context()
    dev = torch.device("cuda", ctx.device)
    o = make_options(kernel, h, path, precision, norm, trunc_R, tol)
    rc = lib().ncf_corr_batch_host(ctx.handle, pox, _ptr(t), _ptr(x), poy, _ptr(s), _ptr(y), B,
                                   _ptr(lags), K, ctypes.byref(o), _ptr(out["c"]), _ptr(out.get("b")),
                                   _ptr(out.get("count")), _stream_handle(stream, dev))
    ctx.check(rc)
    return out


def corr_batch_host_multi(offs, t, x, lags, options, offs_y=None, s=None, y=None, ctx: Context | None = None,
                          stream=None, outs=None):
    """Several estimators of one batch from a single upload (ncf_corr_batch_host_multi).
    `options` is a list of dicts of corr_batch's keyword options (kernel, h, path,
    precision, norm, trunc_R, tol); returns one dict(c, b, count) of host tensors
    [B, K] per option set, equal to corr_batch_host with that set."""
    import torch
    L = lib()
    if not getattr(L, "_multi_types", False):
        vp = ctypes.c_void_p
        vpp = ctypes.POINTER(ctypes.c_void_p)
        L.ncf_corr_batch_host_multi.argtypes = [vp, vp, vp, vp, vp, vp, vp, ctypes.c_int64, vp, ctypes.c_int64,
                                                ctypes.POINTER(ncf_options), ctypes.c_int, vpp, vpp, vpp, vp]
        L.ncf_corr_batch_host_multi.restype = ctypes.c_int
        L._multi_types = True
    n = len(options)
    if n < 1:
        raise ValueError("options: at least one option set")
    ox, pox = _host_offs(offs)
    B = ox.size - 1
    acf = s is None
    oy, poy = (None, ctypes.c_void_p(0)) if acf else _host_offs(offs_y)
    t, x, lags, s, y = (_host_array(a) for a in (t, x, lags, s, y))
    K = lags.numel()
    if outs is None:
        outs = [{"c": torch.empty(B, K, dtype=torch.float64), "b": torch.empty(B, K, dtype=torch.float64),
                 "count": torch.empty(B, K, dtype=torch.int64)} for _ in range(n)]
    elif len(outs) != n:
        raise ValueError("outs: one dict of result buffers per option set")
    for o in outs:
        _check_out(o, (B, K), "cpu")
    opts = (ncf_options * n)(*[make_options(**o) for o in options])
    cp = (ctypes.c_void_p * n)(*[o["c"].data_ptr() for o in outs])
    bp = (ctypes.c_void_p * n)(*[o["b"].data_ptr() if o.get("b") is not None else 0 for o in outs])
    np_ = (ctypes.c_void_p * n)(*[o["count"].data_ptr() if o.get("count") is not None else 0 for o in outs])
    ctx = ctx or default_context()
    dev = torch.device("cuda", ctx.device)
    rc = L.ncf_corr_batch_host_multi(ctx.handle, pox, _ptr(t), _ptr(x), poy, _ptr(s), _ptr(y), B, _ptr(lags), K,
                                     opts, n, cp, bp, np_, _stream_handle(stream, dev))
    ctx.check(rc)
    return outs


def corr_batch_multi(offs, t, x, lags, options, offs_y=None, s=None, y=None, ctx: Context | None = None,
                     stream=None, outs=None):
    """Several estimators of one batch of device arrays on one statistics pass
    (ncf_corr_batch_multi).  `options` is a list of dicts of corr_batch's keyword
    options; returns one dict(c, b, count) of device tensors [B, K] per option
    set, equal to corr_batch with that set."""
    import torch
    L = lib()
    if not getattr(L, "_dmulti_types", False):
        vp = ctypes.c_void_p
        vpp = ctypes.POINTER(ctypes.c_void_p)
        L.ncf_corr_batch_multi.argtypes = [vp, vp, vp, vp, vp, vp, vp, ctypes.c_int64, vp, ctypes.c_int64,
                                           ctypes.POINTER(ncf_options), ctypes.c_int, vpp, vpp, vpp, vp]
        L.ncf_corr_batch_multi.restype = ctypes.c_int
        L._dmulti_types = True
    n = len(options)
    if n < 1:
        raise ValueError("options: at least one option set")
    ctx = ctx or default_context()
    dev = torch.device("cuda", ctx.device)
    t, x, lags = _dev(t, dev), _dev(x, dev), _dev(lags, dev)
    ox, pox = _host_offs(offs)
    B = ox.size - 1
    acf = s is None
    oy, poy = (None, ctypes.c_void_p(0)) if acf else _host_offs(offs_y)
    if not acf:
        s, y = _dev(s, dev), _dev(y, dev)
    K = lags.numel()
    if outs is None:
        outs = [{"c": torch.empty(B, K, dtype=torch.float64, device=dev),
                 "b": torch.empty(B, K, dtype=torch.float64, device=dev),
                 "count": torch.empty(B, K, dtype=torch.int64, device=dev)} for _ in range(n)]
    elif len(outs) != n:
        raise ValueError("outs: one dict of result buffers per option set")
    for o in outs:
        _check_out(o, (B, K), dev)
    opts = (ncf_options * n)(*[make_options(**o) for o in options])
    cp = (ctypes.c_void_p * n)(*[o["c"].data_ptr() for o in outs])
    bp = (ctypes.c_void_p * n)(*[o["b"].data_ptr() if o.get("b") is not None else 0 for o in outs])
    np_ = (ctypes.c_void_p * n)(*[o["count"].data_ptr() if o.get("count") is not None else 0 for o in outs])
    rc = L.ncf_corr_batch_multi(ctx.handle, pox, _ptr(t), _ptr(x), poy, _ptr(None if acf else s),
                                _ptr(None if acf else y), B, _ptr(lags), K, opts, n, cp, bp, np_,
                                _stream_handle(stream, dev))
    ctx.check(rc)
    return outs


class Plan:
    """A prepared batch evaluation (ncf_plan): built once from data laid out
    like the data it will be run on; `execute` then only launches kernels on
    the stream (no host synchronisation, no allocation), so it can be captured
    in a CUDA graph.  Device-side checks report through `status()`."""

    def __init__(self, offs, t, x, lags, kernel="gaussian", h=1.0, offs_y=None, s=None, y=None,
                 path="auto", precision="fp64", norm="none", trunc_R=0.0, tol=0.0,
                 ctx: Context | None = None, stream=None):
        import torch
        self.ctx = ctx or default_context()
        dev = torch.device("cuda", self.ctx.device)
        t, x, lags = _dev(t, dev), _dev(x, dev), _dev(lags, dev)
        ox, pox = _host_offs(offs)
        self.B = ox.size - 1
        self.K = lags.numel()
        self.acf = s is None
        oy, poy = (None, ctypes.c_void_p(0)) if self.acf else _host_offs(offs_y)
        if not self.acf:
            s, y = _dev(s, dev), _dev(y, dev)
        self.n_x, self.n_y = t.numel(), (0 if self.acf else s.numel())
        o = make_options(kernel, h, path, precision, norm, trunc_R, tol)
        self._h = ctypes.c_void_p()
        rc = lib().ncf_plan_create(self.ctx.handle, pox, _ptr(t), _ptr(x), poy, _ptr(None if self.acf else s),
                                   _ptr(None if self.acf else y), self.B, _ptr(lags), self.K, ctypes.byref(o),
                                   _stream_handle(stream, dev), ctypes.byref(self._h))
        self.ctx.check(rc)
        self.device = dev

    @property
    def device_bytes(self) -> int:
        return int(lib().ncf_plan_device_bytes(self._h))

    def execute(self, t, x, s=None, y=None, out=None, stream=None):
        """t, x (and s, y for a CCF): contiguous float64 device tensors of the sizes
        the plan was built for; the plan reads them as they are."""
        import torch
        _check_device_input("t", t, self.n_x, self.device)
        _check_device_input("x", x, self.n_x, self.device)
        if self.acf:
            if s is not None or y is not None:
                raise ValueError("this plan is an ACF: s and y are not taken")
        else:
            _check_device_input("s", s, self.n_y, self.device)
            _check_device_input("y", y, self.n_y, self.device)
        if out is None:
            out = {"c": torch.empty(self.B, self.K, dtype=torch.float64, device=self.device),
                   "b": torch.empty(self.B, self.K, dtype=torch.float64, device=self.device),
                   "count": torch.empty(self.B, self.K, dtype=torch.int64, device=self.device)}
        else:
            _check_out(out, (self.B, self.K), self.device)
        rc = lib().ncf_plan_execute(self._h, _ptr(t), _ptr(x), _ptr(s), _ptr(y), _ptr(out["c"]),
                                    _ptr(out.get("b")), _ptr(out.get("count")),
                                    _stream_handle(stream, self.device))
        self.ctx.check(rc)
        return out

    def status(self, stream=None) -> int:
        """Synchronises the stream; returns the status word of the last launch
        (0 = valid results)."""
        f = ctypes.c_int32()
        lib().ncf_plan_status(self._h, _stream_handle(stream, self.device), ctypes.byref(f))
        return int(f.value)

    def close(self):
        if self._h:
            lib().ncf_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MultiPlan:
    """A plan of several estimators on the same batch (ncf_plan_create_multi): one
    statistics pass per `execute`, then every option set's kernels; no host
    synchronisation or allocation in `execute`, so it can be captured in a CUDA
    graph.  `options`: a list of dicts of corr_batch's keyword options."""

    def __init__(self, offs, t, x, lags, options, offs_y=None, s=None, y=None, ctx: Context | None = None,
                 stream=None):
        import torch
        L = lib()
        if not getattr(L, "_mplan_types", False):
            vp = ctypes.c_void_p
            vpp = ctypes.POINTER(ctypes.c_void_p)
            L.ncf_plan_create_multi.argtypes = [vp, vp, vp, vp, vp, vp, vp, ctypes.c_int64, vp, ctypes.c_int64,
                                                ctypes.POINTER(ncf_options), ctypes.c_int, vp,
                                                ctypes.POINTER(vp)]
            L.ncf_plan_create_multi.restype = ctypes.c_int
            L.ncf_plan_execute_multi.argtypes = [vp, vp, vp, vp, vp, vpp, vpp, vpp, vp]
            L.ncf_plan_execute_multi.restype = ctypes.c_int
            L.ncf_plan_option_sets.argtypes = [vp]
            L.ncf_plan_option_sets.restype = ctypes.c_int
            L._mplan_types = True
        self.ctx = ctx or default_context()
        dev = torch.device("cuda", self.ctx.device)
        t, x, lags = _dev(t, dev), _dev(x, dev), _dev(lags, dev)
        ox, pox = _host_offs(offs)
        self.B, self.K, self.acf = ox.size - 1, lags.numel(), s is None
        oy, poy = (None, ctypes.c_void_p(0)) if self.acf else _host_offs(offs_y)
        if not self.acf:
            s, y = _dev(s, dev), _dev(y, dev)
        self.n_x, self.n_y = t.numel(), (0 if self.acf else s.numel())
        self.n = len(options)
        opts = (ncf_options * self.n)(*[make_options(**o) for o in options])
        self._h = ctypes.c_void_p()
        rc = L.ncf_plan_create_multi(self.ctx.handle, pox, _ptr(t), _ptr(x), poy, _ptr(None if self.acf else s),
                                     _ptr(None if self.acf else y), self.B, _ptr(lags), self.K, opts, self.n,
                                     _stream_handle(stream, dev), ctypes.byref(self._h))
        self.ctx.check(rc)
        self.device = dev

    @property
    def device_bytes(self) -> int:
        return int(lib().ncf_plan_device_bytes(self._h))

    def execute(self, t, x, s=None, y=None, outs=None, stream=None):
        import torch
        _check_device_input("t", t, self.n_x, self.device)
        _check_device_input("x", x, self.n_x, self.device)
        if not self.acf:
            _check_device_input("s", s, self.n_y, self.device)
            _check_device_input("y", y, self.n_y, self.device)
        if outs is None:
            outs = [{"c": torch.empty(self.B, self.K, dtype=torch.float64, device=self.device),
                     "b": torch.empty(self.B, self.K, dtype=torch.float64, device=self.device),
                     "count": torch.empty(self.B, self.K, dtype=torch.int64, device=self.device)}
                    for _ in range(self.n)]
        elif len(outs) != self.n:
            raise ValueError("outs: one dict of result buffers per option set")
        for o in outs:
            _check_out(o, (self.B, self.K), self.device)
        cp = (ctypes.c_void_p * self.n)(*[o["c"].data_ptr() for o in outs])
        bp = (ctypes.c_void_p * self.n)(*[o["b"].data_ptr() if o.get("b") is not None else 0 for o in outs])
        np_ = (ctypes.c_void_p * self.n)(*[o["count"].data_ptr() if o.get("count") is not None else 0
                                           for o in outs])
        rc = lib().ncf_plan_execute_multi(self._h, _ptr(t), _ptr(x), _ptr(s), _ptr(y), cp, bp, np_,
                                          _stream_handle(stream, self.device))
        self.ctx.check(rc)
        return outs

    def status(self, stream=None) -> int:
        f = ctypes.c_int32()
        lib().ncf_plan_status(self._h, _stream_handle(stream, self.device), ctypes.byref(f))
        return int(f.value)

    def close(self):
        if self._h:
            lib().ncf_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ncf_request(ctypes.Structure):
    _fields_ = [("t", ctypes.c_void_p), ("x", ctypes.c_void_p), ("nx", ctypes.c_int64),
                ("s", ctypes.c_void_p), ("y", ctypes.c_void_p), ("ny", ctypes.c_int64),
                ("lags", ctypes.c_void_p), ("K", ctypes.c_int64), ("opt", ncf_options),
                ("x_series", ctypes.c_uint64), ("y_series", ctypes.c_uint64)]


class Server:
    """Continuous-batching request loop (ncf_server_*): requests are admitted
    while others run, as slots and the device-memory budget allow; `submit`
    raises NcfError(NCF_EBUSY) when they do not (retry later)."""

    EBUSY = 7

    def __init__(self, device=0, mem_budget_bytes=8 << 30, slots=4):
        L = lib()
        if not getattr(L, "_server_types", False):
            vp = ctypes.c_void_p
            L.ncf_server_create.argtypes = [ctypes.c_int, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(vp)]
            L.ncf_server_create.restype = ctypes.c_int
            L.ncf_server_submit.argtypes = [vp, ctypes.POINTER(ncf_request), ctypes.POINTER(ctypes.c_uint64)]
            L.ncf_server_submit.restype = ctypes.c_int
            L.ncf_server_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]
            L.ncf_server_poll.restype = ctypes.c_int
            L.ncf_server_wait.argtypes = [vp, ctypes.c_uint64, vp, vp, vp, ctypes.POINTER(ctypes.c_double)]
            L.ncf_server_wait.restype = ctypes.c_int
            L.ncf_server_latency.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_uint64)]
            L.ncf_server_latency.restype = ctypes.c_int
            L.ncf_server_put.argtypes = [vp, vp, vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64)]
            L.ncf_server_put.restype = ctypes.c_int
            L.ncf_server_drop.argtypes = [vp, ctypes.c_uint64]
            L.ncf_server_drop.restype = ctypes.c_int
            L.ncf_server_destroy.argtypes = [vp]
            L.ncf_server_destroy.restype = None
            L._server_types = True
        self._h = ctypes.c_void_p()
        rc = L.ncf_server_create(int(device), int(mem_budget_bytes), int(slots), ctypes.byref(self._h))
        if rc != 0:
            raise NcfError(rc, status_name(rc), "ncf_server_create failed")
        self._keep = {}

    def put(self, t, x) -> int:
        """Copies a series to device memory held by the server (charged to its
        budget) and returns its handle for submit(x_series=..., y_series=...)."""
        t = np.ascontiguousarray(t, dtype=np.float64)
        x = np.ascontiguousarray(x, dtype=np.float64)
        h = ctypes.c_uint64()
        rc = lib().ncf_server_put(self._h, t.ctypes.data, x.ctypes.data, t.size, ctypes.byref(h))
        if rc != 0:
            raise NcfError(rc, status_name(rc), "ncf_server_put failed")
        return h.value

    def drop(self, series: int):
        rc = lib().ncf_server_drop(self._h, int(series))
        if rc != 0:
            raise NcfError(rc, status_name(rc), "ncf_server_drop failed")

    def submit(self, t, x, lags, kernel="gaussian", h=1.0, s=None, y=None, path="auto", precision="fp64",
               norm="none", trunc_R=0.0, tol=0.0, x_series=0, y_series=0):
        """t, x (or x_series) and, for a CCF, s, y (or y_series); t, x may be None
        when x_series names a resident series."""
        arrs = [np.ascontiguousarray(a, dtype=np.float64) if a is not None else None for a in (t, x, s, y, lags)]
        t, x, s, y, lags = arrs
        r = ncf_request()
        if t is not None:
            r.t, r.x, r.nx = t.ctypes.data, x.ctypes.data, t.size
        if s is not None:
            r.s, r.y, r.ny = s.ctypes.data, y.ctypes.data, s.size
        r.x_series, r.y_series = int(x_series), int(y_series)
        r.lags, r.K = lags.ctypes.data, lags.size
        r.opt = make_options(kernel, h, path, precision, norm, trunc_R, tol)
        tk = ctypes.c_uint64()
        rc = lib().ncf_server_submit(self._h, ctypes.byref(r), ctypes.byref(tk))
        if rc != 0:
            raise NcfError(rc, status_name(rc), "request not admitted")
        self._keep[tk.value] = (arrs, lags.size)
        return tk.value

    def done(self, ticket) -> bool:
        d = ctypes.c_int()
        lib().ncf_server_poll(self._h, ticket, ctypes.byref(d))
        return bool(d.value)

    def wait(self, ticket):
        """Blocks until the request is done; returns dict(c, b, count, latency_ms) (numpy)."""
        K = self._keep[ticket][1]
        c, b, n = np.empty(K), np.empty(K), np.empty(K, dtype=np.int64)
        lat = ctypes.c_double()
        rc = lib().ncf_server_wait(self._h, ticket, c.ctypes.data, b.ctypes.data, n.ctypes.data, ctypes.byref(lat))
        self._keep.pop(ticket, None)
        if rc != 0:
            raise NcfError(rc, status_name(rc), f"request {ticket} failed")
        return {"c": c, "b": b, "count": n, "latency_ms": lat.value}

    def latency(self):
        p50, p99, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_uint64()
        lib().ncf_server_latency(self._h, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(n))
        return {"p50_ms": p50.value, "p99_ms": p99.value, "completed": int(n.value)}

    def close(self):
        if self._h:
            lib().ncf_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
