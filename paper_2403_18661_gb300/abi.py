"""Thin Python binding of the C ABI in include/aframe_gb.h (argument marshalling only).

Every compute step runs in the CUDA library libaframe_gb.so; this module
only converts torch tensors to device pointers and sizes, passes the current
CUDA stream, and turns non-zero status codes into exceptions.  There is no
fallback: if the library is missing, loading it raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libaframe_gb.so")

AFG_OK = 0
AFG_FP32 = 0
AFG_BF16 = 1
AFG_ERR_ARG, AFG_ERR_CUDA, AFG_ERR_OOM, AFG_ERR_BUDGET = -1, -2, -3, -4
AFG_ERR_TIMEOUT, AFG_ERR_STATE, AFG_ERR_NAN, AFG_ERR_UNSUPPORTED = -5, -6, -7, -8
_ERRORS = {-1: "AFG_ERR_ARG", -2: "AFG_ERR_CUDA", -3: "AFG_ERR_OOM", -4: "AFG_ERR_BUDGET",
           -5: "AFG_ERR_TIMEOUT", -6: "AFG_ERR_STATE", -7: "AFG_ERR_NAN", -8: "AFG_ERR_UNSUPPORTED"}


class AfgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_ERRORS.get(status, status)}: {msg}")
        self.status = status


class AfgNet(ctypes.Structure):
    _fields_ = [("in_ch", ctypes.c_int32), ("stem_k", ctypes.c_int32), ("stem_stride", ctypes.c_int32),
                ("stem_pool", ctypes.c_int32), ("groups", ctypes.c_int32), ("n_stages", ctypes.c_int32),
                ("widths", ctypes.c_int32 * 4), ("blocks", ctypes.c_int32 * 4), ("eps", ctypes.c_float)]


class AfgConfig(ctypes.Structure):
    _fields_ = [("fs", ctypes.c_int32), ("nfft", ctypes.c_int32), ("hop", ctypes.c_int32),
                ("fir_len", ctypes.c_int32), ("f_highpass", ctypes.c_double), ("win_len", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("hbm_budget", ctypes.c_int64), ("net", AfgNet)]


class AfgKernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("timed", ctypes.c_int64),
                ("total_ms", ctypes.c_double), ("algo_flops", ctypes.c_double), ("algo_bytes", ctypes.c_double)]


class AfgRunParams(ctypes.Structure):
    _fields_ = [("n_raw", ctypes.c_int64), ("epoch_len", ctypes.c_int64), ("psd_len", ctypes.c_int64),
                ("stride", ctypes.c_int64), ("n_win", ctypes.c_int64), ("shift", ctypes.c_int64),
                ("n_int", ctypes.c_int32), ("cluster_half", ctypes.c_int32)]


class AfgSegment(ctypes.Structure):
    _fields_ = [("offset", ctypes.c_int64), ("n_raw", ctypes.c_int64)]


class AfgBatchParams(ctypes.Structure):
    _fields_ = [("psd_len", ctypes.c_int64), ("epoch_len", ctypes.c_int64), ("stride", ctypes.c_int64),
                ("shift_step", ctypes.c_int64), ("n_shift", ctypes.c_int32), ("n_int", ctypes.c_int32),
                ("cluster_half", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("shift_first", ctypes.c_int64)]


class AfgStreamParams(ctypes.Structure):
    _fields_ = [("psd_len", ctypes.c_int64), ("epoch_len", ctypes.c_int64), ("stride", ctypes.c_int64),
                ("n_int", ctypes.c_int32), ("max_streams", ctypes.c_int32), ("max_chunk", ctypes.c_int32)]


class AfgStreamResult(ctypes.Structure):
    _fields_ = [("window", ctypes.c_int64), ("stat", ctypes.c_float), ("logit", ctypes.c_float),
                ("t_push", ctypes.c_double), ("t_done", ctypes.c_double)]


class AfgTile(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("layer", "cin", "cout", "lin", "lout", "stride", "taps", "residual",
                                               "orient", "wpc", "kb", "stages", "acc_bufs", "tuned",
                                               "n_candidates")] + \
               [("us_chosen", ctypes.c_float), ("us_default", ctypes.c_float)]


def _tile_dict(t: AfgTile) -> dict:
    return {name: getattr(t, name) for name, _ in AfgTile._fields_}


class AfgFusedTuning(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("epi_warps", "issue_warps", "spin_ns", "tuned", "n_candidates")] + \
               [("us_chosen", ctypes.c_float), ("us_default", ctypes.c_float)]


def _fused_dict(t: AfgFusedTuning) -> dict:
    return {name: getattr(t, name) for name, _ in AfgFusedTuning._fields_}


STREAM_RESULT_DTYPE = np.dtype([("window", np.int64), ("stat", np.float32), ("logit", np.float32),
                                ("t_push", np.float64), ("t_done", np.float64)])


_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32

# every symbol include/aframe_gb.h declares, with its ctypes signature
SIGNATURES = {
    "afg_version": ([], ctypes.c_char_p),
    "afg_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "afg_weights_count": ([ctypes.POINTER(AfgNet), ctypes.POINTER(_i64)], ctypes.c_int),
    "afg_ctx_create": ([ctypes.POINTER(AfgConfig), _vp, _i64, ctypes.POINTER(_vp)], ctypes.c_int),
    "afg_ctx_destroy": ([_vp], ctypes.c_int),
    "afg_last_error": ([_vp], ctypes.c_char_p),
    "afg_ctx_bytes": ([_vp, ctypes.POINTER(_i64)], ctypes.c_int),
    "afg_sync": ([_vp, _vp], ctypes.c_int),
    "afg_wait_check": ([_vp, _i64, _i32, _vp, _vp], ctypes.c_int),
    "afg_psd_estimate": ([_vp, _vp, _i64, _i32, _i64, _i64, _i64, _vp, _vp], ctypes.c_int),
    "afg_whiten": ([_vp, _vp, _i64, _i32, _vp, _i64, _i64, _i64, _i64, _vp, _vp], ctypes.c_int),
    "afg_infer_windows": ([_vp, _vp, _i64, _i64, _i64, _i64, _i64, _vp, _vp], ctypes.c_int),
    "afg_integrate": ([_vp, _vp, _i64, _i32, _i32, _vp, _vp, _i64, _vp, _vp], ctypes.c_int),
    "afg_analyze": ([_vp, _vp, ctypes.POINTER(AfgRunParams), _vp, _vp, _vp, _i64, _vp, _vp], ctypes.c_int),
    "afg_analyze_host": ([_vp, _vp, ctypes.POINTER(AfgRunParams), _vp, _vp, _i64, _vp, _vp], ctypes.c_int),
    "afg_batch_layout": ([_vp, _vp, _i32, ctypes.POINTER(AfgBatchParams), _vp, ctypes.POINTER(_i64),
                          ctypes.POINTER(_i64)], ctypes.c_int),
    "afg_batch_run": ([_vp, _vp, _i64, _vp, _i32, ctypes.POINTER(AfgBatchParams), _vp, _vp, _vp, _i64, _vp, _vp],
                      ctypes.c_int),
    "afg_stream_start": ([_vp, ctypes.POINTER(AfgStreamParams)], ctypes.c_int),
    "afg_stream_open": ([_vp, ctypes.POINTER(_i64)], ctypes.c_int),
    "afg_stream_push": ([_vp, _i64, _vp, _i64, ctypes.POINTER(_i64)], ctypes.c_int),
    "afg_stream_push_many": ([_vp, _i64, _vp, _vp, _i64, _vp], ctypes.c_int),
    "afg_stream_poll": ([_vp, _i64, _vp, _i64, ctypes.POINTER(_i64), ctypes.c_double], ctypes.c_int),
    "afg_stream_flush": ([_vp, ctypes.c_double], ctypes.c_int),
    "afg_stream_close": ([_vp, _i64], ctypes.c_int),
    "afg_stream_stats": ([_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64)], ctypes.c_int),
    "afg_profile_enable": ([_vp, _i32], ctypes.c_int),
    "afg_profile_read": ([_vp, ctypes.POINTER(AfgKernelStat), _i32, ctypes.POINTER(_i32)], ctypes.c_int),
    "afg_autotune": ([_vp, _i64, _vp], ctypes.c_int),
    "afg_tiles_get": ([_vp, ctypes.POINTER(AfgTile), _i32, ctypes.POINTER(_i32)], ctypes.c_int),
    "afg_tile_candidates": ([_vp, _i32, ctypes.POINTER(AfgTile), _i32, ctypes.POINTER(_i32)], ctypes.c_int),
    "afg_tiles_set": ([_vp, ctypes.POINTER(AfgTile), _i32], ctypes.c_int),
    "afg_fused_tuning_get": ([_vp, ctypes.POINTER(AfgFusedTuning)], ctypes.c_int),
    "afg_fused_tuning_candidates": ([_vp, ctypes.POINTER(AfgFusedTuning), _i32, ctypes.POINTER(_i32)], ctypes.c_int),
    "afg_fused_tuning_set": ([_vp, ctypes.POINTER(AfgFusedTuning)], ctypes.c_int),
    "afg_resample": ([_vp, _vp, _i64, _i32, _i64, _i32, _vp, _i64, ctypes.POINTER(_i64), _vp], ctypes.c_int),
    "afg_resample_size": ([_i64, _i32, ctypes.POINTER(_i64), ctypes.POINTER(_i64)], ctypes.c_int),
    "afg_far": ([_vp, _vp, _vp, _vp, _i64, ctypes.c_double, _vp, _i64, _vp, _vp, _vp, _vp], ctypes.c_int),
    "afg_trigger_times": ([_vp, ctypes.POINTER(AfgRunParams), _vp, _i64, ctypes.c_double, ctypes.c_double, _vp, _vp],
                          ctypes.c_int),
    "afg_psd_estimate_noalloc": ([_vp, _i64, _i32, _i64, _i64, _i64, _i32, _i32, _vp, _vp], ctypes.c_int),
}


def load() -> ctypes.CDLL:
    """Load libaframe_gb.so (built in-tree by __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def version() -> str:
    return load().afg_version().decode()


def make_net(spec) -> AfgNet:
    """AfgNet from any object with in_ch, stem_k, stem_stride, stem_pool, widths, blocks, groups, eps."""
    n = AfgNet()
    n.in_ch, n.stem_k, n.stem_stride, n.stem_pool = spec.in_ch, spec.stem_k, spec.stem_stride, spec.stem_pool
    n.groups, n.n_stages = spec.groups, len(spec.widths)
    for i, (w, b) in enumerate(zip(spec.widths, spec.blocks)):
        n.widths[i], n.blocks[i] = w, b
    n.eps = spec.eps
    return n


def weights_count(spec) -> int:
    out = _i64()
    net = make_net(spec)
    rc = load().afg_weights_count(ctypes.byref(net), ctypes.byref(out))
    if rc != AFG_OK:
        raise AfgError(rc, "invalid network description")
    return out.value


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def psd_estimate_noalloc(x, n_psd: int = 1, psd_step: int = 0, psd_span: Optional[int] = None, fs: int = 2048,
                         hop: int = 8192, out=None, stream=None):
    """Welch PSD through afg_psd_estimate_noalloc: no context, no device allocation by the library.

    For hosts that cannot let a library call cudaMalloc; `out` (float64
    [n_det][n_psd][8193], on x's device) may be passed in so that this call
    allocates nothing at all.
    """
    import torch
    n_det, n = x.shape
    if psd_span is None:
        psd_span = n
    if out is None:
        out = torch.empty((n_det, n_psd, 8193), dtype=torch.float64, device=x.device)
    rc = load().afg_psd_estimate_noalloc(_ptr(x), n, n_det, n_psd, psd_step, psd_span, fs, hop, _ptr(out),
                                         _stream(stream))
    if rc != AFG_OK:
        raise AfgError(rc, "afg_psd_estimate_noalloc failed")
    return out


def resample_size(n_in: int, factor: int):
    """(output count, input sample of output 0) of afg_resample."""
    n, f = _i64(), _i64()
    rc = load().afg_resample_size(int(n_in), int(factor), ctypes.byref(n), ctypes.byref(f))
    if rc != AFG_OK:
        raise AfgError(rc, "resample_size: bad arguments")
    return n.value, f.value


class Context:
    """One library context (weights, twiddles, workspaces) on the current CUDA device."""

    def __init__(self, workload, weights: np.ndarray, precision: int = AFG_FP32, hbm_budget: int = 0):
        lib = load()
        cfg = AfgConfig()
        cfg.fs, cfg.nfft, cfg.hop, cfg.fir_len = workload.fs, workload.nfft, workload.hop, workload.fir_len
        cfg.f_highpass, cfg.win_len = workload.f_highpass, workload.win_len
        cfg.precision, cfg.hbm_budget = precision, hbm_budget
        cfg.net = make_net(workload.net)
        w = np.ascontiguousarray(weights, dtype=np.float32)
        h = _vp()
        rc = lib.afg_ctx_create(ctypes.byref(cfg), w.ctypes.data, len(w), ctypes.byref(h))
        if rc != AFG_OK:
            raise AfgError(rc, "afg_ctx_create failed")
        self._h = h
        self._lib = lib
        self.workload = workload
        self.precision = precision

    def close(self):
        if getattr(self, "_h", None):
            self._lib.afg_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int):
        if rc != AFG_OK:
            raise AfgError(rc, self._lib.afg_last_error(self._h).decode())

    @property
    def bytes_held(self) -> int:
        b = _i64()
        self._check(self._lib.afg_ctx_bytes(self._h, ctypes.byref(b)))
        return b.value

    def sync(self, stream=None):
        """Wait for queued work; raise AfgError(AFG_ERR_TIMEOUT) if a kernel's bounded wait gave up."""
        self._check(self._lib.afg_sync(self._h, _stream(stream)))

    def wait_check(self, limit_ns: int, n_blocks: int = 1, stream=None):
        """Launch afg_wait_check (CTAs whose bounded waits must run out) and return the device
        tensor of per-CTA waited nanoseconds; call sync() to read the timeout record."""
        import torch
        waited = torch.zeros(n_blocks, dtype=torch.int64, device="cuda")
        self._check(self._lib.afg_wait_check(self._h, int(limit_ns), int(n_blocks), _ptr(waited), _stream(stream)))
        return waited

    # ---------------------------------------------------------------- profiling
    def profile_enable(self, on: bool = True):
        self._check(self._lib.afg_profile_enable(self._h, 1 if on else 0))

    def profile_read(self) -> list:
        """Per-kernel launches, CUDA-event time and algorithmic work since the last enable/read."""
        cap = 64
        arr = (AfgKernelStat * cap)()
        n = _i32()
        self._check(self._lib.afg_profile_read(self._h, arr, cap, ctypes.byref(n)))
        return [dict(name=a.name.decode(), launches=a.launches, timed=a.timed, total_ms=a.total_ms,
                     algo_flops=a.algo_flops, algo_bytes=a.algo_bytes) for a in arr[:min(n.value, cap)]]

    # ---------------------------------------------------------------- resampling
    def resample(self, x, factor: int, stream=None):
        """Decimate device strain x [n_det][n_in] by `factor`: returns (y [n_det][n_out], first input sample)."""
        import torch
        n_det, n_in = x.shape
        n_out, first = resample_size(n_in, factor)
        y = torch.empty((n_det, max(n_out, 1)), dtype=torch.float32, device=x.device)
        got = _i64()
        self._check(self._lib.afg_resample(self._h, _ptr(x), n_in, n_det, x.stride(0), factor, _ptr(y), y.stride(0),
                                           ctypes.byref(got), _stream(stream)))
        assert got.value == n_out
        return y[:, :n_out], first

    # ---------------------------------------------------------------- false-alarm rates, trigger times
    def far(self, bg_stat, fg, livetime_s: float, bg_idx=None, n_bg=None, bg_cap: Optional[int] = None,
            out=None, stream=None):
        """FAR of each foreground statistic from a background (device tensors).  n_bg: device int64
        tensor holding the count (as afg_batch_run writes it) or a Python int; bg_cap: entries
        the count may reach (default: len(bg_idx) or len(bg_stat)).  Returns (n_above, far, bg_sorted)."""
        import torch
        dev = bg_stat.device
        if bg_cap is None:
            bg_cap = int(bg_idx.numel() if bg_idx is not None else bg_stat.numel())
        if n_bg is None:
            n_bg = bg_cap
        if not torch.is_tensor(n_bg):
            n_bg = torch.tensor([int(n_bg)], dtype=torch.int64, device=dev)
        n_fg = int(fg.numel())
        if out is None:
            out = (torch.empty(max(n_fg, 1), dtype=torch.int64, device=dev),
                   torch.empty(max(n_fg, 1), dtype=torch.float64, device=dev),
                   torch.empty(max(bg_cap, 1), dtype=torch.float32, device=dev))
        n_above, far, bg_sorted = out
        self._check(self._lib.afg_far(self._h, _ptr(bg_stat), _ptr(bg_idx), _ptr(n_bg), bg_cap, float(livetime_s),
                                      _ptr(fg), n_fg, _ptr(n_above), _ptr(far), _ptr(bg_sorted), _stream(stream)))
        return n_above[:n_fg], far[:n_fg], bg_sorted

    def trigger_times(self, idx, n_raw: int, t0: float = 0.0, gap_s: float = 0.75, shift: int = 0):
        """(t_peak, t_c) of statistic indices of a span analysed with this context's workload."""
        idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
        tp = np.empty(len(idx))
        tc = np.empty(len(idx))
        p = self.run_params(n_raw, shift)
        self._check(self._lib.afg_trigger_times(self._h, ctypes.byref(p), idx.ctypes.data, len(idx), float(t0),
                                                float(gap_s), tp.ctypes.data, tc.ctypes.data))
        return tp, tc

    # ---------------------------------------------------------------- conv tiles
    def autotune(self, n_win: int = 1024, stream=None):
        """Time every tile of each layer geometry of the BF16 tensor-core path (or every candidate of the
        fused 16-channel network) and keep the fastest."""
        self._check(self._lib.afg_autotune(self._h, int(n_win), _stream(stream)))

    def fused_tuning(self) -> dict:
        t = AfgFusedTuning()
        self._check(self._lib.afg_fused_tuning_get(self._h, ctypes.byref(t)))
        return _fused_dict(t)

    def fused_tuning_candidates(self) -> list:
        cap = 64
        arr = (AfgFusedTuning * cap)()
        n = _i32()
        self._check(self._lib.afg_fused_tuning_candidates(self._h, arr, cap, ctypes.byref(n)))
        return [_fused_dict(t) for t in arr[:min(n.value, cap)]]

    def set_fused_tuning(self, d: dict):
        """Apply the fused network's knobs given as a dict with the afg_fused_tuning fields."""
        t = AfgFusedTuning()
        for name, _ in AfgFusedTuning._fields_:
            if name in d:
                setattr(t, name, d[name])
        self._check(self._lib.afg_fused_tuning_set(self._h, ctypes.byref(t)))

    def tiles(self) -> list:
        cap = 256
        arr = (AfgTile * cap)()
        n = _i32()
        self._check(self._lib.afg_tiles_get(self._h, arr, cap, ctypes.byref(n)))
        return [_tile_dict(t) for t in arr[:min(n.value, cap)]]

    def tile_candidates(self, layer: int) -> list:
        cap = 256
        arr = (AfgTile * cap)()
        n = _i32()
        self._check(self._lib.afg_tile_candidates(self._h, int(layer), arr, cap, ctypes.byref(n)))
        return [_tile_dict(t) for t in arr[:min(n.value, cap)]]

    def set_tiles(self, tiles: list):
        """Apply tiles given as dicts with the afg_tile fields (e.g. a saved tuning)."""
        arr = (AfgTile * max(1, len(tiles)))()
        for i, d in enumerate(tiles):
            for name, _ in AfgTile._fields_:
                if name in d:
                    setattr(arr[i], name, d[name])
        self._check(self._lib.afg_tiles_set(self._h, arr, len(tiles)))

    # ---------------------------------------------------------------- hot path
    def psd_estimate(self, x, n_psd: int = 1, psd_step: int = 0, psd_span: Optional[int] = None, out=None,
                     stream=None):
        import torch
        n_det, n = x.shape
        if psd_span is None:
            psd_span = n
        if out is None:
            out = torch.empty((n_det, n_psd, self.workload.nfft // 2 + 1), dtype=torch.float64, device=x.device)
        self._check(self._lib.afg_psd_estimate(self._h, _ptr(x), n, n_det, n_psd, psd_step, psd_span, _ptr(out),
                                               _stream(stream)))
        return out

    def whiten(self, x, psd, out_first: int, out_len: int, epoch_len: int = 0, out=None, stream=None):
        import torch
        n_det, n = x.shape
        if out is None:
            out = torch.empty((n_det, out_len), dtype=torch.float32, device=x.device)
        self._check(self._lib.afg_whiten(self._h, _ptr(x), n, n_det, _ptr(psd), psd.shape[1], out_first, out_len,
                                         epoch_len, _ptr(out), _stream(stream)))
        return out

    def infer_windows(self, y, first: int, stride: int, n_win: int, shift: int = 0, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(n_win, dtype=torch.float32, device=y.device)
        self._check(self._lib.afg_infer_windows(self._h, _ptr(y), y.shape[1], first, stride, n_win, shift, _ptr(out),
                                                _stream(stream)))
        return out

    def integrate(self, logits, n_int: int, cluster_half: int, trig_cap: int = 4096, stream=None):
        import torch
        n_win = logits.shape[0]
        stat = torch.empty(n_win - n_int + 1, dtype=torch.float32, device=logits.device)
        trig = torch.empty(max(trig_cap, 1), dtype=torch.int64, device=logits.device)
        n_trig = torch.zeros(1, dtype=torch.int64, device=logits.device)
        self._check(self._lib.afg_integrate(self._h, _ptr(logits), n_win, n_int, cluster_half, _ptr(stat),
                                            _ptr(trig), trig_cap, _ptr(n_trig), _stream(stream)))
        return stat, trig, n_trig

    def run_params(self, n_raw: int, shift: int = 0) -> AfgRunParams:
        wl = self.workload
        p = AfgRunParams()
        p.n_raw, p.epoch_len, p.psd_len = n_raw, wl.epoch_len, wl.psd_len
        p.stride, p.n_win, p.shift = wl.stride, wl.n_win, shift
        p.n_int, p.cluster_half = wl.n_int, wl.cluster_half
        return p

    def analyze(self, x, shift: int = 0, trig_cap: int = 4096, out=None, stream=None):
        """Whole path on device tensor x [2][n_raw]: returns (logits, stat, trig_idx, n_trig) device tensors."""
        import torch
        wl = self.workload
        p = self.run_params(x.shape[1], shift)
        if out is None:
            out = (torch.empty(wl.n_win, dtype=torch.float32, device=x.device),
                   torch.empty(wl.n_win - wl.n_int + 1, dtype=torch.float32, device=x.device),
                   torch.empty(max(trig_cap, 1), dtype=torch.int64, device=x.device),
                   torch.zeros(1, dtype=torch.int64, device=x.device))
        logits, stat, trig, n_trig = out
        self._check(self._lib.afg_analyze(self._h, _ptr(x), ctypes.byref(p), _ptr(logits), _ptr(stat), _ptr(trig),
                                          trig_cap, _ptr(n_trig), _stream(stream)))
        return logits, stat, trig, n_trig

    # ---------------------------------------------------------------- timeslide batches
    def _batch_args(self, segments, n_shift: int, shift_step: int, use_graph: bool, shift_first: int = 1):
        wl = self.workload
        segs = (AfgSegment * len(segments))()
        for i, (off, n) in enumerate(segments):
            segs[i].offset, segs[i].n_raw = off, n
        p = AfgBatchParams()
        p.psd_len, p.epoch_len, p.stride, p.shift_step = wl.psd_len, wl.epoch_len, wl.stride, shift_step
        p.n_shift, p.n_int, p.cluster_half, p.use_graph = n_shift, wl.n_int, wl.cluster_half, int(use_graph)
        p.shift_first = shift_first
        return segs, p

    def batch_layout(self, segments, n_shift: int, shift_step: int, shift_first: int = 1):
        """(windows per timeslide of each segment, total windows, total statistic samples)."""
        segs, p = self._batch_args(segments, n_shift, shift_step, False, shift_first)
        n_win = (ctypes.c_int64 * len(segments))()
        tw, ts = _i64(), _i64()
        self._check(self._lib.afg_batch_layout(self._h, segs, len(segments), ctypes.byref(p), n_win, ctypes.byref(tw),
                                               ctypes.byref(ts)))
        return list(n_win), tw.value, ts.value

    def batch_run(self, x, segments, n_shift: int, shift_step: int, trig_cap: int = 1 << 20, use_graph: bool = False,
                  out=None, stream=None, shift_first: int = 1):
        """Timeslide background over `segments` [(offset, n_raw)] of device strain x [2][x_len], timeslides
        k = shift_first .. shift_first + n_shift - 1: returns (logits, stat, trig_idx, n_trig) device
        tensors, concatenated in series order."""
        import torch
        segs, p = self._batch_args(segments, n_shift, shift_step, use_graph, shift_first)
        _, tw, ts = self.batch_layout(segments, n_shift, shift_step, shift_first)
        if out is None:
            out = (torch.empty(tw, dtype=torch.float32, device=x.device),
                   torch.empty(ts, dtype=torch.float32, device=x.device),
                   torch.empty(max(trig_cap, 1), dtype=torch.int64, device=x.device),
                   torch.zeros(1, dtype=torch.int64, device=x.device))
        logits, stat, trig, n_trig = out
        self._check(self._lib.afg_batch_run(self._h, _ptr(x), x.shape[1], segs, len(segments), ctypes.byref(p),
                                            _ptr(logits), _ptr(stat), _ptr(trig), trig_cap, _ptr(n_trig),
                                            _stream(stream)))
        return logits, stat, trig, n_trig

    # ---------------------------------------------------------------- streams
    def stream_start(self, max_streams: int = 128, max_chunk: int = 4096):
        wl = self.workload
        p = AfgStreamParams()
        p.psd_len, p.epoch_len, p.stride = wl.psd_len, wl.epoch_len or 16384, wl.stride
        p.n_int, p.max_streams, p.max_chunk = wl.n_int, max_streams, max_chunk
        self._check(self._lib.afg_stream_start(self._h, ctypes.byref(p)))

    def stream_open(self) -> int:
        i = _i64()
        self._check(self._lib.afg_stream_open(self._h, ctypes.byref(i)))
        return i.value

    def stream_push(self, sid: int, chunk: np.ndarray) -> int:
        c = np.ascontiguousarray(chunk, dtype=np.float32)
        t = _i64()
        self._check(self._lib.afg_stream_push(self._h, sid, c.ctypes.data, c.shape[1], ctypes.byref(t)))
        return t.value

    def stream_push_many(self, sids, chunks: np.ndarray) -> np.ndarray:
        """Push chunks[k] ([2][n]) to stream sids[k] for every k in one call; returns the tickets."""
        ids = np.ascontiguousarray(np.asarray(sids, dtype=np.int64))
        c = np.ascontiguousarray(chunks, dtype=np.float32)
        assert c.ndim == 3 and c.shape[0] == ids.size and c.shape[1] == 2
        t = np.empty(ids.size, dtype=np.int64)
        self._check(self._lib.afg_stream_push_many(self._h, ids.size, ids.ctypes.data, c.ctypes.data, c.shape[2],
                                                   t.ctypes.data))
        return t

    def stream_poll(self, sid: int, cap: int = 65536, wait_s: float = 0.0) -> np.ndarray:
        out = np.empty(cap, dtype=STREAM_RESULT_DTYPE)
        n = _i64()
        self._check(self._lib.afg_stream_poll(self._h, sid, out.ctypes.data, cap, ctypes.byref(n), wait_s))
        return out[: n.value]

    def stream_flush(self, wait_s: float = 30.0):
        self._check(self._lib.afg_stream_flush(self._h, wait_s))

    def stream_close(self, sid: int):
        self._check(self._lib.afg_stream_close(self._h, sid))

    def stream_stats(self):
        a, b, c = _i64(), _i64(), _i64()
        self._check(self._lib.afg_stream_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return dict(steps=a.value, windows=b.value, samples=c.value)

    def analyze_host(self, x_host: np.ndarray, shift: int = 0, trig_cap: int = 4096, stat_out=None, trig_out=None,
                     stream=None) -> Tuple[np.ndarray, np.ndarray]:
        """Whole path from host strain (numpy or pinned torch CPU tensor) to host statistic and triggers."""
        wl = self.workload
        n_raw = x_host.shape[1]
        p = self.run_params(n_raw, shift)
        stat = stat_out if stat_out is not None else np.empty(wl.n_win - wl.n_int + 1, dtype=np.float32)
        trig = trig_out if trig_out is not None else np.empty(max(trig_cap, 1), dtype=np.int64)
        n_trig = np.zeros(1, dtype=np.int64)
        xp = x_host.data_ptr() if hasattr(x_host, "data_ptr") else x_host.ctypes.data
        sp = stat.data_ptr() if hasattr(stat, "data_ptr") else stat.ctypes.data
        tp = trig.data_ptr() if hasattr(trig, "data_ptr") else trig.ctypes.data
        self._check(self._lib.afg_analyze_host(self._h, xp, ctypes.byref(p), sp, tp, trig_cap, n_trig.ctypes.data,
                                               _stream(stream)))
        return stat, trig[:min(int(n_trig[0]), trig_cap)]
