"""Python face of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package smoke check
and by the benchmark's CPU-baseline leg, never by the product path.  It shares
no code with the CUDA library; the two meet only in the seeded inputs.

Each function cites the passage of arXiv 2403.18661 it restates; the
arithmetic lives in oracle.c (double precision).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_lib: Optional[ctypes.CDLL] = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C, FP64, no contraction, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-shared", "-fPIC", "-o", _SO + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_SO + ".tmp", _SO)
    return _SO


def _load() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            lib.orc_fft.argtypes = [_dp, _dp, ctypes.c_int64, ctypes.c_int]
            lib.orc_welch.argtypes = [_dp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp]
            lib.orc_whitening_taps.argtypes = [_dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_int, _dp]
            lib.orc_fir.argtypes = [_dp, ctypes.c_int64, _dp, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, _dp]
            lib.orc_conv1d.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int]
            lib.orc_conv1d.restype = None
            lib.orc_group_norm.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp,
                                           ctypes.c_double]
            lib.orc_group_norm.restype = None
            lib.orc_network.argtypes = [_ip, ctypes.c_double, _dp, _dp, ctypes.c_int, _dp]
            lib.orc_infer_windows.argtypes = [_ip, ctypes.c_double, _dp, _dp, _dp, ctypes.c_int64, ctypes.c_int,
                                              ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _dp]
            lib.orc_integrate.argtypes = [_dp, ctypes.c_int64, ctypes.c_int, _dp]
            lib.orc_triggers.argtypes = [_dp, ctypes.c_int64, ctypes.c_int, _lp, ctypes.c_int64]
            lib.orc_triggers.restype = ctypes.c_int64
            lib.orc_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _d(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def fft(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """Unnormalised DFT, X_k = sum_n x_n exp(-+2 pi i k n / N) (radix-2, N a power of two)."""
    x = np.asarray(x, dtype=np.complex128)
    re, im = _d(x.real).copy(), _d(x.imag).copy()
    if _load().orc_fft(_ptr(re), _ptr(im), len(re), +1 if inverse else -1) != 0:
        raise ValueError("length must be a power of two")
    return re + 1j * im


def welch(x: np.ndarray, nfft: int, hop: int, fs: float) -> np.ndarray:
    """One-sided Welch PSD density (periodic Hann, mean, no detrend); Sec. IV ("Noise sampling"), Sec. VI."""
    x = _d(x)
    out = np.empty(nfft // 2 + 1)
    if _load().orc_welch(_ptr(x), len(x), nfft, hop, fs, _ptr(out)) < 1:
        raise ValueError("bad Welch arguments")
    return out


def whitening_taps(psd: np.ndarray, nfft: int, fs: float, f_hp: float, fir_len: int) -> np.ndarray:
    """FIR taps g_m, m in [-F/2, F/2): tapered zero-phase inverse ASD with highpass (Sec. IV ("Noise sampling"))."""
    psd = _d(psd)
    taps = np.empty(fir_len)
    if _load().orc_whitening_taps(_ptr(psd), nfft, fs, f_hp, fir_len, _ptr(taps)) != 0:
        raise ValueError("bad filter arguments")
    return taps


def fir(x: np.ndarray, taps: np.ndarray, first: int, length: int) -> np.ndarray:
    """y_j = sum_m g_m x[first + j - m]: whitening evaluated as a direct linear filter."""
    x, taps = _d(x), _d(taps)
    y = np.empty(length)
    if _load().orc_fir(_ptr(x), len(x), _ptr(taps), len(taps), first, length, _ptr(y)) != 0:
        raise ValueError("output range reaches outside the input (crop too small)")
    return y


def conv1d(x: np.ndarray, w: np.ndarray, stride: int, pad: int) -> np.ndarray:
    """x [Cin][L], w [Cout][Cin][k] -> [Cout][Lout], zero padding."""
    x, w = _d(x), _d(w)
    cin, L = x.shape
    cout, cin2, k = w.shape
    assert cin == cin2
    lout = (L + 2 * pad - k) // stride + 1
    out = np.empty((cout, lout))
    _load().orc_conv1d(_ptr(x), cin, L, _ptr(w), cout, k, stride, pad, _ptr(out), lout)
    return out


def group_norm(x: np.ndarray, groups: int, gamma: np.ndarray, beta: np.ndarray, eps: float) -> np.ndarray:
    out = _d(x).copy()
    C, L = out.shape
    _load().orc_group_norm(_ptr(out), C, L, groups, _ptr(_d(gamma)), _ptr(_d(beta)), eps)
    return out


def _spec(net) -> np.ndarray:
    s = [net.in_ch, net.stem_k, net.stem_stride, net.stem_pool, net.groups, len(net.widths)]
    s += list(net.widths) + list(net.blocks)
    return np.asarray(s, dtype=np.int32)


def network(net, weights: np.ndarray, x: np.ndarray) -> float:
    """One window x [2][W] -> logit (Sec. II: 1D ResNet with GroupNorm)."""
    spec = _spec(net)
    w = _d(weights)
    x = _d(x)
    out = np.empty(1)
    rc = _load().orc_network(spec.ctypes.data_as(_ip), net.eps, _ptr(w), _ptr(x), x.shape[1], _ptr(out))
    if rc != 0:
        raise MemoryError("oracle network allocation failed")
    return float(out[0])


def infer_windows(net, weights: np.ndarray, y: np.ndarray, win_len: int, first: int, stride: int,
                  n_win: int, shift: int = 0) -> np.ndarray:
    """Logits of windows j: det0 y[0][first+j*stride:+W], det1 circularly shifted by `shift`."""
    spec = _spec(net)
    w = _d(weights)
    y0, y1 = _d(y[0]), _d(y[1])
    out = np.empty(n_win)
    rc = _load().orc_infer_windows(spec.ctypes.data_as(_ip), net.eps, _ptr(w), _ptr(y0), _ptr(y1), len(y0),
                                   win_len, first, stride, n_win, shift, _ptr(out))
    if rc != 0:
        raise ValueError("bad window arguments")
    return out


def integrate(z: np.ndarray, n_int: int) -> np.ndarray:
    """1 s top-hat moving average, valid mode (Sec. II)."""
    z = _d(z)
    out = np.empty(len(z) - n_int + 1)
    if _load().orc_integrate(_ptr(z), len(z), n_int, _ptr(out)) != 0:
        raise ValueError("series shorter than the integration length")
    return out


def triggers(I: np.ndarray, half: int) -> np.ndarray:
    """Indices of 8 s cluster maxima (Sec. II), earliest index wins ties."""
    I = _d(I)
    cap = len(I) + 1
    idx = np.empty(cap, dtype=np.int64)
    n = _load().orc_triggers(_ptr(I), len(I), half, idx.ctypes.data_as(_lp), cap)
    return idx[:n].copy()


# --------------------------------------------------------------------------
# Whole-path compositions
# --------------------------------------------------------------------------


def psd_epochs(x: np.ndarray, wl, epochs: Sequence[int]) -> np.ndarray:
    """PSD per detector for the given epochs: Welch over raw [e*epoch_len, e*epoch_len + psd_len).

    Plain mode (epoch_len == 0) has one PSD: the Welch estimate of the whole span.
    """
    out = np.empty((x.shape[0], len(epochs), wl.nfft // 2 + 1))
    for d in range(x.shape[0]):
        for i, e in enumerate(epochs):
            if wl.epoch_len == 0:
                seg = x[d]
            else:
                seg = x[d][e * wl.epoch_len: e * wl.epoch_len + wl.psd_len]
            out[d, i] = welch(seg, wl.nfft, wl.hop, wl.fs)
    return out


def whiten(x: np.ndarray, wl, psd: np.ndarray, epochs: Optional[Sequence[int]] = None) -> np.ndarray:
    """Whitened samples per detector.

    Plain mode: whitened sample j is raw sample crop + j (0.5 s cropped at each edge).
    Epoch mode: whitened sample j of epoch e = j // epoch_len is raw sample
    psd_len + j, filtered with the taps built from that epoch's PSD (Sec. VI).
    `epochs` selects which epochs to produce (psd rows in the same order);
    the result then holds only those epochs' samples, concatenated.
    """
    n_det = x.shape[0]
    if wl.epoch_len == 0:
        out = np.empty((n_det, x.shape[1] - 2 * wl.crop))
        for d in range(n_det):
            taps = whitening_taps(psd[d, 0], wl.nfft, wl.fs, wl.f_highpass, wl.fir_len)
            out[d] = fir(x[d], taps, wl.crop, out.shape[1])
        return out
    if epochs is None:
        epochs = range(wl.n_epochs)
    epochs = list(epochs)
    out = np.empty((n_det, len(epochs) * wl.epoch_len))
    for d in range(n_det):
        for i, e in enumerate(epochs):
            taps = whitening_taps(psd[d, i], wl.nfft, wl.fs, wl.f_highpass, wl.fir_len)
            out[d, i * wl.epoch_len:(i + 1) * wl.epoch_len] = fir(
                x[d], taps, wl.psd_len + e * wl.epoch_len, wl.epoch_len)
    return out


def analyze_plain(x: np.ndarray, wl, weights: np.ndarray) -> dict:
    """The whole plain path: Welch PSD -> filter -> whiten+crop -> windows -> logits -> integrate -> triggers."""
    psd = psd_epochs(x, wl, [0])
    white = whiten(x, wl, psd)
    logits = infer_windows(wl.net, weights, white, wl.win_len, 0, wl.stride, wl.n_win)
    stat = integrate(logits, wl.n_int)
    trig = triggers(stat, wl.cluster_half)
    return dict(psd=psd, white=white, logits=logits, stat=stat, triggers=trig)


# --------------------------------------------------------------------------
# Triggers -> false-alarm rates and times
# --------------------------------------------------------------------------


def far(background: np.ndarray, events: np.ndarray, livetime_s: float):
    """False-alarm rate of each event (Sec. IX): the number of background events
    whose detection statistic is greater than the event's, divided by the
    background livetime.  Returns (counts, rates per second)."""
    bg = np.asarray(background, dtype=np.float64)
    ev = np.asarray(events, dtype=np.float64)
    counts = np.array([int(np.count_nonzero(bg > x)) for x in ev], dtype=np.int64)
    return counts, counts / float(livetime_s)


def trigger_times(wl, idx, t0: float, gap_s: float):
    """Time stamp of statistic samples and the coalescence-time estimate.

    Sec. II: statistic sample j averages windows j .. j + n_int - 1 and is
    stamped at the right edge of the newest one; the coalescence time follows
    by removing the integration length and the delay between coalescence and
    full network activation (Fig. 1: 0.75 s, whitening settle-in plus the
    placement of the coalescence in the training kernel).  With a response
    that switches on gap_s after coalescence and stays on for at least the
    integration length, the causal average first peaks n_int - 1 windows
    after the switch-on window.  Window w starts at raw sample base + w*stride
    (base = the 0.5 s crop in plain mode, the PSD look-back in epoch mode).
    """
    j = np.asarray(idx, dtype=np.int64)
    base = wl.crop if wl.epoch_len == 0 else wl.psd_len
    newest = j + wl.n_int - 1
    t_peak = t0 + (base + newest * wl.stride + wl.win_len) / wl.fs
    t_c = t_peak - (wl.n_int - 1) * wl.stride / wl.fs - gap_s
    return t_peak, t_c


# --------------------------------------------------------------------------
# Resampling
# --------------------------------------------------------------------------


def resample_taps(factor: int) -> np.ndarray:
    """Decimation filter for factor M (Sec. IV.A: strain resampled to 2048 Hz;
    the paper names no filter).  Reading: a Kaiser-windowed sinc (beta = 5),
    2L + 1 taps with L = 10 M, cutoff at the output Nyquist frequency, unit
    gain at DC: the design of the common polyphase resampler."""
    M = int(factor)
    L = 10 * M
    k = np.arange(2 * L + 1) - L
    h = np.sinc(k / M) / M * np.kaiser(2 * L + 1, 5.0)
    return h / h.sum()


def resample(x: np.ndarray, factor: int):
    """Valid-mode decimation: output j is the filter centred on input sample
    (j0 + j) M, j0 = ceil(L / M), for every centre whose taps lie inside x.
    Returns (y, first input sample)."""
    M = int(factor)
    L = 10 * M
    h = resample_taps(M)
    x = np.asarray(x, dtype=np.float64)
    n_in = x.shape[-1]
    j0 = -(-L // M)
    n_out = max(0, (n_in - 1 - L) // M - j0 + 1) if n_in - 1 - L >= j0 * M else 0
    if n_out == 0:
        return np.zeros(x.shape[:-1] + (0,)), j0 * M
    win = np.lib.stride_tricks.sliding_window_view(x, 2 * L + 1, axis=-1)
    sel = win[..., j0 * M - L: j0 * M - L + (n_out - 1) * M + 1: M, :]
    return sel @ h, j0 * M
