"""Seeded synthetic inputs for the detection path: strain, chirps, weights, workloads.

The paper analyses open LIGO strain resampled to 2048 Hz (Sec. IV.A) with a
trained network (Sec. II).  Neither is available here, so every input is
generated from a seed:

* coloured Gaussian noise whose one-sided PSD is an analytic
  "power law + bucket" curve (a stand-in for O3 Hanford/Livingston noise);
* leading-order (Newtonian) chirps projected onto two detectors with an
  amplitude, phase and arrival-time offset per detector, scaled to a chosen
  network SNR (the paper's SNR is the two-detector network SNR, Sec. I);
* network weights drawn from a SplitMix64 stream, in the flat layout that
  both the CUDA library and the oracle parse independently;
* workload presets (sizes, strides, network shapes) for the five workloads.

This module holds none of the method's arithmetic (no Welch PSD, no whitening,
no convolution, no integration): it only produces inputs, which the CUDA path
and the oracle both consume.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

FS = 2048  # Hz, Sec. IV.A: strain resampled to 2048 Hz

# --------------------------------------------------------------------------
# Analytic noise PSD and coloured noise
# --------------------------------------------------------------------------


@dataclasses.dataclass(frozen=True)
class NoiseModel:
    """One-sided PSD S(f) = S0 * (a (f/f0)^-4.14 + b + c (f/f0)^2), flat below f_flat."""

    S0: float = 1e-46
    f0: float = 150.0
    a: float = 1.0
    b: float = 1.0
    c: float = 1.0
    f_flat: float = 10.0

    def psd(self, f: np.ndarray) -> np.ndarray:
        fc = np.maximum(np.asarray(f, dtype=np.float64), self.f_flat)
        x = fc / self.f0
        return self.S0 * (self.a * x ** -4.14 + self.b + self.c * x ** 2)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def coloured_noise(n: int, seed: int, model: NoiseModel = NoiseModel(), fs: int = FS) -> np.ndarray:
    """Gaussian noise of length n with one-sided PSD model.psd (float64).

    White N(0,1) samples are shaped in the frequency domain by sqrt(S fs / 2),
    which gives E[2 |DFT(x)_k|^2 / (fs n)] = S(f_k).
    """
    # shaped on a padded length with small prime factors (a fast FFT size); the
    # first n samples of the circulant process are a stationary sample of the same PSD
    m = _fast_len(n)
    w = _rng(seed).standard_normal(m)
    W = np.fft.rfft(w)
    f = np.fft.rfftfreq(m, 1.0 / fs)
    return np.fft.irfft(W * np.sqrt(model.psd(f) * fs / 2.0), m)[:n]


def _fast_len(n: int) -> int:
    """Smallest 2^a 3^b 5^c >= n."""
    best = 1 << max(0, int(n - 1).bit_length())
    p5 = 1
    while p5 < best:
        p35 = p5
        while p35 < best:
            v = p35
            while v < n:
                v *= 2
            best = min(best, v)
            p35 *= 3
        p5 *= 5
    return best


# --------------------------------------------------------------------------
# Newtonian chirps
# --------------------------------------------------------------------------

T_SUN = 4.925490947e-6  # G M_sun / c^3 in seconds


def _chirp_shape(t: np.ndarray, t_c: float, mchirp: float, f_low: float, phase: float) -> np.ndarray:
    """Leading-order quadrupole chirp h(t) ~ f^(2/3) cos(phi), zero outside [f_low, f_isco]."""
    tm = mchirp * T_SUN
    tau = t_c - t
    out = np.zeros_like(t)
    ok = tau > 0
    tau_ok = tau[ok]
    f = (1.0 / (8.0 * math.pi)) * (5.0 / tau_ok) ** 0.375 * tm ** -0.625
    phi = phase - 2.0 * (tau_ok / (5.0 * tm)) ** 0.625
    m_total = mchirp * 4.0 ** 0.6  # equal-mass binary
    f_isco = 1.0 / (6.0 ** 1.5 * math.pi * m_total * T_SUN)
    band = (f >= f_low) & (f <= f_isco)
    h = np.where(band, f ** (2.0 / 3.0) * np.cos(phi), 0.0)
    # Tukey-like cosine ramps over the first and last 10 cycles in band
    ramp_lo = np.clip((f - f_low) / (0.15 * f_low), 0.0, 1.0)
    ramp_hi = np.clip((f_isco - f) / (0.05 * f_isco), 0.0, 1.0)
    h *= 0.5 - 0.5 * np.cos(math.pi * ramp_lo)
    h *= 0.5 - 0.5 * np.cos(math.pi * ramp_hi)
    out[ok] = h
    return out


def chirp_duration(mchirp: float, f_low: float = 20.0) -> float:
    """Time from f_low to coalescence for a Newtonian chirp (seconds)."""
    tm = mchirp * T_SUN
    return 5.0 / 256.0 * (math.pi * f_low) ** (-8.0 / 3.0) * tm ** (-5.0 / 3.0)


def inject_chirp(strain: np.ndarray, t_c: float, mchirp: float, snr: float, seed: int,
                 model: NoiseModel = NoiseModel(), fs: int = FS, f_low: float = 20.0) -> None:
    """Add one two-detector chirp in place (strain has shape [2][n]).

    Each detector gets its own amplitude factor, phase and arrival offset
    (|offset| <= 10 ms, the H1-L1 light travel time of Sec. IX); the pair is
    scaled so that the network SNR sqrt(sum_d 4 sum_k |h_d(f_k)|^2/S(f_k) df)
    equals snr.
    """
    rng = _rng(seed)
    n = strain.shape[1]
    dur = chirp_duration(mchirp, f_low)
    lo = max(0, int((t_c - dur - 1.0) * fs))
    hi = min(n, int((t_c + 0.5) * fs))
    if hi <= lo:
        return
    m = hi - lo
    nfft = 1 << int(math.ceil(math.log2(m)))
    t = (lo + np.arange(nfft)) / fs
    amps = rng.uniform(0.4, 1.0, size=2)
    phases = rng.uniform(0.0, 2.0 * math.pi, size=2)
    delay = rng.uniform(-0.010, 0.010)
    hs = []
    snr2 = 0.0
    f = np.fft.rfftfreq(nfft, 1.0 / fs)
    S = model.psd(f)
    for d in range(2):
        h = amps[d] * _chirp_shape(t, t_c + (delay if d == 1 else 0.0), mchirp, f_low, phases[d])
        H = np.fft.rfft(h) / fs
        snr2 += 4.0 * np.sum(np.abs(H[1:]) ** 2 / S[1:]) * (fs / nfft)
        hs.append(h)
    scale = snr / math.sqrt(snr2) if snr2 > 0 else 0.0
    for d in range(2):
        strain[d, lo:hi] += scale * hs[d][:m]


# --------------------------------------------------------------------------
# Network description and seeded weights
# --------------------------------------------------------------------------


@dataclasses.dataclass(frozen=True)
class NetSpec:
    """1D ResNet with GroupNorm (Sec. II): stem, stages of BasicBlocks, pooled linear head.

    stem: conv(in_ch -> widths[0], kernel stem_k, stride stem_stride, pad stem_k//2),
    GroupNorm, ReLU, then an optional max-pool (k3, s2, p1).  Stage s has
    blocks[s] BasicBlocks of width widths[s]; the first block of every stage
    after the first downsamples by 2 and has a 1x1 conv + GroupNorm shortcut.
    """

    in_ch: int = 2
    stem_k: int = 3
    stem_stride: int = 1
    stem_pool: int = 0
    widths: Tuple[int, ...] = (16,)
    blocks: Tuple[int, ...] = (2,)
    groups: int = 8
    eps: float = 1e-5


TINY_NET = NetSpec()
RESNET34_NET = NetSpec(stem_k=7, stem_stride=2, stem_pool=1, widths=(64, 128, 256, 512),
                       blocks=(3, 4, 6, 3), groups=16)


def weight_shapes(net: NetSpec) -> List[Tuple[str, Tuple[int, ...]]]:
    """Flat fp32 weight layout, in storage order.

    stem.w [C0][in_ch][stem_k], stem.gamma [C0], stem.beta [C0];
    per block: c1.w [C][Cin][3], g1.gamma, g1.beta, c2.w [C][C][3], g2.gamma, g2.beta,
    and, for a downsampling block, sc.w [C][Cin][1], gsc.gamma, gsc.beta;
    fc.w [C_last], fc.b [1].
    """
    shapes: List[Tuple[str, Tuple[int, ...]]] = []
    c0 = net.widths[0]
    shapes += [("stem.w", (c0, net.in_ch, net.stem_k)), ("stem.gamma", (c0,)), ("stem.beta", (c0,))]
    cin = c0
    for s, (width, nb) in enumerate(zip(net.widths, net.blocks)):
        for b in range(nb):
            stride = 2 if (s > 0 and b == 0) else 1
            p = f"s{s}b{b}."
            shapes += [(p + "c1.w", (width, cin, 3)), (p + "g1.gamma", (width,)), (p + "g1.beta", (width,)),
                       (p + "c2.w", (width, width, 3)), (p + "g2.gamma", (width,)), (p + "g2.beta", (width,))]
            if stride != 1 or cin != width:
                shapes += [(p + "sc.w", (width, cin, 1)), (p + "gsc.gamma", (width,)), (p + "gsc.beta", (width,))]
            cin = width
    shapes += [("fc.w", (cin,)), ("fc.b", (1,))]
    return shapes


def n_weights(net: NetSpec) -> int:
    return int(sum(int(np.prod(s)) for _, s in weight_shapes(net)))


_SM_GAMMA = np.uint64(0x9E3779B97F4A7C15)


def splitmix64_uniform(seed: int, n: int) -> np.ndarray:
    """n uniforms in [0,1) from the SplitMix64 sequence started at seed (53-bit mantissa)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * _SM_GAMMA
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def make_weights(net: NetSpec, seed: int) -> np.ndarray:
    """Seeded random-init weights (float32, flat layout of weight_shapes).

    conv / linear weights ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)); GroupNorm
    gamma ~ U(0.5, 1.5), beta ~ U(-0.1, 0.1); fc bias ~ U(-1/sqrt(fan_in), ..).
    """
    shapes = weight_shapes(net)
    total = n_weights(net)
    u = splitmix64_uniform(seed, total)
    out = np.empty(total, dtype=np.float32)
    off = 0
    fan_in_fc = shapes[-2][1][0]
    for name, shape in shapes:
        size = int(np.prod(shape))
        uu = u[off:off + size]
        if name.endswith(".w") and name != "fc.w":
            bound = 1.0 / math.sqrt(shape[1] * shape[2])
            vals = (2.0 * uu - 1.0) * bound
        elif name in ("fc.w", "fc.b"):
            bound = 1.0 / math.sqrt(fan_in_fc)
            vals = (2.0 * uu - 1.0) * bound
        elif name.endswith("gamma"):
            vals = 0.5 + uu
        else:  # beta
            vals = -0.1 + 0.2 * uu
        out[off:off + size] = vals.astype(np.float32)
        off += size
    return out


# --------------------------------------------------------------------------
# Workload presets
# --------------------------------------------------------------------------


@dataclasses.dataclass(frozen=True)
class Workload:
    """One analysis workload: sizes of the path plus the synthetic strain recipe.

    Plain mode (epoch_len == 0): the Welch PSD of the whole span whitens the
    whole span; windows start at the crop.  Epoch mode: whitened output
    sample j (raw sample lead + j) is whitened with the PSD of raw
    [e*epoch_len, e*epoch_len + psd_len), e = j // epoch_len, i.e. the
    64 s immediately before its 8 s epoch (Sec. VI).
    """

    name: str
    duration_s: float            # analysed seconds (windows x stride / fs)
    net: NetSpec
    stride: int                  # window stride in samples (fs / inference rate)
    n_win: int
    fs: int = FS
    nfft: int = 16384            # Welch segment: 8 s
    hop: int = 8192              # 50 % overlap
    fir_len: int = 2048          # 1 s whitening filter
    f_highpass: float = 32.0
    win_len: int = 3072          # 1.5 s windows
    int_s: float = 1.0           # 1 s top-hat integration (Sec. II)
    cluster_s: float = 8.0       # 8 s clustering window (Sec. II)
    epoch_len: int = 0           # 0: plain; else samples per PSD epoch
    psd_len: int = 131072        # 64 s of PSD context (Sec. VI)
    n_chirps: int = 1
    seed: int = 1234
    weight_seed: int = 77

    @property
    def crop(self) -> int:
        return self.fir_len // 2

    @property
    def n_int(self) -> int:
        return int(round(self.int_s * self.fs / self.stride))

    @property
    def cluster_half(self) -> int:
        return int(round(0.5 * self.cluster_s * self.fs / self.stride))

    @property
    def n_epochs(self) -> int:
        if self.epoch_len == 0:
            return 1
        need = (self.n_win - 1) * self.stride + self.win_len
        return -(-need // self.epoch_len)

    @property
    def lead(self) -> int:
        """Raw sample index of whitened sample 0."""
        return self.crop if self.epoch_len == 0 else self.psd_len

    @property
    def n_white(self) -> int:
        """Whitened samples produced per detector."""
        if self.epoch_len == 0:
            return self.n_raw - 2 * self.crop
        return self.n_epochs * self.epoch_len

    @property
    def n_raw(self) -> int:
        if self.epoch_len == 0:
            return int(round(64 * self.fs))
        return self.psd_len + self.n_epochs * self.epoch_len + self.crop


PLAIN_64S = Workload(name="plain-64s-tiny-4Hz", duration_s=61.0, net=TINY_NET, stride=512, n_win=244)
HOUR_RESNET34 = Workload(name="1h-resnet34gn-16Hz", duration_s=3600.0, net=RESNET34_NET, stride=128,
                         n_win=57600, epoch_len=16384, n_chirps=200, seed=4321)


def make_strain(wl: Workload, model: NoiseModel = NoiseModel()) -> Tuple[np.ndarray, List[dict]]:
    """Two-detector float32 strain [2][n_raw] for a workload, plus the injection list."""
    n = wl.n_raw
    x = np.stack([coloured_noise(n, wl.seed * 2 + d, model, wl.fs) for d in range(2)])
    inj = []
    rng = _rng(wl.seed + 99)
    if wl.n_chirps == 0:
        pass
    elif wl.n_chirps == 1:
        # one 30 Msun chirp-mass binary at SNR 12, merging 40 s into the span
        inj.append(dict(t_c=40.0, mchirp=30.0, snr=12.0))
    else:
        t0 = wl.lead / wl.fs
        span = wl.n_win * wl.stride / wl.fs
        spacing = span / wl.n_chirps
        for i in range(wl.n_chirps):
            inj.append(dict(t_c=t0 + (i + 0.5) * spacing + rng.uniform(-0.2, 0.2) * spacing,
                            mchirp=float(rng.uniform(10.0, 60.0)), snr=float(rng.uniform(4.0, 20.0))))
    for i, p in enumerate(inj):
        inject_chirp(x, p["t_c"], p["mchirp"], p["snr"], seed=wl.seed * 1000 + i, model=model, fs=wl.fs)
    return x.astype(np.float32), inj


# --------------------------------------------------------------------------
# Timeslide batch workload
# --------------------------------------------------------------------------


def segment_lengths(n_seg: int = 40, total_s: int = 86400, lo_s: int = 500, hi_s: int = 20000,
                    seed: int = 2024) -> List[int]:
    """Uneven seeded segment lengths in whole seconds: lengths lo + (total - n lo) u_i / sum(u),
    u_i ~ Exp(1), clipped at hi with the excess spread over the others, summing to total."""
    u = _rng(seed).exponential(1.0, size=n_seg)
    free = total_s - n_seg * lo_s
    extra = free * u / u.sum()
    for _ in range(64):
        over = np.maximum(lo_s + extra - hi_s, 0.0)
        if over.sum() <= 0:
            break
        extra -= over
        room = (lo_s + extra) < hi_s
        extra[room] += over.sum() * extra[room] / extra[room].sum()
    lengths = np.floor(lo_s + extra).astype(np.int64)
    lengths[np.argmax(hi_s - lengths)] += total_s - lengths.sum()
    return [int(v) for v in lengths]


TIMESLIDE_DAY = Workload(name="timeslides-40seg-1day-tiny-4Hz-100shifts", duration_s=86400.0, net=TINY_NET,
                         stride=512, n_win=0, epoch_len=16384, seed=777)


def make_segments(lengths_s: Sequence[int], seed: int, model: NoiseModel = NoiseModel(), fs: int = FS,
                  chirp_every_s: float = 0.0, workers: int = 0) -> Tuple[np.ndarray, List[Tuple[int, int]]]:
    """Concatenated two-detector float32 strain [2][sum n] of independent coloured-noise
    segments, plus [(offset, n_raw)] per segment; optional chirps every chirp_every_s.
    workers > 1 generates segments on that many threads (every segment has its own seeds and
    its chirps are drawn first, in order, so the result does not depend on the thread count)."""
    ns = [int(l) * fs for l in lengths_s]
    x = np.empty((2, sum(ns)), dtype=np.float32)
    segs, off = [], 0
    rng = _rng(seed + 5)
    plan = []
    for i, n in enumerate(ns):
        chirps = []
        if chirp_every_s > 0:
            for j in range(int(n / fs // chirp_every_s)):
                t_c = (j + 0.5) * chirp_every_s + rng.uniform(-1, 1)
                chirps.append((t_c, float(rng.uniform(10, 60)), float(rng.uniform(4, 20)), seed * 7919 + i * 131 + j))
        plan.append((i, n, off, chirps))
        segs.append((off, n))
        off += n

    def one(item):
        i, n, o, chirps = item
        seg = np.stack([coloured_noise(n, seed * 1000 + 2 * i + d, model, fs) for d in range(2)])
        for t_c, mc, snr, cs in chirps:
            inject_chirp(seg, t_c, mc, snr, seed=cs, model=model, fs=fs)
        x[:, o:o + n] = seg

    if workers > 1:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(workers) as ex:
            list(ex.map(one, plan))
    else:
        for item in plan:
            one(item)
    return x, segs


SERVING_128 = Workload(name="serving-128streams-0.25s-chunks-16Hz-tiny", duration_s=0.0, net=TINY_NET,
                       stride=128, n_win=0, epoch_len=16384, seed=555)
