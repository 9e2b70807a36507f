"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks one oracle routine against a closed form, a brute-force
evaluation on a tiny input, an invariant, or an independent library routine
(numpy / scipy / torch in float64), so that a plausible slip in oracle.c
(a dropped term, a wrong sign or index, a transposed operand, a wrong window
or scaling) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2403_18661_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- FFT (radix-2)

@pytest.mark.parametrize("n", [1, 2, 4, 8, 64, 512])
def test_fft_matches_bruteforce_dft(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    k = np.arange(n)
    dft = np.exp(-2j * np.pi * np.outer(k, k) / n) @ x
    got = orc.fft(x)
    assert np.max(np.abs(got - dft)) <= 1e-12 * max(1.0, np.max(np.abs(dft)))
    idft = np.exp(+2j * np.pi * np.outer(k, k) / n) @ x
    assert np.max(np.abs(orc.fft(x, inverse=True) - idft)) <= 1e-12 * max(1.0, np.max(np.abs(idft)))


def test_fft_parseval_and_library_at_16384():
    rng = np.random.default_rng(5)
    x = rng.standard_normal(16384)
    X = orc.fft(x)
    assert abs(np.sum(np.abs(X) ** 2) / 16384 - np.sum(x ** 2)) <= 1e-12 * np.sum(x ** 2)
    ref = np.fft.fft(x)
    assert np.max(np.abs(X - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_fft_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        orc.fft(np.ones(12))


# ---------------------------------------------------------------- Welch PSD

def test_welch_matches_scipy():
    sig = pytest.importorskip("scipy.signal")
    x = inputs.coloured_noise(131072, seed=11)
    got = orc.welch(x, 16384, 8192, 2048.0)
    f, ref = sig.welch(x, fs=2048.0, window="hann", nperseg=16384, noverlap=8192, detrend=False,
                       scaling="density", average="mean", return_onesided=True)
    assert got.shape == ref.shape == (8193,)
    assert np.max(np.abs(got - ref) / ref) < 1e-9


def test_welch_bin_centred_sinusoid_closed_form():
    # periodic Hann: a bin-centred cosine of amplitude a puts a^2 N/(3 fs) in its bin,
    # a^2 N/(12 fs) in each neighbour and nothing elsewhere
    N, fs, k0, a = 1024, 2048.0, 37, 3.0
    n = np.arange(4 * N)
    x = a * np.cos(2 * np.pi * k0 * n / N + 0.3)
    P = orc.welch(x, N, N // 2, fs)
    assert P[k0] == pytest.approx(a * a * N / (3 * fs), rel=1e-10)
    assert P[k0 - 1] == pytest.approx(a * a * N / (12 * fs), rel=1e-10)
    assert P[k0 + 1] == pytest.approx(a * a * N / (12 * fs), rel=1e-10)
    rest = np.delete(P, [k0 - 1, k0, k0 + 1])
    assert np.max(rest) < 1e-20 * P[k0] + 1e-24


def test_welch_is_mean_over_segments():
    # non-overlapping segments with amplitudes a_s: the bin holds mean(a_s^2) N/(3 fs)
    N, fs, k0 = 512, 2048.0, 20
    amps = np.array([1.0, 2.0, 5.0])
    n = np.arange(N)
    x = np.concatenate([a * np.cos(2 * np.pi * k0 * n / N) for a in amps])
    P = orc.welch(x, N, N, fs)
    assert P[k0] == pytest.approx(np.mean(amps ** 2) * N / (3 * fs), rel=1e-10)


def test_welch_white_noise_level():
    # white noise of variance s2 has one-sided density 2 s2 / fs
    rng = np.random.default_rng(3)
    s2, fs = 4.0, 2048.0
    x = math.sqrt(s2) * rng.standard_normal(16384 * 16)
    P = orc.welch(x, 16384, 8192, fs)
    body = P[1:-1]
    expect = 2 * s2 / fs
    # 31 segments averaged; relative sd per bin ~ 1/sqrt(31 * ~0.55 effective); mean over 8191 bins
    assert abs(np.mean(body) / expect - 1) < 3 * 0.2 / math.sqrt(8191) * 3
    # DC and Nyquist carry no one-sided doubling
    assert 0.2 < P[0] / (expect / 2) < 5


# ---------------------------------------------------------------- whitening filter

def test_taps_flat_psd_no_highpass_is_scaled_delta():
    S, fs, nfft, F = 2.5e-3, 2048.0, 1024, 256
    taps = orc.whitening_taps(np.full(nfft // 2 + 1, S), nfft, fs, 0.0, F)
    expect = np.zeros(F)
    expect[F // 2] = math.sqrt(2.0 / fs) / math.sqrt(S)
    assert np.max(np.abs(taps - expect)) < 1e-12 * expect[F // 2]


def test_taps_flat_psd_highpass_dirichlet_closed_form():
    # A_k = S^-1/2 for k >= kc: h_m = S^-1/2 (delta_m - D(m)/N), D(m) = sin((kc-1/2) t)/sin(t/2), t = 2 pi m/N
    S, fs, nfft, F, fhp = 1.0, 2048.0, 2048, 512, 32.0
    kc = int(math.ceil(fhp * nfft / fs))
    taps = orc.whitening_taps(np.full(nfft // 2 + 1, S), nfft, fs, fhp, F)
    m = np.arange(F) - F // 2
    th = 2 * np.pi * m / nfft
    with np.errstate(invalid="ignore", divide="ignore"):
        D = np.where(m == 0, 2 * kc - 1, np.sin((kc - 0.5) * th) / np.sin(th / 2))
    h = (np.where(m == 0, 1.0, 0.0) - D / nfft) / math.sqrt(S)
    taper = 0.5 - 0.5 * np.cos(2 * np.pi * np.arange(F) / F)
    expect = math.sqrt(2 / fs) * h * taper
    assert np.max(np.abs(taps - expect)) < 1e-12 * np.max(np.abs(expect))


def test_taps_bruteforce_cosine_sum_small():
    rng = np.random.default_rng(8)
    nfft, fs, F, fhp = 256, 256.0, 64, 10.0
    psd = rng.uniform(0.5, 2.0, nfft // 2 + 1)
    taps = orc.whitening_taps(psd, nfft, fs, fhp, F)
    k = np.arange(nfft // 2 + 1)
    A = np.where(k * fs / nfft >= fhp, psd ** -0.5, 0.0)
    out = np.empty(F)
    for j in range(F):
        m = j - F // 2
        s = A[0] + A[nfft // 2] * (-1) ** m
        for kk in range(1, nfft // 2):
            s += 2 * A[kk] * math.cos(2 * math.pi * kk * m / nfft)
        out[j] = math.sqrt(2 / fs) * s / nfft * (0.5 - 0.5 * math.cos(2 * math.pi * j / F))
    assert np.max(np.abs(taps - out)) < 1e-12 * np.max(np.abs(out))
    # zero-phase: even about m = 0, and the m = -F/2 tap vanishes
    assert taps[0] == 0.0
    assert np.max(np.abs(taps[1:F // 2] - taps[F // 2 + 1:][::-1])) < 1e-15 * np.max(np.abs(taps))


# ---------------------------------------------------------------- whitening (FIR)

def test_fir_matches_numpy_convolve():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(600)
    taps = rng.standard_normal(64)
    y = orc.fir(x, taps, 32, 600 - 64)
    full = np.convolve(x, taps, mode="full")
    assert np.max(np.abs(y - full[32 + 32: 32 + 32 + 600 - 64])) < 1e-12


def test_fir_refuses_uncropped_range():
    with pytest.raises(ValueError):
        orc.fir(np.zeros(100), np.zeros(16), 7, 10)
    with pytest.raises(ValueError):
        orc.fir(np.zeros(100), np.zeros(16), 8, 86)
    orc.fir(np.zeros(100), np.zeros(16), 8, 85)


def test_whitened_coloured_noise_is_flat_and_unit_variance():
    """Whitening with the filter of the analytic PSD gives a flat PSD of level 2/fs
    over the pass band and a variance equal to its exact expectation (near 31/32)."""
    sig = pytest.importorskip("scipy.signal")
    fs, nfft, F, fhp = 2048, 16384, 2048, 32.0
    model = inputs.NoiseModel()
    n = 1 << 20
    x = inputs.coloured_noise(n, seed=21, model=model)
    f = np.arange(nfft // 2 + 1) * fs / nfft
    taps = orc.whitening_taps(model.psd(f), nfft, fs, fhp, F)
    y = orc.fir(x, taps, F // 2, n - F)
    # exact expectation for the circulant-shaped noise: E[y^2] = (1/n) sum_k (S_k fs/2) |G_k|^2
    g = np.zeros(n)
    g[(np.arange(F) - F // 2) % n] = taps
    G = np.fft.fft(g)
    fk = np.fft.fftfreq(n, 1 / fs)
    ey2 = np.sum(model.psd(np.abs(fk)) * fs / 2 * np.abs(G) ** 2) / n
    assert 0.95 < ey2 < 0.975          # 1 - 32/1024 minus taper smoothing
    var = np.var(y)
    assert abs(var - ey2) < 5 * math.sqrt(2.0 / len(y)) * ey2
    fw, P = sig.welch(y, fs=fs, nperseg=4096, noverlap=2048, window="hann", detrend=False)
    band = (fw >= 40) & (fw <= 1000)
    level = P[band] * fs / 2
    nseg = (len(y) - 4096) // 2048 + 1
    se = 1.0 / math.sqrt(nseg * 0.5)
    assert np.max(np.abs(level - 1.0)) < 5 * se
    assert abs(np.mean(level) - 1.0) < 0.01


# ---------------------------------------------------------------- network layers

# ---------------------------------------------------------------- epoch composition (Sec. VI)

def test_epoch_psd_and_whitening_follow_the_64s_lookback():
    """Sec. VI: the first 64 s of state estimate the PSD and the rest is whitened.  In epoch mode
    whitened sample j (raw sample psd_len + j) belongs to epoch e = j // epoch_len, whose PSD is the
    Welch estimate of raw [e epoch_len, e epoch_len + psd_len), the 64 s just before it.

    Input: white Gaussian noise whose variance steps per 8 s block (block b has variance v_b,
    neighbours differing by at least 1.8x).  For independent samples E|X_k|^2 = sum_n w_n^2 v(n) at
    every bin, so each 8 s Welch segment has the flat expected level 2 v / fs, and a segment that
    straddles two blocks averages them (the periodic Hann's squares sum to the same value over
    either half).  Over the 15 segments of epoch e's look-back (blocks e .. e+7) the expected
    level is therefore (2 / fs) (1.5 v_e + 2 (v_{e+1} + .. + v_{e+6}) + 1.5 v_{e+7}) / 15.
    The whitened samples of epoch e come from raw block e + 8, so away from the block edges their
    variance is v_{e+8} sum_m g_m^2 with g the epoch's own taps (white input).  A look-back or an
    epoch-to-block mapping off by one epoch moves either figure by far more than its tolerance."""
    fs, blk = 2048, 16384
    wl = inputs.Workload(name="epoch-pin", duration_s=0.0, net=inputs.TINY_NET, stride=512, n_win=1,
                         epoch_len=blk, n_chirps=0)
    n_ep = 4
    n_blocks = 8 + n_ep
    rng = np.random.default_rng(2403)
    # per detector: variances on a rising trend (x1.35 per block, so a look-back shifted by one
    # epoch changes the level by about that factor) that alternate low/high (x2.5, so neighbouring
    # blocks differ by >= 1.8x), with +-10 % random factors
    b = np.arange(n_blocks)
    v = np.stack([1.35 ** b * np.where((b + d) % 2 == 0, 1.0, 2.5) * rng.uniform(0.9, 1.1, n_blocks)
                  for d in range(2)])
    n = n_blocks * blk + wl.crop
    x = np.empty((2, n))
    for d in range(2):
        z = rng.standard_normal(n)
        sig = np.sqrt(np.repeat(v[d], blk))
        x[d, : n_blocks * blk] = z[: n_blocks * blk] * sig
        x[d, n_blocks * blk:] = z[n_blocks * blk:] * math.sqrt(v[d, -1])
    eps = list(range(n_ep))
    psd = orc.psd_epochs(x, wl, eps)
    white = orc.whiten(x, wl, psd, eps)
    assert psd.shape == (2, n_ep, 8193) and white.shape == (2, n_ep * blk)
    wts = np.array([1.5] + [2.0] * 6 + [1.5]) / 15.0
    # standard error of the bin-averaged level: each bin of a 15-segment Welch mean scatters by
    # about 1/sqrt(15 / 1.2) of its level; bins are nearly independent, 8191 of them are averaged
    se_level = math.sqrt(1.2 / 15 / 8191)
    for d in range(2):
        for e in eps:
            level = psd[d, e, 1:8192].mean() * fs / 2.0
            want = float(wts @ v[d, e:e + 8])
            assert abs(level / want - 1.0) < 6 * se_level, (d, e, level, want)
            for wrong in (e - 1, e + 1):  # a one-epoch slip of the look-back is far outside
                if 0 <= wrong <= n_blocks - 8:
                    assert abs(float(wts @ v[d, wrong:wrong + 8]) / want - 1.0) > 30 * se_level
            taps = orc.whitening_taps(psd[d, e], wl.nfft, wl.fs, wl.f_highpass, wl.fir_len)
            seg = white[d, e * blk + wl.crop:(e + 1) * blk - wl.crop]  # away from block edges
            var = float(np.mean(seg ** 2))
            want_var = v[d, e + 8] * float(np.sum(taps ** 2))
            # the highpassed output is correlated over a few samples: allow 6 standard errors of
            # sqrt(2 / (n / 2))
            se_var = math.sqrt(2.0 / (len(seg) / 2))
            assert abs(var / want_var - 1.0) < 6 * se_var, (d, e, var, want_var)
            for nb in (e + 7, e + 9):  # the neighbouring raw blocks differ by >= 1.8x
                if nb < n_blocks:
                    assert abs(v[d, nb] / v[d, e + 8] - 1.0) > 0.44


def _conv_brute(x, w, stride, pad):
    cin, L = x.shape
    cout, _, k = w.shape
    lout = (L + 2 * pad - k) // stride + 1
    out = np.zeros((cout, lout))
    for co in range(cout):
        for t in range(lout):
            acc = 0.0
            for ci in range(cin):
                for r in range(k):
                    s = t * stride + r - pad
                    if 0 <= s < L:
                        acc += w[co, ci, r] * x[ci, s]
            out[co, t] = acc
    return out


@pytest.mark.parametrize("stride,k,pad", [(1, 3, 1), (2, 3, 1), (2, 1, 0), (2, 7, 3)])
def test_conv1d_bruteforce(stride, k, pad):
    rng = np.random.default_rng(stride * 10 + k)
    x = rng.standard_normal((2, 8))
    w = rng.standard_normal((2, 2, k))
    assert np.max(np.abs(orc.conv1d(x, w, stride, pad) - _conv_brute(x, w, stride, pad))) < 1e-13


def test_conv1d_identity_tap_is_copy():
    x = np.random.default_rng(0).standard_normal((3, 11))
    w = np.zeros((3, 3, 3))
    for c in range(3):
        w[c, c, 1] = 1.0
    assert np.array_equal(orc.conv1d(x, w, 1, 1), x)


def test_conv1d_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(9)
    x = rng.standard_normal((16, 96))
    w = rng.standard_normal((32, 16, 3))
    ref = torch.nn.functional.conv1d(torch.from_numpy(x)[None], torch.from_numpy(w), stride=2, padding=1)[0]
    assert np.max(np.abs(orc.conv1d(x, w, 2, 1) - ref.numpy())) < 1e-12


def test_group_norm_constant_groups_give_beta_and_matches_torch():
    torch = pytest.importorskip("torch")
    C, L, G = 8, 10, 4
    gamma = np.linspace(0.5, 1.5, C)
    beta = np.linspace(-0.1, 0.1, C)
    x = np.repeat(np.arange(G, dtype=np.float64), (C // G) * L).reshape(C, L)
    assert np.allclose(orc.group_norm(x, G, gamma, beta, 1e-5), beta[:, None] * np.ones((1, L)), atol=1e-14)
    rng = np.random.default_rng(2)
    x = rng.standard_normal((C, L)) * 3 + 1
    ref = torch.nn.functional.group_norm(torch.from_numpy(x)[None], G, torch.from_numpy(gamma),
                                         torch.from_numpy(beta), 1e-5)[0].numpy()
    assert np.max(np.abs(orc.group_norm(x, G, gamma, beta, 1e-5) - ref)) < 1e-12


def _torch_resnet(net, w):
    """Independent float64 torch restatement of the 1D ResNet with GroupNorm."""
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    shapes = inputs.weight_shapes(net)
    params, off = {}, 0
    for name, shape in shapes:
        size = int(np.prod(shape))
        params[name] = torch.from_numpy(w[off:off + size].astype(np.float64).reshape(shape))
        off += size

    def fwd(x):
        h = F.conv1d(x, params["stem.w"], stride=net.stem_stride, padding=net.stem_k // 2)
        h = F.relu(F.group_norm(h, net.groups, params["stem.gamma"], params["stem.beta"], net.eps))
        if net.stem_pool:
            h = F.max_pool1d(h, 3, 2, 1)
        cin = net.widths[0]
        for s, (width, nb) in enumerate(zip(net.widths, net.blocks)):
            for b in range(nb):
                stride = 2 if (s > 0 and b == 0) else 1
                p = f"s{s}b{b}."
                o = F.conv1d(h, params[p + "c1.w"], stride=stride, padding=1)
                o = F.relu(F.group_norm(o, net.groups, params[p + "g1.gamma"], params[p + "g1.beta"], net.eps))
                o = F.conv1d(o, params[p + "c2.w"], padding=1)
                o = F.group_norm(o, net.groups, params[p + "g2.gamma"], params[p + "g2.beta"], net.eps)
                if p + "sc.w" in params:
                    sc = F.conv1d(h, params[p + "sc.w"], stride=stride)
                    sc = F.group_norm(sc, net.groups, params[p + "gsc.gamma"], params[p + "gsc.beta"], net.eps)
                else:
                    sc = h
                h = F.relu(o + sc)
                cin = width
        pooled = h.mean(dim=2)
        return pooled @ params["fc.w"] + params["fc.b"]

    return fwd


def test_tiny_network_matches_torch_restatement():
    torch = pytest.importorskip("torch")
    net = inputs.TINY_NET
    w = inputs.make_weights(net, seed=5)
    assert len(w) == 3345
    rng = np.random.default_rng(4)
    xs = rng.standard_normal((4, 2, 3072))
    ref = _torch_resnet(net, w)(torch.from_numpy(xs)).numpy()
    got = np.array([orc.network(net, w, x) for x in xs])
    assert np.max(np.abs(got - ref)) < 1e-11


@pytest.mark.slow
def test_resnet34_network_matches_torch_restatement():
    torch = pytest.importorskip("torch")
    net = inputs.RESNET34_NET
    w = inputs.make_weights(net, seed=6)
    rng = np.random.default_rng(7)
    x = rng.standard_normal((1, 2, 3072))
    ref = _torch_resnet(net, w)(torch.from_numpy(x)).numpy()
    got = orc.network(net, w, x[0])
    assert abs(got - ref[0]) < 1e-10 * max(1.0, abs(ref[0]))


def test_infer_windows_matches_per_window_and_wraps_circularly():
    net = inputs.TINY_NET
    w = inputs.make_weights(net, seed=5)
    rng = np.random.default_rng(12)
    W, n_y = 3072, 3072 * 3
    y = rng.standard_normal((2, n_y))
    shift = 2048 * 2
    got = orc.infer_windows(net, w, y, W, 512, 1024, 5, shift)
    for j in [0, 4]:
        s0 = 512 + j * 1024
        idx1 = (s0 + shift + np.arange(W)) % n_y
        x = np.stack([y[0, s0:s0 + W], y[1, idx1]])
        assert got[j] == pytest.approx(orc.network(net, w, x), abs=1e-13)


# ---------------------------------------------------------------- integration + triggers

def test_integrate_closed_forms():
    assert np.allclose(orc.integrate(np.full(10, 2.5), 4), 2.5)
    ramp = np.arange(20, dtype=np.float64)
    # mean of j..j+3 = j + 1.5
    assert np.allclose(orc.integrate(ramp, 4), np.arange(17) + 1.5)
    imp = np.zeros(12)
    imp[6] = 1.0
    out = orc.integrate(imp, 4)
    assert np.allclose(out, [0, 0, 0, 0.25, 0.25, 0.25, 0.25, 0, 0])


def _triggers_brute(I, half):
    res = []
    for j in range(len(I)):
        lo, hi = max(0, j - half), min(len(I), j + half + 1)
        window = I[lo:hi]
        if I[j] == window.max() and np.argmax(window) + lo == j:
            res.append(j)
    return np.array(res, dtype=np.int64)


def test_triggers_bruteforce_and_ties():
    rng = np.random.default_rng(0)
    I = rng.standard_normal(500)
    for half in [1, 4, 16]:
        assert np.array_equal(orc.triggers(I, half), _triggers_brute(I, half))
    # plateau: earliest index wins
    I = np.array([0, 1, 3, 3, 3, 1, 0, 5.0])
    assert list(orc.triggers(I, 2)) == [2, 7]
    assert list(orc.triggers(np.full(6, 1.0), 2)) == [0]
    assert list(orc.triggers(np.array([1.0, 1, 1, 0, 0, 0, 2, 2]), 2)) == [0, 6]


# ---------------------------------------------------------------- paper window arithmetic

def test_paper_window_arithmetic_golden():
    g = {k: v["value"] for k, v in json.load(open(os.path.join(GOLDEN, "paper_timing.json"))).items()
         if not k.startswith("_")}
    assert g["train_psd_s"] + g["train_whitened_s"] == g["train_window_s"]
    assert g["train_whitened_s"] - 2 * g["crop_each_edge_s"] == g["analysed_window_s"]
    assert 1.0 / g["inference_rate_hz"] == g["window_stride_s"]
    assert g["analysed_window_s"] - g["window_stride_s"] == g["window_overlap_s"]
    assert g["latency_kernel_pad_s"] + g["latency_whitening_wait_s"] == g["fig1_gap_s"]
    assert g["timeslide_step_s"] > g["light_travel_s"]
    fs = g["sample_rate_hz"]
    wl = inputs.PLAIN_64S
    assert wl.fs == fs and wl.win_len == g["analysed_window_s"] * fs
    assert wl.crop == g["crop_each_edge_s"] * fs and wl.nfft == g["train_psd_s"] * fs
    assert wl.stride == g["window_stride_s"] * fs and wl.psd_len == g["online_psd_s"] * fs
    assert wl.n_int == g["integration_s"] * g["inference_rate_hz"]
    assert wl.cluster_half == g["cluster_s"] / 2 * g["inference_rate_hz"]
    # the 64 s plain span fits 247 windows after cropping; the workload analyses 244 of them
    assert (wl.n_raw - 2 * wl.crop - wl.win_len) // wl.stride + 1 == 247
    assert wl.n_win == 244
    h = inputs.HOUR_RESNET34
    assert h.n_win * h.stride == 3600 * fs and h.n_int == 16


# ---------------------------------------------------------------- false-alarm rates and trigger times

def test_far_closed_form_and_ties():
    """Sec. IX: FAR = #(background > event) / livetime; strictly greater, so a
    tie with a background event does not count it."""
    N, T = 1000, 86400.0
    bg = np.arange(1, N + 1, dtype=np.float64)
    ev = np.array([0.5, 1.0, 1.5, 999.0, N, N + 1.0, -np.inf, np.inf, 500.25])
    counts, rates = orc.far(bg, ev, T)
    want = np.array([N, N - 1, N - 1, 1, 0, 0, N, 0, N - 500])
    assert np.array_equal(counts, want)
    assert np.array_equal(rates, want / T)
    c2, _ = orc.far(np.array([3.0, 3.0, 3.0, 1.0]), np.array([2.0, 3.0, 0.0]), 1.0)
    assert list(c2) == [3, 0, 4]
    c3, r3 = orc.far(np.array([]), np.array([0.0, -1.0]), 10.0)
    assert list(c3) == [0, 0] and list(r3) == [0.0, 0.0]


def test_trigger_time_recovers_a_step_response():
    """A response that switches on at the window whose right edge is t_c + 0.75 s
    (Fig. 1) and stays on: integration (Sec. II) and clustering put the first
    maximum n_int - 1 windows later, and the estimate returns exactly t_c."""
    import dataclasses
    for wl in (inputs.PLAIN_64S, dataclasses.replace(inputs.PLAIN_64S, stride=128)):  # 4 Hz and 16 Hz
        n_win = 200
        for w_on in (7, 40, 123):
            z = np.zeros(n_win)
            z[w_on:] = 1.0
            stat = orc.integrate(z, wl.n_int)
            trig = orc.triggers(stat, wl.cluster_half)
            on = [int(j) for j in trig if stat[j] == 1.0]  # (the flat zero stretch before it may cluster too)
            assert on == [w_on]  # earliest index of the plateau
            t0 = 1234.5
            t_c_true = t0 + (wl.crop + w_on * wl.stride + wl.win_len) / wl.fs - 0.75
            t_peak, t_c = orc.trigger_times(wl, on, t0, 0.75)
            assert abs(t_c[0] - t_c_true) < 1e-9
            assert abs(t_peak[0] - (t_c_true + 0.75 + (wl.n_int - 1) * wl.stride / wl.fs)) < 1e-9


# ---------------------------------------------------------------- resampling

@pytest.mark.parametrize("M", [2, 4, 8])
def test_resample_matches_scipy_resample_poly(M):
    """The oracle's decimator is the Kaiser-windowed design of scipy.signal.resample_poly
    (library check on the valid outputs)."""
    scipy_signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(M)
    x = rng.standard_normal((2, 5000 + 37))
    y, first = orc.resample(x, M)
    ref = scipy_signal.resample_poly(x, 1, M, axis=-1, window=("kaiser", 5.0))
    j0 = first // M
    assert first % M == 0 and y.shape[1] > 0
    assert np.max(np.abs(y - ref[:, j0:j0 + y.shape[1]])) < 1e-12


def test_resample_closed_forms():
    """DC passes exactly; a cosine comes out scaled by the filter's response
    H(f) = sum_k h_k cos(2 pi f k / fs_in), which is ~1 in the band and small
    above the new Nyquist frequency."""
    M, fs = 8, 16384.0
    h = orc.resample_taps(M)
    assert abs(h.sum() - 1.0) < 1e-14 and np.allclose(h, h[::-1])
    y, _ = orc.resample(np.full(4000, 3.25), M)
    assert np.max(np.abs(y - 3.25)) < 1e-13
    L = 10 * M
    k = np.arange(-L, L + 1)
    n = np.arange(40000)
    for f in (100.0, 800.0, 1500.0):
        H = float(np.sum(h * np.cos(2 * np.pi * f * k / fs)))
        y, first = orc.resample(np.cos(2 * np.pi * f * n / fs), M)
        t = first + M * np.arange(y.shape[-1])
        assert np.max(np.abs(y - H * np.cos(2 * np.pi * f * t / fs))) < 1e-12
        if f <= 800.0:
            assert abs(H - 1.0) < 2e-3
        else:
            assert abs(H) < 0.02
    y, _ = orc.resample(np.zeros(100), M)  # shorter than the filter
    assert y.shape[-1] == 0
