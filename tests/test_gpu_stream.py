"""Streaming analysis with continuous batching (afg_stream_*) against the FP64
oracle, and the same results alone and in a mix of streams."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc  # noqa: E402
from paper_2403_18661_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

# BF16 16-channel network against the FP64 oracle: three times the measured 5.6e-4
BF16_LOGIT_TOL = 2e-3
# alone vs in the mix: the only difference is the overlap-save block alignment of
# the whitening (FP32 rounding order), so the FP32 logit tolerance applies
MIX_TOL = 1e-4
WL = inputs.SERVING_128


def _strain(seconds, seed):
    n = int(seconds * WL.fs)
    x = np.stack([inputs.coloured_noise(n, seed * 2 + d) for d in range(2)])
    return x.astype(np.float32)


def _push_all(ctx, sid, x, chunk=512):
    for a in range(0, x.shape[1], chunk):
        ctx.stream_push(sid, x[:, a:a + chunk])


def _oracle_stream(x, w, WL=WL):
    """Epoch-mode whitening of everything pushed, windows at the stream stride, 1 s integration."""
    x64 = x.astype(np.float64)
    P = x.shape[1]
    q = P - WL.psd_len - WL.crop + 1  # whitened samples available
    white = np.empty((2, q))
    for e in range((q + WL.epoch_len - 1) // WL.epoch_len):
        lo, hi = e * WL.epoch_len, min(q, (e + 1) * WL.epoch_len)
        for d in range(2):
            psd = orc.welch(x64[d, e * WL.epoch_len: e * WL.epoch_len + WL.psd_len], WL.nfft, WL.hop, WL.fs)
            taps = orc.whitening_taps(psd, WL.nfft, WL.fs, WL.f_highpass, WL.fir_len)
            white[d, lo:hi] = orc.fir(x64[d], taps, WL.psd_len + lo, hi - lo)
    n_win = (q - WL.win_len) // WL.stride + 1
    z = orc.infer_windows(WL.net, w, white, WL.win_len, 0, WL.stride, n_win)
    return z, orc.integrate(z, WL.n_int), white


@pytest.fixture(scope="module")
def weights():
    return inputs.make_weights(WL.net, WL.weight_seed)


def test_stream_matches_oracle(weights, capsys):
    x = _strain(85.0, 3)
    ctx = abi.Context(WL, weights, precision=abi.AFG_BF16)
    ctx.stream_start(max_streams=4)
    sid = ctx.stream_open()
    _push_all(ctx, sid, x)
    ctx.stream_flush()
    r = ctx.stream_poll(sid)
    z, st, white = _oracle_stream(x, weights)
    assert len(r) == len(st) and np.array_equal(r["window"], np.arange(WL.n_int - 1, len(z)))
    err_z = np.abs(r["logit"] - z[WL.n_int - 1:]) / (1 + np.abs(z[WL.n_int - 1:]))
    err_s = np.abs(r["stat"] - st) / (1 + np.abs(st))
    # the same BF16 network over the oracle's whitened strain: only the stream's FP32
    # whitening (rounding ~1e-6 of unit variance) separates the two, so a tolerance ten
    # times the alone-vs-mix one catches any misplaced or mis-scaled whitened sample
    zb = ctx.infer_windows(torch.from_numpy(white.astype(np.float32)).cuda(), 0, WL.stride, len(z)).cpu().numpy()
    err_w = np.abs(r["logit"] - zb[WL.n_int - 1:]) / (1 + np.abs(zb[WL.n_int - 1:]))
    with capsys.disabled():
        print(f"\nstream: {len(r)} results, max |dz|/(1+|z|) = {err_z.max():.3e}, stat {err_s.max():.3e}, "
              f"vs BF16 network on oracle-whitened strain {err_w.max():.3e}")
    assert err_z.max() < BF16_LOGIT_TOL and err_s.max() < BF16_LOGIT_TOL
    assert err_w.max() < 10 * MIX_TOL
    assert np.all(r["t_done"] >= r["t_push"])
    ctx.close()


def test_stream_small_steps_on_clusters(weights):
    """Steps of one 0.25 s push each (4 new windows): the latency-bound network launch, where
    each window is split over a cluster of CTAs that exchange GroupNorm statistics and halo
    rows through distributed shared memory.  The warm-up runs in large steps (one CTA per
    window); every result of both kinds is checked against the oracle and against the same
    BF16 network run on the oracle's whitened strain."""
    x = _strain(74.0, 5)
    ctx = abi.Context(WL, weights, precision=abi.AFG_BF16)
    ctx.stream_start(max_streams=4)
    sid = ctx.stream_open()
    warm = 67 * WL.fs
    _push_all(ctx, sid, x[:, :warm], chunk=4096)
    ctx.stream_flush()
    steps0 = ctx.stream_stats()["steps"]
    n_small = 0
    for a in range(warm, x.shape[1], 512):
        ctx.stream_push(sid, x[:, a:a + 512])
        ctx.stream_flush()  # one push per step
        n_small += 1
    assert ctx.stream_stats()["steps"] - steps0 == n_small
    r = ctx.stream_poll(sid)
    z, st, white = _oracle_stream(x, weights)
    assert len(r) == len(st) and np.array_equal(r["window"], np.arange(WL.n_int - 1, len(z)))
    n_late = int(np.sum(r["window"] >= (warm - WL.psd_len - WL.crop - WL.win_len) // WL.stride))
    assert n_late >= 4 * (n_small - 1)  # results produced by the small steps
    err_z = np.abs(r["logit"] - z[WL.n_int - 1:]) / (1 + np.abs(z[WL.n_int - 1:]))
    err_s = np.abs(r["stat"] - st) / (1 + np.abs(st))
    zb = ctx.infer_windows(torch.from_numpy(white.astype(np.float32)).cuda(), 0, WL.stride, len(z)).cpu().numpy()
    err_w = np.abs(r["logit"] - zb[WL.n_int - 1:]) / (1 + np.abs(zb[WL.n_int - 1:]))
    assert err_z.max() < BF16_LOGIT_TOL and err_s.max() < BF16_LOGIT_TOL
    # the clustered network differs from one CTA per window only in its summation order (the
    # same FP32 and BF16 arithmetic per element): the alone-vs-mix bound applies
    assert err_w.max() < MIX_TOL, err_w.max()
    ctx.close()


def test_stream_long_filter(weights):
    """A 2 s (4096-tap) whitening filter: stream pieces are too long for the 4096-point block, so
    the steps use the 16384-point multi-stream kernel and the separate scatter launch, and the
    filters come from the one-CTA FP64 build (more than 2048 lags)."""
    import dataclasses
    wl = dataclasses.replace(WL, fir_len=4096)
    x = _strain(86.0, 9)
    ctx = abi.Context(wl, weights, precision=abi.AFG_BF16)
    ctx.stream_start(max_streams=4)
    sid = ctx.stream_open()
    _push_all(ctx, sid, x)
    ctx.stream_flush()
    r = ctx.stream_poll(sid)
    z, st, white = _oracle_stream(x, weights, wl)
    assert len(r) == len(st) and len(r) > 100
    err_s = np.abs(r["stat"] - st) / (1 + np.abs(st))
    zb = ctx.infer_windows(torch.from_numpy(white.astype(np.float32)).cuda(), 0, wl.stride, len(z)).cpu().numpy()
    err_w = np.abs(r["logit"] - zb[wl.n_int - 1:]) / (1 + np.abs(zb[wl.n_int - 1:]))
    assert err_s.max() < BF16_LOGIT_TOL
    assert err_w.max() < 10 * MIX_TOL, err_w.max()
    ctx.close()


def test_stream_round_robin_steps_match_alone(weights):
    """Three streams pushed round-robin one 0.25 s chunk at a time, without waiting: the
    engine forms steps of one or a few pushes of different streams, two of them in flight.
    Each stream's results must equal the same stream analysed alone with the same chunking."""
    xs = [_strain(72.0, 40 + i) for i in range(3)]
    warm = 67 * WL.fs

    def run(streams):
        ctx = abi.Context(WL, weights, precision=abi.AFG_BF16)
        ctx.stream_start(max_streams=4)
        sids = [ctx.stream_open() for _ in streams]
        for sid, x in zip(sids, streams):
            _push_all(ctx, sid, x[:, :warm], chunk=4096)
        ctx.stream_flush()
        for a in range(warm, streams[0].shape[1], 512):
            for sid, x in zip(sids, streams):
                ctx.stream_push(sid, x[:, a:a + 512])
        ctx.stream_flush()
        out = [ctx.stream_poll(sid) for sid in sids]
        ctx.close()
        return out

    mixed = run(xs)
    for i, x in enumerate(xs):
        alone = run([x])[0]
        assert np.array_equal(mixed[i]["window"], alone["window"])
        for key in ("logit", "stat"):
            d = np.abs(mixed[i][key] - alone[key]) / (1 + np.abs(alone[key]))
            assert d.max() <= MIX_TOL, (i, key, d.max())


def test_stream_same_alone_and_in_the_mix(weights):
    xa = _strain(80.0, 7)
    ctx = abi.Context(WL, weights, precision=abi.AFG_BF16)
    ctx.stream_start(max_streams=16)
    a = ctx.stream_open()
    _push_all(ctx, a, xa)
    ctx.stream_flush()
    alone = ctx.stream_poll(a)
    ctx.stream_close(a)
    # the same stream again, now interleaved with 11 others of random chunk sizes
    rng = np.random.default_rng(1)
    others = [(ctx.stream_open(), _strain(80.0, 100 + i)) for i in range(11)]
    a = ctx.stream_open()
    cursors = {sid: 0 for sid, _ in others}
    pos_a = 0
    while pos_a < xa.shape[1]:
        for sid, x in others:
            n = int(rng.choice([128, 512, 1000, 2048]))
            c = cursors[sid]
            if c < x.shape[1]:
                ctx.stream_push(sid, x[:, c:c + n])
                cursors[sid] = c + n
        ctx.stream_push(a, xa[:, pos_a:pos_a + 512])
        pos_a += 512
    ctx.stream_flush()
    mixed = ctx.stream_poll(a)
    assert np.array_equal(mixed["window"], alone["window"])
    for key in ("logit", "stat"):
        d = np.abs(mixed[key] - alone[key]) / (1 + np.abs(alone[key]))
        assert d.max() <= MIX_TOL, (key, d.max())
    st = ctx.stream_stats()
    assert st["steps"] > 0 and st["windows"] > len(alone)
    ctx.close()


def test_stream_admission_by_hbm_budget(weights):
    """Admission by HBM budget, with no headroom beyond two streams: everything a step and a
    gains refresh need (the Welch periodograms and the FP64 filter-build transforms) is reserved
    and counted when the engine starts, so the admitted streams then run through several PSD
    refreshes without any allocation, and their results match the oracle."""
    probe = abi.Context(WL, weights, precision=abi.AFG_BF16)
    probe.stream_start(max_streams=8)
    base = probe.bytes_held
    s0 = probe.stream_open()
    per_stream = probe.bytes_held - base
    probe.close()
    ctx = abi.Context(WL, weights, precision=abi.AFG_BF16, hbm_budget=base + 2 * per_stream + 4096)
    ctx.stream_start(max_streams=8)
    assert ctx.bytes_held == base
    s1, s2 = ctx.stream_open(), ctx.stream_open()
    with pytest.raises(abi.AfgError) as e:
        ctx.stream_open()
    assert e.value.status == -4
    ctx.stream_close(s1)
    ctx.stream_flush()
    import time
    deadline = time.time() + 5
    while True:  # the slot's memory is released by the engine once its work is done
        try:
            s3 = ctx.stream_open()
            break
        except abi.AfgError:
            assert time.time() < deadline
            time.sleep(0.05)
    # 72 s into each admitted stream: the first gains and the refreshes every 8 s after them
    xs = {s2: _strain(72.0, 21), s3: _strain(72.0, 22)}
    for a in range(0, 72 * WL.fs, 2048):
        for sid, x in xs.items():
            ctx.stream_push(sid, x[:, a:a + 2048])
    ctx.stream_flush()
    assert ctx.bytes_held <= base + 2 * per_stream + 4096
    for sid, x in xs.items():
        r = ctx.stream_poll(sid)
        z, st, _ = _oracle_stream(x, weights)
        assert len(r) == len(st) > 0
        assert np.max(np.abs(r["stat"] - st) / (1 + np.abs(st))) < BF16_LOGIT_TOL
    ctx.close()


def test_stream_refuses_nan_and_closed_streams(weights):
    ctx = abi.Context(WL, weights, precision=abi.AFG_BF16)
    ctx.stream_start(max_streams=2)
    sid = ctx.stream_open()
    bad = np.zeros((2, 64), dtype=np.float32)
    bad[1, 5] = np.nan
    with pytest.raises(abi.AfgError) as e:
        ctx.stream_push(sid, bad)
    assert e.value.status == -7
    ctx.stream_close(sid)
    with pytest.raises(abi.AfgError) as e:
        ctx.stream_push(sid, np.zeros((2, 64), dtype=np.float32))
    assert e.value.status == -6
    ctx.close()


def test_stream_push_many_matches_single_pushes(weights):
    """afg_stream_push_many (a burst of arrivals in one call) queues the same chunks as single
    pushes in the same order: three streams pushed one round of 0.25 s chunks per call give the
    same windows, and logits and statistics within the mix tolerance, as single round-robin pushes;
    the tickets count each stream's pushes.  A burst with a non-finite sample or a closed stream is
    refused whole: nothing of it is queued (the next ticket continues the count)."""
    xs = [_strain(72.0, 60 + i) for i in range(3)]
    warm = 67 * WL.fs

    def run(many):
        ctx = abi.Context(WL, weights, precision=abi.AFG_BF16)
        ctx.stream_start(max_streams=4)
        sids = [ctx.stream_open() for _ in xs]
        for sid, x in zip(sids, xs):
            _push_all(ctx, sid, x[:, :warm], chunk=4096)
        ctx.stream_flush()
        first = warm // 4096 + (1 if warm % 4096 else 0)
        for r, a in enumerate(range(warm, xs[0].shape[1], 512)):
            if many:
                t = ctx.stream_push_many(sids, np.stack([x[:, a:a + 512] for x in xs]))
                assert t.tolist() == [first + r] * len(sids)
            else:
                for sid, x in zip(sids, xs):
                    ctx.stream_push(sid, x[:, a:a + 512])
        ctx.stream_flush()
        out = [ctx.stream_poll(sid) for sid in sids]
        if many:
            nxt = first + len(range(warm, xs[0].shape[1], 512))
            bad = np.zeros((3, 2, 64), dtype=np.float32)
            bad[2, 1, 7] = np.inf
            with pytest.raises(abi.AfgError) as e:
                ctx.stream_push_many(sids, bad)
            assert e.value.status == -7
            ctx.stream_close(sids[1])
            with pytest.raises(abi.AfgError) as e:
                ctx.stream_push_many(sids, np.zeros((3, 2, 64), dtype=np.float32))
            assert e.value.status == -6
            # nothing of either refused burst was queued
            assert ctx.stream_push(sids[0], np.zeros((2, 64), dtype=np.float32)) == nxt
        ctx.close()
        return out

    single, many = run(False), run(True)
    for i in range(len(xs)):
        assert len(many[i]) == len(single[i]) > 0
        assert np.array_equal(many[i]["window"], single[i]["window"])
        for key in ("logit", "stat"):
            d = np.abs(many[i][key] - single[i][key]) / (1 + np.abs(single[i][key]))
            assert d.max() <= MIX_TOL, (i, key, d.max())


def test_stream_128_streams_sampled(weights, capsys):
    """The serving configuration at its full size: 128 streams (max_streams = 128), staggered so that
    their PSD refreshes fall in different steps and several share one batched refresh, then 0.25 s
    chunks of every stream per afg_stream_push_many burst.  Every stream delivers exactly its windows'
    statistics (windows n_int - 1 .. n_win - 1, finite), and four sampled streams match the oracle's
    streaming analysis within the BF16 tolerance."""
    n_streams = 128
    rng = np.random.default_rng(7)
    lead = [64.0 + 0.25 * int(rng.integers(0, 32)) for _ in range(n_streams)]  # staggered warm-up
    tail_s = 12.0
    xs = [_strain(lead[i] + tail_s, 300 + i) for i in range(n_streams)]
    ctx = abi.Context(WL, weights, precision=abi.AFG_BF16)
    ctx.stream_start(max_streams=n_streams, max_chunk=4096)
    sids = [ctx.stream_open() for _ in range(n_streams)]
    for sid, x, l in zip(sids, xs, lead):
        _push_all(ctx, sid, x[:, :int(l * WL.fs)], chunk=4096)
    for a in range(0, int(tail_s * WL.fs), 512):
        ctx.stream_push_many(sids, np.stack([x[:, int(l * WL.fs) + a:int(l * WL.fs) + a + 512]
                                             for x, l in zip(xs, lead)]))
    ctx.stream_flush(120.0)
    res = [ctx.stream_poll(sid) for sid in sids]
    for x, r in zip(xs, res):
        q = x.shape[1] - WL.psd_len - WL.crop + 1
        n_win = (q - WL.win_len) // WL.stride + 1
        assert np.array_equal(r["window"], np.arange(WL.n_int - 1, n_win))
        assert np.all(np.isfinite(r["stat"])) and np.all(np.isfinite(r["logit"]))
    worst = 0.0
    for i in (0, 37, 85, 127):
        z, st, _ = _oracle_stream(xs[i], weights)
        r = res[i]
        err = max(float(np.max(np.abs(r["logit"] - z[WL.n_int - 1:]) / (1 + np.abs(z[WL.n_int - 1:])))),
                  float(np.max(np.abs(r["stat"] - st) / (1 + np.abs(st)))))
        worst = max(worst, err)
        assert err < BF16_LOGIT_TOL, (i, err)
    stats = ctx.stream_stats()
    with capsys.disabled():
        print(f"\n128 streams: {sum(len(r) for r in res)} results in {stats['steps']} steps; "
              f"4 sampled streams vs the oracle, max |dz|/(1+|z|) = {worst:.3e}")
    ctx.close()
