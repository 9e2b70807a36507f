"""False-alarm rates (Sec. IX) and trigger times (Sec. II, Fig. 1) through the C ABI.

FAR counts are integer work and must equal the oracle's exactly; the rates
are count / livetime in double precision on both sides (IEEE division), so
they are compared exactly too.  The device sort must return the background
in decreasing order, bit for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc  # noqa: E402
from paper_2403_18661_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    wl = inputs.PLAIN_64S
    c = abi.Context(wl, inputs.make_weights(wl.net, wl.weight_seed))
    yield c
    c.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _check(ctx, bg, fg, livetime, **kw):
    n_above, far, srt = ctx.far(_dev(bg) if "bg_stat" not in kw else kw.pop("bg_stat"), _dev(fg), livetime, **kw)
    ctx.sync()
    return n_above.cpu().numpy(), far.cpu().numpy(), srt.cpu().numpy()


def test_far_matches_the_definition(ctx):
    rng = np.random.default_rng(5)
    bg = np.round(rng.standard_normal(200_003), 2).astype(np.float32)  # many ties
    fg = np.concatenate([bg[rng.integers(0, len(bg), 300)], rng.standard_normal(600).astype(np.float32) * 3,
                         np.array([np.inf, -np.inf, 0.0, -0.0, 100.0, -100.0], dtype=np.float32)]).astype(np.float32)
    T = 8_362_200.0
    cnt, far, srt = _check(ctx, bg, fg, T)
    want, rate = orc.far(bg, fg, T)
    assert np.array_equal(cnt, want)
    assert np.array_equal(far, rate)
    assert np.array_equal(srt[:len(bg)].view(np.uint32), np.sort(bg)[::-1].view(np.uint32)) or \
        np.array_equal(srt[:len(bg)], np.sort(bg)[::-1])


def test_far_gathers_through_indices_with_a_device_count(ctx):
    rng = np.random.default_rng(6)
    stat = rng.standard_normal(5000).astype(np.float32)
    idx = rng.integers(0, 5000, 3000).astype(np.int64)
    fg = rng.standard_normal(257).astype(np.float32)
    n_dev = torch.tensor([2500], dtype=torch.int64, device="cuda")
    cnt, far, srt = _check(ctx, None, fg, 10.0, bg_stat=_dev(stat), bg_idx=_dev(idx), n_bg=n_dev, bg_cap=3000)
    bg = stat[idx[:2500]]
    want, rate = orc.far(bg, fg, 10.0)
    assert np.array_equal(cnt, want) and np.array_equal(far, rate)
    assert np.array_equal(srt[:2500], np.sort(bg)[::-1])


def test_far_degenerate_counts(ctx):
    fg = np.array([-1.0, 0.0, 1.0], dtype=np.float32)
    bg = np.array([0.5, 2.0, -3.0, 0.5], dtype=np.float32)
    # an empty background
    cnt, far, _ = _check(ctx, bg, fg, 1.0, n_bg=0)
    assert list(cnt) == [0, 0, 0] and list(far) == [0.0, 0.0, 0.0]
    # a count above the capacity uses the capacity (a truncated trigger list)
    cnt, _, _ = _check(ctx, bg, fg, 1.0, n_bg=1000, bg_cap=3)
    assert list(cnt) == list(orc.far(bg[:3], fg, 1.0)[0])
    # no foreground events
    n_above, far, srt = ctx.far(_dev(bg), _dev(np.zeros(0, dtype=np.float32)), 1.0)
    ctx.sync()
    assert n_above.numel() == 0 and np.array_equal(srt.cpu().numpy()[:4], np.sort(bg)[::-1])
    with pytest.raises(abi.AfgError) as e:
        ctx.far(_dev(bg), _dev(fg), 0.0)
    assert e.value.status == abi.AFG_ERR_ARG


def test_far_sorts_millions(ctx):
    rng = np.random.default_rng(7)
    bg = (rng.standard_normal(3_000_001) * 10).astype(np.float32)
    fg = bg[::10007].copy()
    cnt, _, srt = _check(ctx, bg, fg, 3600.0)
    assert np.array_equal(srt[:len(bg)], np.sort(bg)[::-1])
    want, _ = orc.far(bg, fg, 3600.0)
    assert np.array_equal(cnt, want)


def test_far_of_a_timeslide_background():
    """The background is the trigger list of a timeslide batch, passed on the device as
    afg_batch_run leaves it; the foreground is a few of its own events."""
    wl = inputs.TIMESLIDE_DAY
    x, segs = inputs.make_segments([90, 117, 101], seed=31, chirp_every_s=40.0)
    w = inputs.make_weights(wl.net, wl.weight_seed)
    c = abi.Context(wl, w, precision=abi.AFG_BF16)
    xd = _dev(x)
    n_win, tw, ts = c.batch_layout(segs, 3, 2048)
    logits, stat, trig, n_trig = c.batch_run(xd, segs, 3, 2048, trig_cap=4096)
    livetime = tw * wl.stride / wl.fs
    c.sync()
    n = int(n_trig.item())
    assert 0 < n <= 4096
    fg_stat = stat[trig[:min(8, n)]].clone()  # a few of its own events (indices written by the batch)
    n_above, far, srt = c.far(stat, fg_stat, livetime, bg_idx=trig, n_bg=n_trig, bg_cap=4096)
    c.sync()
    bg = stat.cpu().numpy()[trig.cpu().numpy()[:n]]
    want, rate = orc.far(bg, fg_stat.cpu().numpy(), livetime)
    assert np.array_equal(n_above.cpu().numpy(), want) and np.array_equal(far.cpu().numpy(), rate)
    assert np.array_equal(srt.cpu().numpy()[:n], np.sort(bg)[::-1])
    c.close()


@pytest.mark.parametrize("mode", ["plain", "epoch"])
def test_trigger_times_match_the_oracle(mode):
    import dataclasses
    wl = inputs.PLAIN_64S if mode == "plain" else dataclasses.replace(inputs.HOUR_RESNET34, n_win=64,
                                                                       net=inputs.PLAIN_64S.net)
    c = abi.Context(wl, inputs.make_weights(wl.net, wl.weight_seed))
    idx = np.array([0, 5, 17, wl.n_win - wl.n_int])
    tp, tc = c.trigger_times(idx, n_raw=10**7, t0=1238166018.0, gap_s=0.75)
    want_p, want_c = orc.trigger_times(wl, idx, 1238166018.0, 0.75)
    assert np.allclose(tp, want_p, rtol=0, atol=1e-6) and np.allclose(tc, want_c, rtol=0, atol=1e-6)
    with pytest.raises(abi.AfgError):
        c.trigger_times([wl.n_win - wl.n_int + 1], n_raw=10**7)
    c.close()
