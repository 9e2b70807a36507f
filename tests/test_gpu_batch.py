"""Timeslide batches (Sec. IX) through afg_batch_run against the FP64 oracle.

Three uneven segments, three timeslides each (L1 shifted by 1, 2, 3 s
within the segment's whitened span), tiny network at 4 Hz.  The oracle
whitens each segment in epoch mode on its own and evaluates every window of
every series directly; tolerances are those of the single-series tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import trigger_match  # noqa: E402
from oracle import oracle as orc  # noqa: E402
from paper_2403_18661_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

LOGIT_TOL = 1e-4
BF16_LOGIT_TOL = 2e-3  # three times the measured 6.1e-4 of this batch
N_SHIFT = 3
SHIFT_STEP = 2048


@pytest.fixture(scope="module")
def batch_case():
    wl = inputs.TIMESLIDE_DAY
    lengths = [90, 117, 101]
    x, segs = inputs.make_segments(lengths, seed=31, chirp_every_s=40.0)
    w = inputs.make_weights(wl.net, wl.weight_seed)
    ref = []  # per segment: list over shifts of (logits, stat, triggers)
    for off, n in segs:
        xs = x[:, off:off + n].astype(np.float64)
        n_ep = (n - wl.psd_len - wl.crop) // wl.epoch_len
        eps = list(range(n_ep))
        psd = orc.psd_epochs(xs, wl, eps)
        white = orc.whiten(xs, wl, psd, eps)
        n_win = (white.shape[1] - wl.win_len) // wl.stride + 1
        per = []
        for k in range(1, N_SHIFT + 1):
            z = orc.infer_windows(wl.net, w, white, wl.win_len, 0, wl.stride, n_win, k * SHIFT_STEP)
            st = orc.integrate(z, wl.n_int)
            per.append((z, st, orc.triggers(st, wl.cluster_half)))
        ref.append(per)
    return wl, x, segs, w, ref


def _check(wl, segs, ref, logits, stat, trig, n_trig, tol):
    lg, st = logits.cpu().numpy(), stat.cpu().numpy()
    tr = trig.cpu().numpy()[: int(n_trig.item())]
    assert np.all(np.diff(tr) > 0)
    lo = so = 0
    worst = 0.0
    tot = dict(oracle=0, gpu=0, identical=True, decisive=0, near_tie=0, near_tie_same=0, near_tie_moved=0,
               near_ties=[])
    for per in ref:
        for z, s_ref, t_ref in per:
            got = lg[lo:lo + len(z)]
            err = np.abs(got - z) / (1 + np.abs(z))
            worst = max(worst, float(err.max()))
            assert err.max() < tol
            s_got = st[so:so + len(s_ref)]
            # this series' triggers (global statistic indices) against the oracle's, both directions
            mine = np.array([int(t) - so for t in tr if so <= t < so + len(s_ref)], dtype=np.int64)
            c = trigger_match.compare(s_got, s_ref, mine, t_ref, wl.cluster_half, tol)
            for k in tot:
                tot[k] = (tot[k] and c[k]) if k == "identical" else tot[k] + c[k]
            lo += len(z)
            so += len(s_ref)
    assert lo == len(lg) and so == len(st)
    return worst, tot


@pytest.mark.parametrize("precision,tol", [(abi.AFG_FP32, LOGIT_TOL), (abi.AFG_BF16, BF16_LOGIT_TOL)])
def test_batch_matches_oracle(batch_case, precision, tol, capsys):
    wl, x, segs, w, ref = batch_case
    ctx = abi.Context(wl, w, precision=precision)
    n_win, tw, ts = ctx.batch_layout(segs, N_SHIFT, SHIFT_STEP)
    assert n_win == [len(per[0][0]) for per in ref]
    out = ctx.batch_run(torch.from_numpy(x).cuda(), segs, N_SHIFT, SHIFT_STEP)
    ctx.sync()
    worst, c = _check(wl, segs, ref, *out, tol)
    with capsys.disabled():
        print(f"\nbatch precision {precision}: {tw} windows, max |dz|/(1+|z|) = {worst:.3e}; "
              f"{trigger_match.summary(c)}")
    # every trigger was checked: decisive ones index for index, near-ties (with the BF16 tolerance
    # almost all maxima of this near-flat random-weight statistic) at the same index or tied
    assert c["oracle"] > 0 and c["decisive"] + c["near_tie_same"] + c["near_tie_moved"] == c["oracle"] + c["gpu"]
    ctx.close()


def test_batch_graph_replay_is_identical(batch_case):
    wl, x, segs, w, ref = batch_case
    ctx = abi.Context(wl, w, precision=abi.AFG_BF16)
    xd = torch.from_numpy(x).cuda()
    direct = [t.clone() for t in ctx.batch_run(xd, segs, N_SHIFT, SHIFT_STEP)]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        out = None
        for _ in range(3):  # capture, then two replays into the same buffers
            out = ctx.batch_run(xd, segs, N_SHIFT, SHIFT_STEP, use_graph=True, out=out, stream=s)
    s.synchronize()
    ctx.sync()
    for a, b in zip(direct, out):
        assert torch.equal(a, b)
    ctx.close()


def test_batch_rejects_short_segments(batch_case):
    wl, x, segs, w, ref = batch_case
    ctx = abi.Context(wl, w, precision=abi.AFG_BF16)
    with pytest.raises(abi.AfgError) as e:
        ctx.batch_layout([(0, 60 * 2048)], N_SHIFT, SHIFT_STEP)  # shorter than the 64 s look-back
    assert e.value.status == -1
    ctx.close()


def test_batch_shift_ranges_concatenate(batch_case):
    """A background split into timeslide ranges (shift_first, as the ranks of a multi-GPU job take
    them) gives, series by series, exactly the logits, statistics and triggers of the whole batch."""
    wl, x, segs, w, ref = batch_case
    ctx = abi.Context(wl, w, precision=abi.AFG_BF16)
    xd = torch.from_numpy(x).cuda()
    n_win, _, _ = ctx.batch_layout(segs, N_SHIFT, SHIFT_STEP)
    full = [t.cpu().numpy() for t in ctx.batch_run(xd, segs, N_SHIFT, SHIFT_STEP)]
    parts = [(1, 1), (2, N_SHIFT - 1)]
    got = {}
    for k_first, n_k in parts:
        lg, st, tr, nt = [t.cpu().numpy() for t in ctx.batch_run(xd, segs, n_k, SHIFT_STEP, shift_first=k_first)]
        tr = tr[: int(nt[0])]
        lo = so = 0
        for i, nw in enumerate(n_win):
            for k in range(k_first, k_first + n_k):
                ns = nw - wl.n_int + 1
                got[(i, k)] = (lg[lo:lo + nw], st[so:so + ns], tr[(tr >= so) & (tr < so + ns)] - so)
                lo += nw
                so += ns
    ctx.sync()
    lg, st, tr, nt = full
    tr = tr[: int(nt[0])]
    lo = so = 0
    for i, nw in enumerate(n_win):
        for k in range(1, N_SHIFT + 1):
            ns = nw - wl.n_int + 1
            a_lg, a_st, a_tr = got[(i, k)]
            assert np.array_equal(a_lg, lg[lo:lo + nw]) and np.array_equal(a_st, st[so:so + ns])
            assert np.array_equal(a_tr, tr[(tr >= so) & (tr < so + ns)] - so)
            lo += nw
            so += ns
    with pytest.raises(abi.AfgError):  # the largest timeslide must fit the shortest segment
        ctx.batch_layout(segs, 1, SHIFT_STEP, shift_first=10 ** 6)
    ctx.close()


def _series_slices(n_win, n_shift, n_int):
    """(logit, statistic) start offsets of every (segment, timeslide) series, in series order."""
    lo = so = 0
    out = {}
    for i, nw in enumerate(n_win):
        for k in range(n_shift):
            out[(i, k)] = (lo, so, nw, nw - n_int + 1)
            lo += nw
            so += nw - n_int + 1
    return out


def test_batch_full_day_sampled(capsys):
    """The batching workload at its full size, in the configuration the bench times: 40 uneven
    segments (about 1 day) x 100 timeslides of 1 s in one persistent launch, BF16.  At this size
    the oracle checks samples and the rest is checked by properties that hold at any size:
    * series of the two shortest segments at timeslides 1, 2, 50 and 100, recomputed as small
      batches (shift_first ranges), are bit-identical to the same series of the full launch;
    * 16 windows of each of those series, spread over the series, match the oracle's logits
      (whitening of the segment on its own, then the network) within the BF16 tolerance;
    * each sampled series' statistic is the 1 s moving average of its logits, and its triggers
      are exactly the clustering of its own statistic."""
    wl = inputs.TIMESLIDE_DAY
    n_shift, step = 100, wl.fs
    lengths = inputs.segment_lengths(n_seg=40, total_s=86400)
    x, segs = inputs.make_segments(lengths, seed=wl.seed, chirp_every_s=300.0, workers=16)
    w = inputs.make_weights(wl.net, wl.weight_seed)
    ctx = abi.Context(wl, w, precision=abi.AFG_BF16)
    xd = torch.from_numpy(x).cuda()
    n_win, tw, ts = ctx.batch_layout(segs, n_shift, step)
    lg, st, tr, nt = [t.cpu().numpy() for t in ctx.batch_run(xd, segs, n_shift, step)]
    ctx.sync()
    assert len(lg) == tw == sum(n_win) * n_shift and len(st) == ts
    tr = tr[: int(nt[0])]
    assert np.all(np.diff(tr) > 0)
    sl = _series_slices(n_win, n_shift, wl.n_int)
    picks = sorted(range(len(segs)), key=lambda i: segs[i][1])[:2]
    sub_segs = [segs[i] for i in picks]
    sub_n_win, _, _ = ctx.batch_layout(sub_segs, 1, step)
    worst, checked = 0.0, 0
    rng = np.random.default_rng(5)
    for j, i in enumerate(picks):
        off, n = segs[i]
        xs = x[:, off:off + n].astype(np.float64)
        eps = list(range((n - wl.psd_len - wl.crop) // wl.epoch_len))
        white = orc.whiten(xs, wl, orc.psd_epochs(xs, wl, eps), eps)
        for k_first, n_k in ((1, 2), (50, 1), (100, 1)):
            s_lg, s_st, s_tr, s_nt = [t.cpu().numpy() for t in
                                      ctx.batch_run(xd, sub_segs, n_k, step, shift_first=k_first)]
            s_tr = s_tr[: int(s_nt[0])]
            s_sl = _series_slices(sub_n_win, n_k, wl.n_int)
            for kk in range(n_k):
                k = k_first + kk
                lo, so, nw, ns = sl[(i, k - 1)]
                a_lo, a_so, a_nw, a_ns = s_sl[(j, kk)]
                assert (a_nw, a_ns) == (nw, ns) == (n_win[i], n_win[i] - wl.n_int + 1)
                z, s = lg[lo:lo + nw], st[so:so + ns]
                assert np.array_equal(z, s_lg[a_lo:a_lo + nw]) and np.array_equal(s, s_st[a_so:a_so + ns])
                mine = tr[(tr >= so) & (tr < so + ns)] - so
                assert np.array_equal(mine, s_tr[(s_tr >= a_so) & (s_tr < a_so + ns)] - a_so)
                # properties: the statistic is the moving average of the logits; the triggers cluster it
                ma = np.convolve(z.astype(np.float64), np.ones(wl.n_int) / wl.n_int, mode="valid")
                assert np.max(np.abs(s - ma) / (1 + np.abs(ma))) < 1e-5
                assert np.array_equal(orc.triggers(s.astype(np.float64), wl.cluster_half), mine)
                # sampled windows against the oracle
                for w0 in sorted(rng.choice(nw, size=16, replace=False).tolist()):
                    ref = orc.infer_windows(wl.net, w, white, wl.win_len, w0 * wl.stride, wl.stride, 1, k * step)
                    e = abs(float(z[w0]) - float(ref[0])) / (1 + abs(float(ref[0])))
                    worst = max(worst, e)
                    checked += 1
                    assert e < BF16_LOGIT_TOL, (i, k, w0, e)
    with capsys.disabled():
        print(f"\nfull-day batch: {tw} windows, {len(tr)} triggers; {checked} sampled windows of "
              f"{len(picks)} segments x 4 timeslides vs the oracle, max |dz|/(1+|z|) = {worst:.3e}")
    ctx.close()
