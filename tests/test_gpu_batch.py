"""Timeslide batches (Sec. IX) through afg_batch_run against the FP64 oracle.

Three uneven segments, three timeslides each (L1 shifted by 1, 2, 3 s
within the segment's whitened span), tiny network at 4 Hz.  The oracle
whitens each segment in epoch mode on its own and evaluates every window of
every series directly; tolerances are those of the single-series tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc  # noqa: E402
from paper_2403_18661_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

LOGIT_TOL = 1e-4
BF16_LOGIT_TOL = 5e-2
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
    lo = so = 0
    worst = 0.0
    for per in ref:
        for z, s_ref, t_ref in per:
            got = lg[lo:lo + len(z)]
            err = np.abs(got - z) / (1 + np.abs(z))
            worst = max(worst, float(err.max()))
            assert err.max() < tol
            s_got = st[so:so + len(s_ref)]
            assert np.max(np.abs(s_got - s_ref) / (1 + np.abs(s_ref))) < tol
            # triggers of this series (global statistic indices) must be the oracle's,
            # except near-ties, which may move by one sample
            mine = set(int(t) - so for t in tr if so <= t < so + len(s_ref))
            for j in t_ref:
                lo_j, hi_j = max(0, j - wl.cluster_half), min(len(s_ref), j + wl.cluster_half + 1)
                nb = np.delete(s_ref[lo_j:hi_j], j - lo_j)
                margin = s_ref[j] - (nb.max() if len(nb) else -np.inf)
                if margin > 2 * tol * (1 + abs(s_ref[j])):
                    assert j in mine or (j - 1) in mine or (j + 1) in mine
            lo += len(z)
            so += len(s_ref)
    assert lo == len(lg) and so == len(st)
    return worst


@pytest.mark.parametrize("precision,tol", [(abi.AFG_FP32, LOGIT_TOL), (abi.AFG_BF16, BF16_LOGIT_TOL)])
def test_batch_matches_oracle(batch_case, precision, tol, capsys):
    wl, x, segs, w, ref = batch_case
    ctx = abi.Context(wl, w, precision=precision)
    n_win, tw, ts = ctx.batch_layout(segs, N_SHIFT, SHIFT_STEP)
    assert n_win == [len(per[0][0]) for per in ref]
    out = ctx.batch_run(torch.from_numpy(x).cuda(), segs, N_SHIFT, SHIFT_STEP)
    ctx.sync()
    worst = _check(wl, segs, ref, *out, tol)
    with capsys.disabled():
        print(f"\nbatch precision {precision}: {tw} windows, max |dz|/(1+|z|) = {worst:.3e}")
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
