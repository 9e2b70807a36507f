"""World-size-2 check of the multi-GPU bookkeeping on CPU (gloo): per-rank seeds
differ, and the job throughput is the units of all ranks over the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2403_18661_gb300 import dist as pdist
    w, r, lr = pdist.env()
    seconds = [2.0, 3.0][rank]
    units = [3600.0, 3600.0][rank]
    rate, total, t = pdist.job_throughput(units, seconds, world)
    q.put((r, w, pdist.rank_seed(4321, r), rate, total, t))
    dist.barrier()
    dist.destroy_process_group()


def test_job_throughput_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, s0, rate0, tot0, t0), (r1, w1, s1, rate1, tot1, t1) = out
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert s0 != s1
    assert tot0 == tot1 == 7200.0 and t0 == t1 == 3.0
    assert rate0 == rate1 == pytest.approx(2400.0)


def test_single_process_needs_no_collective():
    from paper_2403_18661_gb300 import dist as pdist
    assert pdist.job_throughput(3600.0, 3.0, 1) == (1200.0, 3600.0, 3.0)


# ------------------------------------------------------------------ one background over two ranks

SHARD_LENGTHS, SHARD_SHIFTS = [75, 80], 6


def _shard_series(k_first, n_k):
    """Background statistics (the cluster maxima of every series) and livetime of timeslides
    k_first .. k_first + n_k - 1 of a two-segment case, computed with the oracle (Sec. IX)."""
    import numpy as np

    from oracle import oracle as orc
    from paper_2403_18661_gb300 import inputs
    wl = inputs.TIMESLIDE_DAY
    x, segs = inputs.make_segments(SHARD_LENGTHS, seed=17, chirp_every_s=30.0)
    w = inputs.make_weights(wl.net, wl.weight_seed)
    bg, live = [], 0.0
    for off, n in segs:
        xs = x[:, off:off + n].astype(np.float64)
        eps = list(range((n - wl.psd_len - wl.crop) // wl.epoch_len))
        white = orc.whiten(xs, wl, orc.psd_epochs(xs, wl, eps), eps)
        n_win = (white.shape[1] - wl.win_len) // wl.stride + 1
        for k in range(k_first, k_first + n_k):
            z = orc.infer_windows(wl.net, w, white, wl.win_len, 0, wl.stride, n_win, k * wl.fs)
            st = orc.integrate(z, wl.n_int)
            bg.append(st[orc.triggers(st, wl.cluster_half)])
            live += n_win * wl.stride / wl.fs
    return np.concatenate(bg).astype(np.float32), live


def _shard_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np

    from oracle import oracle as orc
    from paper_2403_18661_gb300 import dist as pdist
    k_first, n_k = pdist.shift_range(SHARD_SHIFTS, world, rank)
    bg, live = _shard_series(k_first, n_k)
    gathered = pdist.gather_background(torch.from_numpy(bg), world).numpy()
    livetime = pdist.sum_over_ranks(live, world)
    fg = np.linspace(float(gathered.min()), float(gathered.max()), 17)
    counts, far = orc.far(gathered, fg, livetime)
    q.put((rank, (k_first, n_k), gathered, livetime, counts, far))
    dist.barrier()
    dist.destroy_process_group()


def test_timeslides_split_over_two_ranks_match_one_process():
    """Two gloo ranks each take half of the timeslides of one background (shift_range), gather
    their background triggers (gather_background) and livetimes, and rank the same foreground:
    the gathered background equals the single-process one (as a multiset: the order differs),
    and the false-alarm counts and rates are identical."""
    import numpy as np

    from oracle import oracle as orc
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=600) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [(1, 3), (4, 3)]
    ref_bg, ref_live = _shard_series(1, SHARD_SHIFTS)
    for rank, _, gathered, livetime, counts, far in out:
        assert np.array_equal(np.sort(gathered), np.sort(ref_bg))
        assert livetime == ref_live
        fg = np.linspace(float(ref_bg.min()), float(ref_bg.max()), 17)
        ref_counts, ref_far = orc.far(ref_bg, fg, ref_live)
        assert np.array_equal(counts, ref_counts) and np.array_equal(far, ref_far)
    assert np.array_equal(out[0][2], out[1][2])  # every rank holds the same gathered background
