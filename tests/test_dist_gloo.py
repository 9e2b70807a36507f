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
