"""Failure detection on the GPU without a fault: the library's bounded device-side waits.

The tensor-core kernels wait on mbarriers with a time limit; a wait that gives up is
recorded on the device, the kernel leaves early and afg_sync reports AFG_ERR_TIMEOUT.
afg_wait_check runs CTAs whose waits, through the same helper and record, are on an
mbarrier nothing arrives on, so each ends by its limit with nothing in flight.  The test
checks the status, that the record clears, that the waits lasted their limit, and that the
context keeps working afterwards (a normal analysis still matches the oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc  # noqa: E402
from paper_2403_18661_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_the_context_recovers():
    wl = inputs.PLAIN_64S
    x, _ = inputs.make_strain(wl)
    w = inputs.make_weights(wl.net, wl.weight_seed)
    ctx = abi.Context(wl, w, precision=abi.AFG_BF16)
    ctx.sync()  # nothing recorded yet
    limit = 50_000_000  # 50 ms
    waited = ctx.wait_check(limit, n_blocks=8)
    with pytest.raises(abi.AfgError) as e:
        ctx.sync()
    assert e.value.status == abi.AFG_ERR_TIMEOUT
    ns = waited.cpu().numpy()
    assert np.all(ns >= limit) and np.all(ns < 20 * limit), ns
    ctx.sync()  # the record was cleared by the call that reported it
    # a zero limit gives up at once
    ctx.wait_check(0, n_blocks=1)
    with pytest.raises(abi.AfgError) as e:
        ctx.sync()
    assert e.value.status == abi.AFG_ERR_TIMEOUT
    # the context still works: the BF16 path on the 64 s span against the oracle
    ref = orc.analyze_plain(x.astype(np.float64), wl, w)
    logits = ctx.analyze(torch.from_numpy(x).cuda())[0]
    ctx.sync()
    z = logits.cpu().numpy()
    assert np.max(np.abs(z - ref["logits"]) / (1 + np.abs(ref["logits"]))) < 2e-3
    with pytest.raises(abi.AfgError) as e:
        ctx.wait_check(-1)
    assert e.value.status == abi.AFG_ERR_ARG
    ctx.close()
