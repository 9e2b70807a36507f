"""The allocation-free Welch PSD entry point against the regular one.

afg_psd_estimate_noalloc serves hosts that cannot let a library call
cudaMalloc (an application that owns all device memory through its own
pool, or a latency-critical loop that cannot afford cudaMalloc's implicit
synchronisation).  It keeps its scratch in a static device array instead of
a context workspace; this checks, through the C ABI, that two calls in a row
give exactly the PSD that afg_psd_estimate gives, also after a call that
filled the whole scratch, and that oversize requests are refused before
anything runs.  Collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2403_18661_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu



def _ref_and_noalloc(ctx, xd, fs, hop, **case):
    ref = ctx.psd_estimate(xd, **case)
    out = torch.full_like(ref, float("nan"))
    abi.psd_estimate_noalloc(xd, fs=fs, hop=hop, out=out, **case)
    torch.cuda.synchronize()
    return ref, out


def test_noalloc_psd_matches_context_psd_on_two_calls():
    """Both entry points run the same kernels with the same arguments, so the PSDs must be
    bit-identical; each layout is called twice in a row on the shared scratch."""
    wl = inputs.PLAIN_64S
    x, _ = inputs.make_strain(wl)
    xd = torch.from_numpy(x).cuda()
    ctx = abi.Context(wl, inputs.make_weights(wl.net, wl.weight_seed))
    cases = [dict(n_psd=3, psd_step=16384, psd_span=98304), dict(n_psd=1, psd_step=0, psd_span=131072)]
    for case in cases:
        for _ in range(2):
            ref, out = _ref_and_noalloc(ctx, xd, wl.fs, wl.hop, **case)
            assert torch.isfinite(out).all()
            assert torch.equal(out, ref)
    ctx.close()


def test_noalloc_psd_after_a_larger_call_and_one_detector():
    """The scratch keeps the last call's contents: a call that fills all 64 periodograms is
    followed by smaller calls with other segment layouts (and one detector), each of which must
    still equal afg_psd_estimate exactly."""
    wl = inputs.PLAIN_64S
    n = 16384 + 31 * 8192  # 32 segments per detector: 2 x 32 = 64 periodograms, the whole scratch
    x = np.stack([inputs.coloured_noise(n, 70 + d) for d in range(2)]).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    ctx = abi.Context(wl, inputs.make_weights(wl.net, wl.weight_seed))
    cases = [(xd, dict(n_psd=1, psd_step=0, psd_span=n)),                          # 64 periodograms
             (xd, dict(n_psd=5, psd_step=24576, psd_span=65536)),                  # 2 x 19
             (xd[:1].contiguous(), dict(n_psd=2, psd_step=8192, psd_span=32768)),  # 1 x 4
             (xd[1:].contiguous(), dict(n_psd=1, psd_step=0, psd_span=16384))]     # 1 x 1
    for xin, case in cases:
        ref, out = _ref_and_noalloc(ctx, xin, wl.fs, wl.hop, **case)
        assert torch.isfinite(out).all()
        assert torch.equal(out, ref), case
    ctx.close()


def test_noalloc_psd_refuses_more_periodograms_than_its_scratch():
    n = 16384 + 32 * 8192  # 33 segments x 2 detectors = 66 > 64
    xd = torch.zeros((2, n), device="cuda")
    out = torch.zeros((2, 1, 8193), dtype=torch.float64, device="cuda")
    with pytest.raises(abi.AfgError) as e:
        abi.psd_estimate_noalloc(xd, out=out)
    assert e.value.status == -4
    # one detector (33 periodograms) fits
    abi.psd_estimate_noalloc(xd[:1].contiguous(), out=out[:1].contiguous())
    torch.cuda.synchronize()
