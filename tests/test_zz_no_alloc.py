"""The allocation-free Welch PSD entry point against the regular one.

afg_psd_estimate_noalloc serves hosts that cannot let a library call
cudaMalloc (an application that owns all device memory through its own
pool, or a latency-critical loop that cannot afford cudaMalloc's implicit
synchronisation).  It keeps its scratch in a static device array instead of
a context workspace; this checks, through the C ABI, that two calls in a row
give the PSD that afg_psd_estimate gives, and that oversize requests are
refused before anything runs.  Collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2403_18661_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

PSD_RTOL = 1e-4  # the PSD tolerance of the parity tests


def test_noalloc_psd_matches_context_psd_on_two_calls():
    wl = inputs.PLAIN_64S
    x, _ = inputs.make_strain(wl)
    xd = torch.from_numpy(x).cuda()
    ctx = abi.Context(wl, inputs.make_weights(wl.net, wl.weight_seed))
    cases = [dict(n_psd=3, psd_step=16384, psd_span=98304), dict(n_psd=1, psd_step=0, psd_span=131072)]
    for case in cases:
        ref = ctx.psd_estimate(xd, **case)
        for _ in range(2):
            out = torch.full_like(ref, float("nan"))
            abi.psd_estimate_noalloc(xd, fs=wl.fs, hop=wl.hop, out=out, **case)
            torch.cuda.synchronize()
            assert torch.isfinite(out).all()
            rel = ((out - ref).abs() / ref).max().item()
            assert rel <= PSD_RTOL, rel
    ctx.close()


def test_noalloc_psd_refuses_more_periodograms_than_its_scratch():
    n = 16384 + 32 * 8192  # 33 segments x 2 detectors = 66 > 64
    xd = torch.zeros((2, n), device="cuda")
    out = torch.zeros((2, 1, 8193), dtype=torch.float64, device="cuda")
    with pytest.raises(abi.AfgError) as e:
        abi.psd_estimate_noalloc(xd, out=out)
    assert e.value.status == -4
    # one detector fits
    abi.psd_estimate_noalloc(xd[:1].contiguous(), out=out[:1].contiguous())
    torch.cuda.synchronize()
