"""Decimation to the analysis rate (Sec. IV.A) through afg_resample against the FP64 oracle.

Tolerance: each output accumulates 2L + 1 <= 321 FP32 products of taps
(sum |h| ~ 1.2) and inputs bounded by X, so its rounding error is at most
(2L + 1) u sum|h| X ~ 2.3e-5 X; the test uses 2e-5 max|x| (typical errors are
~1e-6 X).  Output counts and the first input sample are integer work: exact.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc  # noqa: E402
from paper_2403_18661_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 2e-5


@pytest.fixture(scope="module")
def ctx():
    wl = inputs.PLAIN_64S
    c = abi.Context(wl, inputs.make_weights(wl.net, wl.weight_seed))
    yield c
    c.close()


@pytest.mark.parametrize("M,n_in", [(2, 16384 * 3 + 37), (4, 70001), (8, 16384 * 10 + 5), (16, 40000), (8, 161),
                                    (8, 160)])
def test_resample_matches_oracle(ctx, M, n_in, capsys):
    rng = np.random.default_rng(M * 1000 + n_in)
    x = (rng.standard_normal((2, n_in)) * 1e-21).astype(np.float32)  # strain-like magnitudes
    y, first = ctx.resample(torch.from_numpy(x).cuda(), M)
    ctx.sync()
    want, first_o = orc.resample(x.astype(np.float64), M)
    assert first == first_o and y.shape[1] == want.shape[1]
    if want.shape[1]:
        err = np.max(np.abs(y.cpu().numpy() - want)) / np.max(np.abs(x))
        with capsys.disabled():
            print(f"\nresample M={M} n_in={n_in}: {want.shape[1]} outputs, max |dy|/max|x| = {err:.2e}")
        assert err < TOL


def test_resample_strided_rows_and_errors(ctx):
    rng = np.random.default_rng(3)
    big = rng.standard_normal((2, 30000)).astype(np.float32)
    xd = torch.from_numpy(big).cuda()[:, :25000]  # row stride 30000 > n_in
    y, first = ctx.resample(xd, 8)
    ctx.sync()
    want, _ = orc.resample(big[:, :25000].astype(np.float64), 8)
    assert np.max(np.abs(y.cpu().numpy() - want)) / np.max(np.abs(big)) < TOL
    for bad in (1, 17):
        with pytest.raises(abi.AfgError):
            ctx.resample(xd, bad)
