"""Conv tile autotuning of the BF16 tensor-core path (ResNet34-GN).

Every tile the tuner may pick must compute the same network: each candidate
of each layer geometry is applied and the logits are compared with the FP32
path (the ResNet34-GN BF16 logit tolerance, 2e-2 (1 + |z|): three times the
measured 5.9e-3 of BF16 operand rounding through 36 GroupNorm'd convolutions)
and with the default tiles, within 8e-3 (1 + |z|): three times the measured
2.5e-3 (tiles differ only in the FP32 accumulation order inside a layer,
which moves a BF16 rounding of an activation now and then).  37 windows leave partial tiles for every
windows-per-tile count from 2 to 5.
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2403_18661_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

BF16_LOGIT_TOL = 2e-2
TILE_TOL = 8e-3


@pytest.fixture(scope="module")
def resnet():
    wl = dataclasses.replace(inputs.HOUR_RESNET34, n_win=37, n_chirps=1, name="resnet34-37win")
    x, _ = inputs.make_strain(wl)
    w = inputs.make_weights(wl.net, wl.weight_seed)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    c32 = abi.Context(wl, w, precision=abi.AFG_FP32)
    z32 = c32.analyze(xd)[0].cpu().numpy()
    c32.close()
    c16 = abi.Context(wl, w, precision=abi.AFG_BF16)
    z16 = c16.analyze(xd)[0].cpu().numpy()
    c16.sync()
    yield wl, w, xd, z32, z16, c16
    c16.close()


def _geometry(t):
    return (t["cin"], t["cout"], t["lin"], t["lout"], t["stride"], t["taps"], t["residual"])


def test_every_tile_candidate_computes_the_same_network(resnet, capsys):
    wl, w, xd, z32, z16, ctx = resnet
    default = ctx.tiles()
    groups = {}
    for t in default:
        groups.setdefault(_geometry(t), []).append(t["layer"])
    n_runs, worst32, worst16 = 0, 0.0, 0.0
    for geo, layers in groups.items():
        cands = ctx.tile_candidates(layers[0])
        assert cands, f"no tile fits layer geometry {geo}"
        for c in cands:
            ctx.set_tiles([dict(c, layer=l) for l in layers])
            z = ctx.analyze(xd)[0].cpu().numpy()
            ctx.sync()
            d32 = float(np.max(np.abs(z - z32) / (1 + np.abs(z32))))
            d16 = float(np.max(np.abs(z - z16) / (1 + np.abs(z16))))
            knobs = {k: c[k] for k in ("orient", "wpc", "kb", "stages", "acc_bufs")}
            assert np.all(np.isfinite(z)), (geo, knobs)
            assert d32 < BF16_LOGIT_TOL, (geo, knobs, d32)
            assert d16 < TILE_TOL, (geo, knobs, d16)
            worst32, worst16 = max(worst32, d32), max(worst16, d16)
            n_runs += 1
        ctx.set_tiles(default)
    with capsys.disabled():
        print(f"\n{n_runs} tiles over {len(groups)} geometries: vs FP32 max {worst32:.3e}, "
              f"vs default tiles max {worst16:.3e}")


def test_autotune_picks_the_fastest_measured_tile(resnet, capsys):
    wl, w, xd, z32, z16, ctx = resnet
    default = ctx.tiles()
    ctx.autotune(n_win=256)
    tiles = ctx.tiles()
    assert len(tiles) == len(default)
    tot_c = tot_d = 0.0
    for t in tiles:
        assert t["tuned"] == 1
        assert t["n_candidates"] >= len(ctx.tile_candidates(t["layer"]))
        assert 0.0 < t["us_chosen"] <= t["us_default"], t
        tot_c += t["us_chosen"]
        tot_d += t["us_default"]
    z = ctx.analyze(xd)[0].cpu().numpy()
    ctx.sync()
    d32 = float(np.max(np.abs(z - z32) / (1 + np.abs(z32))))
    with capsys.disabled():
        print(f"\nautotune (256 windows): sum over layers {tot_d:.0f} us default -> {tot_c:.0f} us chosen; "
              f"vs FP32 max {d32:.3e}")
        for t in tiles:
            print("  layer {layer:2d} {cin:3d}->{cout:3d} L{lout:3d} s{stride} k{taps} res{residual}: "
                  "orient {orient} wpc {wpc} kb {kb:3d} stages {stages} acc {acc_bufs} "
                  "{us_chosen:8.1f} us (default {us_default:8.1f})".format(**t))
    assert d32 < BF16_LOGIT_TOL
    ctx.set_tiles(default)


def test_tiles_set_rejects_knobs_that_do_not_fit(resnet):
    wl, w, xd, z32, z16, ctx = resnet
    before = ctx.tiles()
    wide = next(t for t in before if t["cout"] >= 256)
    bad = [dict(wide, wpc=0), dict(wide, kb=48), dict(wide, stages=9), dict(wide, acc_bufs=3),
           dict(wide, orient=0, kb=wide["cin"]), dict(wide, wpc=6, acc_bufs=1), dict(wide, layer=0),
           dict(wide, layer=len(before) + 1)]
    for b in bad:
        with pytest.raises(abi.AfgError) as ei:
            ctx.set_tiles([before[0], b])
        assert ei.value.status == abi.AFG_ERR_ARG
        assert ctx.tiles() == before  # nothing applied


def test_autotune_is_refused_without_a_tensor_core_plan():
    wl = inputs.PLAIN_64S
    w = inputs.make_weights(wl.net, wl.weight_seed)
    ctx = abi.Context(wl, w, precision=abi.AFG_FP32)
    with pytest.raises(abi.AfgError) as ei:
        ctx.autotune(64)
    assert ei.value.status == abi.AFG_ERR_UNSUPPORTED
    ctx.close()


def test_fused_network_candidates_compute_the_same_network(capsys):
    """Every tuning candidate of the fused 16-channel network (8 or 12 epilogue warps, 1 or 2 issue warps,
    polling sleep) computes the same network: each candidate's logits against the oracle within the BF16
    tolerance of that network (2e-3 (1 + |z|)), and bit-identical to the default where only the issue warps
    or the polling sleep differ (the arithmetic and its order are the same).  afg_autotune then keeps the
    fastest, and the context computes the same logits with it."""
    from oracle import oracle as orc
    wl = inputs.PLAIN_64S
    w = inputs.make_weights(wl.net, wl.weight_seed)
    rng = np.random.default_rng(7)
    y = rng.standard_normal((2, 40000))
    stride, n_win = 131, 200
    want = orc.infer_windows(wl.net, w, y, wl.win_len, 0, stride, n_win)
    yd = torch.from_numpy(y.astype(np.float32)).cuda()
    ctx = abi.Context(wl, w, precision=abi.AFG_BF16)
    cands = ctx.fused_tuning_candidates()
    assert len(cands) >= 4 and cands[0]["epi_warps"] == 12 and cands[0]["issue_warps"] == 2
    got = {}
    for c in cands:
        ctx.set_fused_tuning(c)
        z = ctx.infer_windows(yd, 0, stride, n_win).cpu().numpy()
        ctx.sync()
        err = np.abs(z - want) / (1 + np.abs(want))
        with capsys.disabled():
            print(f"\nfused candidate {c['epi_warps']} epilogue / {c['issue_warps']} issue warps, "
                  f"{c['spin_ns']} ns: max |dz|/(1+|z|) vs oracle = {err.max():.2e}")
        assert err.max() < 2e-3, (c, err.max())
        got[(c["epi_warps"], c["issue_warps"], c["spin_ns"])] = z
    for k, z in got.items():
        same_order = next(v for kk, v in got.items() if kk[0] == k[0])
        assert np.array_equal(z, same_order), k
    ctx.autotune(1024)
    t = ctx.fused_tuning()
    assert t["tuned"] == 1 and t["n_candidates"] == len(cands) and 0 < t["us_chosen"] <= t["us_default"]
    z = ctx.infer_windows(yd, 0, stride, n_win).cpu().numpy()
    ctx.sync()
    assert np.array_equal(z, got[(t["epi_warps"], t["issue_warps"], t["spin_ns"])])
    with capsys.disabled():
        print(f"fused tuning: {t}")
    with pytest.raises(abi.AfgError) as ei:
        ctx.set_fused_tuning({"epi_warps": 16, "issue_warps": 2, "spin_ns": 64})
    assert ei.value.status == abi.AFG_ERR_ARG
    ctx.close()
    ctx32 = abi.Context(wl, w, precision=abi.AFG_FP32)
    with pytest.raises(abi.AfgError) as ei:
        ctx32.fused_tuning()
    assert ei.value.status == abi.AFG_ERR_UNSUPPORTED
    ctx32.close()
