"""Host-side checks of the C ABI (no GPU needed): the library loads and
exports every symbol include/aframe_gb.h declares, and host-only entry points
behave as documented."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2403_18661_gb300 import abi, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            text = open(os.path.join(inc, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(afg_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2403_18661_gb300 import build
    build.build()
    return abi.load()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared_symbols()
    assert len(declared) >= 12
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
        assert name in abi.SIGNATURES, f"{name} has no binding signature"


def test_binding_covers_only_declared_symbols():
    assert set(abi.SIGNATURES) <= _declared_symbols()


def test_version_and_status_strings(lib):
    assert "sm_103a" in abi.version()
    assert lib.afg_status_string(0) == b"AFG_OK"
    assert lib.afg_status_string(-4) == b"AFG_ERR_BUDGET"
    assert lib.afg_status_string(-99) == b"AFG_ERR_UNKNOWN"


@pytest.mark.parametrize("net", [inputs.TINY_NET, inputs.RESNET34_NET])
def test_weights_count_matches_flat_layout(lib, net):
    assert abi.weights_count(net) == inputs.n_weights(net)


def test_weights_count_rejects_bad_nets(lib):
    import dataclasses
    for bad in [dict(in_ch=3), dict(stem_k=4), dict(widths=(20,)), dict(widths=(48,)), dict(groups=3),
                dict(stem_stride=3)]:
        spec = dataclasses.replace(inputs.TINY_NET, **bad)
        with pytest.raises(abi.AfgError):
            abi.weights_count(spec)


def test_null_context_is_refused(lib):
    assert lib.afg_ctx_destroy(None) == -1
    assert lib.afg_psd_estimate(None, None, 0, 0, 0, 0, 0, None, None) == -1
    assert lib.afg_analyze(None, None, None, None, None, None, 0, None, None) == -1


def test_resample_size_matches_the_oracle():
    """Host-only sizing of the decimator (no GPU): output count and first input sample."""
    from oracle import oracle as orc
    for M in (2, 4, 8, 16):
        for n_in in (0, 10 * M * 2, 10 * M * 2 + 1, 10 * M * 2 + M, 12345, 16384 * 8 + 3):
            n, first = abi.resample_size(n_in, M)
            y, first_o = orc.resample(np.zeros(n_in), M)
            assert n == y.shape[-1] and first == first_o
    with pytest.raises(abi.AfgError):
        abi.resample_size(100, 1)
