"""The two-directional trigger-list comparison used by the GPU parity tests, on the CPU.

A statistic perturbed within the tolerance must be accepted with its own trigger list; a
list with a decisive trigger dropped, added or moved, or a near-tie resolved to a point
that is not tied, must be rejected.  Both lists come from the oracle's clustering."""
import numpy as np
import pytest

import trigger_match
from oracle import oracle as orc


def _series(n=4000, seed=0):
    rng = np.random.default_rng(seed)
    z = np.convolve(rng.standard_normal(n), np.ones(16) / 16, mode="same")
    return z


def test_within_tolerance_is_accepted_and_counted():
    tol, half = 1e-3, 64
    s_ref = _series()
    rng = np.random.default_rng(1)
    s_gpu = s_ref + rng.uniform(-0.9, 0.9, s_ref.shape) * tol * (1 + np.abs(s_ref))
    t_ref, t_gpu = orc.triggers(s_ref, half), orc.triggers(s_gpu, half)
    c = trigger_match.compare(s_gpu, s_ref, t_gpu, t_ref, half, tol)
    assert c["oracle"] == len(t_ref) and c["gpu"] == len(t_gpu)
    assert c["decisive"] > 0 and c["decisive"] + c["near_tie"] == len(t_ref) + len(t_gpu)


def test_near_tie_resolved_to_a_tied_neighbour_is_listed():
    tol, half = 1e-3, 8
    s_ref = np.zeros(100)
    s_ref[40], s_ref[44] = 1.0, 1.0 - 1e-4  # a tie within the tolerance
    s_gpu = s_ref.copy()
    s_gpu[44] = 1.0 + 1e-4  # the GPU resolves it to the other point
    c = trigger_match.compare(s_gpu, s_ref, orc.triggers(s_gpu, half), orc.triggers(s_ref, half), half, tol)
    assert c["near_tie_moved"] == 2
    assert {(side, j, k) for side, j, k, _, _ in c["near_ties"]} == {("oracle", 40, 44), ("gpu", 44, 40)}


@pytest.mark.parametrize("mistake", ["drop", "add", "move"])
def test_decisive_mismatch_is_rejected(mistake):
    """A GPU statistic that differs from the oracle's beyond the tolerance at one decisive peak
    (lowered, raised elsewhere, or shifted by one sample) changes the GPU's own clustering there;
    the comparison rejects it even with a generous tolerance on everything else."""
    tol, half = 1e-3, 64
    s = _series(seed=2)
    t = orc.triggers(s, half)
    m = trigger_match.margins(s, t, half)
    j = int(t[np.argmax(m)])  # the most decisive trigger
    g = s.copy()
    if mistake == "drop":
        g[j] -= 2 * m.max()
    elif mistake == "add":
        g[j + half // 2] = s[j] + 1.0
    else:
        g[j + 1] = s[j] + m.max() / 2
    with pytest.raises(AssertionError):
        trigger_match.compare(g, s, orc.triggers(g, half), t, half, 10 * tol)


def test_wrong_list_for_its_own_statistic_is_rejected():
    s = _series(seed=4)
    t = orc.triggers(s, 64)
    with pytest.raises(AssertionError):
        trigger_match.compare(s, s, t[1:], t, 64, 1e-3)


def test_statistic_outside_tolerance_is_rejected():
    s = _series(seed=3)
    t = orc.triggers(s, 32)
    g = s.copy()
    g[100] += 0.1
    with pytest.raises(AssertionError):
        trigger_match.compare(g, s, t, t, 32, 1e-3)


def test_untied_partner_is_rejected():
    tol, half = 1e-3, 8
    s_ref = np.zeros(100)
    s_ref[40], s_ref[44] = 1.0, 0.99  # not a tie: 1e-2 apart, more than 2 tol
    s_gpu = s_ref.copy()
    s_gpu[44] = 1.0 + 1e-4  # only possible with a statistic error of 1e-2: rejected
    with pytest.raises(AssertionError):
        trigger_match.compare(s_gpu, s_ref, orc.triggers(s_gpu, half), orc.triggers(s_ref, half), half, tol)
