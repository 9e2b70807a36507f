"""Two-directional comparison of trigger lists (Sec. II: a trigger is the maximum of the
integrated statistic over an 8 s window; ties go to the earliest index).

Both sides cluster their own statistic with the same rule.  First, each side's list must be
exactly the clustering of its own statistic (the oracle's clustering applied to the GPU's
statistic reproduces the GPU's list index for index).  Then, if the two statistics agree
element-wise within tol (1 + |I|), the lists are forced to agree wherever a maximum is
decisive: a trigger j whose value beats every other value within +-half by more than
2 tol (1 + |I_j|) on one side is, on the other side, still strictly above every neighbour,
hence a trigger at the same index.  So:

* every decisive trigger of either list must be in the other list at the same index;
* every other trigger (a near-tie) that the other list lacks must be explained by a tie:
  the other side's largest value within +-half of it sits at an index k whose oracle value
  lies within 2 tol (1 + |I|) of the trigger's.  Near-ties are counted and listed, with
  the distance to the nearest trigger of the other list.

`compare` returns the counts so that the tests can print them.
"""
from __future__ import annotations

import numpy as np


def margins(stat: np.ndarray, trig: np.ndarray, half: int) -> np.ndarray:
    """Value of each trigger minus the largest other value within +-half."""
    out = np.empty(len(trig))
    for n, j in enumerate(trig):
        lo, hi = max(0, j - half), min(len(stat), j + half + 1)
        nb = np.delete(stat[lo:hi], j - lo)
        out[n] = stat[j] - (nb.max() if len(nb) else -np.inf)
    return out


def compare(stat_gpu, stat_ref, trig_gpu, trig_ref, half: int, tol: float) -> dict:
    """Check the GPU trigger list against the oracle's (see the module docstring).
    Raises AssertionError on a mismatch; returns counts and the near-tie list."""
    from oracle import oracle as orc

    sg = np.asarray(stat_gpu, dtype=np.float64)
    so = np.asarray(stat_ref, dtype=np.float64)
    tg = np.asarray(trig_gpu, dtype=np.int64)
    to = np.asarray(trig_ref, dtype=np.int64)
    assert sg.shape == so.shape
    assert np.array_equal(orc.triggers(sg, half), tg), "GPU triggers are not the clustering of its own statistic"
    assert np.array_equal(orc.triggers(so, half), to), "oracle triggers are not the clustering of its statistic"
    err = np.abs(sg - so) / (1 + np.abs(so))
    assert err.size == 0 or err.max() <= tol, f"statistic differs by {err.max():.3g} > {tol}"
    set_g, set_o = set(tg.tolist()), set(to.tolist())
    counts = dict(oracle=len(to), gpu=len(tg), identical=bool(np.array_equal(tg, to)), decisive=0, near_tie=0,
                  near_tie_same=0, near_tie_moved=0, near_ties=[])
    for side, trig, stat, other, other_stat, other_list in (("oracle", to, so, set_g, sg, tg),
                                                            ("gpu", tg, sg, set_o, so, to)):
        for j, m in zip(trig.tolist(), margins(stat, trig, half)):
            if m > 2 * tol * (1 + abs(stat[j])):
                counts["decisive"] += 1
                assert j in other, f"decisive {side} trigger {j} (margin {m:.3g}) missing on the other side"
                continue
            counts["near_tie"] += 1
            if j in other:
                counts["near_tie_same"] += 1
                continue
            lo, hi = max(0, j - half), min(len(other_stat), j + half + 1)
            win = other_stat[lo:hi].copy()
            win[j - lo] = -np.inf
            k = lo + int(np.argmax(win))
            assert other_stat[k] >= other_stat[j], f"{side} trigger {j} missing on the other side, undominated"
            gap = abs(so[j] - so[k])
            assert gap <= 2 * tol * (1 + abs(so[j])), (
                f"{side} trigger {j} lost to {k} on the other side: oracle values differ by {gap:.3g}, not a tie")
            dist = int(np.min(np.abs(other_list - j))) if len(other_list) else -1
            counts["near_tie_moved"] += 1
            counts["near_ties"].append((side, j, k, dist, float(m)))
    return counts


def summary(c: dict) -> str:
    return (f"triggers oracle {c['oracle']} gpu {c['gpu']} (identical lists: {c['identical']}): "
            f"{c['decisive']} decisive (exact), "
            f"{c['near_tie']} near-ties ({c['near_tie_same']} same index, {c['near_tie_moved']} resolved "
            f"to a tied point: (side, index, tied point, distance to the other list's nearest trigger, "
            f"margin) {c['near_ties']})")
