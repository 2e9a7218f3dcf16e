"""The lemma behind first-pass inheritance, checked on the CPU.

The refinement kernel lets a side S of a cut skip its own first contraction
pass and take its parent's contraction sets on S.  It does this when three
things hold: S's members are positions 0 .. |S|-1 of the parent's
first-pass order, nothing in S peels, and S has the parent's kcap.  This
test restates the first pass (capped maximum-adjacency order, ties to the
smallest id, an entry a -> j contracted iff j's key reached kcap no later
than a's pick; Nagamochi-Ibaraki with k = T + 1; tests/_helpers.py)
independently of both the kernel and the oracle.  On seeded graphs of dense
blocks joined by a few edges, split on the oracle's canonical cut, it checks
the claim:
  * no contracted entry crosses the cut when a side is a prefix;
  * the side's own first pass, on its induced subgraph with ids renumbered
    in order, builds exactly the parent's sets restricted to it.
"""
import numpy as np
import pytest

import oracle
from tests._helpers import capped_pass, contracted, nbr_lists, sets_of


def block_graph(rng):
    sizes = rng.integers(12, 70, size=int(rng.integers(2, 5)))
    n = int(sizes.sum())
    perm = rng.permutation(n)  # ids not ordered by block
    starts = np.concatenate([[0], np.cumsum(sizes)])
    eu, ev = [], []
    for b, s in enumerate(sizes):
        p = float(rng.uniform(0.25, 0.7))
        iu, iv = np.triu_indices(int(s), 1)
        keep = rng.random(len(iu)) < p
        eu += list(starts[b] + iu[keep])
        ev += list(starts[b] + iv[keep])
        if b + 1 < len(sizes):
            for _ in range(int(rng.integers(1, 3))):
                eu.append(int(starts[b] + rng.integers(0, s)))
                ev.append(int(starts[b + 1] + rng.integers(0, sizes[b + 1])))
    eu, ev = perm[np.array(eu)], perm[np.array(ev)]
    lo, hi = np.minimum(eu, ev), np.maximum(eu, ev)
    key = np.unique(lo.astype(np.int64) * n + hi)
    return n, (key // n).astype(np.int32), (key % n).astype(np.int32)


RULES = {"log10": (oracle.RULE_LOG10, 1, 1, 10), "log2": (oracle.RULE_LOG2, 1, 1, 5),
         "sqrt": (oracle.RULE_SQRT, 1, 1, 0), "linear": (oracle.RULE_LINEAR, 1, 20, 0)}


@pytest.mark.parametrize("rule", list(RULES))
def test_prefix_side_inherits_the_parent_first_pass(rule):
    # sqrt and linear thresholds change with almost every size, so a side
    # rarely keeps its parent's kcap there and nothing is inherited; the
    # no-crossing half of the lemma holds under every rule
    kind, num, den, min_exercised = RULES[rule]
    rng = np.random.default_rng(2509)
    exercised = prefix_sides = differs_without_prefix = 0
    for _ in range(60):
        n0, eu0, ev0 = block_graph(rng)
        alive = oracle.peel(n0, eu0, ev0, kind, num, den)
        ids = np.nonzero(alive)[0]
        loc = -np.ones(n0, np.int64)
        loc[ids] = np.arange(len(ids))
        m = alive[eu0] & alive[ev0]
        n, eu, ev = len(ids), loc[eu0[m]], loc[ev0[m]]
        if n < 4 or oracle.components(n, eu, ev).max() > 0:
            continue
        T = oracle.threshold(n, kind, num, den)
        accepted, lam, side, _ = oracle.item_cut(n, eu.astype(np.int32), ev.astype(np.int32), T)
        if accepted:
            continue
        assert lam <= T
        pos, sat = capped_pass(n, nbr_lists(n, eu, ev), T + 1)
        cmask = contracted(eu, ev, pos, sat)
        parent_sets = sets_of(n, eu, ev, cmask)
        for s in (side, ~side):
            size = int(s.sum())
            if int(pos[s].max()) >= size:
                # not a prefix: the parent's sets need not be the side's own
                # (the condition the kernel checks is not a formality)
                members = np.nonzero(s)[0]
                sl = -np.ones(n, np.int64)
                sl[members] = np.arange(size)
                inside = s[eu] & s[ev]
                su, sv = sl[eu[inside]], sl[ev[inside]]
                cpos, csat = capped_pass(size, nbr_lists(size, su, sv), T + 1)
                own = sets_of(size, su, sv, contracted(su, sv, cpos, csat))
                roots = parent_sets[members]
                if not s[roots].all() or not np.array_equal(own, sl[roots]):
                    differs_without_prefix += 1
                continue
            prefix_sides += 1
            # no contracted entry crosses the cut
            assert not np.any(cmask & (s[eu] != s[ev]))
            members = np.nonzero(s)[0]  # ascending: a monotone renumbering
            sl = -np.ones(n, np.int64)
            sl[members] = np.arange(size)
            inside = s[eu] & s[ev]
            su, sv = sl[eu[inside]], sl[ev[inside]]
            if not oracle.peel(size, su.astype(np.int32), sv.astype(np.int32), kind, num, den).all():
                continue
            if oracle.threshold(size, kind, num, den) != T:
                continue
            exercised += 1
            cpos, csat = capped_pass(size, nbr_lists(size, su, sv), T + 1)
            # the side's own pass is the parent's order prefix, step for step
            assert np.array_equal(cpos, pos[members])
            child_sets = sets_of(size, su, sv, contracted(su, sv, cpos, csat))
            inherited = sl[parent_sets[members]]
            assert np.array_equal(child_sets, inherited)
    assert prefix_sides >= 20 and exercised >= min_exercised, (prefix_sides, exercised)
    assert differs_without_prefix >= 10, differs_without_prefix
