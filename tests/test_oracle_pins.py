"""Pins for the CPU oracle (no GPU).

Each check ties the oracle to something other than itself: closed forms,
brute-force enumeration of every bipartition, hand-traced cases
(tests/golden/hand_traced.json), scipy / networkx routines, and invariants
of the whole refinement (Algorithms 1-3).
"""
import json
import math
import os

import networkx as nx
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

import oracle
import synth
from tests._helpers import (brute_min_cut, capped_pass, clusters_of, contract_passes, contracted,
                            cut_value, induced_edges, is_connected, min_labels, nbr_lists, sets_of)

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_traced.json")))


# ---------------------------------------------------------------- threshold
def test_threshold_log10_powers_of_ten():
    # floor(log10 n) = number of decimal digits - 1; the off-by-one values
    # around every power of ten are where floating log10 can misround
    for k in range(0, 16):
        p = 10 ** k
        for n in (p - 1, p, p + 1):
            if n >= 1:
                assert oracle.threshold(n) == len(str(n)) - 1, n


def test_threshold_log10_random():
    rng = np.random.default_rng(1)
    for n in rng.integers(1, 2**62, 2000):
        assert oracle.threshold(int(n)) == len(str(int(n))) - 1


def test_threshold_other_rules():
    rng = np.random.default_rng(2)
    for n in list(range(1, 300)) + [int(x) for x in rng.integers(1, 2**40, 500)]:
        assert oracle.threshold(n, oracle.RULE_LOG2) == n.bit_length() - 1
        assert oracle.threshold(n, oracle.RULE_SQRT) == math.isqrt(n)
        assert oracle.threshold(n, oracle.RULE_LINEAR, 3, 20) == (3 * n) // 20
    assert oracle.threshold(0) == -1


# ---------------------------------------------------------------- CSR build
def test_build_csr_matches_set_definition():
    rng = np.random.default_rng(3)
    n = 200
    src = rng.integers(0, n, 3000).astype(np.int32)
    dst = rng.integers(0, n, 3000).astype(np.int32)
    off, adj = oracle.build_csr(n, src, dst)
    nbrs = [set() for _ in range(n)]
    for a, b in zip(src, dst):
        if a != b:
            nbrs[a].add(int(b)); nbrs[b].add(int(a))
    for v in range(n):
        assert list(adj[off[v]:off[v + 1]]) == sorted(nbrs[v])


def test_build_csr_rejects_bad_ids():
    with pytest.raises(ValueError):
        oracle.build_csr(3, [0, 3], [1, 1])


# ---------------------------------------------------------------- components
def test_components_match_scipy():
    rng = np.random.default_rng(4)
    for trial in range(30):
        n = int(rng.integers(1, 120))
        m = int(rng.integers(0, 2 * n))
        eu = rng.integers(0, n, m).astype(np.int32)
        ev = rng.integers(0, n, m).astype(np.int32)
        comp = oracle.components(n, eu, ev)
        A = sp.coo_matrix((np.ones(m), (eu, ev)), shape=(n, n))
        nc, lab = connected_components(A, directed=False)
        assert len(np.unique(comp)) == nc
        for c in range(nc):
            members = np.nonzero(lab == c)[0]
            assert np.all(comp[members] == members.min())


# ---------------------------------------------------------------- Stoer-Wagner
@pytest.mark.parametrize("case", GOLDEN["stoer_wagner"], ids=lambda c: c["name"])
def test_stoer_wagner_hand_traced(case):
    e = np.array(case["edges"], np.int32)
    lam, side = oracle.stoer_wagner(case["n"], e[:, 0], e[:, 1], case.get("weights"))
    assert lam == case["lambda"]
    assert sorted(np.nonzero(side)[0].tolist()) == case["side"]


def test_stoer_wagner_brute_force():
    rng = np.random.default_rng(5)
    checked = 0
    while checked < 150:
        n = int(rng.integers(2, 13))
        iu, ju = np.triu_indices(n, 1)
        keep = rng.random(len(iu)) < rng.uniform(0.2, 0.9)
        eu, ev = iu[keep].astype(np.int32), ju[keep].astype(np.int32)
        if not is_connected(n, eu, ev):
            continue
        w = rng.integers(1, 5, len(eu)) if checked % 2 else None
        lam, side = oracle.stoer_wagner(n, eu, ev, w)
        best, _ = brute_min_cut(n, eu, ev, w)
        assert lam == best
        assert cut_value(eu, ev, side, w) == best
        assert not side[0] and side.any()
        checked += 1


@pytest.mark.parametrize("fam,args,lam", [
    ("complete", (7,), 6), ("complete", (12,), 11), ("cycle", (9,), 2), ("cycle", (30,), 2),
    ("path", (10,), 1), ("tree", (25,), 1), ("hypercube", (3,), 3), ("hypercube", (5,), 5),
    ("bipartite", (3, 5), 3), ("bipartite", (6, 4), 4), ("two_cliques", (6, 3), 3),
    ("two_cliques", (8, 1), 1),
])
def test_stoer_wagner_closed_forms(fam, args, lam):
    n, eu, ev = synth.tiny_family(fam, *args)
    got, side = oracle.stoer_wagner(n, eu, ev)
    assert got == lam
    assert cut_value(eu, ev, side) == lam


def test_stoer_wagner_matches_networkx_value():
    rng = np.random.default_rng(6)
    for trial in range(20):
        n = int(rng.integers(15, 60))
        eu, ev = synth.random_gnp(n, float(rng.uniform(0.1, 0.4)), rng)
        if not is_connected(n, eu, ev):
            continue
        w = rng.integers(1, 4, len(eu))
        G = nx.Graph()
        G.add_nodes_from(range(n))
        for a, b, c in zip(eu, ev, w):
            G.add_edge(int(a), int(b), weight=int(c))
        ref, _ = nx.stoer_wagner(G)
        lam, side = oracle.stoer_wagner(n, eu, ev, w)
        assert lam == ref
        assert cut_value(eu, ev, side, w) == lam


# ---------------------------------------------------------------- peel
def test_peel_hand_traced_path12():
    case = GOLDEN["peel"][0]
    n, eu, ev = synth.tiny_family("path", case["n"])
    alive = oracle.peel(n, eu, ev)
    assert np.nonzero(alive)[0].tolist() == case["alive"]


def test_peel_fixpoint_invariant_and_small_connected():
    rng = np.random.default_rng(7)
    for trial in range(40):
        n = int(rng.integers(2, 400))
        eu, ev = synth.random_gnp(n, float(rng.uniform(0.002, 0.05)), rng)
        alive = oracle.peel(n, eu, ev)
        na = int(alive.sum())
        deg = np.zeros(n, np.int64)
        both = alive[eu] & alive[ev]
        np.add.at(deg, eu[both], 1)
        np.add.at(deg, ev[both], 1)
        T = oracle.threshold(na) if na else -1
        assert np.all(deg[alive] > T)
        # a removed vertex had at most T(n_round) <= T(n) alive neighbours when
        # it went, and the survivors are a subset of that round's alive set
        nb_alive = np.zeros(n, np.int64)
        np.add.at(nb_alive, eu[alive[ev]], 1)
        np.add.at(nb_alive, ev[alive[eu]], 1)
        assert np.all(nb_alive[~alive] <= oracle.threshold(n))
    # connected graphs on fewer than 10 vertices have T = 0 and minimum degree 1
    for n in range(2, 10):
        _, eu, ev = synth.tiny_family("tree", n, seed=n)
        assert oracle.peel(n, eu, ev).all()


# ---------------------------------------------------------------- item cut
def _clique_graph(case):
    eu, ev = [], []
    for cl in case["cliques"]:
        for i in range(len(cl)):
            for j in range(i + 1, len(cl)):
                eu.append(cl[i]); ev.append(cl[j])
    for a, b in case["extra_edges"]:
        eu.append(a); ev.append(b)
    return np.array(eu, np.int32), np.array(ev, np.int32)


@pytest.mark.parametrize("case", GOLDEN["item_cut"], ids=lambda c: c["name"])
def test_item_cut_hand_traced(case):
    eu, ev = _clique_graph(case)
    acc, lam, side, rep = oracle.item_cut(case["n"], eu, ev, case["T"])
    assert acc == case["accepted"]
    if not acc:
        assert lam == case["lambda"]
        assert np.nonzero(side)[0].tolist() == case["side"]
        assert rep.tolist() == case["rep"]


@pytest.mark.parametrize("case", [c for c in GOLDEN["item_cut"] if "plain_sw_side" in c],
                         ids=lambda c: c["name"])
def test_cut_rule_contraction_changes_the_side(case):
    """Reading R5 runs canonical Stoer-Wagner after the capped contraction;
    the plain canonical Stoer-Wagner on the uncontracted item (the other
    reading) can return another minimum cut.  Both sides, hand-traced, have
    the minimum value; the oracle's item cut is the R5 one."""
    eu, ev = _clique_graph(case)
    lam, side = oracle.stoer_wagner(case["n"], eu, ev)
    assert lam == case["lambda"]
    assert np.nonzero(side)[0].tolist() == case["plain_sw_side"] != case["side"]
    for s in (case["side"], case["plain_sw_side"]):
        mask = np.zeros(case["n"], bool)
        mask[s] = True
        assert cut_value(eu, ev, mask) == case["lambda"]


def test_item_cut_decision_and_side_brute_force():
    """accept <=> lambda > T; on failure lambda is exact and the side is a
    minimum cut not containing vertex 0; the contraction never splits a cut
    of value <= T (every such bipartition keeps each super-vertex whole)."""
    rng = np.random.default_rng(8)
    n_fail = n_acc = 0
    while n_fail + n_acc < 300:
        n = int(rng.integers(2, 14))
        iu, ju = np.triu_indices(n, 1)
        keep = rng.random(len(iu)) < rng.uniform(0.15, 0.8)
        eu, ev = iu[keep].astype(np.int32), ju[keep].astype(np.int32)
        if not is_connected(n, eu, ev):
            continue
        T = int(rng.integers(0, 5))
        acc, lam, side, rep = oracle.item_cut(n, eu, ev, T)
        best, masks = brute_min_cut(n, eu, ev)
        assert acc == (best > T)
        if acc:
            n_acc += 1
            continue
        n_fail += 1
        assert lam == best
        assert cut_value(eu, ev, side) == best
        assert not side[0] and side.any()
        assert np.all(rep <= np.arange(n)) and np.all(rep[rep] == rep)
        # every cut of value <= T keeps each super-vertex on one side
        eu64, ev64 = eu.astype(np.int64), ev.astype(np.int64)
        all_masks = np.arange(1, 1 << (n - 1), dtype=np.int64) << 1
        bits_u = (all_masks[:, None] >> eu64[None, :]) & 1
        bits_v = (all_masks[:, None] >> ev64[None, :]) & 1
        small = all_masks[(bits_u != bits_v).sum(axis=1) <= T]
        bits = (small[:, None] >> np.arange(n)[None, :]) & 1
        assert np.all(bits == bits[:, rep])
    assert n_fail > 50 and n_acc > 50


def _random_connected(rng, n_lo, n_hi):
    while True:
        n = int(rng.integers(n_lo, n_hi + 1))
        if rng.random() < 0.5:
            iu, ju = np.triu_indices(n, 1)
            keep = rng.random(len(iu)) < rng.uniform(0.1, 0.7)
            eu, ev = iu[keep], ju[keep]
        else:  # dense blocks joined by a few edges, ids shuffled
            sizes = rng.integers(3, max(4, n // 2), size=int(rng.integers(2, 5)))
            n = int(sizes.sum())
            starts = np.concatenate([[0], np.cumsum(sizes)])
            eu, ev = [], []
            for b, s in enumerate(sizes):
                iu, ju = np.triu_indices(int(s), 1)
                keep = rng.random(len(iu)) < rng.uniform(0.4, 0.9)
                eu += list(starts[b] + iu[keep]); ev += list(starts[b] + ju[keep])
                if b + 1 < len(sizes):
                    for _ in range(int(rng.integers(1, 4))):
                        eu.append(int(starts[b] + rng.integers(0, s)))
                        ev.append(int(starts[b + 1] + rng.integers(0, sizes[b + 1])))
            perm = rng.permutation(n)
            eu, ev = perm[np.array(eu)], perm[np.array(ev)]
            lo, hi = np.minimum(eu, ev), np.maximum(eu, ev)
            key = np.unique(lo.astype(np.int64) * n + hi)
            eu, ev = key // n, key % n
        eu, ev = np.asarray(eu, np.int32), np.asarray(ev, np.int32)
        if len(eu) and is_connected(n, eu, ev):
            return n, eu, ev


def test_item_cut_contraction_matches_restated_passes():
    """The contraction the oracle's cut step ends with (rep) equals the
    passes restated from their definition in tests/_helpers.py (capped
    maximum-adjacency order from the smallest id, ties to the smallest id,
    an edge contracted when the later end's key reached k = T+1 by the
    earlier end's pick; repeated on the contracted multigraph until one
    super-vertex is left or a pass contracts nothing).  A wrong tie rule in
    any pass changes rep on some of these graphs."""
    rng = np.random.default_rng(11)
    n_multi = n_fail = 0
    for trial in range(1200):
        n, eu, ev = _random_connected(rng, 4, 40)
        T = int(rng.integers(0, 6))
        acc, lam, side, rep = oracle.item_cut(n, eu, ev, T)
        want, passes = contract_passes(n, eu, ev, T + 1)
        assert np.array_equal(rep, want), (trial, n, T)
        assert acc == (len(np.unique(want)) == 1)
        n_multi += passes >= 3
        n_fail += not acc
    assert n_multi >= 100 and n_fail >= 200, (n_multi, n_fail)


def test_first_contraction_pass_sets_match_restatement():
    """The oracle's contraction after a first pass that leaves one
    super-vertex or merges nothing is exactly that first pass's sets, so on
    those graphs rep equals the first pass restated alone (capped_pass,
    contracted, sets_of)."""
    rng = np.random.default_rng(12)
    checked = 0
    for _ in range(1500):
        n, eu, ev = _random_connected(rng, 4, 30)
        T = int(rng.integers(0, 5))
        pos, sat = capped_pass(n, nbr_lists(n, eu, ev), T + 1)
        mask = contracted(eu.astype(np.int64), ev.astype(np.int64), pos, sat)
        first = sets_of(n, eu, ev, mask)
        nsv = len(np.unique(first))
        if nsv != 1 and mask.any():
            # a second pass may merge more; it must only coarsen the first
            _, _, _, rep = oracle.item_cut(n, eu, ev, T)
            assert np.array_equal(rep[first], rep)
            continue
        _, _, _, rep = oracle.item_cut(n, eu, ev, T)
        assert np.array_equal(rep, first)
        checked += 1
    assert checked >= 300, checked


# ---------------------------------------------------------------- whole refinement
def _wcc_invariants(w, out, T_of=oracle.threshold):
    off, adj = oracle.build_csr(w.n, w.src, w.dst)
    inp = w.labels
    outc = clusters_of(out)
    ids = sorted(outc)
    assert ids == list(range(len(ids)))
    mins = [int(outc[i].min()) for i in ids]
    assert mins == sorted(mins)  # ids ascending by smallest vertex id
    for i in ids:
        vs = outc[i]
        assert len(vs) >= max(w.min_size, 2)
        assert len(np.unique(inp[vs])) == 1 and inp[vs[0]] >= 0  # subset of one input cluster
        eu, ev = induced_edges(off, adj, vs)
        assert is_connected(len(vs), eu, ev)
        T = T_of(len(vs))
        if len(vs) <= 14:
            lam, _ = brute_min_cut(len(vs), eu, ev)
        else:
            G = nx.Graph()
            G.add_nodes_from(range(len(vs)))
            G.add_edges_from(zip(eu.tolist(), ev.tolist()))
            lam = nx.stoer_wagner(G)[0] if len(vs) <= 400 else None
        if lam is not None:
            assert lam > T
        # accepted clusters have minimum degree > T (peeling is a no-op on them)
        deg = np.bincount(np.concatenate([eu, ev]), minlength=len(vs))
        assert deg.min() > T
    return off, adj


def test_wcc_planted_1k_shape_and_invariants():
    w = synth.planted_1k(0)
    off, adj = oracle.build_csr(w.n, w.src, w.dst)
    out, st = oracle.wcc(w.n, off, adj, w.labels, w.min_size)
    _wcc_invariants(w, out)
    assert st["in_clusters"] == 20
    # four bridged blocks split into their halves (bridge cut 1 <= T(50) = 1)
    assert st["out_clusters"] == 24 and st["splits"] == 4
    sizes = sorted(len(v) for v in clusters_of(out).values())
    # 8 halves of at most 25 vertices (a few low-degree members peeled), 16 whole blocks
    assert sum(1 for x in sizes if x <= 25) == 8 and min(sizes) >= 20
    # the 10 pendant vertices (degree 1 inside their cluster) are peeled
    deg_in = np.zeros(w.n, np.int64)
    same = w.labels[w.src] == w.labels[w.dst]
    np.add.at(deg_in, w.src[same], 1)
    np.add.at(deg_in, w.dst[same], 1)
    assert np.all(out[deg_in <= 1] == -1)


def test_wcc_random_small_against_brute_force():
    rng = np.random.default_rng(9)
    for trial in range(25):
        n = int(rng.integers(20, 120))
        k = int(rng.integers(1, 6))
        lab = rng.integers(0, k, n).astype(np.int32)
        lab[rng.random(n) < 0.05] = -1
        src, dst = [], []
        for c in range(k):
            vs = np.nonzero(lab == c)[0]
            if len(vs) < 2:
                continue
            a, b = synth.random_gnp(len(vs), float(rng.uniform(0.05, 0.5)), rng)
            src.append(vs[a]); dst.append(vs[b])
        a, b = synth.random_gnp(n, 0.01, rng)
        src.append(a); dst.append(b)
        s, d = synth.graphs._dedup(n, np.concatenate(src), np.concatenate(dst))
        w = synth.Workload("rand", n, s, d, lab, int(rng.integers(2, 6)))
        off, adj = oracle.build_csr(n, s, d)
        out, _ = oracle.wcc(n, off, adj, lab, w.min_size)
        _wcc_invariants(w, out)


def test_wcc_idempotent_and_relabel_invariant():
    w = synth.planted_1k(0)
    off, adj = oracle.build_csr(w.n, w.src, w.dst)
    out, _ = oracle.wcc(w.n, off, adj, w.labels, w.min_size)
    again, _ = oracle.wcc(w.n, off, adj, out, w.min_size)
    assert np.array_equal(again, out)
    # permuting the input label values changes nothing
    vals = np.unique(w.labels[w.labels >= 0])
    lut = dict(zip(vals.tolist(), (np.random.default_rng(1).permutation(len(vals)) * 7 + 3).tolist()))
    lab2 = np.array([lut.get(int(x), -1) if x >= 0 else -1 for x in w.labels], np.int32)
    out2, _ = oracle.wcc(w.n, off, adj, lab2, w.min_size)
    assert np.array_equal(out2, out)
    # a monotone relabelling of vertex ids (interleaving unclustered isolated
    # vertices) maps the result accordingly
    newid = np.arange(w.n) * 2 + 1
    n2 = 2 * w.n + 1
    off2, adj2 = oracle.build_csr(n2, newid[w.src], newid[w.dst])
    lab3 = np.full(n2, -1, np.int32)
    lab3[newid] = w.labels
    out3, _ = oracle.wcc(n2, off2, adj2, lab3, w.min_size)
    assert np.array_equal(out3[newid], out)
    assert np.all(out3[np.setdiff1d(np.arange(n2), newid)] == -1)


def test_wcc_min_id_mode_and_label_subset():
    w = synth.lfr_like(4000, seed=3)
    off, adj = oracle.build_csr(w.n, w.src, w.dst)
    out, _ = oracle.wcc(w.n, off, adj, w.labels, w.min_size)
    outm, _ = oracle.wcc(w.n, off, adj, w.labels, w.min_size, out_mode=1)
    assert np.array_equal(min_labels(out), outm)
    # refining a subset of input clusters gives the same clusters on them
    only = np.zeros(int(w.labels.max()) + 1, np.uint8)
    pick = np.unique(w.labels[w.labels >= 0])[::3]
    only[pick] = 1
    sub, _ = oracle.wcc(w.n, off, adj, w.labels, w.min_size, only_labels=only, out_mode=1)
    mask = np.isin(w.labels, pick)
    assert np.array_equal(sub[mask], outm[mask])
    assert np.all(sub[~mask] == -1)


def test_wcc_edge_cases():
    off, adj = oracle.build_csr(0, [], [])
    out, st = oracle.wcc(0, off, adj, np.zeros(0, np.int32), 2)
    assert len(out) == 0 and st["in_clusters"] == 0
    # no clusters at all
    n, eu, ev = synth.tiny_family("complete", 6)
    off, adj = oracle.build_csr(n, eu, ev)
    out, st = oracle.wcc(n, off, adj, np.full(n, -1, np.int32), 2)
    assert np.all(out == -1)
    # one clique cluster: accepted whole (lambda = 5 > T(6) = 0)
    out, st = oracle.wcc(n, off, adj, np.zeros(n, np.int32), 2)
    assert np.all(out == 0)
    # singletons and edgeless clusters are dropped (CCR keeps parts >= 2)
    out, _ = oracle.wcc(n, off, adj, np.arange(n, dtype=np.int32), 2)
    assert np.all(out == -1)
    # min_size larger than every cluster drops everything
    out, _ = oracle.wcc(n, off, adj, np.zeros(n, np.int32), 7)
    assert np.all(out == -1)
    # min_size below 2 behaves as 2
    o1, _ = oracle.wcc(n, off, adj, np.zeros(n, np.int32), 0)
    assert np.all(o1 == 0)
