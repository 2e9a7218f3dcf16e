"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer work: the refined clustering must be bit-identical to the oracle's
on the same seeded inputs (both BATCHED and PLAIN schedules, host and device
buffers).
"""
import numpy as np
import pytest

import oracle
import synth
from tests._helpers import min_labels

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wcc():
    import paper_2509_02590_gb300 as w
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return w


def _oracle(w, rule="log10", num=1, den=1, min_size=None):
    kind = {"log10": oracle.RULE_LOG10, "log2": oracle.RULE_LOG2, "sqrt": oracle.RULE_SQRT,
            "linear": oracle.RULE_LINEAR}[rule]
    off, adj = oracle.build_csr(w.n, w.src, w.dst)
    out, st = oracle.wcc(w.n, off, adj, w.labels, w.min_size if min_size is None else min_size,
                         kind, num, den)
    return out, st, off, adj


def _gpu(wcc, w, mode="batched", device=True, rule="log10", num=1, den=1, min_size=None,
         from_edges=True):
    ms = w.min_size if min_size is None else min_size
    if from_edges:
        g = wcc.WccGraph.from_edges(torch.from_numpy(w.src).cuda(), torch.from_numpy(w.dst).cuda(),
                                    w.n)
    else:
        off, adj = oracle.build_csr(w.n, w.src, w.dst)
        g = wcc.WccGraph.from_csr(off, adj)
    with g:
        if device:
            out, st = g.run(torch.from_numpy(w.labels).cuda(), min_size=ms, rule=rule, num=num,
                            den=den, mode=mode, stats=True)
            out = out.cpu().numpy()
        else:
            out, st = g.run(w.labels, min_size=ms, rule=rule, num=num, den=den, mode=mode,
                            stats=True)
    return out, st


@pytest.mark.parametrize("builder", ["rows", "radix"])
def test_csr_builder_matches_oracle(wcc, monkeypatch, builder):
    """Both CSR builders (every row sorted on chip; all entries sorted at
    once) give the oracle's CSR."""
    monkeypatch.setenv("WCC_CSR_BUILDER", builder)
    w = synth.lfr_like(20000, seed=1)
    off, adj = oracle.build_csr(w.n, w.src, w.dst)
    # duplicate and reversed edges plus self-loops in the input are dropped
    rng = np.random.default_rng(0)
    extra = rng.integers(0, w.m, 500)
    src = np.concatenate([w.src, w.dst[extra], np.arange(50, dtype=np.int32)])
    dst = np.concatenate([w.dst, w.src[extra], np.arange(50, dtype=np.int32)])
    with wcc.WccGraph.from_edges(src, dst, w.n) as g:
        goff, gadj = g.csr()
    assert np.array_equal(goff, off) and np.array_equal(gadj, adj)


@pytest.mark.parametrize("builder", ["rows", "radix"])
@pytest.mark.parametrize("hubs", ["to_16384", "to_40000"])
@pytest.mark.parametrize("dups", [False, True])
def test_csr_builder_rows_of_every_length(wcc, monkeypatch, dups, hubs, builder):
    """Rows of 1, 31-33, 63-65, 16383-16384 entries (hubs among short rows;
    with "to_40000" also rows of 16385, 20000 and 40000, longer than one CTA
    sorts on chip, so the row builder hands the graph to the full sort),
    with and without duplicate, reversed and self-loop edges, against the
    oracle's CSR, for both builders."""
    monkeypatch.setenv("WCC_CSR_BUILDER", builder)
    rng = np.random.default_rng(7 + dups)
    n = 60_000
    src, dst = [], []
    rows = [(0, 16_384), (1, 65), (2, 64), (3, 16_383), (4, 33), (5, 32), (6, 31), (7, 1),
            (8, 63)]
    if hubs == "to_40000":
        rows = [(0, 40_000), (1, 16_385), (2, 16_384), (3, 16_383), (4, 33), (5, 32), (6, 31),
                (7, 1), (8, 20_000)]
    for h, d in rows:
        nb = rng.choice(np.arange(100, n), size=d, replace=False)
        src.append(np.full(d, h)); dst.append(nb)
    a = rng.integers(100, n, 200_000)
    b = rng.integers(100, n, 200_000)
    src.append(a); dst.append(b)
    if dups:
        src.append(b[:30_000]); dst.append(a[:30_000])           # reversed copies
        src.append(np.arange(20)); dst.append(np.arange(20))     # self-loops
        src.append(np.zeros(6000, np.int64)); dst.append(dst[0][:6000].copy())  # hub repeats
        k = min(500, len(dst[1]))
        src.append(dst[1][:k].copy()); dst.append(np.ones(k, np.int64))
    src = np.concatenate(src).astype(np.int32)
    dst = np.concatenate(dst).astype(np.int32)
    off, adj = oracle.build_csr(n, src, dst)
    with wcc.WccGraph.from_edges(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n) as g:
        goff, gadj = g.csr()
    assert np.array_equal(goff, off) and np.array_equal(gadj, adj)


def test_planted_1k_all_modes(wcc):
    w = synth.planted_1k(0)
    ref, rst, _, _ = _oracle(w)
    for mode in ("batched", "plain"):
        for device in (True, False):
            out, st = _gpu(wcc, w, mode=mode, device=device)
            assert np.array_equal(out, ref), (mode, device)
            assert st["out_clusters"] == rst["out_clusters"]
            assert st["splits"] == rst["splits"]
            assert st["peeled"] == rst["peeled"]


def test_lfr_100k_full(wcc):
    w = synth.lfr_like(100_000, seed=0)
    ref, rst, _, _ = _oracle(w)
    out, st = _gpu(wcc, w)
    assert np.array_equal(out, ref)
    assert st["in_clusters"] == rst["in_clusters"]
    assert st["out_clusters"] == rst["out_clusters"]


def test_lfr_plain_equals_batched(wcc):
    w = synth.lfr_like(30_000, seed=2)
    ref, _, _, _ = _oracle(w)
    a, _ = _gpu(wcc, w, mode="batched")
    b, _ = _gpu(wcc, w, mode="plain", from_edges=False)
    assert np.array_equal(a, ref) and np.array_equal(b, ref)


@pytest.mark.parametrize("seed", range(6))
def test_random_instances(wcc, seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(200, 3000))
    k = int(rng.integers(2, 40))
    lab = rng.integers(0, k, n).astype(np.int32)
    lab[rng.random(n) < 0.1] = -1
    src, dst = [], []
    for c in range(k):
        vs = np.nonzero(lab == c)[0]
        if len(vs) < 2:
            continue
        a, b = synth.random_gnp(len(vs), float(rng.uniform(0.02, 0.4)), rng)
        src.append(vs[a]); dst.append(vs[b])
    a, b = synth.random_gnp(n, 3.0 / n, rng)
    src.append(a); dst.append(b)
    s, d = synth.graphs._dedup(n, np.concatenate(src), np.concatenate(dst))
    w = synth.Workload("rand", n, s, d, lab, int(rng.integers(2, 8)))
    ref, _, _, _ = _oracle(w)
    out, _ = _gpu(wcc, w)
    assert np.array_equal(out, ref)


@pytest.mark.parametrize("rule,num,den", [("log2", 1, 1), ("sqrt", 1, 1), ("linear", 1, 20)])
def test_other_rules(wcc, rule, num, den):
    w = synth.lfr_like(8000, seed=4)
    ref, _, _, _ = _oracle(w, rule, num, den)
    out, _ = _gpu(wcc, w, rule=rule, num=num, den=den)
    assert np.array_equal(out, ref)


def _block_chains(seed):
    """Input clusters that are chains of dense blocks joined by one or two
    edges: every split cuts one link, and the side holding the smallest id
    is usually a prefix of the parent's first contraction pass, so its own
    sides inherit again, several levels deep.  Ids are either in block order
    or shuffled within each cluster."""
    rng = np.random.default_rng(seed)
    src, dst, lab = [], [], []
    n = 0
    for c in range(int(rng.integers(6, 12))):
        nb = int(rng.integers(1, 8))
        sizes = rng.integers(40, 400, size=nb)
        tot = int(sizes.sum())
        perm = rng.permutation(tot) if rng.random() < 0.5 else np.arange(tot)
        starts = np.concatenate([[0], np.cumsum(sizes)])
        for b in range(nb):
            a, d = synth.random_gnp(int(sizes[b]), float(rng.uniform(0.06, 0.3)), rng)
            src.append(n + perm[starts[b] + a]); dst.append(n + perm[starts[b] + d])
            if b + 1 < nb:
                k = int(rng.integers(1, 3))
                src.append(n + perm[starts[b] + rng.integers(0, sizes[b], k)])
                dst.append(n + perm[starts[b + 1] + rng.integers(0, sizes[b + 1], k)])
        lab.append(np.full(tot, c, np.int32))
        n += tot
    s, d = synth.graphs._dedup(n, np.concatenate(src), np.concatenate(dst))
    return synth.Workload("chains", n, s, d, np.concatenate(lab), 2)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_block_chains_split_with_inherited_passes(wcc, seed):
    w = _block_chains(seed)
    ref, rst, _, _ = _oracle(w)
    assert rst["splits"] > 0
    for mode in ("batched", "plain"):
        out, st = _gpu(wcc, w, mode=mode)
        assert np.array_equal(out, ref), mode
        assert st["splits"] == rst["splits"] and st["peeled"] == rst["peeled"]


def test_dc_planted_small(wcc):
    w = synth.dc_planted(200_000, 2_000_000, seed=5, size_max=5000)
    ref, _, _, _ = _oracle(w)
    out, _ = _gpu(wcc, w)
    assert np.array_equal(out, ref)


def test_edge_cases(wcc):
    n, eu, ev = synth.tiny_family("complete", 6)
    off, adj = oracle.build_csr(n, eu, ev)
    with wcc.WccGraph.from_csr(off, adj) as g:
        assert np.all(g.run(np.full(n, -1, np.int32)) == -1)           # no clusters
        assert np.all(g.run(np.zeros(n, np.int32)) == 0)               # one clique
        assert np.all(g.run(np.arange(n, dtype=np.int32)) == -1)       # singletons
        assert np.all(g.run(np.zeros(n, np.int32), min_size=7) == -1)  # too small
        assert np.all(g.run(np.zeros(n, np.int32), min_size=0) == 0)   # min_size < 2 acts as 2
        big = np.full(n, 2**31 - 1, np.int32)
        assert np.all(g.run(big) == 0)                                 # arbitrary label values
        with pytest.raises(wcc.WccError):
            g.run(np.full(n, -5, np.int32))                            # labels below -1
    # empty graph with clusters: everything is a singleton after CCR
    with wcc.WccGraph.from_edges(np.zeros(0, np.int32), np.zeros(0, np.int32), 10) as g:
        assert np.all(g.run(np.zeros(10, np.int32)) == -1)


def test_invalid_graphs_rejected(wcc):
    with pytest.raises(wcc.WccError):   # asymmetric
        wcc.WccGraph.from_csr(np.array([0, 1, 1], np.int64), np.array([1], np.int32))
    with pytest.raises(wcc.WccError):   # self-loop
        wcc.WccGraph.from_csr(np.array([0, 1], np.int64), np.array([0], np.int32))
    with pytest.raises(wcc.WccError):   # id out of range
        wcc.WccGraph.from_edges(np.array([0], np.int32), np.array([5], np.int32), 3)


def test_hand_traced_items(wcc):
    # two K5 joined by one edge, one cluster of 10: T(10) = 1, cut 1 -> split
    eu, ev = [], []
    for base in (0, 5):
        for i in range(5):
            for j in range(i + 1, 5):
                eu.append(base + i); ev.append(base + j)
    eu.append(4); ev.append(5)
    w = synth.Workload("k5k5", 10, np.array(eu, np.int32), np.array(ev, np.int32),
                       np.zeros(10, np.int32), 2)
    out, _ = _gpu(wcc, w)
    assert out.tolist() == [0] * 5 + [1] * 5


def test_min_labels_consistent(wcc):
    w = synth.lfr_like(5000, seed=7)
    ref, _, _, _ = _oracle(w)
    out, _ = _gpu(wcc, w)
    assert np.array_equal(min_labels(out), min_labels(ref))


def _random_workload(seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(500, 4000))
    k = int(rng.integers(2, 12))
    lab = rng.integers(0, k, n).astype(np.int32)
    src, dst = [], []
    for c in range(k):
        vs = np.nonzero(lab == c)[0]
        if len(vs) < 2:
            continue
        a, b = synth.random_gnp(len(vs), float(rng.uniform(0.01, 0.2)), rng)
        src.append(vs[a]); dst.append(vs[b])
    a, b = synth.random_gnp(n, 2.0 / n, rng)
    src.append(a); dst.append(b)
    s, d = synth.graphs._dedup(n, np.concatenate(src), np.concatenate(dst))
    return synth.Workload("rand", n, s, d, lab, 2)


# Internal strategy switches (each must leave the result unchanged): the
# sparse passes only, the forest acceptance test on every item, working
# memory in the global slab instead of shared memory, small items on a whole
# CTA instead of one warp each, and small items forced onto single warps
# (a run with no more input clusters than CTAs otherwise gives every item a
# CTA).
@pytest.mark.parametrize("env", [{"WCC_DENSE_NSV": "0"}, {"WCC_FOREST_MIN_N": "2"},
                                 {"WCC_SMEM_KB": "40"}, {"WCC_TINY_N": "0"},
                                 {"WCC_TINY_N": "64"}, {"WCC_TINY_N": "32"},
                                 {"WCC_DENSE_NSV": "0", "WCC_FOREST_MIN_N": "2", "WCC_SMEM_KB": "40",
                                  "WCC_TINY_N": "0"}])
def test_strategy_switches_keep_results(wcc, monkeypatch, env):
    cases = [synth.planted_1k(0), synth.lfr_like(12000, seed=8)] + [_random_workload(s) for s in range(3)]
    refs = [_oracle(w)[0] for w in cases]
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    for w, ref in zip(cases, refs):
        out, _ = _gpu(wcc, w)
        assert np.array_equal(out, ref), (w.name, env)
        out, _ = _gpu(wcc, w, mode="plain", device=False)
        assert np.array_equal(out, ref), (w.name, env, "plain")
