"""Pins of the oracle's CM refinement (Section 2.4, Algorithms 4-5) and of
its community step (GetCommunities with a CPM local-moving rule), against
hand-traced cases, closed forms, and properties that follow from the
definitions rather than from the code:

- the hand-traced cases of tests/golden/hand_traced.json (tie rules,
  strict improvement, the empty community);
- a resolution above every degree leaves singletons; disjoint cliques at a
  small resolution come out as the cliques;
- the local-moving result is a local optimum when the sweeps converge: no
  vertex gains by moving to a neighbouring or an empty community;
- the connected step splits each local-moving community into exactly the
  components of its induced subgraph;
- CM on a cluster made of two dense blocks joined by many edges plus a
  pendant block returns the three blocks, where WCC keeps the two dense
  blocks together; CM output clusters are connected, above the threshold
  (brute-force cuts), and inside one input cluster.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from tests._helpers import TAKEN_ID_CASE

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = json.load(open(os.path.join(HERE, "golden", "hand_traced.json")))


@pytest.mark.parametrize("case", GOLDEN["cpm"], ids=[c["name"] for c in GOLDEN["cpm"]])
def test_cpm_hand_traced(case):
    comm = oracle.cpm_communities(case["n"], case["eu"], case["ev"], case["gnum"], case["gden"])
    assert comm.tolist() == case["comm"]


def _random_graph(rng, n, p):
    eu, ev = [], []
    for u in range(n):
        for v in range(u + 1, n):
            if rng.random() < p:
                eu.append(u)
                ev.append(v)
    return np.array(eu, np.int32), np.array(ev, np.int32)


def _adj(n, eu, ev):
    nb = [[] for _ in range(n)]
    for u, v in zip(eu, ev):
        nb[u].append(v)
        nb[v].append(u)
    return nb


def test_cpm_large_resolution_leaves_singletons():
    rng = np.random.default_rng(0)
    for t in range(30):
        n = int(rng.integers(2, 40))
        eu, ev = _random_graph(rng, n, float(rng.uniform(0.05, 0.6)))
        dmax = max([0] + [len(x) for x in _adj(n, eu, ev)])
        # joining any community gains at most deg - gamma * 1 < 0 = staying alone
        comm = oracle.cpm_communities(n, eu, ev, dmax + 1, 1)
        assert comm.tolist() == list(range(n))


def test_cpm_disjoint_cliques_come_out_whole():
    rng = np.random.default_rng(1)
    for t in range(20):
        sizes = rng.integers(3, 13, size=int(rng.integers(1, 6)))
        perm = rng.permutation(int(sizes.sum()))
        eu, ev, members, b = [], [], [], 0
        for s in sizes:
            ids = perm[b:b + s]
            members.append(sorted(int(x) for x in ids))
            for i, j in itertools.combinations(ids, 2):
                eu.append(int(i))
                ev.append(int(j))
            b += s
        n = int(sizes.sum())
        comm = oracle.cpm_communities(n, np.array(eu, np.int32), np.array(ev, np.int32), 1, 100)
        for mem in members:
            assert {int(comm[v]) for v in mem} == {mem[0]}


def _gains_ok(n, nb, comm, gnum, gden):
    """True iff no vertex has a move whose gain (k(v,c)*gden - gnum*n_c, n_c
    without v; an empty community gains 0) is strictly above staying."""
    size = {}
    for v in range(n):
        size[comm[v]] = size.get(comm[v], 0) + 1
    for v in range(n):
        c0 = comm[v]
        k = {}
        for u in nb[v]:
            k[comm[u]] = k.get(comm[u], 0) + 1
        stay = k.get(c0, 0) * gden - gnum * (size[c0] - 1)
        best = 0 if size[c0] > 1 else None
        for c, kc in k.items():
            if c == c0:
                continue
            g = kc * gden - gnum * size[c]
            best = g if best is None or g > best else best
        if best is not None and best > stay:
            return False
    return True


def test_cpm_local_moving_ends_at_a_local_optimum():
    rng = np.random.default_rng(2)
    checked = 0
    for t in range(150):
        n = int(rng.integers(2, 60))
        eu, ev = _random_graph(rng, n, float(rng.uniform(0.03, 0.5)))
        gnum, gden = int(rng.integers(0, 4)), int(rng.integers(1, 9))
        comm = oracle.cpm_communities(n, eu, ev, gnum, gden, connected=False)
        assert _gains_ok(n, _adj(n, eu, ev), comm.tolist(), gnum, gden)
        checked += 1
    assert checked == 150


def test_cpm_connected_step_is_the_components_of_each_community():
    rng = np.random.default_rng(3)
    for t in range(100):
        n = int(rng.integers(2, 50))
        eu, ev = _random_graph(rng, n, float(rng.uniform(0.02, 0.3)))
        gnum, gden = int(rng.integers(0, 3)), int(rng.integers(1, 6))
        raw = oracle.cpm_communities(n, eu, ev, gnum, gden, connected=False)
        con = oracle.cpm_communities(n, eu, ev, gnum, gden, connected=True)
        # components of the graph keeping only edges inside a raw community
        keep = raw[eu] == raw[ev] if len(eu) else np.zeros(0, bool)
        comp = oracle.components(n, eu[keep], ev[keep])
        assert con.tolist() == comp.tolist()


def _blocks_graph():
    """Cluster 0: dense blocks A (0..19) and B (20..39), 12 edges between
    them, and a block C (40..51) hanging on A by one edge; cluster 1: a
    clique D (52..63)."""
    rng = np.random.default_rng(4)
    eu, ev = [], []

    def dense(lo, hi, p):
        for i in range(lo, hi):
            for j in range(i + 1, hi):
                if rng.random() < p:
                    eu.append(i)
                    ev.append(j)

    dense(0, 20, 0.8)
    dense(20, 40, 0.8)
    dense(40, 52, 0.9)
    dense(52, 64, 1.0)
    for t in range(12):  # A-B: 12 disjoint edges, far above T(40) = 1
        eu.append(t)
        ev.append(20 + t)
    eu.append(5)
    ev.append(45)  # C hangs on A by one edge
    labels = np.zeros(64, np.int32)
    labels[52:] = 1
    return 64, np.array(eu, np.int32), np.array(ev, np.int32), labels


def test_cm_splits_what_wcc_keeps():
    n, eu, ev, labels = _blocks_graph()
    off, adj = oracle.build_csr(n, eu, ev)
    wcc_out, _ = oracle.wcc(n, off, adj, labels, 2)
    cm_out, st = oracle.cm(n, off, adj, labels, 2, 1, 4)
    # WCC: the bridge to C is cut; A and B stay together (12 edges > T)
    assert len(set(wcc_out[:40].tolist())) == 1
    assert wcc_out[40] != wcc_out[0] and len(set(wcc_out[40:52].tolist())) == 1
    # CM: the side A u B goes through the community step and comes out as A, B
    assert len(set(cm_out[:20].tolist())) == 1 and len(set(cm_out[20:40].tolist())) == 1
    assert cm_out[0] != cm_out[20]
    assert len(set(cm_out[40:52].tolist())) == 1 and cm_out[40] not in (cm_out[0], cm_out[20])
    assert len(set(cm_out[52:].tolist())) == 1
    # ids: ranks of the smallest members (0, 20, 40, 52)
    assert [cm_out[0], cm_out[20], cm_out[40], cm_out[52]] == [0, 1, 2, 3]
    assert st["splits"] >= 1


def _brute_min_cut(n, nb):
    best = None
    for mask in range(1, 1 << (n - 1)):
        s = {v for v in range(n) if (mask >> v) & 1}
        cut = sum(1 for v in s for u in nb[v] if u not in s)
        best = cut if best is None or cut < best else best
    return best


def test_cm_output_invariants_on_random_planted_graphs():
    """Every CM output cluster is inside one input cluster, connected, and
    (up to 14 vertices, by enumerating all bipartitions) has min cut > T."""
    rng = np.random.default_rng(5)
    for t in range(25):
        k = int(rng.integers(2, 5))
        sizes = rng.integers(5, 15, size=k)
        n = int(sizes.sum())
        blk = np.repeat(np.arange(k), sizes)
        eu, ev = [], []
        for i in range(n):
            for j in range(i + 1, n):
                p = 0.6 if blk[i] == blk[j] else 0.05
                if rng.random() < p:
                    eu.append(i)
                    ev.append(j)
        eu, ev = np.array(eu, np.int32), np.array(ev, np.int32)
        labels = (blk // 2).astype(np.int32)  # pairs of blocks form the input clusters
        off, adj = oracle.build_csr(n, eu, ev)
        out, _ = oracle.cm(n, off, adj, labels, 3, int(rng.integers(1, 4)), 10)
        nb = _adj(n, eu, ev)
        for c in set(out.tolist()) - {-1}:
            mem = [v for v in range(n) if out[v] == c]
            assert len({int(labels[v]) for v in mem}) == 1
            idx = {v: i for i, v in enumerate(mem)}
            sub = [[idx[u] for u in nb[v] if u in idx] for v in mem]
            comp = oracle.components(len(mem), *_edge_list(sub))
            assert len(set(comp.tolist())) == 1
            if len(mem) <= 14:
                assert _brute_min_cut(len(mem), sub) > oracle.threshold(len(mem))


def _edge_list(sub):
    eu, ev = [], []
    for v, row in enumerate(sub):
        for u in row:
            if v < u:
                eu.append(v)
                ev.append(u)
    return np.array(eu, np.int32), np.array(ev, np.int32)



def test_cpm_local_optimum_where_the_id_n_plus_v_is_taken():
    """The 17-vertex graph of tests/_helpers.py: a vertex comes to share the
    id n + v with vertices that joined it there while its best move is to be
    alone; the empty community offered must then be another, empty id, or
    the vertex stays where it gains less than alone and the sweeps never
    settle (the local optimum fails)."""
    c = TAKEN_ID_CASE
    eu, ev = np.array(c["eu"], np.int32), np.array(c["ev"], np.int32)
    comm = oracle.cpm_communities(c["n"], eu, ev, c["gnum"], c["gden"], connected=False)
    assert _gains_ok(c["n"], _adj(c["n"], eu, ev), comm.tolist(), c["gnum"], c["gden"])


def _restated_local_moving(n, nb, gnum, gden, max_sweeps=64):
    """R12 written out from its statement: sweeps in ascending id; v leaves
    c0; candidates are its neighbours' other communities and, when c0 keeps
    members, an empty community (n + v when free, else the smallest free
    id); the largest gain wins, ties to the smallest id; v moves only on a
    strictly larger gain than staying.  Returns each vertex's community as
    the smallest member of it."""
    comm = list(range(n))
    size = [1] * n + [0] * n
    for _ in range(max_sweeps):
        moved = False
        for v in range(n):
            c0 = comm[v]
            k = {}
            for u in nb[v]:
                k[comm[u]] = k.get(comm[u], 0) + 1
            size[c0] -= 1
            stay = k.get(c0, 0) * gden - gnum * size[c0]
            cands = [(kc * gden - gnum * size[c], c) for c, kc in k.items() if c != c0]
            if size[c0] > 0:
                e = n + v if size[n + v] == 0 else next(i for i in range(2 * n) if size[i] == 0)
                cands.append((0, e))
            target = c0
            if cands:
                g, c = max(cands, key=lambda t: (t[0], -t[1]))
                if g > stay:
                    target = c
                    moved = True
            comm[v] = target
            size[target] += 1
        if not moved:
            break
    first = {}
    for v in range(n):
        first.setdefault(comm[v], v)
    return [first[comm[v]] for v in range(n)]


def test_cpm_sweeps_match_a_restatement():
    """The oracle's local moving equals the restatement above, community for
    community, on 2,000 seeded random graphs over a range of densities and
    resolutions (including the 17-vertex taken-id graph)."""
    rng = np.random.default_rng(9)
    cases = [(TAKEN_ID_CASE["n"], np.array(TAKEN_ID_CASE["eu"], np.int32),
              np.array(TAKEN_ID_CASE["ev"], np.int32), TAKEN_ID_CASE["gnum"], TAKEN_ID_CASE["gden"])]
    for t in range(2000):
        n = int(rng.integers(2, 40))
        eu, ev = _random_graph(rng, n, float(rng.uniform(0.03, 0.6)))
        cases.append((n, eu, ev, int(rng.integers(0, 6)), int(rng.integers(1, 9))))
    for n, eu, ev, gnum, gden in cases:
        got = oracle.cpm_communities(n, eu, ev, gnum, gden, connected=False).tolist()
        assert got == _restated_local_moving(n, _adj(n, eu, ev), gnum, gden), (n, gnum, gden)


def test_cm_idempotent():
    """CM output clusters are well connected (lambda > T after no peel), so
    CM run again on its own output accepts each of them whole: no cut
    split, so no community step, and the same clusters come back."""
    rng = np.random.default_rng(6)
    for t in range(20):
        k = int(rng.integers(2, 6))
        sizes = rng.integers(6, 30, size=k)
        n = int(sizes.sum())
        blk = np.repeat(np.arange(k), sizes)
        iu, ju = np.triu_indices(n, 1)
        pr = np.where(blk[iu] == blk[ju], float(rng.uniform(0.3, 0.8)), float(rng.uniform(0.0, 0.05)))
        keep = rng.random(len(iu)) < pr
        eu, ev = iu[keep].astype(np.int32), ju[keep].astype(np.int32)
        labels = (blk // 2).astype(np.int32)
        gnum, gden = int(rng.integers(1, 4)), int(rng.choice([10, 100]))
        off, adj = oracle.build_csr(n, eu, ev)
        out, _ = oracle.cm(n, off, adj, labels, 2, gnum, gden)
        again, st = oracle.cm(n, off, adj, out, 2, gnum, gden)
        assert again.tolist() == out.tolist()
        assert st["splits"] == 0
