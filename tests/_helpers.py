"""Test-only helpers: brute-force minimum cuts and refinement invariants.

Nothing here is part of the CUDA path or of the oracle; these are the
independent checks the oracle is pinned against.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components


def brute_min_cut(n: int, eu, ev, w=None):
    """Minimum over all 2^(n-1)-1 bipartitions (vertex 0 fixed on side A).
    Returns (value, list of minimising side masks as int bitmasks of B)."""
    eu = np.asarray(eu, np.int64)
    ev = np.asarray(ev, np.int64)
    w = np.ones(len(eu), np.int64) if w is None else np.asarray(w, np.int64)
    masks = np.arange(1, 1 << (n - 1), dtype=np.int64) << 1  # bit v set => v in B; bit 0 never set
    bu = (masks[:, None] >> eu[None, :]) & 1
    bv = (masks[:, None] >> ev[None, :]) & 1
    cut = ((bu != bv) * w[None, :]).sum(axis=1)
    best = int(cut.min())
    return best, [int(x) for x in masks[cut == best]]


def cut_value(eu, ev, side, w=None):
    eu = np.asarray(eu)
    ev = np.asarray(ev)
    side = np.asarray(side, bool)
    w = np.ones(len(eu), np.int64) if w is None else np.asarray(w, np.int64)
    return int(((side[eu] != side[ev]) * w).sum())


def induced_edges(off, adj, verts):
    """Edge list (local ids, u < v) of G[verts] for an ascending vertex array."""
    verts = np.asarray(verts, np.int64)
    pos = {int(v): i for i, v in enumerate(verts)}
    eu, ev = [], []
    for i, v in enumerate(verts):
        for u in adj[off[v]:off[v + 1]]:
            j = pos.get(int(u))
            if j is not None and i < j:
                eu.append(i); ev.append(j)
    return np.array(eu, np.int32), np.array(ev, np.int32)


def is_connected(n, eu, ev) -> bool:
    if n <= 1:
        return True
    A = sp.coo_matrix((np.ones(len(eu)), (eu, ev)), shape=(n, n))
    return connected_components(A, directed=False)[0] == 1


def clusters_of(labels):
    """dict label -> ascending vertex array (labels >= 0 only)."""
    labels = np.asarray(labels)
    idx = np.nonzero(labels >= 0)[0]
    order = idx[np.argsort(labels[idx], kind="stable")]
    lab = labels[order]
    if len(order) == 0:
        return {}
    cuts = np.nonzero(np.diff(lab))[0] + 1
    return {int(lab[a]): order[a:b] for a, b in zip(np.r_[0, cuts], np.r_[cuts, len(order)])}


def min_labels(labels):
    """Replace each output id by the smallest vertex id of its cluster."""
    labels = np.asarray(labels)
    out = np.full(len(labels), -1, np.int64)
    for _, vs in clusters_of(labels).items():
        out[vs] = vs.min()
    return out


# ---- capped maximum-adjacency passes, restated from their definition ----
# (Nagamochi-Ibaraki with threshold k: keys capped at k, largest key first,
# ties to the smallest id; an edge whose key reaches k is contracted.)  These
# restate the contraction independently of the oracle and of the kernel.

def nbr_lists(n, eu, ev):
    """Neighbour lists with one entry per edge (repeated for parallel edges)."""
    nb = [[] for _ in range(n)]
    for x, y in zip(eu, ev):
        nb[int(x)].append(int(y))
        nb[int(y)].append(int(x))
    return nb


def capped_pass(n, nbrs, k):
    """(pos, sat): pick step of every vertex and the step at which its key
    reached k (n + 1 if never)."""
    key = np.zeros(n, np.int64)
    added = np.zeros(n, bool)
    pos = np.full(n, -1, np.int64)
    sat = np.full(n, n + 1, np.int64)
    for step in range(n):
        v = int(np.argmax(np.where(added, -1, key)))  # largest key, smallest id
        added[v] = True
        pos[v] = step
        for u in nbrs[v]:
            if not added[u] and key[u] < k:
                key[u] += 1
                if key[u] == k:
                    sat[u] = step
    return pos, sat


def contracted(eu, ev, pos, sat):
    """Mask of contracted edges: the later end's key had reached k by the
    time the earlier end was picked."""
    a = np.where(pos[eu] < pos[ev], eu, ev)
    j = np.where(pos[eu] < pos[ev], ev, eu)
    return sat[j] <= pos[a]


def sets_of(n, eu, ev, mask):
    """Smallest member of each vertex's set under the masked edges."""
    p = np.arange(n)

    def find(x):
        while p[x] != x:
            p[x] = p[p[x]]
            x = p[x]
        return x

    for x, y in zip(eu[mask], ev[mask]):
        rx, ry = find(int(x)), find(int(y))
        if rx != ry:
            p[max(rx, ry)] = min(rx, ry)
    return np.array([find(x) for x in range(n)])


def contract_passes(n, eu, ev, k):
    """Passes of capped_pass on the contracted multigraph (super-vertices
    renumbered 0.. in ascending order of their smallest member, which keeps
    every tie) until one super-vertex is left or a pass contracts nothing.
    Returns (rep, passes): rep[v] = smallest member of v's super-vertex."""
    eu = np.asarray(eu, np.int64)
    ev = np.asarray(ev, np.int64)
    rep = np.arange(n)
    passes = 0
    while True:
        svs = np.unique(rep)
        if len(svs) <= 1:
            break
        idx = np.searchsorted(svs, rep)
        qu, qv = idx[eu], idx[ev]
        keep = qu != qv
        qu, qv = qu[keep], qv[keep]
        passes += 1
        pos, sat = capped_pass(len(svs), nbr_lists(len(svs), qu, qv), k)
        mask = contracted(qu, qv, pos, sat)
        if not mask.any():
            break
        rep = svs[sets_of(len(svs), qu, qv, mask)[idx]]
    return rep, passes


# A 17-vertex graph, found by a seeded search over random graphs, on which
# CPM local moving at resolution 2/5 brings a vertex v to share the id n + v
# with vertices that joined it there while v's best move is to be alone
# (the corner case of the empty-community candidate).
TAKEN_ID_CASE = dict(
    n=17, gnum=2, gden=5,
    eu=[0, 0, 0, 0, 1, 2, 2, 2, 2, 2, 3, 3, 3, 3, 3, 4, 4, 4, 4, 5, 5, 5, 6, 6, 6, 6, 7, 8, 8, 8,
        8, 9, 10, 10, 10, 11, 12, 12, 14],
    ev=[8, 9, 14, 15, 14, 3, 7, 8, 9, 14, 5, 9, 12, 14, 16, 7, 8, 11, 12, 10, 13, 14, 9, 10, 14,
        16, 10, 9, 11, 12, 13, 14, 11, 14, 16, 14, 14, 16, 15])


def taken_id_cm_input(clique: int = 5):
    """One input cluster: TAKEN_ID_CASE's graph joined to a clique on the
    next `clique` ids by the single edge 1-17, so that the cut split hands
    the 17-vertex graph to the community step whole.  Returns
    (n, src, dst, labels, min_size, gnum, gden)."""
    c = TAKEN_ID_CASE
    n = c["n"] + clique
    eu, ev = list(c["eu"]), list(c["ev"])
    for i in range(c["n"], n):
        for j in range(i + 1, n):
            eu.append(i)
            ev.append(j)
    eu.append(1)
    ev.append(c["n"])
    return (n, np.array(eu, np.int32), np.array(ev, np.int32), np.zeros(n, np.int32), 2,
            c["gnum"], c["gden"])
