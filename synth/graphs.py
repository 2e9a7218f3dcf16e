"""Seeded synthetic graphs and input clusterings.

Every generator returns a :class:`Workload`: ``n`` vertices, an undirected
simple edge list (``src[i] < dst[i]`` after dedup, int32, each edge once) and
an input clustering ``labels`` (int32, ``-1`` = unclustered).  Vertex ids and
label values are randomly permuted, so clusters are never contiguous id
ranges and label values are arbitrary non-negative integers.

The real graphs and Leiden clusterings of the paper's experiments are not
available here; these generators stand in for them (planted clusters over
power-law graphs).  Recipes are documented on each function.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    n: int
    src: np.ndarray
    dst: np.ndarray
    labels: np.ndarray
    min_size: int
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(len(self.src))

    @property
    def n_clusters(self) -> int:
        lab = self.labels[self.labels >= 0]
        return int(len(np.unique(lab))) if len(lab) else 0


def _dedup(n: int, u: np.ndarray, v: np.ndarray):
    """Drop self-loops and repeated edges; return (min, max) endpoint arrays."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    keep = u != v
    a = np.minimum(u[keep], v[keep])
    b = np.maximum(u[keep], v[keep])
    key = a * n + b
    key.sort()
    if len(key):
        key = key[np.concatenate(([True], key[1:] != key[:-1]))]
    return (key // n).astype(np.int32), (key % n).astype(np.int32)


def _permute(rng, n, src, dst, labels):
    """Random vertex relabelling and random relabelling of cluster values."""
    perm = rng.permutation(n).astype(np.int64)
    s, d = perm[src], perm[dst]
    lab = np.full(n, -1, dtype=np.int64)
    lab[perm] = labels
    vals = np.unique(lab[lab >= 0])
    if len(vals):
        newv = rng.permutation(len(vals) * 3)[:len(vals)]  # sparse, arbitrary values
        lut = np.full(int(vals.max()) + 1, -1, dtype=np.int64)
        lut[vals] = newv
        lab = np.where(lab >= 0, lut[np.maximum(lab, 0)], -1)
    s2, d2 = _dedup(n, s, d)
    return s2, d2, lab.astype(np.int32)


def _powerlaw(rng, expo: float, lo: float, hi: float, size: int) -> np.ndarray:
    """Continuous power law p(x) ~ x^-expo on [lo, hi] by inverse transform."""
    u = rng.random(size)
    a, b = lo ** (1.0 - expo), hi ** (1.0 - expo)
    return (a + u * (b - a)) ** (1.0 / (1.0 - expo))


def _powerlaw_mean(expo: float, lo: float, hi: float) -> float:
    if abs(expo - 2.0) < 1e-12:
        num = np.log(hi / lo)
    else:
        num = (hi ** (2 - expo) - lo ** (2 - expo)) / (2 - expo)
    den = (hi ** (1 - expo) - lo ** (1 - expo)) / (1 - expo)
    return float(num / den)


def _fit_lo(expo: float, hi: float, mean: float) -> float:
    """Lower cut-off giving the requested mean (bisection)."""
    lo_, hi_ = 1.0, hi
    for _ in range(100):
        mid = 0.5 * (lo_ + hi_)
        if _powerlaw_mean(expo, mid, hi) < mean:
            lo_ = mid
        else:
            hi_ = mid
    return 0.5 * (lo_ + hi_)


def _fit_expo(lo: float, hi: float, mean: float) -> float:
    """Power-law exponent giving the requested mean on [lo, hi] (bisection)."""
    a, b = 1.01, 10.0
    for _ in range(200):
        mid = 0.5 * (a + b)
        if _powerlaw_mean(mid, lo, hi) > mean:
            a = mid
        else:
            b = mid
    return 0.5 * (a + b)


def _sizes(rng, n: int, expo: float, lo: int, hi: int) -> np.ndarray:
    """Cluster sizes drawn from a power law until they cover n vertices; the
    last size is trimmed and a too-small remainder is folded into the others."""
    out = []
    total = 0
    while total < n:
        s = np.rint(_powerlaw(rng, expo, lo, hi, 4096)).astype(np.int64)
        out.append(s)
        total += int(s.sum())
    s = np.concatenate(out)
    c = np.cumsum(s)
    k = int(np.searchsorted(c, n)) + 1
    s = s[:k].copy()
    s[-1] -= int(s.sum()) - n
    if s[-1] < lo and k > 1:
        rem = int(s[-1])
        s = s[:-1]
        idx = rng.integers(0, len(s), size=rem)
        np.add.at(s, idx, 1)
    return s


def _members(comm: np.ndarray, k: int):
    """Vertices grouped by community: (order, start offsets)."""
    order = np.argsort(comm, kind="stable")
    cnt = np.bincount(comm, minlength=k)
    start = np.zeros(k + 1, dtype=np.int64)
    np.cumsum(cnt, out=start[1:])
    return order, start


def planted_1k(seed: int = 0) -> Workload:
    """Planted partition, 1,000 vertices in 20 blocks of 50, p_in = 0.2,
    p_out = 0.002.  Blocks 0-3 are two halves of 25 (p_in only inside a half)
    joined by one uniformly drawn edge; blocks 4 and 5 each get 5 pendant
    vertices (ids 1000..1009 before relabelling) with one edge to a uniform
    member of their block and in that block's input cluster.  Input
    clustering = the blocks; min size 11."""
    rng = np.random.default_rng(seed)
    n0, bs = 1000, 50
    iu, ju = np.triu_indices(n0, 1)
    bi, bj = iu // bs, ju // bs
    same = bi == bj
    bridged = bi < 4
    same_half = (iu % bs) // 25 == (ju % bs) // 25
    p = np.where(same, np.where(bridged & ~same_half, 0.0, 0.2), 0.002)
    keep = rng.random(len(iu)) < p
    src = [iu[keep]]
    dst = [ju[keep]]
    for b in range(4):
        src.append(np.array([b * bs + rng.integers(0, 25)]))
        dst.append(np.array([b * bs + 25 + rng.integers(0, 25)]))
    labels = np.concatenate([np.arange(n0) // bs, np.repeat([4, 5], 5)])
    pend = np.arange(n0, n0 + 10)
    hosts = np.concatenate([4 * bs + rng.integers(0, bs, 5), 5 * bs + rng.integers(0, bs, 5)])
    src.append(pend)
    dst.append(hosts)
    n = n0 + 10
    s, d, lab = _permute(rng, n, np.concatenate(src), np.concatenate(dst), labels)
    return Workload("planted_1k", n, s, d, lab, 11,
                    {"blocks": 20, "block_size": bs, "p_in": 0.2, "p_out": 0.002, "seed": seed})


def lfr_like(n: int = 100_000, seed: int = 0, mean_deg: float = 20.0, deg_exp: float = 2.5,
             max_deg: int = 1000, size_exp: float = 1.5, size_min: int = 20,
             size_max: int = 2000, mu: float = 0.3, merge_frac: float = 0.1,
             min_size: int = 2) -> Workload:
    """LFR-style benchmark graph (written from the published description of
    the LFR benchmark, not from its code).

    Degrees: power law (exponent ``deg_exp``) on [k_min, max_deg], k_min
    fitted so the mean is ``mean_deg``.  Community sizes: power law
    (``size_exp``) on [size_min, size_max] covering n.  Vertices are assigned
    to communities uniformly at random; each gets intra-degree
    round((1-mu) k) capped at its community size - 1, the rest of its degree
    inter-community.  Intra stubs are wired by a configuration model inside
    each community, inter stubs across the graph (same-community inter pairs,
    loops and repeats dropped).  Then ``merge_frac`` of the communities
    (rounded to an even count) are paired at random: the edges between the two
    members of a pair are deleted and 1 or 2 (uniform) bridge edges added, and
    the pair forms one input cluster.  Input clustering = communities with the
    merged pairs."""
    rng = np.random.default_rng(seed)
    kmin = _fit_lo(deg_exp, max_deg, mean_deg)
    deg = np.clip(np.rint(_powerlaw(rng, deg_exp, kmin, max_deg, n)), 1, max_deg).astype(np.int64)
    sizes = _sizes(rng, n, size_exp, size_min, size_max)
    k = len(sizes)
    comm = np.repeat(np.arange(k), sizes)
    rng.shuffle(comm)
    d_in = np.minimum(np.rint((1.0 - mu) * deg).astype(np.int64), sizes[comm] - 1)
    d_out = deg - d_in

    # intra: configuration model per community
    stub_v = np.repeat(np.arange(n), d_in)
    stub_c = comm[stub_v]
    order = np.lexsort((rng.random(len(stub_v)), stub_c))
    stub_v, stub_c = stub_v[order], stub_c[order]
    cnt = np.bincount(stub_c, minlength=k)
    last = np.cumsum(cnt) - 1
    drop = np.zeros(len(stub_v), dtype=bool)
    drop[last[(cnt % 2 == 1)]] = True
    stub_v = stub_v[~drop]
    iu, iv = stub_v[0::2], stub_v[1::2]

    # inter: configuration model over the whole graph
    ost = np.repeat(np.arange(n), d_out)
    rng.shuffle(ost)
    if len(ost) % 2:
        ost = ost[:-1]
    ou, ov = ost[0::2], ost[1::2]
    keep = comm[ou] != comm[ov]
    ou, ov = ou[keep], ov[keep]

    u = np.concatenate([iu, ou])
    v = np.concatenate([iv, ov])

    # merge pairs of communities through 1-2 bridges
    n_merge = 2 * int(round(merge_frac * k / 2.0))
    chosen = rng.choice(k, size=n_merge, replace=False)
    pairs = chosen.reshape(-1, 2)
    partner = np.full(k, -1, dtype=np.int64)
    partner[pairs[:, 0]] = pairs[:, 1]
    partner[pairs[:, 1]] = pairs[:, 0]
    between = partner[comm[u]] == comm[v]
    u, v = u[~between], v[~between]
    order_m, start = _members(comm, k)
    bu, bv = [], []
    for a, b in pairs:
        nb = int(rng.integers(1, 3))
        ma = order_m[start[a]:start[a + 1]]
        mb = order_m[start[b]:start[b + 1]]
        bu.append(ma[rng.integers(0, len(ma), nb)])
        bv.append(mb[rng.integers(0, len(mb), nb)])
    u = np.concatenate([u] + bu)
    v = np.concatenate([v] + bv)
    lab_of_comm = np.arange(k)
    lab_of_comm[pairs[:, 1]] = pairs[:, 0]
    labels = lab_of_comm[comm]
    s, d, lab = _permute(rng, n, u, v, labels)
    return Workload("lfr_like", n, s, d, lab, min_size,
                    {"k_min": kmin, "communities": k, "merged_pairs": len(pairs), "mu": mu,
                     "seed": seed})


def dc_planted(n: int, m: int, seed: int = 0, deg_exp: float = 2.2, max_deg: int | None = None,
               size_exp: float = 1.8, size_min: int = 10, size_max: int = 50_000,
               f_in: float = 0.8, chain_frac: float = 0.05, chain_parts=(2, 4),
               min_size: int = 2) -> Workload:
    """Degree-corrected planted partition with Chung-Lu degrees.

    Weights w_v: power law (``deg_exp``) on [w_min, max_deg] with w_min fitted
    so the mean is 2m/n.  Cluster sizes: power law (``size_exp``) on
    [size_min, size_max] covering n.  A fraction ``chain_frac`` of the
    clusters (those with at least 2*parts*3 members) are chains: their members
    are cut into p equal parts (p uniform in ``chain_parts``), intra edges stay
    inside a part, and 1-2 bridge edges join consecutive parts.  f_in*m intra
    edges are spread over the edge groups (clusters, or chain parts) in
    proportion to their weight, capped at density 0.5, with both endpoints
    drawn in proportion to w inside the group; (1-f_in)*m inter edges draw
    both endpoints in proportion to w over the whole graph (same-cluster
    pairs dropped).  Loops and repeats dropped."""
    rng = np.random.default_rng(seed)
    mean = 2.0 * m / n
    if max_deg is None:
        max_deg = max(int(np.sqrt(n) * 10), 100)
    wmin = _fit_lo(deg_exp, max_deg, mean)
    w = _powerlaw(rng, deg_exp, wmin, max_deg, n)
    sizes = _sizes(rng, n, size_exp, size_min, size_max)
    k = len(sizes)
    comm = np.repeat(np.arange(k), sizes)  # vertices of a cluster contiguous before relabelling
    starts = np.concatenate([[0], np.cumsum(sizes)])

    # edge groups: clusters, with chain clusters split into parts
    grp_start, grp_len, grp_cluster = [], [], []
    bu, bv = [], []
    is_chain = (rng.random(k) < chain_frac)
    for c in range(k):
        s0, sz = int(starts[c]), int(sizes[c])
        p = int(rng.integers(chain_parts[0], chain_parts[1] + 1)) if is_chain[c] else 1
        if p > 1 and sz >= 2 * p * 3:
            plen = sz // p
            bounds = [s0 + i * plen for i in range(p)] + [s0 + sz]
            for i in range(p):
                grp_start.append(bounds[i]); grp_len.append(bounds[i + 1] - bounds[i])
                grp_cluster.append(c)
            for i in range(p - 1):
                nb = int(rng.integers(1, 3))
                bu.append(rng.integers(bounds[i], bounds[i + 1], nb))
                bv.append(rng.integers(bounds[i + 1], bounds[i + 2], nb))
        else:
            is_chain[c] = False
            grp_start.append(s0); grp_len.append(sz); grp_cluster.append(c)
    grp_start = np.asarray(grp_start, dtype=np.int64)
    grp_len = np.asarray(grp_len, dtype=np.int64)
    cw = np.concatenate([[0.0], np.cumsum(w)])
    gw = cw[grp_start + grp_len] - cw[grp_start]
    m_in = f_in * m * gw / gw.sum()
    cap = 0.5 * grp_len * (grp_len - 1) / 2.0
    m_g = np.minimum(np.rint(m_in), np.floor(cap)).astype(np.int64)
    g_of_edge = np.repeat(np.arange(len(grp_len)), m_g)

    def draw(g):
        lo = cw[grp_start[g]]
        hi = cw[grp_start[g] + grp_len[g]]
        x = lo + rng.random(len(g)) * (hi - lo)
        idx = np.searchsorted(cw, x, side="right") - 1
        return np.clip(idx, grp_start[g], grp_start[g] + grp_len[g] - 1)

    iu, iv = draw(g_of_edge), draw(g_of_edge)
    m_out = int(round((1.0 - f_in) * m))
    x1 = rng.random(m_out) * cw[-1]
    x2 = rng.random(m_out) * cw[-1]
    ou = np.clip(np.searchsorted(cw, x1, side="right") - 1, 0, n - 1)
    ov = np.clip(np.searchsorted(cw, x2, side="right") - 1, 0, n - 1)
    keep = comm[ou] != comm[ov]
    u = np.concatenate([iu, ou[keep]] + bu)
    v = np.concatenate([iv, ov[keep]] + bv)
    s, d, lab = _permute(rng, n, u, v, comm)
    return Workload("dc_planted", n, s, d, lab, min_size,
                    {"clusters": k, "chains": int(is_chain.sum()), "w_min": wmin,
                     "f_in_target": f_in, "seed": seed})


def random_gnp(n: int, p: float, rng) -> tuple[np.ndarray, np.ndarray]:
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(len(iu)) < p
    return iu[keep].astype(np.int32), ju[keep].astype(np.int32)


def tiny_family(name: str, *args, seed: int = 0):
    """Small named graphs for closed-form checks: returns (n, eu, ev)."""
    rng = np.random.default_rng(seed)
    if name == "complete":
        (n,) = args
        iu, ju = np.triu_indices(n, 1)
        return n, iu.astype(np.int32), ju.astype(np.int32)
    if name == "cycle":
        (n,) = args
        a = np.arange(n)
        return n, a.astype(np.int32), ((a + 1) % n).astype(np.int32)
    if name == "path":
        (n,) = args
        a = np.arange(n - 1)
        return n, a.astype(np.int32), (a + 1).astype(np.int32)
    if name == "tree":
        (n,) = args
        child = np.arange(1, n)
        parent = np.array([rng.integers(0, c) for c in child])
        return n, parent.astype(np.int32), child.astype(np.int32)
    if name == "hypercube":
        (d,) = args
        n = 1 << d
        u, v = [], []
        for x in range(n):
            for b in range(d):
                y = x ^ (1 << b)
                if x < y:
                    u.append(x); v.append(y)
        return n, np.array(u, np.int32), np.array(v, np.int32)
    if name == "bipartite":
        a, b = args
        u = np.repeat(np.arange(a), b)
        v = np.tile(np.arange(a, a + b), a)
        return a + b, u.astype(np.int32), v.astype(np.int32)
    if name == "two_cliques":
        a, kb = args  # two K_a joined by kb <= a disjoint edges
        iu, ju = np.triu_indices(a, 1)
        u = np.concatenate([iu, iu + a, np.arange(kb)])
        v = np.concatenate([ju, ju + a, a + np.arange(kb)])
        return 2 * a, u.astype(np.int32), v.astype(np.int32)
    raise ValueError(name)


WORKLOADS = {
    "planted_1k": lambda seed=0: planted_1k(seed),
    "lfr_100k": lambda seed=0: lfr_like(100_000, seed),
    "dcpp_10m": lambda seed=0: dc_planted(10_000_000, 200_000_000, seed, deg_exp=2.2,
                                          size_exp=1.8, size_min=10, size_max=50_000,
                                          chain_frac=0.05, chain_parts=(2, 4)),
}
