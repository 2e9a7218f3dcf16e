"""Seeded synthetic graphs generated on the GPU (torch), for the sizes that
numpy would take minutes to hours to draw: the degree-corrected planted
partition with 10M vertices / 200M edges and with 100M vertices / 2B edges.

This module only draws random numbers (torch's Philox generator on the
device, numpy for the small per-cluster tables); it holds no part of the
refinement's arithmetic.  The same recipe as ``graphs.dc_planted``: Chung-Lu
weights with a power-law distribution, power-law cluster sizes, a fraction of
chain clusters cut into 2-4 parts joined by 1-2 bridges, intra edges spread
over the edge groups in proportion to their weight (capped at density 0.5)
with endpoints drawn in proportion to the weights inside the group, the rest
of the m drawn edges (including what the density cap refused) as inter edges
with endpoints drawn in proportion to the weights over the whole graph
(same-cluster pairs dropped), then a random relabelling of vertices and label
values, and removal of loops and repeats.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .graphs import _fit_expo, _fit_lo, _powerlaw, _sizes


@dataclass
class GpuWorkload:
    name: str
    n: int
    src: "object"      # torch int32 [m] on the device (u < v after dedup)
    dst: "object"
    labels: "object"   # torch int32 [n] on the device
    min_size: int
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.src.numel())


def _draw(torch, gen, cw, lo, hi, count):
    """Indices i with cw[i] <= x < cw[i+1] for x uniform in [cw[lo], cw[hi])."""
    a, b = cw[lo], cw[hi]
    x = a + torch.rand(count, generator=gen, device=cw.device, dtype=torch.float64) * (b - a)
    idx = torch.searchsorted(cw, x, right=True) - 1
    return torch.minimum(torch.maximum(idx, lo), hi - 1)


def dc_planted_gpu(n: int, m: int, seed: int = 0, deg_exp: float = 2.2, max_deg: int | None = None,
                   size_exp: float | None = 1.8, size_mean: float | None = None,
                   size_min: int = 10, size_max: int = 50_000, f_in: float = 0.8,
                   chain_frac: float = 0.05, chain_parts=(2, 4), min_size: int = 2,
                   device: str = "cuda", chunk: int = 1 << 27,
                   draw_factor: float = 1.0) -> GpuWorkload:
    """``draw_factor`` scales the number of edges drawn so that the edges left
    after dropping repeats and same-cluster inter pairs come close to m."""
    import torch

    rng = np.random.default_rng(seed)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    if size_exp is None:
        size_exp = _fit_expo(size_min, size_max, size_mean)
    if max_deg is None:
        max_deg = max(int(np.sqrt(n) * 10), 100)
    mean = 2.0 * m / n
    wmin = _fit_lo(deg_exp, max_deg, mean)

    # per-vertex weights (device)
    u = torch.rand(n, generator=gen, device=device, dtype=torch.float64)
    a, b = wmin ** (1.0 - deg_exp), max_deg ** (1.0 - deg_exp)
    w = (a + u * (b - a)) ** (1.0 / (1.0 - deg_exp))
    cw = torch.zeros(n + 1, dtype=torch.float64, device=device)
    cw[1:] = torch.cumsum(w, 0)
    del u, w

    # clusters and edge groups (host tables, vectorised)
    sizes = _sizes(rng, n, size_exp, size_min, size_max)
    k = len(sizes)
    starts = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    parts = rng.integers(chain_parts[0], chain_parts[1] + 1, size=k)
    is_chain = (rng.random(k) < chain_frac) & (sizes >= 2 * parts * 3)
    parts = np.where(is_chain, parts, 1)
    gcount = parts
    g_cluster = np.repeat(np.arange(k), gcount)
    g_index = np.arange(len(g_cluster)) - np.repeat(np.cumsum(gcount) - gcount, gcount)
    plen = sizes[g_cluster] // parts[g_cluster]
    g_start = starts[g_cluster] + g_index * plen
    g_len = np.where(g_index == parts[g_cluster] - 1, starts[g_cluster] + sizes[g_cluster] - g_start,
                     plen)
    # bridges between consecutive parts of chain clusters
    bmask = g_index < parts[g_cluster] - 1
    nb = rng.integers(1, 3, size=int(bmask.sum()))
    b_lo = np.repeat(g_start[bmask], nb)
    b_hi = np.repeat(g_start[bmask] + g_len[bmask], nb)
    b_lo2 = b_hi
    b_hi2 = np.repeat(g_start[np.nonzero(bmask)[0] + 1] + g_len[np.nonzero(bmask)[0] + 1], nb)
    bu = b_lo + (rng.random(len(b_lo)) * (b_hi - b_lo)).astype(np.int64)
    bv = b_lo2 + (rng.random(len(b_lo2)) * (b_hi2 - b_lo2)).astype(np.int64)

    gs = torch.from_numpy(g_start).to(device)
    gl = torch.from_numpy(g_len).to(device)
    gw = cw[gs + gl] - cw[gs]
    m_in = f_in * m * draw_factor * gw / gw.sum()
    cap = 0.5 * gl.double() * (gl.double() - 1) / 2.0
    m_g = torch.minimum(torch.round(m_in), torch.floor(cap)).long()
    comm = torch.repeat_interleave(torch.arange(k, device=device),
                                   torch.from_numpy(sizes).to(device))

    keys = []
    # intra edges, drawn group-chunk by group-chunk to bound memory
    total = int(m_g.sum().item())
    csum = torch.cumsum(m_g, 0)
    done = 0
    while done < total:
        hi_e = min(total, done + chunk)
        first = int(torch.searchsorted(csum, torch.tensor([done], device=device), right=True).item())
        last = int(torch.searchsorted(csum, torch.tensor([hi_e - 1], device=device),
                                      right=True).item())
        sel = torch.arange(first, last + 1, device=device)
        cnt = m_g[sel].clone()
        before = (csum[first] - m_g[first]).item()
        cnt[0] -= done - before
        cnt[-1] -= int(csum[last].item()) - hi_e
        g_of = torch.repeat_interleave(sel, cnt)
        lo, hi = gs[g_of], gs[g_of] + gl[g_of]
        iu = _draw(torch, gen, cw, lo, hi, len(g_of))
        iv = _draw(torch, gen, cw, lo, hi, len(g_of))
        keys.append(_pack(torch, iu, iv, n))
        done = hi_e
    # inter edges: the rest of the draw (intra edges a density cap refused
    # move here, so the total stays m * draw_factor)
    m_out = max(0, int(round(m * draw_factor)) - total)
    done = 0
    zero = torch.zeros((), dtype=torch.long, device=device)
    top = torch.full((), n, dtype=torch.long, device=device)
    while done < m_out:
        c = min(chunk, m_out - done)
        ou = _draw(torch, gen, cw, zero, top, c)
        ov = _draw(torch, gen, cw, zero, top, c)
        keep = comm[ou] != comm[ov]
        keys.append(_pack(torch, ou[keep], ov[keep], n))
        done += c
    keys.append(_pack(torch, torch.from_numpy(bu).to(device), torch.from_numpy(bv).to(device), n))
    del cw

    # random relabelling of vertices and label values, loops and repeats dropped
    perm = torch.randperm(n, generator=gen, device=device)
    lab = torch.empty(n, dtype=torch.int32, device=device)
    newv = torch.from_numpy(rng.permutation(3 * k)[:k].astype(np.int32)).to(device)
    lab[perm] = newv[comm].int()
    del comm
    allk = torch.cat(keys)
    del keys
    su = perm[allk // n]
    sv = perm[allk % n]
    del allk
    mn, mx = torch.minimum(su, sv), torch.maximum(su, sv)
    del su, sv
    key = mn * n + mx
    del mn, mx
    key = key[(key // n) != (key % n)]
    # sort and drop repeats in key-range buckets (a sort takes at most 2^31
    # elements; equal keys always share a bucket)
    nb = max(1, -(-key.numel() // (1 << 30)))
    span = -(-(n * n) // nb)
    srcs, dsts = [], []
    for bi in range(nb):
        part = key[(key >= bi * span) & (key < (bi + 1) * span)] if nb > 1 else key
        part, _ = torch.sort(part)
        if part.numel():
            part = part[torch.cat([torch.ones(1, dtype=torch.bool, device=device),
                                   part[1:] != part[:-1]])]
        srcs.append((part // n).int())
        dsts.append((part % n).int())
        del part
    del key
    src = torch.cat(srcs)
    dst = torch.cat(dsts)
    del srcs, dsts
    return GpuWorkload("dc_planted_gpu", n, src, dst, lab, min_size,
                       {"clusters": k, "chains": int(is_chain.sum()), "w_min": wmin,
                        "intra_drawn": total, "inter_drawn": m_out,
                        "size_exp": size_exp, "seed": seed,
                        "cluster_sizes": sizes, "chain_clusters": np.nonzero(is_chain)[0],
                        "label_of_cluster": newv.cpu().numpy()})


def _pack(torch, u, v, n):
    u = u.long()
    v = v.long()
    return torch.minimum(u, v) * n + torch.maximum(u, v)


def dcpp_10m(seed: int = 0, device: str = "cuda") -> GpuWorkload:
    """10M vertices, about 200M undirected edges (Chung-Lu exponent 2.2, mean
    degree 40), cluster sizes power law (1.8) on [10, 50000], 80% intra edges,
    5% chain clusters of 2-4 parts."""
    return dc_planted_gpu(10_000_000, 200_000_000, seed=seed, deg_exp=2.2, size_exp=1.8,
                          size_min=10, size_max=50_000, f_in=0.8, chain_frac=0.05,
                          chain_parts=(2, 4), device=device, draw_factor=1.285)


def dcpp_1m(seed: int = 0, device: str = "cuda") -> GpuWorkload:
    """The laws of dcpp_10m at a tenth of the size: 1M vertices, about 20M
    undirected edges, cluster sizes on [10, 50000] (a case small enough for
    a profiler capture of one refinement launch)."""
    return dc_planted_gpu(1_000_000, 20_000_000, seed=seed, deg_exp=2.2, size_exp=1.8,
                          size_min=10, size_max=50_000, f_in=0.8, chain_frac=0.05,
                          chain_parts=(2, 4), device=device, draw_factor=1.285)


def dcpp_100m(seed: int = 0, device: str = "cuda") -> GpuWorkload:
    """100M vertices, about 2B undirected edges (Chung-Lu exponent 2.1,
    maximum degree 200k), cluster sizes on [10, 100000] with the exponent
    fitted to a mean of 20 (5M clusters), 80% intra edges, 3% bridged
    2-part chain clusters."""
    return dc_planted_gpu(100_000_000, 2_000_000_000, seed=seed, deg_exp=2.1, max_deg=200_000,
                          size_exp=None, size_mean=20.0, size_min=10, size_max=100_000,
                          f_in=0.8, chain_frac=0.03, chain_parts=(2, 2), device=device,
                          draw_factor=1.19)


def dcpp_10m_b(seed: int = 0, device: str = "cuda") -> GpuWorkload:
    """The second reading of the 10M-vertex configuration: 500k clusters,
    the size exponent fitted to a mean of 20 on [10, 50000]; 10M vertices,
    about 200M undirected edges (Chung-Lu exponent 2.2, mean degree 40), 80%
    intra edges asked for but capped at density 0.5 inside clusters this
    small (the rest are drawn between clusters; meta holds the realised
    split), 5% chain clusters of 2-4 parts."""
    return dc_planted_gpu(10_000_000, 200_000_000, seed=seed, deg_exp=2.2, size_exp=None,
                          size_mean=20.0, size_min=10, size_max=50_000, f_in=0.8,
                          chain_frac=0.05, chain_parts=(2, 4), device=device, draw_factor=1.19)
