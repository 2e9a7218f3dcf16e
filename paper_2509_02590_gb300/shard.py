"""One graph's input clusters refined on several GPUs, one process per GPU.

Algorithms 1-2 of the paper refine every input cluster on its own (the
``forall`` over the clusters of Sections 2.2-2.3), so the input clusters of
one graph can be dealt out to ranks with nothing exchanged while they are
refined.  Each rank holds a full copy of the graph and runs ``wcc_run`` on
its shard (the labels of every other shard set to -1).  The only exchange
is the canonical numbering at the end: every rank turns its result into
cluster minima (per vertex, the smallest vertex id of its output cluster,
``wcc_cluster_minima``); the shards are disjoint, so the element-wise
maximum over ranks -- one all-reduce -- is the minima of the whole run, and
``wcc_number_by_minima`` numbers it exactly as one ``wcc_run`` would.

The shards are planned by longest-processing-time-first on the estimated
work of each input cluster, n_c times the degree sum of its members (an
item's extraction reads every member's row; its cut work grows with n_c).

This module plans and orchestrates; the refinement, the minima and the
numbering run in the library's kernels.
"""
from __future__ import annotations

import heapq

import numpy as np


def cluster_work(labels: np.ndarray, deg: np.ndarray):
    """(values, work): the distinct input labels >= 0 (ascending) and, per
    label, n_c * (sum of its members' degrees)."""
    labels = np.asarray(labels)
    deg = np.asarray(deg, np.int64)
    ok = labels >= 0
    values, inv = np.unique(labels[ok], return_inverse=True)
    n_c = np.bincount(inv, minlength=len(values)).astype(np.int64)
    d_c = np.bincount(inv, weights=deg[ok], minlength=len(values)).astype(np.int64)
    return values.astype(np.int64), n_c * d_c


def lpt_owner(work: np.ndarray, world: int):
    """Longest processing time first: clusters in decreasing work (ties: the
    smaller index first) each go to the least-loaded rank (ties: the lower
    rank).  Returns (owner rank per cluster, load per rank)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    work = np.asarray(work, np.int64)
    order = np.lexsort((np.arange(len(work)), -work))
    owner = np.empty(len(work), np.int32)
    heap = [(0, r) for r in range(world)]
    for c in order:
        load, r = heapq.heappop(heap)
        owner[c] = r
        heapq.heappush(heap, (load + int(work[c]), r))
    loads = np.zeros(world, np.int64)
    np.add.at(loads, owner, work)
    return owner, loads


class ShardPlan:
    """Which rank refines which input cluster."""

    def __init__(self, labels: np.ndarray, deg: np.ndarray, world: int):
        self.world = world
        self.values, self.work = cluster_work(labels, deg)
        self.owner, self.loads = lpt_owner(self.work, world)

    def mask(self, rank: int) -> np.ndarray:
        """Shard of rank as a mask over label values 0..max (for
        ``only_labels``-style selection)."""
        top = int(self.values.max()) + 1 if len(self.values) else 0
        m = np.zeros(top, np.uint8)
        m[self.values[self.owner == rank]] = 1
        return m

    def shard_labels(self, labels, rank: int):
        """labels with every input cluster outside rank's shard set to -1
        (numpy in, numpy out; a CUDA tensor in, a CUDA tensor out)."""
        if type(labels).__module__.startswith("torch"):
            import torch
            dev = labels.device
            values = torch.from_numpy(self.values).to(dev)
            owner = torch.from_numpy(self.owner).to(dev)
            ok = labels >= 0
            idx = torch.searchsorted(values, torch.where(ok, labels, 0).to(torch.int64))
            idx = torch.clamp(idx, max=max(len(self.values) - 1, 0))
            mine = ok & (owner[idx] == rank) if len(self.values) else ok & False
            return torch.where(mine, labels, torch.full_like(labels, -1))
        labels = np.asarray(labels, np.int32)
        out = np.full_like(labels, -1)
        ok = np.nonzero(labels >= 0)[0]
        if len(ok):
            idx = np.searchsorted(self.values, labels[ok])
            sel = ok[self.owner[idx] == rank]
            out[sel] = labels[sel]
        return out


def refine_merged(plan: ShardPlan, rank: int, labels, refine_minima, allreduce_max, number):
    """One rank's part of a sharded refinement.

    refine_minima(shard_labels) -> this shard's cluster minima (-1 outside
    it); allreduce_max(minima) -> the element-wise maximum over all ranks;
    number(minima) -> the canonical labels.  Returns the merged labels (the
    same on every rank)."""
    mine = plan.shard_labels(labels, rank)
    minima = refine_minima(mine)
    merged = allreduce_max(minima)
    return number(merged)


def gpu_refine_sharded(graph, labels, rank: int, plan: ShardPlan, group=None, min_size: int = 2,
                       rule="log10", num: int = 1, den: int = 1, mode="batched"):
    """The sharded refinement on this rank's GPU: labels is a CUDA int32
    tensor (the whole input clustering, the same on every rank), graph a
    WccGraph on this rank's device.  The minima are all-reduced with
    torch.distributed (``group``; no all-reduce when the plan has one
    rank).  Returns the merged refined clustering as a CUDA tensor."""
    import torch

    from . import _binding

    def refine_minima(lab_r):
        out_r = graph.run(lab_r, min_size=min_size, rule=rule, num=num, den=den, mode=mode)
        mn = torch.empty_like(out_r)
        _binding.wcc_cluster_minima(out_r.data_ptr(), out_r.numel(), mn.data_ptr(), 1,
                                    torch.cuda.current_stream(out_r.device).cuda_stream)
        return mn

    def allreduce_max(mn):
        if plan.world > 1:
            import torch.distributed as dist
            dist.all_reduce(mn, op=dist.ReduceOp.MAX, group=group)
        return mn

    def number(mn):
        out = torch.empty_like(mn)
        _binding.wcc_number_by_minima(mn.data_ptr(), mn.numel(), out.data_ptr(), 1,
                                      torch.cuda.current_stream(mn.device).cuda_stream)
        return out

    return refine_merged(plan, rank, labels, refine_minima, allreduce_max, number)
