"""Multi-rank paths on two CPU processes over gloo: bench.py's weak scaling
(one independent instance per rank, max-over-ranks time, summed work), one
graph's input clusters sharded over ranks and merged into the canonical
numbering, and the reference arm's rank rule (rank 0 alone reports)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


CHILD = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import torch, torch.distributed as dist
import bench, synth
dist.init_process_group("gloo")
r = dist.get_rank()
w = synth.lfr_like(3000, seed=r)            # each rank its own instance
ms = 10.0 + 5.0 * r                          # pretend per-rank step times
out = bench.aggregate_ranks(dist, torch, torch.device("cpu"), ms, w.m, w.n_clusters)
print(json.dumps({{"rank": r, "m": w.m, "k": w.n_clusters, "agg": out}}), flush=True)
dist.barrier()
dist.destroy_process_group()
"""


def test_weak_scaling_aggregation_two_ranks():
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r),
                   WORLD_SIZE="2", LOCAL_RANK=str(r))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=300)
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    m_sum = sum(o["m"] for o in outs)
    k_sum = sum(o["k"] for o in outs)
    for o in outs:
        t, m, k = o["agg"]
        assert t == 15.0            # the slowest rank
        assert m == m_sum and k == k_sum
    assert outs[0]["m"] != outs[1]["m"]  # independent instances per rank


def test_reference_arm_only_rank0_reports():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3", "--gpus", "2"], env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_prints_the_contract_line():
    """Rank 0 of the reference arm (the oracle on the host cores) prints one
    JSON line with the keys of the bench contract."""
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "planted_1k", "--steps", "2", "--warmup", "3"], env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3
    assert d["value"] > 0 and d["unit"] == "edges/s" and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("planted_1k")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_oracle_over_all_cores_leaves_no_process():
    """The all-cores oracle figure: disjoint input clusters per spawned
    process, a positive rate, and every worker gone afterwards."""
    import multiprocessing as mp

    sys.path.insert(0, ROOT)
    import bench
    import synth
    w = synth.lfr_like(20_000, seed=0, min_size=2)
    r = bench.cpu_baseline_pool(w, budget_s=1.0)
    assert r["value"] > 0 and r["unit"] == "edges/s" and r["cores"] >= 1
    assert not mp.active_children()
    with pytest.raises(Exception):
        bench.cpu_baseline_pool(w, timeout_s=0.001)  # workers cannot start in time
    assert not mp.active_children()


# ---- one graph's input clusters sharded over ranks -------------------------
SHARD_CHILD = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import numpy as np
import torch, torch.distributed as dist
import oracle, synth
from paper_2509_02590_gb300.shard import ShardPlan, refine_merged
dist.init_process_group("gloo")
r, world = dist.get_rank(), dist.get_world_size()
w = synth.lfr_like(6000, seed=3, min_size=2)      # the same graph on every rank
off, adj = oracle.build_csr(w.n, w.src, w.dst)
plan = ShardPlan(w.labels, np.diff(off), world)

def refine_minima(lab_r):
    # this rank's shard refined alone (labels of other shards are -1), as
    # cluster minima: the oracle's smallest-vertex output form
    out, _ = oracle.wcc(w.n, off, adj, lab_r, w.min_size, out_mode=1)
    return torch.from_numpy(out)

def allreduce_max(t):
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t

def number(mn):
    mn = mn.numpy()
    ids = np.unique(mn[mn >= 0])
    out = np.full(len(mn), -1, np.int32)
    out[mn >= 0] = np.searchsorted(ids, mn[mn >= 0])
    return out

merged = refine_merged(plan, r, w.labels, refine_minima, allreduce_max, number)
ref, _ = oracle.wcc(w.n, off, adj, w.labels, w.min_size)
mine = plan.shard_labels(w.labels, r)
print(json.dumps({{"rank": r, "equal": bool(np.array_equal(merged, ref)),
                   "loads": plan.loads.tolist(), "work_max": int(plan.work.max()),
                   "mine": sorted(set(mine[mine >= 0].tolist()))}}), flush=True)
dist.barrier()
dist.destroy_process_group()
"""


def test_sharded_refinement_equals_one_rank():
    """Two gloo ranks refine disjoint LPT shards of one graph's input
    clusters (the oracle stands in for the GPU refinement on CPU), merge
    their cluster minima with one all-reduce (max) and number them: the
    result equals one rank refining everything."""
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r),
                   WORLD_SIZE="2", LOCAL_RANK=str(r))
        procs.append(subprocess.Popen([sys.executable, "-c", SHARD_CHILD.format(root=ROOT)],
                                      env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=300)
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    assert all(o["equal"] for o in outs)
    a, b = set(outs[0]["mine"]), set(outs[1]["mine"])
    assert a and b and not (a & b)                      # disjoint, both non-empty
    loads = outs[0]["loads"]
    assert max(loads) - min(loads) <= outs[0]["work_max"]  # LPT balance bound


def test_lpt_owner_by_hand():
    sys.path.insert(0, ROOT)
    import numpy as np

    from paper_2509_02590_gb300.shard import lpt_owner
    # 10 -> rank 0, 9 -> rank 1, 8 -> rank 1 (9 < 10), 7 -> rank 0 (10 < 17),
    # 1 -> rank 0 (17 = 17: the lower rank)
    owner, loads = lpt_owner(np.array([10, 9, 8, 7, 1]), 2)
    assert owner.tolist() == [0, 1, 1, 0, 0] and loads.tolist() == [18, 17]
    owner, loads = lpt_owner(np.array([5, 5, 5]), 1)
    assert owner.tolist() == [0, 0, 0] and loads.tolist() == [15]
    owner, loads = lpt_owner(np.array([], np.int64), 3)
    assert len(owner) == 0 and loads.tolist() == [0, 0, 0]
