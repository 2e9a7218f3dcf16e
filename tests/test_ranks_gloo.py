"""The multi-rank path of bench.py (weak scaling: one independent instance
per rank, max-over-ranks time, summed work) on two CPU processes over gloo,
plus the reference arm's rank rule (rank 0 alone reports)."""
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
