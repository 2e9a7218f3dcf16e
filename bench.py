#!/usr/bin/env python
"""Benchmark of the WCC refinement hot path on one GB300 per rank.

One step = the whole path over one synthetic input: device CSR build from the
edge list (wcc_create_graph_from_edges) + the refinement (wcc_run: grouping by
input label, refinement kernel, output numbering).  Inputs (edge list and input
clustering) are resident in HBM when the timed region starts; L2 is flushed
(a 512 MiB device write) before every timed step, outside the step's events.
The line also reports the refinement alone on a resident graph
("graph_resident") and the CSR build time.

Workloads (--workload; the default is the one the driver times):
  lfr_100k   LFR-style graph, 100,000 vertices (power-law degrees, exponent
             2.5, mean 20, max 1,000; power-law community sizes 20-2,000,
             exponent 1.5; mixing 0.3; 10% of communities merged pairwise
             through 1-2 bridges), seed = rank, criterion floor(log10 n), min
             size 2 (s_pre = s_post = 1 as in the paper's experiments);
  planted_1k 1,010-vertex planted partition (20 blocks of 50, 4 bridged, 10
             pendant vertices), min size 11; the plain path is its headline;
  dcpp_10m   degree-corrected planted partition, 10M vertices, ~200M edges,
             power-law cluster sizes 10-50,000 (exponent 1.8), 5% chain clusters;
  dcpp_10m_b the same with 500k clusters (size exponent fitted to a mean of 20);
  dcpp_1m    the laws of dcpp_10m at 1M vertices, ~20M edges (a profiling case);
  dcpp_100m  100M vertices, ~2B edges, 5M clusters on [10, 100,000], 3%
             bridged two-part clusters (about 100 GB of device memory).
The two large ones are generated on the GPU and run with the schedule tuning
that wcc_autotune picks for them during setup; their plain path (one launch
per work item, millions of items) is not run, and their CPU baseline is the
oracle on a seeded sample of input clusters (each refines independently).

Multi-GPU (torchrun): input clusters are independent (Algorithms 1-2 iterate
over them with no exchange), so each rank refines its own instance with no
data-path collective: weak scaling.

``--impl reference`` times the CPU oracle (the plain C refinement used as the
parity reference) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "WCC clusters/s and edges/s at 1 GB300 (batched/served vs plain), %HBM roofline; p50/p99"
WORKLOADS = ("lfr_100k", "planted_1k", "dcpp_1m", "dcpp_10m", "dcpp_10m_b", "dcpp_100m")
LARGE = ("dcpp_1m", "dcpp_10m", "dcpp_10m_b", "dcpp_100m")


def workload(name: str, rank: int):
    import synth
    if name == "lfr_100k":
        return synth.lfr_like(100_000, seed=rank, min_size=2)
    if name == "planted_1k":
        return synth.planted_1k(seed=rank)
    from synth import gpu_graphs
    if name == "dcpp_10m":
        return gpu_graphs.dcpp_10m(seed=rank)
    if name == "dcpp_10m_b":
        return gpu_graphs.dcpp_10m_b(seed=rank)
    if name == "dcpp_1m":
        return gpu_graphs.dcpp_1m(seed=rank)
    return gpu_graphs.dcpp_100m(seed=rank)


def n_clusters(w) -> int:
    return int(w.meta["clusters"]) if w.meta and "clusters" in w.meta else int(w.n_clusters)


def describe(name: str, w) -> dict:
    text = {
        "lfr_100k": f"LFR-style graph, {w.n} vertices, {w.m} undirected edges, {n_clusters(w)} input "
                    "clusters (10% merged pairwise by 1-2 bridges)",
        "planted_1k": f"planted partition, {w.n} vertices, {w.m} edges, 20 blocks of 50 (4 bridged "
                      "halves, 10 pendant vertices)",
        "dcpp_10m": f"degree-corrected planted partition, {w.n} vertices, {w.m} undirected edges, "
                    f"{n_clusters(w)} clusters (sizes 10-50,000, 5% chains of 2-4 parts)",
        "dcpp_1m": f"degree-corrected planted partition, {w.n} vertices, {w.m} undirected edges, "
                   f"{n_clusters(w)} clusters (the 10M graph's laws at a tenth of its size)",
        "dcpp_10m_b": f"degree-corrected planted partition, {w.n} vertices, {w.m} undirected "
                      f"edges, {n_clusters(w)} clusters (sizes 10-50,000 with the exponent fitted "
                      "to a mean of 20, 5% chains of 2-4 parts)",
        "dcpp_100m": f"degree-corrected planted partition, {w.n} vertices, {w.m} undirected edges, "
                     f"{n_clusters(w)} clusters (sizes 10-100,000, 3% bridged two-part clusters)",
    }[name]
    return {"workload": f"{name}: {text}, criterion floor(log10 n), min size {w.min_size}",
            "n": int(w.n), "m": int(w.m), "input_clusters": n_clusters(w), "min_size": int(w.min_size),
            "rule": "log10", "l2": "flushed before every timed step (512 MiB device write)"}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.lines = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={','.join(self.FIELDS)}",
                 "--format=csv,noheader,nounits", "-i", str(gpu_index), "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def wait_first(self, timeout=5.0):
        t0 = time.perf_counter()
        while self.proc and not self.lines and time.perf_counter() - t0 < timeout:
            time.sleep(0.02)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t_begin: float, t_end: float):
        if not self.proc:
            return None
        rows = [l for (t, l) in self.lines if t_begin <= t <= t_end]
        if not rows:
            rows = [l for (_, l) in self.lines[-3:]]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            parts = [p.strip() for p in r.split(",")]
            if len(parts) < len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() in ("active", "1", "yes"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ peaks
def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ------------------------------------------------------------------ oracle
def oracle_step(w):
    import oracle
    off, adj = oracle.build_csr(w.n, w.src, w.dst)
    out, st = oracle.wcc(w.n, off, adj, w.labels, w.min_size)
    return out


def cluster_sample(w, max_edges: int = 1_500_000, seed: int = 0):
    """A seeded sample of whole input clusters of a large device-generated
    workload, as a small host workload: the subgraph they induce, with vertex
    ids renumbered monotonically (refinement depends only on each cluster's
    induced subgraph, and a monotone renumbering keeps every tie-break)."""
    import numpy as np
    import torch
    import synth
    rng = np.random.default_rng(seed)
    lab_of = w.meta["label_of_cluster"]
    sizes = w.meta["cluster_sizes"]
    order = rng.permutation(len(sizes))
    # about max_edges / mean intra-degree vertices' worth of clusters
    deg = 2.0 * w.m / w.n
    budget_v = max_edges / max(deg * 0.4, 1.0)
    take = order[np.cumsum(sizes[order]) <= budget_v]
    sample = torch.from_numpy(np.unique(lab_of[take]).astype(np.int32)).to(w.labels.device)
    in_s = torch.isin(w.labels, sample)
    ids = torch.nonzero(in_s).flatten()
    keep = in_s[w.src.long()] & in_s[w.dst.long()] & (w.labels[w.src.long()] == w.labels[w.dst.long()])
    su = torch.searchsorted(ids, w.src[keep].long()).to(torch.int32).cpu().numpy()
    sv = torch.searchsorted(ids, w.dst[keep].long()).to(torch.int32).cpu().numpy()
    lab = w.labels[ids].cpu().numpy()
    s = synth.Workload("sample", int(ids.numel()), su, sv, lab, int(w.min_size))
    return s, int(sample.numel())


def cpu_baseline(name, w, budget_s: float = 12.0):
    """The oracle as it stands, single-threaded, repeated until ~budget_s of
    CPU time: edges/s.  Small workloads run in full; large ones on a seeded
    sample of whole input clusters."""
    import oracle
    oracle.build()
    if name in LARGE:
        sw, k = cluster_sample(w)
        what = f"{k} whole input clusters of {name} sampled ({sw.n} vertices, {sw.m} intra-cluster edges)"
    else:
        sw, k = w, n_clusters(w)
        what = f"the full {name} workload"
    times = []
    t_all = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        oracle_step(sw)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_all > budget_s or len(times) >= 50:
            break
    mean = sum(times) / len(times)
    out = {"value": sw.m / mean, "unit": "edges/s", "cores": 1, "kind": "oracle",
           "sample": f"{what} (CSR build + refinement), {len(times)} repetitions, "
                     f"mean {mean * 1e3:.1f} ms each",
           "clusters_per_s": k / mean}
    # the all-cores figure beside it, where a step is long enough to share out
    if mean >= 0.02 and host_cores() > 1:
        try:
            out["all_cores"] = cpu_baseline_pool(sw)
        except Exception as e:  # the single-core baseline stands on its own
            out["all_cores"] = {"error": f"{type(e).__name__}: {e}"[:200]}
    return out


# ---- the oracle over disjoint sets of input clusters, one process each -----
def host_cores() -> int:
    """Cores this process may run on (its affinity mask), at most 64."""
    try:
        n = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        n = os.cpu_count() or 1
    return max(1, min(n, 64))


def _pool_worker(conn):
    """Receives (off, adj, labels, min_size, mask) once, then times one oracle
    run over its input clusters per "run" message until "stop"."""
    import oracle
    off, adj, labels, min_size, mask = conn.recv()
    conn.send("ready")
    while conn.recv() == "run":
        t0 = time.perf_counter()
        oracle.wcc(len(labels), off, adj, labels, min_size, only_labels=mask)
        conn.send(time.perf_counter() - t0)


def cpu_baseline_pool(sw, budget_s: float = 8.0, timeout_s: float = 120.0):
    """The same oracle, unchanged, run on disjoint sets of input clusters in
    one spawned process per host core (Algorithm 2 refines every input
    cluster independently).  The sets are balanced greedily by cluster work
    (members plus intra-cluster edges), largest first.  A step is the CSR
    build (one process, timed on its own) plus the wall time until every
    process has finished its set.  Every wait has a deadline; on any failure
    the processes are killed and the error is raised."""
    import multiprocessing as mp
    import numpy as np
    import oracle
    cores = host_cores()
    lab = np.asarray(sw.labels)
    ok = lab >= 0
    nlab = int(lab[ok].max()) + 1 if ok.any() else 0
    src, dst = np.asarray(sw.src), np.asarray(sw.dst)
    intra = (lab[src] == lab[dst]) & (lab[src] >= 0)
    work = np.bincount(lab[src[intra]], minlength=nlab) + np.bincount(lab[ok], minlength=nlab)
    load = np.zeros(cores)
    masks = [np.zeros(nlab, np.uint8) for _ in range(cores)]
    for c in np.argsort(-work, kind="stable"):
        p = int(np.argmin(load))
        masks[p][c] = 1
        load[p] += work[c]
    masks = [m for m in masks if m.any()]
    t0 = time.perf_counter()
    off, adj = oracle.build_csr(sw.n, sw.src, sw.dst)
    t_csr = time.perf_counter() - t0
    ctx = mp.get_context("spawn")
    procs, conns = [], []

    def recv(c):
        if not c.poll(timeout_s):
            raise TimeoutError("oracle worker did not answer")
        return c.recv()

    def send_quietly(c, obj):
        try:
            c.send(obj)
        except (OSError, EOFError):
            pass  # the worker is gone; its "ready" never comes

    try:
        for m in masks:
            a, b = ctx.Pipe()
            pr = ctx.Process(target=_pool_worker, args=(b,), daemon=True)
            pr.start()
            b.close()  # the worker's end: a worker that dies closes the pipe
            procs.append(pr)
            conns.append(a)
            # the arrays go from a thread, so that a worker that never reads
            # cannot hold this one past the deadline below
            threading.Thread(target=send_quietly, args=(a, (off, adj, lab, int(sw.min_size), m)),
                             daemon=True).start()
        for c in conns:
            if recv(c) != "ready":
                raise RuntimeError("oracle worker failed to start")

        def step():
            for c in conns:
                c.send("run")
            return max(recv(c) for c in conns)

        step()  # warm-up
        times = []
        t_all = time.perf_counter()
        while True:
            t0 = time.perf_counter()
            step()
            times.append(time.perf_counter() - t0)
            if time.perf_counter() - t_all > budget_s or len(times) >= 50:
                break
        for c in conns:
            c.send("stop")
        stopped = True
    except BaseException:
        stopped = False
        raise
    finally:
        for pr in procs:
            if stopped:
                pr.join(5)
            if pr.is_alive():
                pr.kill()
                pr.join(5)
    mean = t_csr + sum(times) / len(times)
    return {"value": sw.m / mean, "unit": "edges/s", "cores": len(masks),
            "sample": f"the same sample; {len(masks)} processes over disjoint input clusters "
                      f"(largest set {int(load.max())} of {int(work.sum())} work units), CSR build "
                      f"{t_csr * 1e3:.1f} ms on one core, {len(times)} repetitions, "
                      f"mean {mean * 1e3:.1f} ms each"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    w = workload(args.workload, 0)
    if args.workload in LARGE:
        sw, k = cluster_sample(w)
        what = f"{k} whole input clusters of {args.workload} per step ({sw.m} intra-cluster edges)"
    else:
        sw, k = w, n_clusters(w)
        what = f"the full {args.workload} workload per step"
    for _ in range(args.warmup):
        oracle_step(sw)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_step(sw)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = sw.m * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "edges/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": describe(args.workload, w),
            "clusters_per_s": k * args.steps / total,
            "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle",
                             "sample": what},
            "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ traffic
def profiled_traffic():
    """DRAM bytes per k_refine launch from the committed ncu capture, or None
    when the kernel sources have changed since the counters were taken."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", "k_refine_lfr_100k.traffic.json")
    try:
        rec = json.load(open(prof))
        h = hashlib.sha256()
        for src in rec["kernel_sources"]:
            h.update(open(os.path.join(ROOT, src), "rb").read())
        if h.hexdigest() != rec["kernel_sources_sha256"]:
            return None
        return rec["traffic_bytes_per_launch"]
    except (OSError, ValueError, KeyError):
        return None


# ------------------------------------------------------------------ roofline
# Algorithmic bytes (what the method must move at least, not what the
# kernels happen to move):
#   CSR build: the edge list read (8 B per edge), the CSR written (8 B per
#     row offset, 4 B per directed entry);
#   refinement kernel: 8 B per member of an input cluster (its row offsets)
#     and 8 B per adjacency entry of every extracted item (the neighbour id
#     and its label), counted by the kernel itself;
#   a whole step: the CSR build, the labels read (4 B per vertex), the
#     refinement kernel's bytes and the labels written (4 B per vertex).
def csr_bytes(n, m):
    return 8.0 * m + 8.0 * (n + 1) + 4.0 * (2 * m)


def kernel_roofline(alg_bytes, ms, peak, peak_kind, step_ms):
    achieved = alg_bytes / (ms / 1e3) / 1e9
    return {"kernel": "k_refine", "bound": "hbm", "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "traffic": None, "peak_source": peak_kind,
            "alg_bytes_per_launch": alg_bytes, "ms_per_launch": ms, "share_of_step": ms / step_ms}


def step_roofline(n, m, refine_bytes, step_ms, peak):
    b = csr_bytes(n, m) + 4.0 * n + refine_bytes + 4.0 * n
    gbs = b / (step_ms / 1e3) / 1e9
    return {"alg_bytes": b, "achieved": gbs, "unit": "GB/s", "frac": gbs / peak}


def csr_roofline(n, m, ms, peak):
    try:
        b = csr_bytes(n, m)
        gbs = b / (ms / 1e3) / 1e9
        return {"bound": "hbm", "alg_bytes": b, "achieved": gbs, "peak": peak, "unit": "GB/s",
                "frac": gbs / peak}
    except (TypeError, ValueError, ZeroDivisionError):
        return None


# ------------------------------------------------------------------ a large configuration
def large_record(wcc, torch, dev, flush, stream, peak, peak_kind, name="dcpp_10m", steps=5,
                 warmup=3, resident_runs=5):
    """A bounded measurement of a large configuration beside the headline
    workload: the same step (CSR build + refinement, inputs resident, L2
    flushed before each), the refinement on a resident graph, the CSR build
    alone and the rooflines, with the default schedule tuning."""
    w = workload(name, 0)
    src, dst, lab = w.src.to(dev), w.dst.to(dev), w.labels.to(dev)
    out = torch.empty_like(lab)

    def step():
        g = wcc.WccGraph.from_edges(src, dst, w.n)
        try:
            _, st = g.run(lab, min_size=w.min_size, out=out, stats=True)
        finally:
            g.close()
        return st

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    step_ms, r_ms, r_bytes = [], [], []
    for k in range(steps):
        flush.fill_(k & 0xff)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st = step()
        b.record(stream)
        torch.cuda.synchronize()
        step_ms.append(a.elapsed_time(b))
        r_ms.append(st["ms_refine"])
        r_bytes.append(st["alg_bytes"])
    res_ms, csr_ms = [], None
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.fill_(1)
    a.record(stream)
    g = wcc.WccGraph.from_edges(src, dst, w.n)
    b.record(stream)
    torch.cuda.synchronize()
    csr_ms = a.elapsed_time(b)
    with g:
        g.run(lab, min_size=w.min_size, out=out)
        for k in range(resident_runs):
            flush.fill_(k & 0xff)
            a.record(stream)
            g.run(lab, min_size=w.min_size, out=out)
            b.record(stream)
            torch.cuda.synchronize()
            res_ms.append(a.elapsed_time(b))
    sm = sorted(step_ms)
    mean = sum(step_ms) / len(step_ms)
    rm = sum(res_ms) / len(res_ms)
    rk = sum(r_ms) / len(r_ms)
    rb = sum(r_bytes) / len(r_bytes)
    k_in = n_clusters(w)
    rec = {"workload": describe(name, w)["workload"], "n": int(w.n), "m": int(w.m),
           "input_clusters": k_in, "steps": steps, "warmup": warmup, "ms_per_step": mean,
           "p50_ms": sm[len(sm) // 2], "p99_ms": sm[-1],
           "edges_per_s": w.m / (mean / 1e3), "clusters_per_s": k_in / (mean / 1e3),
           "graph_resident": {"ms_per_run": rm, "edges_per_s": w.m / (rm / 1e3),
                              "clusters_per_s": k_in / (rm / 1e3), "runs": len(res_ms)},
           "csr_build_ms": csr_ms,
           "roofline": kernel_roofline(rb, rk, peak, peak_kind, mean),
           "step_roofline": step_roofline(w.n, w.m, rb, mean, peak),
           "csr_roofline": csr_roofline(w.n, w.m, csr_ms, peak),
           "tuning": wcc.get_tuning()}
    del src, dst, lab, out, w
    torch.cuda.empty_cache()
    return rec


# ------------------------------------------------------------------ CM
def cm_record(wcc, torch, w, src_d, dst_d, lab_d, flush, runs=5):
    """CM (WCC whose split parts go through the CPM community step) on the
    workload's resident graph at the two resolutions the paper's inputs use
    (CPM 0.001 and 0.01): mean time per run, edges/s, and the counters."""
    out = torch.empty_like(lab_d)
    rec = {"runs": runs}
    with wcc.WccGraph.from_edges(src_d, dst_d, w.n) as g:
        for gnum, gden in ((1, 1000), (1, 100)):
            for _ in range(2):
                g.run_cm(lab_d, (gnum, gden), min_size=w.min_size, out=out)
            ts, st = [], None
            for k in range(runs):
                flush.fill_(k & 0xff)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                _, st = g.run_cm(lab_d, (gnum, gden), min_size=w.min_size, out=out, stats=True)
                b.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            ms = sum(ts) / len(ts)
            rec[f"cpm_{gnum}/{gden}"] = {
                "ms_per_run": ms, "edges_per_s": w.m / (ms / 1e3),
                "items": st["items"], "splits": st["splits"], "out_clusters": st["out_clusters"]}
    return rec


def latency_by_size(edges, lat_ms, cuts=(10 ** 5, 10 ** 6)):
    """p50/p99 latency (ms) of the requests in each edge-count band: below
    cuts[0], [cuts[0], cuts[1]), and from cuts[1] up.  edges and lat_ms are
    per request, in the same order; empty bands are left out."""
    def short(x):
        return f"{x // 10 ** 6}M" if x % 10 ** 6 == 0 else f"{x // 1000}k" if x % 1000 == 0 else str(x)

    bands = ((0, cuts[0], f"<{short(cuts[0])}"),
             (cuts[0], cuts[1], f"{short(cuts[0])}-{short(cuts[1])}"),
             (cuts[1], None, f">={short(cuts[1])}"))
    out = {}
    for lo, hi, name in bands:
        sel = sorted(l for e, l in zip(edges, lat_ms) if e >= lo and (hi is None or e < hi))
        if sel:
            q = lambda f: sel[min(len(sel) - 1, int(round(f * (len(sel) - 1))))]
            out[name + " edges"] = {"requests": len(sel), "p50_ms": q(0.5), "p99_ms": q(0.99)}
    return out


# ------------------------------------------------------------------ ranks
def aggregate_ranks(dist, torch, dev, total_ms: float, m: int, clusters: int):
    """Weak scaling across ranks: every rank refines its own instance with no
    data-path collective; the job time is the slowest rank's and the work is
    the sum over ranks.  Returns (max total_ms, sum of edges, sum of input
    clusters).  dist may be None (one rank)."""
    if dist is None:
        return total_ms, float(m), float(clusters)
    t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    mw = torch.tensor([float(m), float(clusters)], dtype=torch.float64, device=dev)
    dist.all_reduce(mw)
    return float(t.item()), float(mw[0].item()), float(mw[1].item())


# ------------------------------------------------------------------ serving
def serving_bench(wcc, np, torch, n_requests: int = 10_000, pool_size: int = 200, seed: int = 0,
                  budget: int = 80 << 30, tight_budget: int = 2 << 30, tight_requests: int = 1000):
    """The request stream: requests whose graphs are degree-corrected planted
    partitions with log-uniform edge counts in [1e3, 1e7] (n = m/10, cluster
    sizes power law 1.5 on [20, 2000], degree exponent 2.5), drawn from a
    pool of distinct seeded graphs held in pinned host memory.  Every
    request brings its graph as a host edge list (wcc_submit_edges): the
    server uploads it, builds the CSR, refines, returns the result and frees
    the graph, all under its memory budget.  Capacity is the throughput of a
    burst of all requests; then the same requests arrive as a Poisson
    process at 0.5 and at 0.8 of that capacity (0.8 is the headline) and
    the latency of each (submit to result, wcc_stats.ms_total) is recorded.
    A last burst under a tight budget shows the admission control binding."""
    import time as _t

    from synth import gpu_graphs
    rng = np.random.default_rng(seed)
    pool = []
    t_gen = _t.perf_counter()
    for i in range(pool_size):
        m = int(10 ** rng.uniform(3, 7))
        n = max(m // 10, 200)
        w = gpu_graphs.dc_planted_gpu(n, m, seed=1000 + i, deg_exp=2.5, size_exp=1.5,
                                      size_min=20, size_max=2000, f_in=0.8, chain_frac=0.05,
                                      chain_parts=(2, 2))
        pool.append((w.src.cpu().pin_memory(), w.dst.cpu().pin_memory(), int(w.n),
                     w.labels.cpu().numpy(), int(w.m)))
        del w
    gen_s = _t.perf_counter() - t_gen
    picks = rng.integers(0, pool_size, n_requests)
    edges = sum(pool[k][4] for k in picks)

    def stream(rate, bud, count):
        """Submit the first count picks (all at once when rate is None, else
        Poisson arrivals at rate); returns (seconds, sorted latencies in ms,
        server counters)."""
        gaps = rng.exponential(1.0 / rate, count) if rate else np.zeros(count)
        with wcc.WccServer(bud) as srv:
            tickets, req_edges = [], []
            t0 = _t.perf_counter()
            nxt = t0
            for k, gap in zip(picks[:count], gaps):
                nxt += gap
                while _t.perf_counter() < nxt:
                    pass
                s, d, n, lab, m = pool[k]
                tickets.append(srv.submit_edges(s, d, n, lab))
                req_edges.append(m)
            lat = []
            for t in tickets:
                _, st = srv.wait(t)
                lat.append(st["ms_total"])
            took = _t.perf_counter() - t0
            info = dict(srv.info())
        info["by_size"] = latency_by_size(req_edges, lat)
        return took, sorted(lat), info

    def p(lat, q):
        return lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]

    burst_s, _, burst_info = stream(None, budget, n_requests)
    cap_rps = n_requests / burst_s
    loads = {}
    for load in (0.5, 0.8):
        run_s, lat, info = stream(load * cap_rps, budget, n_requests)
        loads[str(load)] = {"offered_requests_per_s": load * cap_rps,
                            "requests_per_s": n_requests / run_s, "edges_per_s": edges / run_s,
                            "p50_ms": p(lat, 0.5), "p99_ms": p(lat, 0.99),
                            "by_size": info["by_size"],
                            "peak_active": info["peak_active"],
                            "peak_used_bytes": info["peak_used_bytes"]}
    tight_edges = sum(pool[k][4] for k in picks[:tight_requests])
    t_s, t_lat, t_info = stream(None, tight_budget, tight_requests)
    tight = {"budget_bytes": tight_budget, "requests": tight_requests,
             "requests_per_s": tight_requests / t_s, "edges_per_s": tight_edges / t_s,
             "p50_ms": p(t_lat, 0.5), "p99_ms": p(t_lat, 0.99),
             "budget_waits": t_info["budget_waits"], "peak_active": t_info["peak_active"],
             "peak_used_bytes": t_info["peak_used_bytes"],
             "budget_left_for_requests": t_info["budget_bytes"]}
    head = loads["0.8"]
    return {"requests": n_requests, "edges": int(edges), "load": 0.8,
            "capacity_requests_per_s": cap_rps, "capacity_edges_per_s": edges / burst_s,
            "requests_per_s": head["requests_per_s"], "edges_per_s": head["edges_per_s"],
            "p50_ms": head["p50_ms"], "p99_ms": head["p99_ms"], "loads": loads,
            "burst": {"peak_active": burst_info["peak_active"],
                      "peak_used_bytes": burst_info["peak_used_bytes"],
                      "budget_waits": burst_info["budget_waits"],
                      "slot_waits": burst_info["slot_waits"]},
            "tight_budget": tight,
            "mean_edges_per_request": edges / n_requests, "pool_generation_s": gen_s,
            "sample": f"{n_requests} requests drawn from {pool_size} distinct seeded graphs "
                      "(log-uniform 1e3..1e7 edges) in pinned host memory; every request "
                      "uploads its edge list, has its CSR built, refined and freed by the "
                      f"server under a {budget >> 30} GB budget; capacity = a burst of all "
                      "requests, then Poisson arrivals at 0.5 and 0.8 of it; latency = "
                      "submit to result; a burst of the first "
                      f"{tight_requests} under a {tight_budget >> 30} GB budget"}


# ------------------------------------------------------------------ GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lfr_100k", choices=WORKLOADS)
    ap.add_argument("--plain-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--resident-steps", type=int, default=50)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=10_000)
    ap.add_argument("--serving-pool", type=int, default=200)
    ap.add_argument("--no-autotune", action="store_true",
                    help="run the large configurations with the default tuning")
    ap.add_argument("--no-cm", action="store_true",
                    help="skip the CM record (the CPM community step after every split)")
    ap.add_argument("--no-large-record", action="store_true",
                    help="skip the bounded 10M-vertex record beside the default workload")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    import paper_2509_02590_gb300 as wcc

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    name = args.workload
    large = name in LARGE
    w = workload(name, rank)
    dev = torch.device("cuda", local)
    as_dev = (lambda x: x.to(dev)) if torch.is_tensor(w.src) else (lambda x: torch.from_numpy(x).to(dev))
    src_d, dst_d, lab_d = as_dev(w.src), as_dev(w.dst), as_dev(w.labels)
    out_d = torch.empty_like(lab_d)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    k_in = n_clusters(w)

    # the large configurations run with the schedule's autotuned setting
    # (setup, outside the timed region); the others with the defaults
    tuning = wcc.get_tuning()
    if large and not args.no_autotune:
        with wcc.WccGraph.from_edges(src_d, dst_d, w.n) as g_t:
            tuning, _ = wcc.autotune(g_t, lab_d, min_size=w.min_size)

    def step(mode="batched"):
        g = wcc.WccGraph.from_edges(src_d, dst_d, w.n)
        try:
            _, st = g.run(lab_d, min_size=w.min_size, mode=mode, out=out_d, stats=True)
        finally:
            g.close()
        return st

    for _ in range(args.warmup):
        step()
    barrier()

    sampler = ClockSampler(local)
    sampler.wait_first()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    refine_ms, refine_bytes = [], []
    barrier()
    l0 = wcc.wcc_kernel_launches()
    t_begin = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        ev[k][0].record(stream)
        st = step()
        ev[k][1].record(stream)
        refine_ms.append(st["ms_refine"])
        refine_bytes.append(st["alg_bytes"])
    barrier()
    t_end = time.perf_counter()
    launches = wcc.wcc_kernel_launches() - l0
    sampler.stop()
    clocks = sampler.summary(t_begin, t_end)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms, m_all, k_all = aggregate_ranks(dist, torch, dev, sum(step_ms), w.m, k_in)
    value = m_all * args.steps / (total_ms / 1e3)
    clusters_per_s = k_all * args.steps / (total_ms / 1e3)

    def pct(v, q):
        v = sorted(v)
        return v[min(len(v) - 1, int(round(q * (len(v) - 1))))]

    # the refinement alone on a resident graph, and the CSR build alone
    csr_ms, res_ms = [], []
    g_res = None
    for k in range(max(args.resident_steps, 0) + 2 if args.resident_steps > 0 else 0):
        flush.fill_(k & 0xff)
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(stream)
        if g_res is None:
            g_res = wcc.WccGraph.from_edges(src_d, dst_d, w.n)
            b.record(stream)
        else:
            b.record(stream)
        g_res.run(lab_d, min_size=w.min_size, out=out_d)
        c.record(stream)
        torch.cuda.synchronize()
        if k == 0:
            csr_ms.append(a.elapsed_time(b))
        elif k >= 2:
            res_ms.append(b.elapsed_time(c))
    resident = None
    if res_ms:
        rm = sum(res_ms) / len(res_ms)
        resident = {"edges_per_s": w.m / (rm / 1e3), "clusters_per_s": k_in / (rm / 1e3),
                    "ms_per_run": rm, "p50_ms": pct(res_ms, 0.5), "p99_ms": pct(res_ms, 0.99),
                    "runs": len(res_ms), "csr_build_ms": csr_ms[0] if csr_ms else None}
        g_res.close()

    # plain path (one kernel launch per work item), same workload
    plain = None
    if args.plain_steps > 0 and not large:
        pms = []
        for k in range(args.plain_steps):
            flush.fill_(k & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step("plain")
            b.record(stream)
            torch.cuda.synchronize()
            pms.append(a.elapsed_time(b))
        pm = sum(pms) / len(pms)
        plain = {"edges_per_s": w.m / (pm / 1e3), "clusters_per_s": k_in / (pm / 1e3),
                 "ms_per_step": pm, "steps": len(pms)}
    ref_out = out_d.clone()

    # end to end through the public API with pinned host buffers
    src_h = src_d.cpu().pin_memory()
    dst_h = dst_d.cpu().pin_memory()
    lab_h = lab_d.cpu().pin_memory()
    out_h = torch.empty_like(lab_h).pin_memory()
    e2e_steps = min(args.e2e_steps, 2) if large else args.e2e_steps
    e2e_t = []
    for k in range(e2e_steps + 2 if e2e_steps > 0 else 1):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with wcc.WccGraph.from_edges(src_h, dst_h, w.n) as g:
            g.run(lab_h, min_size=w.min_size, out=out_h)
        e2e_t.append(time.perf_counter() - t0)
    e2e_t = e2e_t[2:] or e2e_t
    e2e_mean = sum(e2e_t) / len(e2e_t)
    e2e_local = torch.tensor([e2e_mean], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(e2e_local, op=dist.ReduceOp.MAX)
    e2e_value = m_all / float(e2e_local.item())
    # the result must match the device-buffer run
    ok = bool(torch.equal(out_h, ref_out.cpu()))

    # roofline of the dominant kernel (the refinement kernel) and of the step
    peak, peak_kind = hbm_peak()
    r_ms = sum(refine_ms) / len(refine_ms)
    r_bytes = sum(refine_bytes) / len(refine_bytes)
    roofline = kernel_roofline(r_bytes, r_ms, peak, peak_kind, total_ms / args.steps)
    if name == "lfr_100k":
        roofline["traffic"] = profiled_traffic()
    roofline["step"] = step_roofline(w.n, w.m, r_bytes, total_ms / args.steps, peak)
    if resident and resident.get("csr_build_ms"):
        resident["csr_roofline"] = csr_roofline(w.n, w.m, resident["csr_build_ms"], peak)

    # a bounded record of the 10M-vertex configuration beside the headline
    large_rec = None
    if name == "lfr_100k" and not args.no_large_record:
        try:
            large_rec = large_record(wcc, torch, dev, flush, stream, peak, peak_kind)
        except Exception as e:  # the headline stands on its own
            large_rec = {"error": f"{type(e).__name__}: {e}"[:300]}

    cm = None
    if name in ("lfr_100k", "planted_1k") and not args.no_cm:
        try:
            cm = cm_record(wcc, torch, w, src_d, dst_d, lab_d, flush)
        except Exception as e:  # the headline stands on its own
            cm = {"error": f"{type(e).__name__}: {e}"[:300]}

    serving = None
    if args.serving_requests > 0 and name == "lfr_100k":
        serving = serving_bench(wcc, np, torch, n_requests=args.serving_requests,
                                pool_size=args.serving_pool, seed=rank)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": describe(name, w),
                "schedule": {"mode": "batched", "parallelism": f"independent x{world}",
                             "tuning": tuning | {"autotuned": large and not args.no_autotune}},
                "clusters_per_s": clusters_per_s, "p50_ms": pct(step_ms, 0.5),
                "p99_ms": pct(step_ms, 0.99),
                "graph_resident": resident,
                "plain": plain,
                "batched_over_plain": (value / (plain["edges_per_s"] * world)) if plain else None,
                "e2e": {"value": e2e_value, "unit": "edges/s",
                        "h2d_bytes_per_step": int(8 * w.m + 4 * w.n),
                        "d2h_bytes_per_step": int(4 * w.n), "ms_per_step": 1e3 * e2e_mean,
                        "steps": len(e2e_t), "matches_device_run": ok},
                "gpu_launches": int(launches), "roofline": roofline, "clocks": clocks,
                "dcpp_10m": large_rec, "cm": cm, "serving": serving}
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(name, w)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
