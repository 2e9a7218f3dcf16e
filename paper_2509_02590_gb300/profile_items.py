"""Per-item profile of one BATCHED refinement, binned by item size.

    python -m paper_2509_02590_gb300.profile_items WORKLOAD [key=value,...]

WORKLOAD is one of lfr_100k, dcpp_10m, dcpp_10m_b, dcpp_100m (seed 0); the
optional key=value pairs set the schedule tuning (wcc_set_tuning fields).
The library records every item of one run when WCC_PROFILE_ITEMS names a
file (phase cycles of the CTA path, start and end times; items refined on a
single warp are recorded whole), plus the time split of every CTA between
claiming, warp batches and CTA items.  Profiling slows the run; the times
printed first are of unprofiled runs.
"""
from __future__ import annotations

import csv
import os
import sys
import tempfile
import time

BINS = [(0, 32), (33, 64), (65, 128), (129, 256), (257, 512), (513, 1024), (1025, 2048),
        (2049, 8192), (8193, 65534), (65535, 1 << 31)]
PHASES = ["load", "extract", "ccr", "peel", "cc", "contract", "sw", "out"]


def _workload(name):
    import torch
    if name == "lfr_100k":
        import synth
        w = synth.lfr_like(100_000, seed=0, min_size=2)
        return (w.n, torch.from_numpy(w.src).cuda(), torch.from_numpy(w.dst).cuda(),
                torch.from_numpy(w.labels).cuda(), w.min_size)
    from synth import gpu_graphs
    w = getattr(gpu_graphs, name)(seed=0)
    return w.n, w.src.cuda(), w.dst.cuda(), w.labels.cuda(), w.min_size


def main(argv):
    import torch

    import paper_2509_02590_gb300 as wcc
    name = argv[0]
    if len(argv) > 1:
        kv = dict(x.split("=") for x in argv[1].split(","))
        wcc.set_tuning(**{k: int(v) for k, v in kv.items()})
    torch.cuda.set_device(0)
    n, src, dst, lab, min_size = _workload(name)
    print(f"{name}: n={n} m={src.numel()} tuning {wcc.get_tuning()}")
    g = wcc.WccGraph.from_edges(src, dst, n)
    out = torch.empty_like(lab)
    for _ in range(2):
        g.run(lab, min_size=min_size, out=out)
    ms = []
    for _ in range(3):
        _, st = g.run(lab, min_size=min_size, out=out, stats=True)
        ms.append(round(st["ms_refine"], 2))
    print(f"refinement (unprofiled) ms {ms}; items {st['items']}, splits {st['splits']}")
    fd, path = tempfile.mkstemp(suffix=".csv")
    os.close(fd)
    os.remove(path)
    os.environ["WCC_PROFILE_ITEMS"] = path
    try:
        _, st2 = g.run(lab, min_size=min_size, out=out, stats=True)
    finally:
        del os.environ["WCC_PROFILE_ITEMS"]
    print(f"profiled run ms {st2['ms_refine']:.2f}")
    rows = list(csv.DictReader(open(path)))
    cta = [r for r in rows if int(r["outcome"]) != 100]
    warp = [r for r in rows if int(r["outcome"]) == 100]
    print(f"items recorded: {len(rows)} ({len(cta)} on the CTA, {len(warp)} on single warps; "
          "the record holds at most 2^20)")
    tot = sum(int(r["t_end"]) - int(r["t_begin"]) for r in cta) or 1
    print("CTA items by size | items | vertices | CTA-ms | share | ns/vertex | phase shares "
          + " ".join(PHASES))
    for lo, hi in BINS:
        rs = [r for r in cta if lo <= int(r["n"]) <= hi]
        if not rs:
            continue
        t = sum(int(r["t_end"]) - int(r["t_begin"]) for r in rs)
        nv = sum(int(r["n"]) for r in rs)
        cyc = [sum(int(r[p]) for r in rs) for p in PHASES]
        c = max(sum(cyc), 1)
        print(f"{lo}-{hi} | {len(rs)} | {nv} | {t / 1e6:.1f} | {t / tot:.3f} | {t / nv:.0f} | "
              + " ".join(f"{x / c:.2f}" for x in cyc))
    for r in sorted(cta, key=lambda r: int(r["t_begin"]) - int(r["t_end"]))[:5]:
        print(f"longest: n {r['n']} entries {r['E']} {(int(r['t_end']) - int(r['t_begin'])) / 1e6:.2f}"
              f" ms, outcome {r['outcome']}, global slab {r['slab']}, passes {r['passes']}, "
              f"super-vertices after the first pass {r['nsv1']}")
    if warp:
        d = sorted(int(r["t_end"]) - int(r["t_begin"]) for r in warp)
        print(f"single-warp items: median {d[len(d) // 2] / 1e3:.1f} us, "
              f"p90 {d[int(0.9 * (len(d) - 1))] / 1e3:.1f} us")
    cpath = path + ".cta"
    if os.path.exists(cpath):
        cr = list(csv.DictReader(open(cpath)))
        cl = sum(int(r["claim"]) for r in cr)
        ti = sum(int(r["tiny"]) for r in cr)
        ct = sum(int(r["cta_time"]) for r in cr)
        s = max(cl + ti + ct, 1)
        b = sum(int(r["batches"]) for r in cr)
        tis = sum(int(r["tiny_items"]) for r in cr)
        print(f"CTA cycles: claiming {cl / s:.3f}, warp batches {ti / s:.3f}, CTA items "
              f"{ct / s:.3f}; {b} batches holding {tis} single-warp items "
              f"({tis / max(b, 1):.2f} each)")
        os.remove(cpath)
    os.remove(path)


if __name__ == "__main__":
    main(sys.argv[1:])
