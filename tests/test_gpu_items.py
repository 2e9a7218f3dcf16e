"""Parity of the CUDA path with the oracle on item shapes that take specific
routes through the refinement kernel:

  * input clusters made of several components, and clusters that a peel
    disconnects: the largest component is refined in place by the CTA that
    found it while the others are queued;
  * long chains of dense blocks: after the first contraction pass dozens of
    super-vertices are left, which the dense finish takes up to 128 of
    (several widths forced through WCC_DENSE_NSV; 0 forces the sparse passes).

The refined clustering must be bit-identical to the oracle's.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wcc():
    import paper_2509_02590_gb300 as w
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return w


def _dense_block(rng, base, size, p):
    iu, ju = np.triu_indices(size, 1)
    keep = rng.random(len(iu)) < p
    return list(base + iu[keep]), list(base + ju[keep])


def _finish(rng, n, eu, ev, lab, min_size, name):
    perm = rng.permutation(n)  # clusters are not id ranges
    eu, ev = perm[np.array(eu, np.int64)], perm[np.array(ev, np.int64)]
    labels = np.empty(n, np.int32)
    labels[perm] = np.asarray(lab, np.int32)
    s, d = synth.graphs._dedup(n, eu.astype(np.int32), ev.astype(np.int32))
    return synth.Workload(name, n, s, d, labels, min_size)


def split_workload(seed):
    """Input clusters that CCR splits (2-5 dense components, some below
    min_size), clusters that a peel splits (two dense blocks of 50-90
    vertices joined through a path of degree-2 vertices, which go once
    T(n) = 2), and such clusters whose large part then fails its cut."""
    rng = np.random.default_rng(seed)
    eu, ev, lab = [], [], []
    n = 0
    c = 0
    for _ in range(30):
        kind = int(rng.integers(0, 3))
        if kind == 0:
            for _ in range(int(rng.integers(2, 6))):
                size = int(rng.integers(3, 60))
                a, b = _dense_block(rng, n, size, float(rng.uniform(0.3, 0.9)))
                eu += a; ev += b
                lab += [c] * size
                n += size
        else:
            sizes = [int(rng.integers(50, 90)) for _ in range(2 if kind == 1 else 3)]
            starts = []
            for size in sizes:
                a, b = _dense_block(rng, n, size, float(rng.uniform(0.2, 0.5)))
                eu += a; ev += b
                starts.append(n)
                lab += [c] * size
                n += size
            # blocks 0 and 1: a path of 3 degree-2 vertices (peeled at T = 2)
            path = list(range(n, n + 3))
            lab += [c] * 3
            n += 3
            chain = [starts[0] + int(rng.integers(0, sizes[0]))] + path + \
                    [starts[1] + int(rng.integers(0, sizes[1]))]
            eu += chain[:-1]; ev += chain[1:]
            if kind == 2:  # block 2 hangs off block 1 by one edge: the cut splits it
                eu.append(starts[1] + int(rng.integers(0, sizes[1])))
                ev.append(starts[2] + int(rng.integers(0, sizes[2])))
        c += 1
    # a few edges between clusters
    for _ in range(n // 20):
        eu.append(int(rng.integers(0, n))); ev.append(int(rng.integers(0, n)))
    return _finish(rng, n, eu, ev, lab, 5, f"split{seed}")


def long_chains(seed, blocks=(40, 70, 120)):
    """One input cluster per entry of blocks: a chain of that many dense
    blocks of 6-12 vertices, consecutive blocks joined by 1-2 edges.  The
    first contraction pass leaves about one super-vertex per block."""
    rng = np.random.default_rng(seed)
    eu, ev, lab = [], [], []
    n = 0
    for c, nb in enumerate(blocks):
        prev = None
        for _ in range(nb):
            size = int(rng.integers(6, 13))
            a, b = _dense_block(rng, n, size, 0.9)
            eu += a; ev += b
            lab += [c] * size
            if prev is not None:
                for _ in range(int(rng.integers(1, 3))):
                    eu.append(prev[0] + int(rng.integers(0, prev[1])))
                    ev.append(n + int(rng.integers(0, size)))
            prev = (n, size)
            n += size
    return _finish(rng, n, eu, ev, lab, 2, f"chains{seed}")


def _check(wcc, w, modes=("batched", "plain")):
    off, adj = oracle.build_csr(w.n, w.src, w.dst)
    ref, rst = oracle.wcc(w.n, off, adj, w.labels, w.min_size)
    with wcc.WccGraph.from_edges(torch.from_numpy(w.src).cuda(), torch.from_numpy(w.dst).cuda(),
                                 w.n) as g:
        for mode in modes:
            out, st = g.run(torch.from_numpy(w.labels).cuda(), min_size=w.min_size, mode=mode,
                            stats=True)
            assert np.array_equal(out.cpu().numpy(), ref), (w.name, mode)
            assert st["splits"] == rst["splits"] and st["peeled"] == rst["peeled"], (w.name, mode)
    return rst


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_split_children_continue_in_place(wcc, seed):
    w = split_workload(seed)
    rst = _check(wcc, w)
    assert rst["peeled"] > 0 and rst["splits"] > 0


@pytest.mark.parametrize("dense", [None, "64", "32", "0"])
def test_long_chains_through_each_finish(wcc, monkeypatch, dense):
    if dense is not None:
        monkeypatch.setenv("WCC_DENSE_NSV", dense)
    for seed in (0, 1):
        rst = _check(wcc, long_chains(seed))
        assert rst["splits"] >= 60


def big_items(seed, sizes=(66_000, 33_000)):
    """Input clusters above the 16-bit local-id limit (65,535 vertices): one
    random graph of sizes[0] vertices (mean degree 12; the peel takes its
    low-degree vertices), and one cluster of two random halves of sizes[1]
    vertices joined by a single edge, which splits on that bridge; plus
    small clusters."""
    rng = np.random.default_rng(seed)
    eu, ev, lab = [], [], []
    n = 0

    def gnp(size, mean):
        m = int(size * mean / 2)
        a = rng.integers(0, size, m)
        b = rng.integers(0, size, m)
        return list(n + a), list(n + b)

    big, half = sizes
    a, b = gnp(big, 12.0)
    eu += a; ev += b; lab += [0] * big; n += big
    h0 = n
    a, b = gnp(half, 14.0)
    eu += a; ev += b; n += half
    h1 = n
    a, b = gnp(half, 14.0)
    eu += a; ev += b; n += half
    lab += [1] * (2 * half)
    eu.append(h0 + int(rng.integers(0, half))); ev.append(h1 + int(rng.integers(0, half)))
    for c in range(2, 40):
        size = int(rng.integers(5, 200))
        a, b = _dense_block(rng, n, size, float(rng.uniform(0.1, 0.6)))
        eu += a; ev += b; lab += [c] * size; n += size
    return _finish(rng, n, eu, ev, lab, 2, f"big{seed}")


def test_items_with_32bit_local_ids(wcc):
    w = big_items(0)
    rst = _check(wcc, w, modes=("batched",))
    assert rst["splits"] >= 1 and rst["peeled"] > 0


def test_bounded_queue_wait_times_out_then_recovers(wcc, monkeypatch):
    """A CTA with nothing to claim while other items are still running waits
    at most WCC_WAIT_LIMIT_MS.  At 1 ms the idle CTAs of a run whose largest
    item takes longer than that give up: the run ends with WCC_ERR_TIMEOUT
    instead of waiting, every CTA leaves, and the next run on the same graph
    (with the default limit) returns the oracle's result."""
    w = big_items(1, sizes=(20_000, 8_000))
    off, adj = oracle.build_csr(w.n, w.src, w.dst)
    ref, _ = oracle.wcc(w.n, off, adj, w.labels, w.min_size)
    lab = torch.from_numpy(w.labels).cuda()
    with wcc.WccGraph.from_edges(torch.from_numpy(w.src).cuda(), torch.from_numpy(w.dst).cuda(),
                                 w.n) as g:
        monkeypatch.setenv("WCC_WAIT_LIMIT_MS", "1")
        with pytest.raises(wcc.WccError) as e:
            g.run(lab, min_size=w.min_size)
        assert e.value.status == -4  # WCC_ERR_TIMEOUT
        monkeypatch.delenv("WCC_WAIT_LIMIT_MS")
        out = g.run(lab, min_size=w.min_size)
        assert np.array_equal(out.cpu().numpy(), ref)
        out = g.run(lab, min_size=w.min_size, mode="plain")
        assert np.array_equal(out.cpu().numpy(), ref)
