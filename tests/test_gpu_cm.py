"""GPU CM refinement (wcc_run_cm: Section 2.4, Algorithms 4-5, with the CPM
community step after every cut split) against the oracle's CM, element by
element: the planted case where CM splits what WCC keeps, random planted
partitions over a range of resolutions, LFR-style and degree-corrected
graphs whose parts are large enough for the community step's global-memory
path, host and device buffers, and the argument checks."""
import numpy as np
import pytest

import oracle
import synth
from tests._helpers import taken_id_cm_input

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wcc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2509_02590_gb300 as w
    return w


def _both(wcc, n, src, dst, labels, min_size, gnum, gden, rule="log10"):
    kind = {"log10": oracle.RULE_LOG10, "log2": oracle.RULE_LOG2, "sqrt": oracle.RULE_SQRT}[rule]
    off, adj = oracle.build_csr(n, src, dst)
    ref, rst = oracle.cm(n, off, adj, labels, min_size, gnum, gden, kind)
    with wcc.WccGraph.from_edges(src, dst, n) as g:
        got, st = g.run_cm(labels, (gnum, gden), min_size=min_size, rule=rule, stats=True)
    return ref, rst, got, st


def _blocks():
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
    for t in range(12):
        eu.append(t)
        ev.append(20 + t)
    eu.append(5)
    ev.append(45)
    labels = np.zeros(64, np.int32)
    labels[52:] = 1
    return 64, np.array(eu, np.int32), np.array(ev, np.int32), labels


def test_cm_blocks_case(wcc):
    n, src, dst, labels = _blocks()
    ref, rst, got, st = _both(wcc, n, src, dst, labels, 2, 1, 4)
    assert np.array_equal(got, ref)
    assert ref.max() == 3  # A, B, C and D
    assert st["splits"] == rst["splits"] and st["out_clusters"] == rst["out_clusters"]


@pytest.mark.parametrize("seed", range(8))
def test_cm_random_planted(wcc, seed):
    rng = np.random.default_rng(100 + seed)
    k = int(rng.integers(4, 12))
    sizes = rng.integers(8, 60, size=k)
    n = int(sizes.sum())
    blk = np.repeat(np.arange(k), sizes)
    p_in, p_out = float(rng.uniform(0.2, 0.6)), float(rng.uniform(0.002, 0.02))
    iu, ju = np.triu_indices(n, 1)
    pr = np.where(blk[iu] == blk[ju], p_in, p_out)
    keep = rng.random(len(iu)) < pr
    src, dst = iu[keep].astype(np.int32), ju[keep].astype(np.int32)
    labels = (blk // int(rng.integers(2, 4))).astype(np.int32)  # merged blocks as input clusters
    gnum, gden = int(rng.integers(0, 5)), int(rng.choice([1, 10, 100]))
    ref, _, got, _ = _both(wcc, n, src, dst, labels, int(rng.choice([2, 3, 5])), gnum, gden)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("gamma", [(1, 1000), (1, 100), (1, 10)])
def test_cm_lfr(wcc, gamma):
    w = synth.lfr_like(20_000, seed=3, min_size=2)
    ref, rst, got, st = _both(wcc, w.n, w.src, w.dst, w.labels, w.min_size, *gamma)
    assert np.array_equal(got, ref)
    assert st["items"] == rst["items"] and st["splits"] == rst["splits"]


def test_cm_large_parts(wcc):
    """Input clusters up to 3,000 vertices: parts whose induced subgraph and
    community state do not fit in shared memory take the global path."""
    w = synth.dc_planted(60_000, 600_000, seed=11, size_max=3000)
    ref, rst, got, st = _both(wcc, w.n, w.src, w.dst, w.labels, w.min_size, 1, 100)
    assert np.array_equal(got, ref)
    assert rst["splits"] > 0


def test_cm_device_buffers_and_resolution_checks(wcc):
    w = synth.lfr_like(5_000, seed=8, min_size=2)
    off, adj = oracle.build_csr(w.n, w.src, w.dst)
    ref, _ = oracle.cm(w.n, off, adj, w.labels, 2, 1, 100)
    with wcc.WccGraph.from_edges(w.src, w.dst, w.n) as g:
        lab_d = torch.from_numpy(w.labels).cuda()
        out_d = g.run_cm(lab_d, (1, 100))
        torch.cuda.synchronize()
        assert np.array_equal(out_d.cpu().numpy(), ref)
        assert np.array_equal(g.run_cm(w.labels, (1, 100)), ref)
        # the plain WCC run on the same graph is untouched by CM's state
        assert np.array_equal(g.run(w.labels), oracle.wcc(w.n, off, adj, w.labels, 2)[0])
        for bad in [(-1, 1), (1, 0)]:
            with pytest.raises(wcc.WccError) as ei:
                g.run_cm(w.labels, bad)
            assert ei.value.status == -1


def test_cm_empty_community_when_n_plus_v_is_taken(wcc):
    """A part on which a vertex's best move is to be alone while the id n + v
    is held by vertices that joined it there: the kernel offers the smallest
    empty id instead, as the oracle does (the result differs from offering
    n + v itself)."""
    n, src, dst, labels, min_size, gnum, gden = taken_id_cm_input()
    ref, rst, got, st = _both(wcc, n, src, dst, labels, min_size, gnum, gden)
    assert rst["splits"] >= 1
    assert np.array_equal(got, ref)
