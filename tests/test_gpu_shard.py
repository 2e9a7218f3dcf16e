"""One graph's input clusters split into shards (as on several GPUs, here
one after the other on one GPU), merged through cluster minima: the merged
result must equal one wcc_run over everything, bit for bit.  Also the two
merge entry points on their own (host and device buffers, rejection of
malformed minima)."""
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


def _minima(b, out):
    mn = torch.empty_like(out)
    b.wcc_cluster_minima(out.data_ptr(), out.numel(), mn.data_ptr(), 1,
                         torch.cuda.current_stream().cuda_stream)
    return mn


def _number(b, mn):
    out = torch.empty_like(mn)
    k = b.wcc_number_by_minima(mn.data_ptr(), mn.numel(), out.data_ptr(), 1,
                               torch.cuda.current_stream().cuda_stream)
    return out, k


@pytest.mark.parametrize("world", [2, 3, 5])
def test_shards_merged_equal_one_run(wcc, world):
    from paper_2509_02590_gb300 import _binding as b
    from paper_2509_02590_gb300.shard import ShardPlan, gpu_refine_sharded
    w = synth.lfr_like(20_000, seed=4, min_size=2)
    off, _ = oracle.build_csr(w.n, w.src, w.dst)
    lab = torch.from_numpy(w.labels).cuda()
    with wcc.WccGraph.from_edges(torch.from_numpy(w.src).cuda(), torch.from_numpy(w.dst).cuda(),
                                 w.n) as g:
        full = g.run(lab, min_size=w.min_size)
        plan = ShardPlan(w.labels, np.diff(off), world)
        parts = []
        for r in range(world):
            lab_r = plan.shard_labels(lab, r)
            assert torch.equal(lab_r.cpu(), torch.from_numpy(plan.shard_labels(w.labels, r)))
            parts.append(_minima(b, g.run(lab_r, min_size=w.min_size)))
        merged = torch.stack(parts).max(dim=0).values  # what the all-reduce (max) computes
        out, k = _number(b, merged)
        assert torch.equal(out, full)
        assert k == int(full.max().item()) + 1
        # a one-rank plan through the package's driver (no all-reduce)
        one = gpu_refine_sharded(g, lab, 0, ShardPlan(w.labels, np.diff(off), 1),
                                 min_size=w.min_size)
        assert torch.equal(one, full)


def test_minima_and_numbering_round_trip(wcc):
    from paper_2509_02590_gb300 import _binding as b
    w = synth.planted_1k(0)
    off, adj = oracle.build_csr(w.n, w.src, w.dst)
    ref, _ = oracle.wcc(w.n, off, adj, w.labels, w.min_size)
    ref_min, _ = oracle.wcc(w.n, off, adj, w.labels, w.min_size, out_mode=1)
    out = torch.from_numpy(ref).cuda()
    mn = _minima(b, out)
    assert np.array_equal(mn.cpu().numpy(), ref_min)
    back, k = _number(b, mn)
    assert np.array_equal(back.cpu().numpy(), ref) and k == int(ref.max()) + 1
    # host buffers
    mh = np.empty(w.n, np.int32)
    b.wcc_cluster_minima(ref.ctypes.data, w.n, mh.ctypes.data, 0, 0)
    assert np.array_equal(mh, ref_min)
    oh = np.empty(w.n, np.int32)
    assert b.wcc_number_by_minima(mh.ctypes.data, w.n, oh.ctypes.data, 0, 0) == k
    assert np.array_equal(oh, ref)
    # malformed input is refused
    bad = mh.copy()
    v = int(np.nonzero(bad >= 0)[0][0])
    bad[v] = v + 1  # a minimum above its own vertex
    with pytest.raises(wcc.WccError) as e:
        b.wcc_number_by_minima(bad.ctypes.data, w.n, oh.ctypes.data, 0, 0)
    assert e.value.status == -1
    badl = ref.copy()
    badl[3] = w.n  # a label outside [-1, n)
    with pytest.raises(wcc.WccError) as e:
        b.wcc_cluster_minima(badl.ctypes.data, w.n, mh.ctypes.data, 0, 0)
    assert e.value.status == -1
