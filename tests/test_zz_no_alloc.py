"""wcc_build_csr_no_alloc: the CSR build for callers that cannot allocate
device memory (for example code running under an allocator that owns the
whole device, or a framework that forbids allocation after start-up).

Through the C ABI, its output must equal the CSR of the existing entry point
(wcc_create_graph_from_edges + wcc_graph_export_csr) exactly -- integer
work -- on two calls in a row, the second one smaller than the first so that
leftovers from the first call in the shared scratch array would show.  This
file is collected last on purpose.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _existing_csr(wcc, src, dst, n):
    with wcc.WccGraph.from_edges(src, dst, n) as g:
        return g.csr()


def _no_alloc_csr(binding, src, dst, n):
    m = len(src)
    s = torch.from_numpy(np.ascontiguousarray(src, np.int32)).cuda()
    d = torch.from_numpy(np.ascontiguousarray(dst, np.int32)).cuda()
    row_off = torch.full((n + 1,), -7, dtype=torch.int64, device="cuda")
    cols = torch.full((max(2 * m, 1),), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    nnz = binding.wcc_build_csr_no_alloc(s.data_ptr(), d.data_ptr(), m, n, row_off.data_ptr(),
                                         cols.data_ptr(), stream)
    return row_off.cpu().numpy(), cols[:nnz].cpu().numpy()


def test_no_alloc_csr_matches_existing_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2509_02590_gb300 as wcc
    from paper_2509_02590_gb300 import _binding

    big = synth.lfr_like(10_000, seed=21)
    rng = np.random.default_rng(5)
    extra = rng.integers(0, big.m, 300)
    big_src = np.concatenate([big.src, big.dst[extra], np.arange(20, dtype=np.int32)])
    big_dst = np.concatenate([big.dst, big.src[extra], np.arange(20, dtype=np.int32)])
    small = synth.planted_1k(0)
    cases = [(big_src, big_dst, big.n), (small.src, small.dst, small.n)]
    assert len(big_src) <= 1 << 17

    for src, dst, n in cases:  # two calls in a row, the second one smaller
        ref_off, ref_adj = _existing_csr(wcc, src, dst, n)
        off, adj = _no_alloc_csr(_binding, src, dst, n)
        assert np.array_equal(off, ref_off)
        assert np.array_equal(adj, ref_adj)

    # later calls make no device allocation: the library's own count of
    # cudaMalloc calls does not move, and neither does the free memory
    s = torch.from_numpy(small.src).cuda()
    d = torch.from_numpy(small.dst).cuda()
    row_off = torch.empty(small.n + 1, dtype=torch.int64, device="cuda")
    cols = torch.empty(2 * small.m, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    allocs_before = _binding.wcc_device_allocations()
    for _ in range(3):
        _binding.wcc_build_csr_no_alloc(s.data_ptr(), d.data_ptr(), small.m, small.n,
                                        row_off.data_ptr(), cols.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert allocs_before > 0  # the count is live: the graphs built above allocated
    assert _binding.wcc_device_allocations() == allocs_before
    assert torch.cuda.mem_get_info()[0] == free_before


def test_no_alloc_rejects_sizes_beyond_the_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2509_02590_gb300 as wcc
    from paper_2509_02590_gb300 import _binding

    with pytest.raises(wcc.WccError) as ei:
        _binding.wcc_build_csr_no_alloc(0, 0, (1 << 17) + 1, 10, 0, 0, 0)
    assert "m must be in [0, 131072]" in str(ei.value)
    with pytest.raises(wcc.WccError) as ei:
        _binding.wcc_build_csr_no_alloc(0, 0, 0, (1 << 22) + 1, 0, 0, 0)
    assert "n must be in [0, 4194304]" in str(ei.value)
