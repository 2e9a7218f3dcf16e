"""Serving (wcc_server_create / wcc_submit / wcc_poll / wcc_wait): requests
refined together in one persistent kernel must each give exactly the
result they give alone (wcc_run), whatever else is in the mix; the oracle
checks a subset directly.  Also: poll before completion, budget refusal,
concurrent submitters, and destroying a server with uncollected work."""
import threading

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wcc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2509_02590_gb300 as w
    return w


def _workloads():
    ws = [synth.planted_1k(0)]
    for i, n in enumerate((2_000, 5_000, 12_000, 30_000)):
        ws.append(synth.lfr_like(n, seed=40 + i))
    ws.append(synth.dc_planted(50_000, 500_000, seed=7, size_max=3000))
    return ws


def test_serving_alone_equals_mix(wcc):
    wl = _workloads()
    graphs = [wcc.WccGraph.from_edges(w.src, w.dst, w.n) for w in wl]
    rng = np.random.default_rng(3)
    reqs = []
    for k in range(36):
        gi = int(rng.integers(0, len(wl)))
        ms = int(rng.choice([2, 3, wl[gi].min_size]))
        rule = ["log10", "log10", "log2", "sqrt"][k % 4]
        reqs.append((gi, ms, rule))
    alone = [graphs[gi].run(wl[gi].labels, min_size=ms, rule=rule) for gi, ms, rule in reqs]
    results = [None] * len(reqs)
    with wcc.WccServer(8 << 30) as srv:
        tickets = [None] * len(reqs)
        # submit from three host threads at once
        def submitter(lo):
            for i in range(lo, len(reqs), 3):
                gi, ms, rule = reqs[i]
                tickets[i] = srv.submit(graphs[gi], wl[gi].labels, min_size=ms, rule=rule)
        th = [threading.Thread(target=submitter, args=(j,)) for j in range(3)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for i, t in enumerate(tickets):
            out, st = srv.wait(t, timeout_ms=120_000)
            results[i] = out
            assert st["ms_total"] >= st["ms_refine"] >= 0
    for i, (gi, ms, rule) in enumerate(reqs):
        assert np.array_equal(results[i], alone[i]), (i, reqs[i])
    # a few directly against the oracle
    for i in range(0, len(reqs), 9):
        gi, ms, rule = reqs[i]
        w = wl[gi]
        off, adj = oracle.build_csr(w.n, w.src, w.dst)
        kind = {"log10": oracle.RULE_LOG10, "log2": oracle.RULE_LOG2, "sqrt": oracle.RULE_SQRT}[rule]
        ref, _ = oracle.wcc(w.n, off, adj, w.labels, ms, kind)
        assert np.array_equal(results[i], ref)
    for g in graphs:
        g.close()


def test_serving_poll_then_collect_once(wcc):
    w = synth.lfr_like(20_000, seed=9)
    with wcc.WccGraph.from_edges(w.src, w.dst, w.n) as g, wcc.WccServer(2 << 30) as srv:
        t = srv.submit(g, w.labels)
        got = None
        for _ in range(200_000):
            got = srv.poll(t)
            if got is not None:
                break
        assert got is not None
        assert np.array_equal(got[0], g.run(w.labels))
        with pytest.raises(KeyError):
            srv.poll(t)  # collected once; the ticket is gone


def test_serving_budget_refuses_what_never_fits(wcc):
    big = synth.lfr_like(100_000, seed=1)
    with wcc.WccGraph.from_edges(big.src, big.dst, big.n) as g:
        srv = wcc.WccServer(160 << 20)  # fixed structures fit, a 100k-vertex request does not
        try:
            with pytest.raises(wcc.WccError) as ei:
                srv.submit(g, big.labels)
            assert ei.value.status == -5  # WCC_ERR_BUSY
        finally:
            srv.close()
    with pytest.raises(wcc.WccError):
        wcc.WccServer(1 << 20)  # below the fixed structures


def test_serving_destroy_with_uncollected_requests(wcc):
    w = synth.lfr_like(10_000, seed=5)
    with wcc.WccGraph.from_edges(w.src, w.dst, w.n) as g:
        srv = wcc.WccServer(2 << 30)
        for _ in range(5):
            srv.submit(g, w.labels)
        srv.close()  # finishes them and discards the results
