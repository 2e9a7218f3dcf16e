"""Serving (wcc_server_create / wcc_submit / wcc_submit_edges / wcc_poll /
wcc_wait): requests refined together in one persistent kernel must each
give exactly the result they give alone (wcc_run), whatever else is in the
mix; the oracle checks a subset directly.  Also: requests that bring their
graph as an edge list, a budget that makes requests wait for memory, poll
before completion, budget refusal, concurrent submitters, and destroying a
server with uncollected work."""
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


def _noisy_edges(w, rng):
    """The workload's edge list with a few repeated and reversed edges and
    self-loops added (the server's graph builder drops them)."""
    k = min(200, w.m)
    pick = rng.integers(0, w.m, k)
    loops = rng.integers(0, w.n, 20).astype(np.int32)
    src = np.concatenate([w.src, w.dst[pick], loops]).astype(np.int32)
    dst = np.concatenate([w.dst, w.src[pick], loops]).astype(np.int32)
    return src, dst


def test_serving_edge_requests_alone_equals_mix(wcc):
    """Requests that bring their graph as a host edge list (the server
    builds, holds and releases it) mixed with requests on resident graphs,
    from three threads: every result equals wcc_run alone, a subset the
    oracle."""
    wl = _workloads()
    graphs = [wcc.WccGraph.from_edges(w.src, w.dst, w.n) for w in wl]
    rng = np.random.default_rng(11)
    reqs = []
    for k in range(30):
        gi = int(rng.integers(0, len(wl)))
        ms = int(rng.choice([2, 3, wl[gi].min_size]))
        rule = ["log10", "log2", "log10", "sqrt"][k % 4]
        reqs.append((gi, ms, rule, k % 3 != 0))  # two in three bring edges
    edges = [_noisy_edges(w, rng) for w in wl]
    alone = [graphs[gi].run(wl[gi].labels, min_size=ms, rule=rule) for gi, ms, rule, _ in reqs]
    results = [None] * len(reqs)
    with wcc.WccServer(8 << 30) as srv:
        tickets = [None] * len(reqs)

        def submitter(lo):
            for i in range(lo, len(reqs), 3):
                gi, ms, rule, by_edges = reqs[i]
                if by_edges:
                    s, d = edges[gi]
                    tickets[i] = srv.submit_edges(s, d, wl[gi].n, wl[gi].labels, min_size=ms,
                                                  rule=rule)
                else:
                    tickets[i] = srv.submit(graphs[gi], wl[gi].labels, min_size=ms, rule=rule)
        th = [threading.Thread(target=submitter, args=(j,)) for j in range(3)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for i, t in enumerate(tickets):
            results[i], _ = srv.wait(t, timeout_ms=120_000)
        info = srv.info()
    assert info["admitted"] == len(reqs) and info["used_bytes"] == 0
    for i in range(len(reqs)):
        assert np.array_equal(results[i], alone[i]), (i, reqs[i])
    for i in range(1, len(reqs), 7):
        gi, ms, rule, _ = reqs[i]
        w = wl[gi]
        off, adj = oracle.build_csr(w.n, w.src, w.dst)
        kind = {"log10": oracle.RULE_LOG10, "log2": oracle.RULE_LOG2, "sqrt": oracle.RULE_SQRT}[rule]
        ref, _ = oracle.wcc(w.n, off, adj, w.labels, ms, kind)
        assert np.array_equal(results[i], ref)
    for g in graphs:
        g.close()


def test_serving_budget_binds_admission(wcc):
    """With a budget that holds about two edge requests at once (their CSR
    and working memory, plus the builder's transient memory), the others
    wait for memory to free up: the waits are counted, the bytes held never
    exceed the budget, and every result is still exact."""
    w = synth.lfr_like(30_000, seed=12)
    with wcc.WccGraph.from_edges(w.src, w.dst, w.n) as g:
        ref = g.run(w.labels)
    # one request: 240 B per vertex + 1 MB, CSR 2 x (8 B per vertex + 8 B per
    # edge), builder 2 x (56 B per edge + 8 B per vertex) + 1 MB
    one = 240 * w.n + (1 << 20) + 2 * (8 * (w.n + 1) + 8 * w.m)
    build = 2 * (56 * w.m + 8 * w.n) + (1 << 20)
    want = 2 * one + build + (4 << 20)  # room for two requests, not three

    def fixed_part(b):
        probe = wcc.WccServer(b)
        left = probe.info()["budget_bytes"]
        probe.close()
        return b - left

    budget = fixed_part(400 << 20) + want
    budget = fixed_part(budget) + want  # the queue is sized from the budget
    with wcc.WccServer(budget) as srv:
        tickets = [srv.submit_edges(w.src, w.dst, w.n, w.labels) for _ in range(8)]
        outs = [srv.wait(t, timeout_ms=120_000)[0] for t in tickets]
        info = srv.info()
    for out in outs:
        assert np.array_equal(out, ref)
    assert info["budget_waits"] > 0
    assert info["peak_used_bytes"] <= info["budget_bytes"]
    assert 1 <= info["peak_active"] <= 2


def test_serving_edge_request_refusals(wcc):
    w = synth.lfr_like(5_000, seed=2)
    with wcc.WccServer(2 << 30) as srv:
        with pytest.raises(wcc.WccError) as ei:   # can never fit the budget
            srv.submit_edges(w.src, w.dst, 10_000_000, np.zeros(10_000_000, np.int32))
        assert ei.value.status == -5
        bad = w.dst.copy()
        bad[7] = w.n + 3                           # an id outside [0, n)
        t = srv.submit_edges(w.src, bad, w.n, w.labels)
        with pytest.raises(wcc.WccError) as ei:
            srv.wait(t, timeout_ms=60_000)
        assert ei.value.status == -1
        t = srv.submit_edges(w.src, w.dst, w.n, w.labels)  # the server still serves
        out, _ = srv.wait(t, timeout_ms=60_000)
    with wcc.WccGraph.from_edges(w.src, w.dst, w.n) as g:
        assert np.array_equal(out, g.run(w.labels))


def test_serving_submit_does_not_wait_for_the_device(wcc):
    """A submission while the kernel is busy returns at once: nothing on the
    submit path waits for the whole device (pinning host memory per request
    did, and stalled every submission until the backlog had drained)."""
    from synth import gpu_graphs
    big = gpu_graphs.dcpp_1m(seed=0)
    small = synth.lfr_like(5_000, seed=4)
    with wcc.WccGraph.from_edges(big.src, big.dst, big.n) as gb, \
            wcc.WccGraph.from_edges(small.src, small.dst, small.n) as gs:
        _, st = gb.run(big.labels, min_size=big.min_size, stats=True)
        busy_ms = st["ms_refine"]
        ref_small = gs.run(small.labels)
        lab_big = big.labels.cpu().numpy()
        import time
        with wcc.WccServer(16 << 30) as srv:
            tb = srv.submit(gb, lab_big, min_size=big.min_size)
            times, tickets = [], []
            for _ in range(10):
                t0 = time.perf_counter()
                tickets.append(srv.submit(gs, small.labels))
                times.append((time.perf_counter() - t0) * 1e3)
            outs = [srv.wait(t, timeout_ms=120_000)[0] for t in tickets]
            srv.wait(tb, timeout_ms=120_000)
    assert max(times) < busy_ms / 2, (times, busy_ms)
    for out in outs:
        assert np.array_equal(out, ref_small)
