"""Resumable runs (wcc_job_*): a refinement stopped at item boundaries,
checkpointed to a file and resumed -- in the same job or in a job loaded from
the file -- gives exactly the clustering wcc_run gives (and the oracle's)."""
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


def _case():
    w = synth.dc_planted(60_000, 900_000, seed=11, size_max=4000)
    off, adj = oracle.build_csr(w.n, w.src, w.dst)
    ref, _ = oracle.wcc(w.n, off, adj, w.labels, w.min_size)
    return w, ref


def test_steps_then_finish_equal_run(wcc):
    w, ref = _case()
    with wcc.WccGraph.from_edges(w.src, w.dst, w.n) as g:
        assert np.array_equal(g.run(w.labels, min_size=w.min_size), ref)
        with wcc.WccJob.start(g, w.labels, min_size=w.min_size) as job:
            steps = 0
            while not job.step(0):  # stop as soon as possible each time
                steps += 1
                assert steps < 100_000
            out, st = job.finish(stats=True)
        assert np.array_equal(out, ref)
        assert st["out_clusters"] == int(out.max()) + 1


def test_checkpoint_and_resume_in_a_new_job(wcc, tmp_path):
    w, ref = _case()
    path = tmp_path / "queue.wccjob"
    with wcc.WccGraph.from_edges(w.src, w.dst, w.n) as g:
        job = wcc.WccJob.start(g, w.labels, min_size=w.min_size)
        finished = job.step(0)
        job.save(path)
        if not finished:
            with pytest.raises(wcc.WccError) as ei:
                job.finish()  # work left: not yet
            assert ei.value.status == -5  # WCC_ERR_BUSY
        job.close()
        with wcc.WccJob.load(g, path) as job2:
            while not job2.step(1):
                pass
            assert np.array_equal(job2.finish(), ref)
        # a second load of the same checkpoint gives the same again
        with wcc.WccJob.load(g, path) as job3:
            assert job3.step(-1)
            assert np.array_equal(job3.finish(), ref)


def test_load_rejects_foreign_and_corrupt_files(wcc, tmp_path):
    w, _ = _case()
    path = tmp_path / "queue.wccjob"
    with wcc.WccGraph.from_edges(w.src, w.dst, w.n) as g:
        with wcc.WccJob.start(g, w.labels, min_size=w.min_size) as job:
            job.save(path)
        other = synth.lfr_like(5000, seed=2)
        with wcc.WccGraph.from_edges(other.src, other.dst, other.n) as g2:
            with pytest.raises(wcc.WccError):
                wcc.WccJob.load(g2, path)  # another graph
        data = bytearray(path.read_bytes())
        data[len(data) // 2] ^= 0xFF
        bad = tmp_path / "bad.wccjob"
        bad.write_bytes(bytes(data))
        with pytest.raises(wcc.WccError):
            wcc.WccJob.load(g, bad)  # checksum
        bad.write_bytes(path.read_bytes()[:100])
        with pytest.raises(wcc.WccError):
            wcc.WccJob.load(g, bad)  # truncated


def _fnv1a(data: bytes) -> int:
    h = 1469598103934665603
    for b in data:
        h = ((h ^ b) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def _parse(blob: bytes):
    """Offsets of the fields of a job file (layout of wcc_job_save)."""
    import struct
    n = struct.unpack_from("<q", blob, 8)[0]
    hdr = 8 + 5 * 8 + 2 * 4 + 2 * 8 + 7 * 8
    P, M = struct.unpack_from("<qq", blob, hdr)
    items = hdr + 16
    members = items + 8 * P
    lmin = members + 4 * M
    return n, P, M, hdr, items, members, lmin


def _reseal(body: bytearray) -> bytes:
    import struct
    return bytes(body) + struct.pack("<Q", _fnv1a(bytes(body)))


def test_load_checks_contents_not_only_the_checksum(wcc, tmp_path):
    import struct
    w, ref = _case()
    path = tmp_path / "queue.wccjob"
    with wcc.WccGraph.from_edges(w.src, w.dst, w.n) as g:
        with wcc.WccJob.start(g, w.labels, min_size=w.min_size) as job:
            job.save(path)
        blob = path.read_bytes()
        body = bytearray(blob[:-8])
        assert _reseal(body) == blob  # the test's reading of the format is the library's
        n, P, M, hdr, items, members, lmin = _parse(blob)
        assert P > 1 and M > 1
        bad = tmp_path / "bad.wccjob"
        # a vertex listed twice
        b1 = bytearray(body)
        b1[members + 4:members + 8] = b1[members:members + 4]
        bad.write_bytes(_reseal(b1))
        with pytest.raises(wcc.WccError):
            wcc.WccJob.load(g, bad)
        # a cluster minimum outside [-1, n)
        b2 = bytearray(body)
        struct.pack_into("<i", b2, lmin, n)
        bad.write_bytes(_reseal(b2))
        with pytest.raises(wcc.WccError):
            wcc.WccJob.load(g, bad)
        # a header that understates the largest item and degree sum: the
        # working memory is sized from the items, so the run is unchanged
        b3 = bytearray(body)
        struct.pack_into("<qq", b3, 8 + 3 * 8, 1, 1)
        bad.write_bytes(_reseal(b3))
        with wcc.WccJob.load(g, bad) as job:
            assert job.step(-1)
            assert np.array_equal(job.finish(), ref)
