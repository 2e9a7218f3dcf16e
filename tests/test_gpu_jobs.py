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
