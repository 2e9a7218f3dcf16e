"""The process-wide tuning of the refinement schedule (host logic: needs no
GPU) and, on a GPU, the autotuner: whatever tuning it picks, the refined
clustering is the oracle's."""
import json

import numpy as np
import pytest

import oracle
import synth

wcc = pytest.importorskip("paper_2509_02590_gb300")

DEFAULT = {"tiny_max": 64, "tiny_max_deg": 4096, "dense_max": 128, "forest_min_n": 0, "smem_kb": 0}


@pytest.fixture(autouse=True)
def _restore():
    yield
    wcc.set_tuning(**DEFAULT)


def test_defaults_and_round_trip():
    assert wcc.get_tuning() == DEFAULT
    t = wcc.set_tuning(tiny_max=16, tiny_max_deg=300, dense_max=8, forest_min_n=64, smem_kb=100)
    assert wcc.get_tuning() == t == {"tiny_max": 16, "tiny_max_deg": 300, "dense_max": 8,
                                     "forest_min_n": 64, "smem_kb": 100}


@pytest.mark.parametrize("field,value", [("tiny_max", 65), ("tiny_max", -1), ("dense_max", 129),
                                         ("tiny_max_deg", -5), ("smem_kb", -1),
                                         ("forest_min_n", -2)])
def test_out_of_range_rejected(field, value):
    with pytest.raises(wcc.WccError) as ei:
        wcc.set_tuning(**{field: value})
    assert ei.value.status == -1
    assert wcc.get_tuning() == DEFAULT  # nothing changed


def test_load_tuning_file(tmp_path):
    p = tmp_path / "tune.json"
    rec = {"device": "test device", "sms": 152, "n": 10, "nnz": 20, "ms": 1.5, "tiny_max": 16,
           "tiny_max_deg": 512, "dense_max": 24, "forest_min_n": 0, "smem_kb": 160}
    p.write_text(json.dumps(rec))
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        # a file naming another device model is refused on a GPU
        with pytest.raises(wcc.WccError):
            wcc.load_tuning(str(p))
        return
    got = wcc.load_tuning(str(p))
    assert got == {k: rec[k] for k in DEFAULT}
    assert wcc.get_tuning() == got


def test_load_tuning_rejects_bad_files(tmp_path):
    with pytest.raises(wcc.WccError):
        wcc.load_tuning(str(tmp_path / "missing.json"))
    p = tmp_path / "bad.json"
    p.write_text('{"device": "x", "tiny_max": 16}')  # fields missing
    with pytest.raises(wcc.WccError):
        wcc.load_tuning(str(p))
    p.write_text('{"device": "x", "tiny_max": 99, "tiny_max_deg": 1, "dense_max": 1, '
                 '"forest_min_n": 0, "smem_kb": 0}')  # out of range
    with pytest.raises(wcc.WccError):
        wcc.load_tuning(str(p))
    assert wcc.get_tuning() == DEFAULT


@pytest.mark.gpu
def test_autotune_keeps_results(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = synth.lfr_like(12000, seed=3)
    off, adj = oracle.build_csr(w.n, w.src, w.dst)
    ref, _ = oracle.wcc(w.n, off, adj, w.labels, w.min_size)
    cache = tmp_path / "tune.json"
    with wcc.WccGraph.from_edges(w.src, w.dst, w.n) as g:
        best, ms = wcc.autotune(g, w.labels, min_size=w.min_size, cache_path=str(cache))
        assert ms > 0 and best == wcc.get_tuning()
        assert np.array_equal(g.run(w.labels, min_size=w.min_size), ref)
        rec = json.loads(cache.read_text())
        assert {k: rec[k] for k in DEFAULT} == best and rec["sms"] > 0
        wcc.set_tuning(**DEFAULT)
        assert wcc.load_tuning(str(cache)) == best  # same device model
        lab = torch.from_numpy(w.labels).cuda()  # device labels work too
        best2, _ = wcc.autotune(g, lab, min_size=w.min_size)
        assert np.array_equal(g.run(lab, min_size=w.min_size).cpu().numpy(), ref)
