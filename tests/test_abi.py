"""The C-ABI library loads and exports every function include/wcc.h declares
(no GPU needed: nothing is computed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(wcc_\w+)\s*\(", text))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("wcc_create_graph", "wcc_create_graph_from_edges", "wcc_run",
                     "wcc_destroy_graph", "wcc_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    lib_path = __graft_entry__._builder().build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_has_the_same_names():
    import paper_2509_02590_gb300._binding as b
    missing = [n for n in sorted(_declared()) if not hasattr(b, n)]
    assert not missing, missing


def test_no_gpu_fails_loudly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np

    import paper_2509_02590_gb300 as w
    with pytest.raises(w.WccError) as ei:
        w.WccGraph.from_csr(np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32))
    assert ei.value.status == -3  # WCC_ERR_CUDA, never a CPU fallback
