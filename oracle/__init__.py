"""Plain CPU oracle for WCC refinement -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
path never imports, links or executes anything here, and this package shares
no code with it.

The arithmetic lives in ``wcc_oracle.c`` (plain C, single-threaded); this
module only compiles it with ``gcc`` and marshals numpy arrays through ctypes.
What each function computes, and which part of the paper it follows, is
stated in ``wcc_oracle.h``.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, brute-force enumeration of all bipartitions, hand-traced
cases, library cross-checks and whole-refinement invariants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wcc_oracle.c")
_LIB = os.path.join(_HERE, "libwcc_oracle.so")

RULE_LOG10, RULE_LOG2, RULE_SQRT, RULE_LINEAR = 0, 1, 2, 3


class Stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "in_clusters", "out_clusters", "items", "splits", "peeled", "ni_passes", "sw_phases")]

    def as_dict(self):
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libwcc_oracle.so`` (gcc, -O2)."""
    hdr = os.path.join(_HERE, "wcc_oracle.h")
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(hdr))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-Wall", "-Wextra", "-fPIC", "-shared",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        L.wo_threshold.argtypes = [i32, i64, i64, i64]
        L.wo_threshold.restype = i64
        L.wo_build_csr.argtypes = [i64, i64, i32p, i32p, i64p, i32p, i64p]
        L.wo_build_csr.restype = ctypes.c_int
        L.wo_components.argtypes = [i64, i64, i32p, i32p, i32p]
        L.wo_components.restype = i64
        L.wo_peel.argtypes = [i64, i64, i32p, i32p, i32, i64, i64, u8p]
        L.wo_peel.restype = i64
        L.wo_stoer_wagner.argtypes = [i64, i64, i32p, i32p, i64p, u8p]
        L.wo_stoer_wagner.restype = i64
        L.wo_item_cut.argtypes = [i64, i64, i32p, i32p, i64, i32p, u8p, i64p]
        L.wo_item_cut.restype = ctypes.c_int
        L.wo_wcc.argtypes = [i64, i64p, i32p, i32p, i32, i64, i64, i32, u8p, i64, i32, i32p,
                             ctypes.POINTER(Stats)]
        L.wo_wcc.restype = ctypes.c_int
        L.wo_cm.argtypes = [i64, i64p, i32p, i32p, i32, i64, i64, i32, i64, i64, u8p, i64, i32,
                            i32p, ctypes.POINTER(Stats)]
        L.wo_cm.restype = ctypes.c_int
        L.wo_cpm_communities.argtypes = [i64, i64, i32p, i32p, i64, i64, i32, i32p]
        L.wo_cpm_communities.restype = i64
        _lib = L
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _edges(eu, ev):
    eu = np.ascontiguousarray(eu, dtype=np.int32)
    ev = np.ascontiguousarray(ev, dtype=np.int32)
    assert eu.shape == ev.shape
    return eu, ev


def threshold(n: int, kind: int = RULE_LOG10, num: int = 1, den: int = 1) -> int:
    return int(lib().wo_threshold(kind, num, den, n))


def build_csr(n: int, src, dst):
    """Simple symmetric CSR (int64 offsets, int32 sorted columns)."""
    src, dst = _edges(src, dst)
    off = np.zeros(n + 1, dtype=np.int64)
    adj = np.zeros(max(2 * len(src), 1), dtype=np.int32)
    nnz = ctypes.c_int64(0)
    rc = lib().wo_build_csr(n, len(src), _p(src, ctypes.c_int32), _p(dst, ctypes.c_int32),
                            _p(off, ctypes.c_int64), _p(adj, ctypes.c_int32), ctypes.byref(nnz))
    if rc != 0:
        raise ValueError("edge endpoint outside [0, n)")
    return off, adj[:nnz.value].copy()


def components(n: int, eu, ev) -> np.ndarray:
    eu, ev = _edges(eu, ev)
    comp = np.empty(n, dtype=np.int32)
    lib().wo_components(n, len(eu), _p(eu, ctypes.c_int32), _p(ev, ctypes.c_int32),
                        _p(comp, ctypes.c_int32))
    return comp


def peel(n: int, eu, ev, kind: int = RULE_LOG10, num: int = 1, den: int = 1) -> np.ndarray:
    eu, ev = _edges(eu, ev)
    alive = np.empty(n, dtype=np.uint8)
    lib().wo_peel(n, len(eu), _p(eu, ctypes.c_int32), _p(ev, ctypes.c_int32), kind, num, den,
                  _p(alive, ctypes.c_uint8))
    return alive.astype(bool)


def stoer_wagner(n: int, eu, ev, w=None):
    """Canonical Stoer-Wagner: returns (min cut value, side mask)."""
    eu, ev = _edges(eu, ev)
    side = np.zeros(n, dtype=np.uint8)
    wp = None
    if w is not None:
        w = np.ascontiguousarray(w, dtype=np.int64)
        wp = _p(w, ctypes.c_int64)
    lam = lib().wo_stoer_wagner(n, len(eu), _p(eu, ctypes.c_int32), _p(ev, ctypes.c_int32), wp,
                                _p(side, ctypes.c_uint8))
    return int(lam), side.astype(bool)


def item_cut(n: int, eu, ev, T: int):
    """Cut step of one item: returns (accepted, lambda or None, side mask, rep)."""
    eu, ev = _edges(eu, ev)
    rep = np.empty(n, dtype=np.int32)
    side = np.zeros(n, dtype=np.uint8)
    lam = ctypes.c_int64(-1)
    rc = lib().wo_item_cut(n, len(eu), _p(eu, ctypes.c_int32), _p(ev, ctypes.c_int32), T,
                           _p(rep, ctypes.c_int32), _p(side, ctypes.c_uint8), ctypes.byref(lam))
    if rc < 0:
        raise RuntimeError(f"wo_item_cut failed ({rc})")
    return bool(rc == 1), (None if rc == 1 else int(lam.value)), side.astype(bool), rep


def wcc(n: int, off: np.ndarray, adj: np.ndarray, labels: np.ndarray, min_size: int,
        kind: int = RULE_LOG10, num: int = 1, den: int = 1,
        only_labels: Optional[np.ndarray] = None, out_mode: int = 0):
    """Whole refinement.  Returns (label_out int32[n], stats dict)."""
    off = np.ascontiguousarray(off, dtype=np.int64)
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    assert off.shape == (n + 1,) and labels.shape == (n,)
    out = np.empty(n, dtype=np.int32)
    st = Stats()
    only_p, n_only = None, 0
    if only_labels is not None:
        only = np.ascontiguousarray(only_labels, dtype=np.uint8)
        only_p, n_only = _p(only, ctypes.c_uint8), len(only)
    adj_p = _p(adj if len(adj) else np.zeros(1, np.int32), ctypes.c_int32)
    rc = lib().wo_wcc(n, _p(off, ctypes.c_int64), adj_p, _p(labels, ctypes.c_int32), kind, num,
                      den, min_size, only_p, n_only, out_mode, _p(out, ctypes.c_int32),
                      ctypes.byref(st))
    if rc != 0:
        raise RuntimeError(f"wo_wcc failed ({rc})")
    return out, st.as_dict()


def cpm_communities(n: int, eu, ev, gnum: int, gden: int, connected: bool = True) -> np.ndarray:
    """CPM local moving, then (connected) the connected parts of every
    community: comm[v] = smallest id of v's community (the community step
    of CM)."""
    eu, ev = _edges(eu, ev)
    comm = np.empty(n, dtype=np.int32)
    r = lib().wo_cpm_communities(n, len(eu), _p(eu, ctypes.c_int32), _p(ev, ctypes.c_int32),
                                 gnum, gden, int(bool(connected)), _p(comm, ctypes.c_int32))
    if r < 0:
        raise ValueError("bad input")
    return comm


def cm(n: int, off: np.ndarray, adj: np.ndarray, labels: np.ndarray, min_size: int,
       gnum: int, gden: int, kind: int = RULE_LOG10, num: int = 1, den: int = 1,
       only_labels: Optional[np.ndarray] = None, out_mode: int = 0):
    """CM refinement (WCC with the CPM community step after every split).
    Returns (label_out int32[n], stats dict)."""
    off = np.ascontiguousarray(off, dtype=np.int64)
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    assert off.shape == (n + 1,) and labels.shape == (n,)
    out = np.empty(n, dtype=np.int32)
    st = Stats()
    only_p, n_only = None, 0
    if only_labels is not None:
        only = np.ascontiguousarray(only_labels, dtype=np.uint8)
        only_p, n_only = _p(only, ctypes.c_uint8), len(only)
    adj_p = _p(adj if len(adj) else np.zeros(1, np.int32), ctypes.c_int32)
    rc = lib().wo_cm(n, _p(off, ctypes.c_int64), adj_p, _p(labels, ctypes.c_int32), kind, num,
                     den, min_size, gnum, gden, only_p, n_only, out_mode, _p(out, ctypes.c_int32),
                     ctypes.byref(st))
    if rc != 0:
        raise RuntimeError(f"wo_cm failed ({rc})")
    return out, st.as_dict()
