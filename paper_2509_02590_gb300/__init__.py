"""GB300 Well-Connected Clusters refinement (WCC, arXiv 2509.02590).

The refinement runs in the CUDA library ``libwcc_gb300.so`` behind the C ABI
of ``include/wcc.h``.  ``_binding`` exposes that ABI under the same names;
:class:`WccGraph` below only marshals numpy arrays (host buffers) or CUDA
torch tensors (device buffers, ordered on torch's current stream) into it.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _binding
from ._binding import (WCC_MODE_BATCHED, WCC_MODE_PLAIN, WCC_RULE_LINEAR,  # noqa: F401
                       WCC_RULE_LOG2, WCC_RULE_LOG10, WCC_RULE_SQRT, WccError,
                       wcc_build_csr_no_alloc, wcc_create_graph,
                       wcc_create_graph_from_edges, wcc_destroy_graph, wcc_graph_export_csr,
                       wcc_graph_nnz, wcc_graph_num_vertices, wcc_kernel_launches, wcc_device_allocations,
                       wcc_last_error, wcc_poll, wcc_run, wcc_run_cm, wcc_server_create,
                       wcc_server_destroy, wcc_submit, wcc_wait,
                       wcc_stats, wcc_threshold_rule, wcc_tuning, wcc_get_tuning,
                       wcc_set_tuning, wcc_autotune, wcc_load_tuning, wcc_job_start,
                       wcc_job_step, wcc_job_save, wcc_job_load, wcc_job_finish,
                       wcc_job_destroy)

_RULES = {"log10": WCC_RULE_LOG10, "log2": WCC_RULE_LOG2, "sqrt": WCC_RULE_SQRT,
          "linear": WCC_RULE_LINEAR}
_MODES = {"batched": WCC_MODE_BATCHED, "plain": WCC_MODE_PLAIN}


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _buf(x, dtype):
    """(pointer, on_device, stream, keepalive) for a numpy array or torch tensor."""
    if _is_torch(x):
        import torch
        tdt = {np.int32: torch.int32, np.int64: torch.int64}[dtype]
        if x.dtype != tdt or not x.is_contiguous():
            raise TypeError(f"expected a contiguous {tdt} tensor")
        if x.is_cuda:
            return x.data_ptr(), 1, torch.cuda.current_stream(x.device).cuda_stream, x
        return x.data_ptr(), 0, 0, x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, 0, 0, a


def rule_struct(rule="log10", num: int = 1, den: int = 1) -> wcc_threshold_rule:
    kind = _RULES[rule] if isinstance(rule, str) else int(rule)
    return wcc_threshold_rule(kind, 0, num, den)


class WccGraph:
    """A graph resident on the GPU (owns a ``wcc_graph`` handle)."""

    def __init__(self, handle: int):
        self.handle = handle

    @classmethod
    def from_csr(cls, row_off, cols, n: int | None = None) -> "WccGraph":
        po, dev_o, st, ko = _buf(row_off, np.int64)
        pc, dev_c, _, kc = _buf(cols, np.int32)
        if dev_o != dev_c:
            raise TypeError("row_off and cols must both be host or both be device buffers")
        n = (len(ko) - 1) if n is None else n
        return cls(wcc_create_graph(po, pc, n, len(kc), dev_o, st))

    @classmethod
    def from_edges(cls, src, dst, n: int) -> "WccGraph":
        ps, dev_s, st, ks = _buf(src, np.int32)
        pd, dev_d, _, kd = _buf(dst, np.int32)
        if dev_s != dev_d or len(ks) != len(kd):
            raise TypeError("src and dst must match in length and placement")
        return cls(wcc_create_graph_from_edges(ps, pd, len(ks), n, dev_s, st))

    @property
    def n(self) -> int:
        return wcc_graph_num_vertices(self.handle)

    @property
    def nnz(self) -> int:
        return wcc_graph_nnz(self.handle)

    def csr(self, device: bool = False):
        """The graph's CSR (row offsets, columns): numpy arrays, or CUDA
        tensors on the current device when ``device``."""
        if device:
            import torch
            off = torch.empty(self.n + 1, dtype=torch.int64, device="cuda")
            adj = torch.empty(max(self.nnz, 1), dtype=torch.int32, device="cuda")
            wcc_graph_export_csr(self.handle, off.data_ptr(), adj.data_ptr(), 1,
                                 torch.cuda.current_stream().cuda_stream)
            torch.cuda.current_stream().synchronize()
            return off, adj[:self.nnz]
        off = np.empty(self.n + 1, np.int64)
        adj = np.empty(max(self.nnz, 1), np.int32)
        wcc_graph_export_csr(self.handle, off.ctypes.data, adj.ctypes.data, 0, 0)
        return off, adj[:self.nnz]

    def run(self, labels, min_size: int = 2, rule="log10", num: int = 1, den: int = 1,
            mode="batched", out=None, stats: bool = False):
        """Refine ``labels`` (numpy -> numpy on the host path, CUDA tensor ->
        CUDA tensor on the device path).  Returns ``out`` (and a stats dict
        when ``stats``)."""
        pin, dev, stream, kin = _buf(labels, np.int32)
        if out is None:
            if _is_torch(labels):
                import torch
                out = torch.empty_like(labels)
            else:
                out = np.empty(len(kin), np.int32)
        pout, dev_o, _, kout = _buf(out, np.int32)
        if dev_o != dev:
            raise TypeError("labels and out must both be host or both be device buffers")
        st = wcc_stats() if stats else None
        r = rule_struct(rule, num, den)
        m = _MODES[mode] if isinstance(mode, str) else int(mode)
        wcc_run(self.handle, pin, r, min_size, m, pout, dev, stream, st)
        if out is not kout and not _is_torch(out):
            out[...] = kout
        return (out, st.as_dict()) if stats else out

    def run_cm(self, labels, resolution=(1, 1000), min_size: int = 2, rule="log10",
               num: int = 1, den: int = 1, out=None, stats: bool = False):
        """CM refinement (WCC whose split parts go through the CPM community
        step at resolution = (cpm_num, cpm_den)); buffers as ``run``."""
        pin, dev, stream, kin = _buf(labels, np.int32)
        if out is None:
            if _is_torch(labels):
                import torch
                out = torch.empty_like(labels)
            else:
                out = np.empty(len(kin), np.int32)
        pout, dev_o, _, kout = _buf(out, np.int32)
        if dev_o != dev:
            raise TypeError("labels and out must both be host or both be device buffers")
        st = wcc_stats() if stats else None
        r = rule_struct(rule, num, den)
        gnum, gden = resolution
        wcc_run_cm(self.handle, pin, r, min_size, int(gnum), int(gden), pout, dev, stream, st)
        if out is not kout and not _is_torch(out):
            out[...] = kout
        return (out, st.as_dict()) if stats else out

    def close(self):
        if self.handle:
            wcc_destroy_graph(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class WccServer:
    """A continuous-batching refinement server (owns a ``wcc_server``).

    Requests carry host (numpy) clusterings; results come back as numpy
    arrays.  A graph passed to ``submit`` must stay open until its requests
    are collected; ``submit_edges`` hands the server an edge list instead."""

    def __init__(self, mem_budget_bytes: int):
        self.handle = wcc_server_create(int(mem_budget_bytes))
        self._n = {}
        self._keep = {}  # edge lists of requests not collected yet

    def submit(self, graph: WccGraph, labels, min_size: int = 2, rule="log10", num: int = 1,
               den: int = 1) -> int:
        lab = np.ascontiguousarray(labels, dtype=np.int32)
        if len(lab) != graph.n:
            raise ValueError("labels must have one entry per vertex")
        t = wcc_submit(self.handle, graph.handle, lab.ctypes.data, rule_struct(rule, num, den),
                       min_size)
        self._n[t] = graph.n
        return t

    def submit_edges(self, src, dst, n: int, labels, min_size: int = 2, rule="log10",
                     num: int = 1, den: int = 1) -> int:
        """Queue a request that brings its graph as a host edge list (numpy
        arrays or CPU tensors, pinned ones upload fastest); the server builds
        the graph on admission and releases it afterwards.  The edge arrays
        are held here until the request is collected."""
        ps, dev_s, _, ks = _buf(src, np.int32)
        pd, dev_d, _, kd = _buf(dst, np.int32)
        if dev_s or dev_d:
            raise TypeError("submit_edges takes host edge lists")
        lab = np.ascontiguousarray(labels, dtype=np.int32)
        m = len(ks)
        if len(kd) != m or len(lab) != n:
            raise ValueError("src and dst must match; labels must have one entry per vertex")
        t = _binding.wcc_submit_edges(self.handle, ps, pd, m, int(n), lab.ctypes.data,
                                      rule_struct(rule, num, den), min_size)
        self._n[t] = int(n)
        self._keep[t] = (ks, kd)
        return t

    def info(self) -> dict:
        """Admission counters (budget, bytes held, waits, requests at once)."""
        return _binding.wcc_server_info(self.handle)

    def _collect(self, fn, ticket, *args):
        n = self._n[ticket]
        out = np.empty(max(n, 1), np.int32)
        st = wcc_stats()
        try:
            r = fn(self.handle, ticket, *args, out.ctypes.data, st)
        except WccError:
            self._n.pop(ticket, None)
            self._keep.pop(ticket, None)
            raise
        if r != _binding.WCC_OK:
            return None
        self._n.pop(ticket, None)
        self._keep.pop(ticket, None)
        return out[:n], st.as_dict()

    def poll(self, ticket: int):
        """(labels, stats) when finished, else None."""
        return self._collect(wcc_poll, ticket)

    def wait(self, ticket: int, timeout_ms: int = 600_000):
        """(labels, stats) once finished, or None after timeout_ms."""
        return self._collect(wcc_wait, ticket, int(timeout_ms))

    def close(self):
        if self.handle:
            wcc_server_destroy(self.handle)
            self.handle = 0
        self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class WccJob:
    """A refinement in resumable steps (owns a ``wcc_job``): ``step`` runs for
    a time budget, ``save`` / ``WccJob.load`` checkpoint the queue to a file,
    ``finish`` gives the refined clustering once ``step`` has returned True.
    Host (numpy) clusterings; the graph must stay open while the job lives."""

    def __init__(self, handle: int, graph: WccGraph):
        self.handle = handle
        self.graph = graph

    @classmethod
    def start(cls, graph: WccGraph, labels, min_size: int = 2, rule="log10", num: int = 1,
              den: int = 1) -> "WccJob":
        lab = np.ascontiguousarray(labels, dtype=np.int32)
        if len(lab) != graph.n:
            raise ValueError("labels must have one entry per vertex")
        return cls(wcc_job_start(graph.handle, lab.ctypes.data, rule_struct(rule, num, den),
                                 min_size, 0, 0), graph)

    @classmethod
    def load(cls, graph: WccGraph, path: str) -> "WccJob":
        return cls(wcc_job_load(graph.handle, str(path), 0), graph)

    def step(self, time_budget_ms: int = -1) -> bool:
        """True once the queue is empty."""
        return wcc_job_step(self.handle, int(time_budget_ms), 0) == _binding.WCC_OK

    def save(self, path: str) -> None:
        wcc_job_save(self.handle, str(path), 0)

    def finish(self, stats: bool = False):
        out = np.empty(max(self.graph.n, 1), np.int32)
        st = wcc_stats() if stats else None
        wcc_job_finish(self.handle, out.ctypes.data, 0, 0, st)
        out = out[:self.graph.n]
        return (out, st.as_dict()) if stats else out

    def close(self):
        if self.handle:
            wcc_job_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def get_tuning() -> dict:
    """The process-wide tuning of the refinement schedule (see include/wcc.h)."""
    return wcc_get_tuning().as_dict()


def set_tuning(**fields) -> dict:
    """Changes fields of the process-wide tuning; returns the new tuning."""
    t = wcc_get_tuning()
    for k, v in fields.items():
        if k not in t.as_dict():
            raise KeyError(k)
        setattr(t, k, int(v))
    wcc_set_tuning(t)
    return t.as_dict()


def autotune(graph: "WccGraph", labels, min_size: int = 2, rule="log10", num: int = 1,
             den: int = 1, cache_path: str | None = None):
    """Times candidate tunings on this graph and clustering, sets the fastest
    and returns (tuning dict, ms per run)."""
    pin, dev, stream, _keep = _buf(labels, np.int32)
    best, ms = wcc_autotune(graph.handle, pin, rule_struct(rule, num, den), min_size, dev, stream,
                            cache_path)
    return best.as_dict(), ms


def load_tuning(cache_path: str) -> dict:
    """Sets the tuning that autotune wrote to cache_path; returns it."""
    return wcc_load_tuning(cache_path).as_dict()


__all__ = ["WccServer", "WccGraph", "WccError", "rule_struct", "wcc_create_graph",
           "wcc_create_graph_from_edges", "wcc_run", "wcc_destroy_graph", "wcc_last_error",
           "wcc_graph_num_vertices", "wcc_graph_nnz", "wcc_kernel_launches", "wcc_build_csr_no_alloc", "wcc_graph_export_csr", "wcc_stats",
           "wcc_threshold_rule", "WCC_MODE_BATCHED", "WCC_MODE_PLAIN", "wcc_server_create",
           "wcc_submit", "wcc_poll", "wcc_wait", "wcc_server_destroy", "wcc_tuning",
           "wcc_get_tuning", "wcc_set_tuning", "wcc_autotune", "wcc_load_tuning", "get_tuning",
           "set_tuning", "autotune", "load_tuning", "WccJob", "wcc_job_start", "wcc_job_step",
           "wcc_job_save", "wcc_job_load", "wcc_job_finish", "wcc_job_destroy"]
_ = ctypes
