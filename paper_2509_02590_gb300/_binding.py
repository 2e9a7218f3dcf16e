"""ctypes binding of the C ABI in ``include/wcc.h`` (argument marshalling only).

Every function here forwards to ``libwcc_gb300.so``; no step of the
refinement runs in Python.  If the library is missing or cannot be loaded,
importing this module raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwcc_gb300.so")

WCC_OK = 0
WCC_PENDING = 1
WCC_ERR_INVALID = -1
WCC_ERR_OOM = -2
WCC_ERR_CUDA = -3
WCC_ERR_TIMEOUT = -4
WCC_ERR_BUSY = -5
WCC_ERR_INTERNAL = -6

WCC_RULE_LOG10, WCC_RULE_LOG2, WCC_RULE_SQRT, WCC_RULE_LINEAR = 0, 1, 2, 3
WCC_MODE_BATCHED, WCC_MODE_PLAIN = 0, 1

STATUS_NAMES = {0: "WCC_OK", 1: "WCC_PENDING", -1: "WCC_ERR_INVALID", -2: "WCC_ERR_OOM",
                -3: "WCC_ERR_CUDA", -4: "WCC_ERR_TIMEOUT", -5: "WCC_ERR_BUSY",
                -6: "WCC_ERR_INTERNAL"}


class wcc_threshold_rule(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("num", ctypes.c_int64), ("den", ctypes.c_int64)]


class wcc_stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in (
        "in_clusters", "out_clusters", "items", "splits", "peeled", "ni_passes", "sw_phases",
        "max_item", "alg_bytes")] + [(f, ctypes.c_double) for f in (
            "ms_membership", "ms_refine", "ms_output", "ms_total")]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class wcc_tuning(ctypes.Structure):
    _fields_ = [("tiny_max", ctypes.c_int32), ("tiny_max_deg", ctypes.c_int32),
                ("dense_max", ctypes.c_int32), ("forest_min_n", ctypes.c_int32),
                ("smem_kb", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved"}


class wcc_server_counters(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "budget_bytes", "used_bytes", "peak_used_bytes", "admitted", "budget_waits", "slot_waits",
        "peak_active", "max_active")]

    def as_dict(self):
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


class WccError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (nvcc, sm_103a). "
            "There is no CPU fallback.")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
    gpp = ctypes.POINTER(ctypes.c_void_p)
    L.wcc_create_graph.argtypes = [vp, vp, i64, i64, c_int, vp, gpp]
    L.wcc_create_graph.restype = c_int
    L.wcc_create_graph_from_edges.argtypes = [vp, vp, i64, i64, c_int, vp, gpp]
    L.wcc_create_graph_from_edges.restype = c_int
    L.wcc_graph_num_vertices.argtypes = [vp]
    L.wcc_graph_num_vertices.restype = i64
    L.wcc_graph_nnz.argtypes = [vp]
    L.wcc_graph_nnz.restype = i64
    L.wcc_graph_export_csr.argtypes = [vp, vp, vp, c_int, vp]
    L.wcc_graph_export_csr.restype = c_int
    L.wcc_run.argtypes = [vp, vp, ctypes.POINTER(wcc_threshold_rule), i32, i32, vp, c_int, vp,
                          ctypes.POINTER(wcc_stats)]
    L.wcc_run.restype = c_int
    L.wcc_run_cm.argtypes = [vp, vp, ctypes.POINTER(wcc_threshold_rule), i32, i64, i64, vp, c_int,
                             vp, ctypes.POINTER(wcc_stats)]
    L.wcc_run_cm.restype = c_int
    L.wcc_destroy_graph.argtypes = [vp]
    L.wcc_destroy_graph.restype = None
    L.wcc_server_create.argtypes = [i64, gpp]
    L.wcc_server_create.restype = c_int
    L.wcc_submit.argtypes = [vp, vp, vp, ctypes.POINTER(wcc_threshold_rule), i32,
                             ctypes.POINTER(ctypes.c_uint64)]
    L.wcc_submit.restype = c_int
    L.wcc_poll.argtypes = [vp, ctypes.c_uint64, vp, ctypes.POINTER(wcc_stats)]
    L.wcc_poll.restype = c_int
    L.wcc_wait.argtypes = [vp, ctypes.c_uint64, i64, vp, ctypes.POINTER(wcc_stats)]
    L.wcc_wait.restype = c_int
    L.wcc_server_destroy.argtypes = [vp]
    L.wcc_server_destroy.restype = None
    L.wcc_build_csr_no_alloc.argtypes = [vp, vp, i64, i64, vp, vp, ctypes.POINTER(i64), vp]
    L.wcc_build_csr_no_alloc.restype = c_int
    L.wcc_kernel_launches.argtypes = []
    L.wcc_kernel_launches.restype = i64
    L.wcc_device_allocations.argtypes = []
    L.wcc_device_allocations.restype = i64
    L.wcc_submit_edges.argtypes = [vp, vp, vp, i64, i64, vp,
                                   ctypes.POINTER(wcc_threshold_rule), i32,
                                   ctypes.POINTER(ctypes.c_uint64)]
    L.wcc_submit_edges.restype = c_int
    L.wcc_server_info.argtypes = [vp, ctypes.POINTER(wcc_server_counters)]
    L.wcc_server_info.restype = c_int
    L.wcc_cluster_minima.argtypes = [vp, i64, vp, c_int, vp]
    L.wcc_cluster_minima.restype = c_int
    L.wcc_number_by_minima.argtypes = [vp, i64, vp, ctypes.POINTER(i64), c_int, vp]
    L.wcc_number_by_minima.restype = c_int
    L.wcc_last_error.argtypes = []
    L.wcc_last_error.restype = ctypes.c_char_p
    tp = ctypes.POINTER(wcc_tuning)
    L.wcc_get_tuning.argtypes = [tp]
    L.wcc_get_tuning.restype = c_int
    L.wcc_set_tuning.argtypes = [tp]
    L.wcc_set_tuning.restype = c_int
    L.wcc_autotune.argtypes = [vp, vp, ctypes.POINTER(wcc_threshold_rule), i32, c_int, vp,
                               ctypes.c_char_p, tp, ctypes.POINTER(ctypes.c_double)]
    L.wcc_autotune.restype = c_int
    L.wcc_load_tuning.argtypes = [ctypes.c_char_p, tp]
    L.wcc_load_tuning.restype = c_int
    L.wcc_job_start.argtypes = [vp, vp, ctypes.POINTER(wcc_threshold_rule), i32, c_int, vp,
                                ctypes.POINTER(vp)]
    L.wcc_job_start.restype = c_int
    L.wcc_job_step.argtypes = [vp, i64, vp]
    L.wcc_job_step.restype = c_int
    L.wcc_job_save.argtypes = [vp, ctypes.c_char_p, vp]
    L.wcc_job_save.restype = c_int
    L.wcc_job_load.argtypes = [vp, ctypes.c_char_p, vp, ctypes.POINTER(vp)]
    L.wcc_job_load.restype = c_int
    L.wcc_job_finish.argtypes = [vp, vp, c_int, vp, ctypes.POINTER(wcc_stats)]
    L.wcc_job_finish.restype = c_int
    L.wcc_job_destroy.argtypes = [vp]
    L.wcc_job_destroy.restype = None
    return L


lib = _load()


def wcc_server_create(mem_budget_bytes: int) -> int:
    out = ctypes.c_void_p()
    _check(lib.wcc_server_create(mem_budget_bytes, ctypes.byref(out)))
    return out.value


def wcc_submit(server: int, g: int, clustering_in: int, rule: wcc_threshold_rule | None,
               min_size: int) -> int:
    t = ctypes.c_uint64(0)
    _check(lib.wcc_submit(server, g, clustering_in,
                          ctypes.byref(rule) if rule is not None else None, min_size,
                          ctypes.byref(t)))
    return int(t.value)


def wcc_submit_edges(server: int, src: int, dst: int, m: int, n: int, clustering_in: int,
                     rule: wcc_threshold_rule | None, min_size: int) -> int:
    t = ctypes.c_uint64(0)
    _check(lib.wcc_submit_edges(server, src, dst, m, n, clustering_in,
                                ctypes.byref(rule) if rule is not None else None, min_size,
                                ctypes.byref(t)))
    return int(t.value)


def wcc_server_info(server: int) -> dict:
    c = wcc_server_counters()
    _check(lib.wcc_server_info(server, ctypes.byref(c)))
    return c.as_dict()


def wcc_poll(server: int, ticket: int, clustering_out: int,
             stats: wcc_stats | None = None) -> int:
    """WCC_OK or WCC_PENDING (raises on the request's error)."""
    return _check(lib.wcc_poll(server, ticket, clustering_out,
                               ctypes.byref(stats) if stats is not None else None))


def wcc_wait(server: int, ticket: int, timeout_ms: int, clustering_out: int,
             stats: wcc_stats | None = None) -> int:
    """WCC_OK or WCC_PENDING after timeout_ms (raises on the request's error)."""
    return _check(lib.wcc_wait(server, ticket, timeout_ms, clustering_out,
                               ctypes.byref(stats) if stats is not None else None))


def wcc_server_destroy(server: int) -> None:
    lib.wcc_server_destroy(server)


def wcc_build_csr_no_alloc(src: int, dst: int, m: int, n: int, row_off: int, cols: int,
                           stream: int) -> int:
    """Device-buffer CSR build that allocates nothing; returns nnz."""
    nnz = ctypes.c_int64(0)
    _check(lib.wcc_build_csr_no_alloc(src, dst, m, n, row_off, cols, ctypes.byref(nnz), stream))
    return int(nnz.value)


def wcc_kernel_launches() -> int:
    return int(lib.wcc_kernel_launches())


def wcc_device_allocations() -> int:
    return int(lib.wcc_device_allocations())


def wcc_cluster_minima(labels: int, n: int, minima: int, on_device: int, stream: int) -> None:
    _check(lib.wcc_cluster_minima(labels, n, minima, on_device, stream))


def wcc_number_by_minima(minima: int, n: int, labels_out: int, on_device: int,
                         stream: int) -> int:
    k = ctypes.c_int64(0)
    _check(lib.wcc_number_by_minima(minima, n, labels_out, ctypes.byref(k), on_device, stream))
    return int(k.value)


def wcc_last_error() -> str:
    return lib.wcc_last_error().decode(errors="replace")


def _check(status: int) -> int:
    if status not in (WCC_OK, WCC_PENDING):
        raise WccError(status, wcc_last_error())
    return status


def wcc_create_graph(row_off: int, cols: int, n: int, nnz: int, on_device: int,
                     stream: int) -> int:
    out = ctypes.c_void_p()
    _check(lib.wcc_create_graph(row_off, cols, n, nnz, on_device, stream, ctypes.byref(out)))
    return out.value


def wcc_create_graph_from_edges(src: int, dst: int, m: int, n: int, on_device: int,
                                stream: int) -> int:
    out = ctypes.c_void_p()
    _check(lib.wcc_create_graph_from_edges(src, dst, m, n, on_device, stream, ctypes.byref(out)))
    return out.value


def wcc_graph_num_vertices(g: int) -> int:
    return int(lib.wcc_graph_num_vertices(g))


def wcc_graph_nnz(g: int) -> int:
    return int(lib.wcc_graph_nnz(g))


def wcc_graph_export_csr(g: int, row_off: int, cols: int, on_device: int, stream: int) -> None:
    _check(lib.wcc_graph_export_csr(g, row_off, cols, on_device, stream))


def wcc_run(g: int, clustering_in: int, rule: wcc_threshold_rule | None, min_size: int,
            mode: int, clustering_out: int, on_device: int, stream: int,
            stats: wcc_stats | None = None) -> None:
    _check(lib.wcc_run(g, clustering_in, ctypes.byref(rule) if rule is not None else None,
                       min_size, mode, clustering_out, on_device, stream,
                       ctypes.byref(stats) if stats is not None else None))


def wcc_run_cm(g: int, clustering_in: int, rule: wcc_threshold_rule | None, min_size: int,
               cpm_num: int, cpm_den: int, clustering_out: int, on_device: int, stream: int,
               stats: wcc_stats | None = None) -> None:
    _check(lib.wcc_run_cm(g, clustering_in, ctypes.byref(rule) if rule is not None else None,
                          min_size, cpm_num, cpm_den, clustering_out, on_device, stream,
                          ctypes.byref(stats) if stats is not None else None))


def wcc_destroy_graph(g: int) -> None:
    lib.wcc_destroy_graph(g)


def wcc_get_tuning() -> wcc_tuning:
    t = wcc_tuning()
    _check(lib.wcc_get_tuning(ctypes.byref(t)))
    return t


def wcc_set_tuning(t: wcc_tuning) -> None:
    _check(lib.wcc_set_tuning(ctypes.byref(t)))


def wcc_autotune(g: int, clustering_in: int, rule: wcc_threshold_rule | None, min_size: int,
                 on_device: int, stream: int, cache_path: str | None):
    """(best tuning, ms of one run with it)."""
    best = wcc_tuning()
    ms = ctypes.c_double()
    _check(lib.wcc_autotune(g, clustering_in, ctypes.byref(rule) if rule is not None else None,
                            min_size, on_device, stream,
                            cache_path.encode() if cache_path else None, ctypes.byref(best),
                            ctypes.byref(ms)))
    return best, ms.value


def wcc_load_tuning(cache_path: str) -> wcc_tuning:
    t = wcc_tuning()
    _check(lib.wcc_load_tuning(cache_path.encode(), ctypes.byref(t)))
    return t


def wcc_job_start(g: int, clustering_in: int, rule: wcc_threshold_rule | None, min_size: int,
                  on_device: int, stream: int) -> int:
    out = ctypes.c_void_p()
    _check(lib.wcc_job_start(g, clustering_in, ctypes.byref(rule) if rule is not None else None,
                             min_size, on_device, stream, ctypes.byref(out)))
    return out.value


def wcc_job_step(job: int, time_budget_ms: int, stream: int) -> int:
    """WCC_OK (queue drained) or WCC_PENDING (time up, work left)."""
    return _check(lib.wcc_job_step(job, time_budget_ms, stream))


def wcc_job_save(job: int, path: str, stream: int) -> None:
    _check(lib.wcc_job_save(job, path.encode(), stream))


def wcc_job_load(g: int, path: str, stream: int) -> int:
    out = ctypes.c_void_p()
    _check(lib.wcc_job_load(g, path.encode(), stream, ctypes.byref(out)))
    return out.value


def wcc_job_finish(job: int, clustering_out: int, on_device: int, stream: int,
                   stats: wcc_stats | None) -> None:
    _check(lib.wcc_job_finish(job, clustering_out, on_device, stream,
                              ctypes.byref(stats) if stats is not None else None))


def wcc_job_destroy(job: int) -> None:
    lib.wcc_job_destroy(job)
