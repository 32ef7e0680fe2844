"""Thin ctypes binding of libmpld (include/mpld.h): argument marshalling only.

Every step of the decomposition runs inside the library (host C++ for the
simplification, split, packing and recovery; CUDA kernels for the search).
There is no CPU fallback: if ``libmpld.so`` is missing or cannot be loaded,
importing the library raises.

Streams are CUDA stream handles as integers (for example
``torch.cuda.current_stream().cuda_stream``); 0 is the legacy default stream.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

MPLD_OK = 0
MPLD_BUDGET = 1
MPLD_TIMEOUT = 2
MPLD_E_INVALID = -1
MPLD_E_OOM = -2
MPLD_E_CUDA = -3
MPLD_E_TIMEOUT = -4
MPLD_E_TOO_LARGE = -5
MPLD_E_STATE = -6
MPLD_NO_SIMPLIFY = 1
MPLD_SINGLE_INSTANCE = 2
MPLD_HOST_ONLY = 4
MPLD_COLUMN_BFS = 8
MPLD_BICONNECTED = 16
MPLD_CLIQUE_BOUND = 32
MPLD_PARALLEL_EXACT = 64
MPLD_SPLIT_BUDGET = 128
MPLD_DENSITY_BALANCE = 256
MPLD_MAX_INSTANCE_SEGMENTS = 65535

_P = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64


class mpld_graph(ctypes.Structure):
    _fields_ = [("n_seg", _i32), ("k", _i32), ("n_conf", _i32), ("conf_u", _P), ("conf_v", _P),
                ("n_stitch", _i32), ("st_u", _P), ("st_v", _P), ("polygon_of", _P),
                ("cost_conflict", _i32), ("cost_stitch", _i32)]


class mpld_params(ctypes.Structure):
    _fields_ = [("node_budget", _i64), ("time_limit_ms", _i64), ("flags", ctypes.c_uint32),
                ("warps_per_cta", _i32), ("slot_bytes", _i32), ("cta_segments", _i32)]


class mpld_result(ctypes.Structure):
    _fields_ = [("status", _i32), ("n_components", _i32), ("n_conflicts", _i64),
                ("n_stitches", _i64), ("cost", _i64), ("nodes", _i64),
                ("n_removed_segments", _i64), ("max_component", _i32),
                ("n_budget_components", _i32), ("work", _i64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class mpld_info(ctypes.Structure):
    _fields_ = [("n_seg", _i32), ("k", _i32), ("n_components", _i32), ("max_component", _i32),
                ("n_removed_segments", _i64), ("arena_bytes", _i64), ("state_bytes", _i64),
                ("instance_segments", _i64)]


class mpld_device_instance(ctypes.Structure):
    _fields_ = [("n", _i32), ("k", _i32), ("n_conf_entries", _i32), ("n_stitch_entries", _i32),
                ("conf_ptr", _P), ("conf_nbr", _P), ("st_ptr", _P), ("st_nbr", _P),
                ("cost_conflict", _i32), ("cost_stitch", _i32)]


class mpld_server_config(ctypes.Structure):
    _fields_ = [("arena_bytes", _i64), ("result_pool_bytes", _i64), ("max_in_flight", _i32),
                ("streams", _i32), ("warps_per_cta", _i32), ("worker_threads", _i32)]


class mpld_server_stats(ctypes.Structure):
    _fields_ = [(f, _i64) for f in ("submitted", "built", "admitted", "completed", "failed",
                                    "waiting", "in_flight", "arena_used_bytes",
                                    "arena_peak_bytes", "instances_launched", "kernel_launches",
                                    "max_concurrent")]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class mpld_tune(ctypes.Structure):
    _fields_ = [("warps_per_cta", _i32), ("slot_bytes", _i32), ("ctas_per_sm", _i32),
                ("n_instances_spilled", _i32), ("ms", ctypes.c_float)]


# name -> (argtypes, restype); the names are those of include/mpld.h
_SIGS = {
    "mpld_build_matrix": ([ctypes.POINTER(mpld_graph), ctypes.POINTER(mpld_params), _P,
                           ctypes.POINTER(_P)], _i32),
    "mpld_solve": ([_P, ctypes.POINTER(mpld_params), _P, ctypes.POINTER(mpld_result), _P], _i32),
    "mpld_solve_batch": ([ctypes.POINTER(_P), _i32, ctypes.POINTER(mpld_params), ctypes.POINTER(_P),
                          ctypes.POINTER(mpld_result), _P], _i32),
    "mpld_search_batch_async": ([ctypes.POINTER(_P), _i32, ctypes.POINTER(mpld_params), _P], _i32),
    "mpld_fetch": ([_P, _P, ctypes.POINTER(mpld_result), _P], _i32),
    "mpld_search_plain_async": ([_P, ctypes.POINTER(mpld_params), _P], _i32),
    "mpld_shard_instances": ([_P, _i32, _P], _i32),
    "mpld_instance_sizes": ([_P, _P], _i32),
    "mpld_search_subset_async": ([_P, ctypes.POINTER(mpld_params), _P, _i32, _P], _i32),
    "mpld_fetch_instances": ([_P, _P, _P, _P, _P, _P], _i32),
    "mpld_finish_from": ([_P, _P, _P, _P, _P, _P, ctypes.POINTER(mpld_result)], _i32),
    "mpld_free": ([_P], None),
    "mpld_status_string": ([_i32], ctypes.c_char_p),
    "mpld_problem_info": ([_P, ctypes.POINTER(mpld_info)], _i32),
    "mpld_component_results": ([_P, _P, _P, _P, _P], _i32),
    "mpld_export_matrix": ([_P, _i32, _P, _P], _i32),
    "mpld_autotune": ([ctypes.POINTER(_P), _i32, ctypes.POINTER(mpld_params), _P,
                       ctypes.POINTER(mpld_tune)], _i32),
    "mpld_search_instance_noalloc": ([ctypes.POINTER(mpld_device_instance),
                                      ctypes.POINTER(mpld_params), _P, _P, _P], _i32),
    "mpld_server_create": ([ctypes.POINTER(mpld_server_config), ctypes.POINTER(mpld_params),
                            ctypes.POINTER(_P)], _i32),
    "mpld_server_submit": ([_P, ctypes.POINTER(mpld_graph), ctypes.c_uint32,
                            ctypes.POINTER(_i64)], _i32),
    "mpld_server_poll": ([_P, _P, _i32, ctypes.POINTER(_i32)], _i32),
    "mpld_server_result": ([_P, _i64, _P, ctypes.POINTER(mpld_result)], _i32),
    "mpld_server_stats_get": ([_P, ctypes.POINTER(mpld_server_stats)], _i32),
    "mpld_server_destroy": ([_P], None),
}

MPLD_NOALLOC_SCRATCH_BYTES = 8 << 20

_lib = None


def library(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libmpld.so (building it first if asked); raises if unavailable."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise ImportError(f"libmpld.so not built ({path}); run paper_2303_14335_gb300/build.py")
        lib = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


_probe = None


def probe_library() -> ctypes.CDLL:
    """Load libmpld_probe.so, the integer-pipe throughput probe the benchmark
    reports beside its roofline (measurement support; not part of libmpld)."""
    global _probe
    if _probe is None:
        library()   # builds both libraries when they are missing
        if not os.path.exists(_build.PROBE_LIB):
            raise ImportError(f"libmpld_probe.so not built ({_build.PROBE_LIB})")
        lib = ctypes.CDLL(_build.PROBE_LIB)
        lib.mpld_probe_int_peak.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        lib.mpld_probe_int_peak.restype = ctypes.c_int
        _probe = lib
    return _probe


class MpldError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {mpld_status_string(code)} ({code})")
        self.code = code


def _check(code: int, what: str) -> int:
    if code < 0:
        raise MpldError(code, what)
    return code


def _arr(a, dtype=np.int32) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def _ptr(a: np.ndarray | None):
    return a.ctypes.data_as(_P) if a is not None and a.size else None


def make_params(node_budget: int = 0, time_limit_ms: int = 0, flags: int = 0,
                warps_per_cta: int = 0, slot_bytes: int = 0, cta_segments: int = 0) -> mpld_params:
    return mpld_params(node_budget, time_limit_ms, flags, warps_per_cta, slot_bytes, cta_segments)


# ------------------------------------------------------------------ ABI names

def mpld_status_string(code: int) -> str:
    return library().mpld_status_string(code).decode()


def mpld_build_matrix(layout, params: mpld_params | None = None, stream: int = 0) -> "Problem":
    """Simplify, split and pack a layout; returns the handle (see Problem)."""
    n = int(layout.n_seg)
    keep = dict(cu=_arr(layout.conf_u), cv=_arr(layout.conf_v), su=_arr(layout.st_u),
                sv=_arr(layout.st_v))
    poly = getattr(layout, "polygon_of", None)
    keep["poly"] = _arr(poly) if poly is not None else None
    g = mpld_graph(n, int(layout.k), len(keep["cu"]), _ptr(keep["cu"]), _ptr(keep["cv"]),
                   len(keep["su"]), _ptr(keep["su"]), _ptr(keep["sv"]), _ptr(keep["poly"]),
                   int(getattr(layout, "cost_conflict", 10)), int(getattr(layout, "cost_stitch", 1)))
    h = _P()
    prm = params if params is not None else make_params()
    _check(library().mpld_build_matrix(ctypes.byref(g), ctypes.byref(prm), _P(stream), ctypes.byref(h)),
           "mpld_build_matrix")
    return Problem(h, n, int(layout.k))


def mpld_solve(p: "Problem", params: mpld_params | None = None, stream: int = 0):
    """Plain path: one launch per instance; returns (status, masks, result)."""
    mask = np.empty(max(p.n_seg, 1), dtype=np.int8)
    res = mpld_result()
    prm = params if params is not None else make_params()
    rc = _check(library().mpld_solve(p.handle, ctypes.byref(prm), _ptr(mask), ctypes.byref(res),
                                     _P(stream)), "mpld_solve")
    return rc, mask[:p.n_seg], res


def mpld_solve_batch(ps, params: mpld_params | None = None, stream: int = 0):
    """Batched path over several problems; returns (status, [masks], [results])."""
    ps = list(ps)
    masks = [np.empty(max(p.n_seg, 1), dtype=np.int8) for p in ps]
    hs = (_P * len(ps))(*[p.handle for p in ps])
    mp = (_P * len(ps))(*[_ptr(m) for m in masks])
    res = (mpld_result * len(ps))()
    prm = params if params is not None else make_params()
    rc = _check(library().mpld_solve_batch(hs, len(ps), ctypes.byref(prm), mp, res, _P(stream)),
                "mpld_solve_batch")
    return rc, [m[:p.n_seg] for m, p in zip(masks, ps)], list(res)


def mpld_search_batch_async(ps, params: mpld_params | None = None, stream: int = 0) -> int:
    ps = list(ps)
    hs = (_P * len(ps))(*[p.handle for p in ps])
    prm = params if params is not None else make_params()
    return _check(library().mpld_search_batch_async(hs, len(ps), ctypes.byref(prm), _P(stream)),
                  "mpld_search_batch_async")


def mpld_search_plain_async(p: "Problem", params: mpld_params | None = None, stream: int = 0) -> int:
    prm = params if params is not None else make_params()
    return _check(library().mpld_search_plain_async(p.handle, ctypes.byref(prm), _P(stream)),
                  "mpld_search_plain_async")


def mpld_fetch(p: "Problem", stream: int = 0):
    mask = np.empty(max(p.n_seg, 1), dtype=np.int8)
    res = mpld_result()
    rc = _check(library().mpld_fetch(p.handle, _ptr(mask), ctypes.byref(res), _P(stream)), "mpld_fetch")
    return rc, mask[:p.n_seg], res


def mpld_free(p: "Problem") -> None:
    p.close()


def mpld_problem_info(p: "Problem") -> mpld_info:
    info = mpld_info()
    _check(library().mpld_problem_info(p.handle, ctypes.byref(info)), "mpld_problem_info")
    return info


def mpld_component_results(p: "Problem", results: bool = True):
    """(nodes, cost, status, comp_of) of the last fetch, per search instance.

    With ``results=False`` only ``comp_of`` is filled (no fetch needed) and
    the other three are None.
    """
    info = mpld_problem_info(p)
    C = info.n_components
    comp_of = np.zeros(max(p.n_seg, 1), dtype=np.int32)
    if not results:
        _check(library().mpld_component_results(p.handle, None, None, None, _ptr(comp_of)),
               "mpld_component_results")
        return None, None, None, comp_of[:p.n_seg]
    nodes = np.zeros(max(C, 1), dtype=np.int64)
    cost = np.zeros(max(C, 1), dtype=np.int64)
    status = np.zeros(max(C, 1), dtype=np.int32)
    _check(library().mpld_component_results(p.handle, _ptr(nodes), _ptr(cost), _ptr(status),
                                            _ptr(comp_of)), "mpld_component_results")
    return nodes[:C], cost[:C], status[:C], comp_of[:p.n_seg]


def mpld_shard_instances(p: "Problem", world: int) -> np.ndarray:
    """Rank of every search instance (longest processing time first)."""
    C = mpld_problem_info(p).n_components
    owner = np.zeros(max(C, 1), dtype=np.int32)
    _check(library().mpld_shard_instances(p.handle, world, _ptr(owner)), "mpld_shard_instances")
    return owner[:C]


def mpld_instance_sizes(p: "Problem") -> np.ndarray:
    C = mpld_problem_info(p).n_components
    sizes = np.zeros(max(C, 1), dtype=np.int32)
    _check(library().mpld_instance_sizes(p.handle, _ptr(sizes)), "mpld_instance_sizes")
    return sizes[:C]


def mpld_search_subset_async(p: "Problem", instances, params: mpld_params | None = None,
                             stream: int = 0) -> int:
    inst = _arr(instances)
    prm = params or make_params()
    return _check(library().mpld_search_subset_async(p.handle, ctypes.byref(prm), _ptr(inst),
                                                     len(inst), _P(stream)),
                  "mpld_search_subset_async")


def mpld_fetch_instances(p: "Problem", stream: int = 0):
    """(nodes, cost, status, instance masks) of the last search, per instance."""
    info = mpld_problem_info(p)
    C = info.n_components
    nodes = np.zeros(max(C, 1), dtype=np.int64)
    cost = np.zeros(max(C, 1), dtype=np.int64)
    status = np.zeros(max(C, 1), dtype=np.int32)
    masks = np.zeros(max(info.instance_segments, 1), dtype=np.int8)
    _check(library().mpld_fetch_instances(p.handle, _ptr(nodes), _ptr(cost), _ptr(status),
                                          _ptr(masks), _P(stream)), "mpld_fetch_instances")
    return nodes[:C], cost[:C], status[:C], masks[:info.instance_segments]


def mpld_finish_from(p: "Problem", nodes, cost, status, inst_masks):
    """Recovery and counts from per-instance results (e.g. gathered from several ranks)."""
    nodes, cost = _arr(nodes, np.int64), _arr(cost, np.int64)
    status, inst_masks = _arr(status, np.int32), _arr(inst_masks, np.int8)
    mask = np.empty(max(p.n_seg, 1), dtype=np.int8)
    res = mpld_result()
    rc = _check(library().mpld_finish_from(p.handle, _ptr(nodes), _ptr(cost), _ptr(status),
                                           _ptr(inst_masks), _ptr(mask), ctypes.byref(res)),
                "mpld_finish_from")
    return rc, mask[:p.n_seg], res


def mpld_export_matrix(p: "Problem", comp: int) -> np.ndarray:
    """Dense 0/1 EC matrix of instance ``comp`` decoded from the packed arena."""
    dims = np.zeros(3, dtype=np.int32)
    _check(library().mpld_export_matrix(p.handle, comp, None, _ptr(dims)), "mpld_export_matrix")
    n, k, ne = (int(x) for x in dims)
    out = np.zeros((n * k, 1 + n + k * ne), dtype=np.uint8)
    _check(library().mpld_export_matrix(p.handle, comp, _ptr(out), _ptr(dims)), "mpld_export_matrix")
    return out


def mpld_autotune(ps, params: mpld_params | None = None, stream: int = 0) -> mpld_tune:
    ps = list(ps)
    hs = (_P * len(ps))(*[p.handle for p in ps])
    prm = params if params is not None else make_params()
    t = mpld_tune()
    _check(library().mpld_autotune(hs, len(ps), ctypes.byref(prm), _P(stream), ctypes.byref(t)),
           "mpld_autotune")
    return t


def mpld_search_instance_noalloc(n: int, k: int, conf_ptr: int, conf_nbr: int, n_conf_entries: int,
                                 st_ptr: int, st_nbr: int, n_stitch_entries: int, mask_out: int,
                                 result_out: int, params: mpld_params | None = None,
                                 stream: int = 0, cost_conflict: int = 10,
                                 cost_stitch: int = 1) -> int:
    """Allocation-free search of one instance given in device CSR buffers.

    Every pointer is a device address the caller owns (for example
    ``tensor.data_ptr()``): int32 CSR offsets and neighbours of the conflict
    and stitch adjacency, an int8 mask buffer of n entries and a 32-byte
    result record (int64 cost, int64 nodes, int32 status, int32 unused,
    int64 work).  The library allocates nothing: its packed copy of the
    instance and the search stacks live in a fixed array inside the
    library.  Enqueues on ``stream`` and returns without waiting.
    """
    inst = mpld_device_instance(n, k, n_conf_entries, n_stitch_entries, _P(conf_ptr),
                                _P(conf_nbr) if conf_nbr else None, _P(st_ptr),
                                _P(st_nbr) if st_nbr else None, cost_conflict, cost_stitch)
    prm = params if params is not None else make_params()
    return _check(library().mpld_search_instance_noalloc(ctypes.byref(inst), ctypes.byref(prm),
                                                          _P(mask_out), _P(result_out), _P(stream)),
                  "mpld_search_instance_noalloc")


def _graph_struct(layout):
    keep = dict(cu=_arr(layout.conf_u), cv=_arr(layout.conf_v), su=_arr(layout.st_u),
                sv=_arr(layout.st_v))
    poly = getattr(layout, "polygon_of", None)
    keep["poly"] = _arr(poly) if poly is not None else None
    g = mpld_graph(int(layout.n_seg), int(layout.k), len(keep["cu"]), _ptr(keep["cu"]),
                   _ptr(keep["cv"]), len(keep["su"]), _ptr(keep["su"]), _ptr(keep["sv"]),
                   _ptr(keep["poly"]), int(getattr(layout, "cost_conflict", 10)),
                   int(getattr(layout, "cost_stitch", 1)))
    return g, keep


def mpld_server_create(config: mpld_server_config | None = None,
                       search: mpld_params | None = None) -> "Server":
    """Start a server (device arena, ring, pinned result pool, workers)."""
    h = _P()
    cfg = config if config is not None else mpld_server_config()
    prm = search if search is not None else make_params()
    _check(library().mpld_server_create(ctypes.byref(cfg), ctypes.byref(prm), ctypes.byref(h)),
           "mpld_server_create")
    return Server(h)


def mpld_server_submit(server: "Server", layout, flags: int = 0) -> int:
    g, keep = _graph_struct(layout)
    t = _i64()
    _check(library().mpld_server_submit(server.handle, ctypes.byref(g), flags, ctypes.byref(t)),
           "mpld_server_submit")
    server.n_seg[t.value] = int(layout.n_seg)
    return t.value


def mpld_server_poll(server: "Server", max_done: int = 1024) -> list:
    buf = (_i64 * max(max_done, 1))()
    n = _i32()
    _check(library().mpld_server_poll(server.handle, ctypes.cast(buf, _P), max_done, ctypes.byref(n)),
           "mpld_server_poll")
    return [buf[i] for i in range(n.value)]


def mpld_server_result(server: "Server", ticket: int):
    """(status or error code, masks, result) of a finished ticket; releases it."""
    n = server.n_seg.pop(ticket, 0)
    mask = np.empty(max(n, 1), dtype=np.int8)
    res = mpld_result()
    rc = library().mpld_server_result(server.handle, ticket, _ptr(mask), ctypes.byref(res))
    return rc, mask[:n], res


def mpld_server_stats_get(server: "Server") -> mpld_server_stats:
    st = mpld_server_stats()
    _check(library().mpld_server_stats_get(server.handle, ctypes.byref(st)), "mpld_server_stats_get")
    return st


def mpld_server_destroy(server: "Server") -> None:
    server.close()


class Server:
    """Owning wrapper of an ``mpld_server*``."""

    def __init__(self, handle):
        self.handle = handle
        self.n_seg = {}

    def close(self):
        if self.handle is not None and self.handle.value:
            library().mpld_server_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Problem:
    """Owning wrapper of an ``mpld_problem*`` handle."""

    def __init__(self, handle: ctypes.c_void_p, n_seg: int, k: int):
        self.handle = handle
        self.n_seg = n_seg
        self.k = k

    def close(self):
        if self.handle is not None and self.handle.value:
            library().mpld_free(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
