"""GB300-native BLEST breadth-first search: thin Python binding of ``libblest.so``.

Every function below has the name of the C entry point it marshals (declared in
``include/blest.h``); none of them computes any part of the traversal.  Arrays
are numpy int32 on the host; the ``*_device`` calls take CUDA int32 tensors (or
raw device pointers) and an optional CUDA stream.  A non-OK status raises
:class:`BlestError`.  If the compiled library is missing it is built in-tree;
if it cannot be built or loaded the import of any entry point fails loudly --
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

__all__ = [
    "BlestError", "Stats", "RunInfo",
    "BLEST_ORDER_NONE", "BLEST_ORDER_COMPRESS", "BLEST_ORDER_BANDWIDTH", "BLEST_ORDER_AUTO",
    "BLEST_UPDATE_AUTO", "BLEST_UPDATE_EAGER", "BLEST_UPDATE_LAZY", "BLEST_PULL_POPC", "BLEST_PULL_MMA",
    "blest_graph_create", "blest_graph_create_ex", "blest_batch_create", "blest_destroy", "blest_set_option",
    "blest_get_stats", "blest_bfs", "blest_bfs_parents", "blest_msbfs", "blest_bfs_multiroot", "blest_batch_bfs",
    "blest_batch_graph_capture", "blest_batch_graph_launch", "blest_bfs_device",
    "blest_msbfs_device", "blest_bfs_multiroot_device", "blest_sync", "blest_get_run_info", "blest_get_level_times",
    "blest_get_level_arrivals", "blest_distance_stats", "blest_graph_save", "blest_graph_load",
    "blest_export",
    "blest_autotune", "blest_autotune_msbfs", "blest_autotune_multiroot", "blest_shard_begin", "blest_shard_pull",
    "blest_shard_merge", "blest_shard_finish", "blest_shard_sweep", "blest_shard_more", "blest_export_size", "blest_compute_order", "blest_is_social",
    "blest_debug_pull",
    "blest_bfs_static_scratch", "blest_server_create", "blest_server_submit", "blest_server_wait",
    "blest_server_pause", "blest_server_get_stats", "blest_server_destroy", "lib", "EXPORTED_SYMBOLS",
]

BLEST_OK = 0
STATUS_NAMES = {0: "BLEST_OK", 1: "BLEST_ERR_INVALID_ARG", 2: "BLEST_ERR_NOT_SYMMETRIC", 3: "BLEST_ERR_TOO_LARGE",
                4: "BLEST_ERR_OOM", 5: "BLEST_ERR_CUDA", 6: "BLEST_ERR_TIMEOUT", 7: "BLEST_ERR_INTERNAL"}
(BLEST_ERR_INVALID_ARG, BLEST_ERR_NOT_SYMMETRIC, BLEST_ERR_TOO_LARGE, BLEST_ERR_OOM, BLEST_ERR_CUDA,
 BLEST_ERR_TIMEOUT, BLEST_ERR_INTERNAL) = 1, 2, 3, 4, 5, 6, 7
BLEST_ORDER_NONE, BLEST_ORDER_COMPRESS, BLEST_ORDER_BANDWIDTH, BLEST_ORDER_AUTO = 0, 1, 2, 3
BLEST_UPDATE_AUTO, BLEST_UPDATE_EAGER, BLEST_UPDATE_LAZY = 0, 1, 2
BLEST_PULL_POPC, BLEST_PULL_MMA = 0, 1
BLEST_OPT_UPDATE, BLEST_OPT_PULL, BLEST_OPT_BLOCKS_PER_SM, BLEST_OPT_BARRIER_TIMEOUT_US = 0, 1, 2, 3
BLEST_OPT_RECORD_LEVELS, BLEST_OPT_UNROLL, BLEST_OPT_TEST_PHANTOM_BLOCK = 4, 5, 6
BLEST_OPT_VISITED_FILTER, BLEST_OPT_MIN_BLOCKS, BLEST_OPT_STAGE_DEPTH, BLEST_OPT_LAYOUT = 7, 8, 9, 10
BLEST_OPT_SCHEDULE = 11
BLEST_OPT_MS_PULL, BLEST_OPT_MS_CHUNK, BLEST_OPT_MS_BLOCKS_PER_SM, BLEST_OPT_MS_LEVELS = 12, 13, 14, 15
BLEST_OPT_MS_VISITED_FILTER = 16
BLEST_ARRAY_REAL_PTRS, BLEST_ARRAY_VIRTUAL_TO_REAL, BLEST_ARRAY_ROW_IDS = 0, 1, 2
BLEST_ARRAY_MASKS, BLEST_ARRAY_NEW_ID, BLEST_ARRAY_VSS_COUNT = 3, 4, 5
BLEST_ARRAY_COMPACT_OFFSETS, BLEST_ARRAY_COMPACT_ROWS, BLEST_ARRAY_COMPACT_MASKS = 6, 7, 8

EXPORTED_SYMBOLS = [
    "blest_graph_create", "blest_graph_create_ex", "blest_batch_create", "blest_destroy", "blest_set_option",
    "blest_get_stats", "blest_bfs", "blest_bfs_parents", "blest_msbfs", "blest_bfs_multiroot", "blest_batch_bfs",
    "blest_batch_graph_capture",
    "blest_batch_graph_launch", "blest_bfs_device", "blest_msbfs_device", "blest_bfs_multiroot_device", "blest_sync",
    "blest_get_run_info", "blest_get_level_times", "blest_get_level_arrivals", "blest_distance_stats", "blest_graph_save", "blest_graph_load",
    "blest_autotune", "blest_autotune_msbfs", "blest_autotune_multiroot", "blest_shard_begin",
    "blest_shard_pull", "blest_shard_merge", "blest_shard_finish", "blest_shard_sweep", "blest_shard_more",
    "blest_export_size", "blest_export", "blest_compute_order", "blest_is_social", "blest_debug_pull",
    "blest_server_create", "blest_server_submit", "blest_server_wait", "blest_server_pause", "blest_server_get_stats",
    "blest_server_destroy", "blest_bfs_static_scratch", "blest_status_string", "blest_last_error",
]


class BlestError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        self.name = STATUS_NAMES.get(status, f"status {status}")
        super().__init__(f"{where}: {self.name}: {message}")


class CreateParams(ctypes.Structure):
    _fields_ = [("window", ctypes.c_int32), ("threads", ctypes.c_int32), ("skip_symmetry_check", ctypes.c_int32),
                ("prepass", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("num_slice_sets", ctypes.c_int64),
                ("num_vss", ctypes.c_int64), ("num_slices", ctypes.c_int64), ("unpadded_slices", ctypes.c_int64),
                ("connectivity_bits", ctypes.c_int64), ("update_divergence", ctypes.c_double),
                ("compression_ratio", ctypes.c_double), ("bvss_bytes", ctypes.c_int64),
                ("state_bytes", ctypes.c_int64), ("order", ctypes.c_int32), ("update", ctypes.c_int32),
                ("order_seconds", ctypes.c_double), ("build_seconds", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class TuneResult(ctypes.Structure):
    _fields_ = [("update", ctypes.c_int32), ("pull", ctypes.c_int32), ("unroll", ctypes.c_int32),
                ("min_blocks", ctypes.c_int32), ("visited_filter", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("stage_depth", ctypes.c_int32), ("layout", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("best_ms", ctypes.c_double), ("rule_ms", ctypes.c_double)]


class MsTuneResult(ctypes.Structure):
    _fields_ = [("pull", ctypes.c_int32), ("chunk", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("levels", ctypes.c_int32), ("visited_filter", ctypes.c_int32), ("candidates", ctypes.c_int32), ("best_ms", ctypes.c_double), ("popc_ms", ctypes.c_double),
                ("mma_ms", ctypes.c_double)]


class ServerParams(ctypes.Structure):
    _fields_ = [("memory_cap_bytes", ctypes.c_int64), ("max_batch_sources", ctypes.c_int32),
                ("max_inflight", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("max_queries_per_launch", ctypes.c_int32), ("narrow_sms", ctypes.c_int32),
                ("narrow_levels", ctypes.c_int32), ("long_slots", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("sources_launched", ctypes.c_int64), ("queries_done", ctypes.c_int64),
                ("queries_waiting", ctypes.c_int64), ("memory_in_use", ctypes.c_int64), ("memory_peak", ctypes.c_int64)]


class RunInfo(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("update", ctypes.c_int32), ("pull", ctypes.c_int32),
                ("grid_blocks", ctypes.c_int32), ("threads_per_block", ctypes.c_int32), ("recorded", ctypes.c_int32),
                ("output_path", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None
_i32p = ctypes.POINTER(ctypes.c_int32)
_vp = ctypes.c_void_p


def lib():
    """Load (building in-tree if needed) ``libblest.so`` and declare its ABI."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        L = ctypes.CDLL(path)
        sig = {
            "blest_graph_create": (ctypes.c_int, [ctypes.c_int32, _i32p, _i32p, ctypes.c_int, ctypes.POINTER(_vp)]),
            "blest_graph_create_ex": (ctypes.c_int, [ctypes.c_int32, _i32p, _i32p, ctypes.c_int,
                                                     ctypes.POINTER(CreateParams), ctypes.POINTER(_vp)]),
            "blest_batch_create": (ctypes.c_int, [ctypes.c_int32, _i32p, ctypes.POINTER(_i32p), ctypes.POINTER(_i32p),
                                                  _i32p, ctypes.POINTER(CreateParams), ctypes.POINTER(_vp)]),
            "blest_destroy": (None, [_vp]),
            "blest_set_option": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int64]),
            "blest_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(Stats)]),
            "blest_bfs": (ctypes.c_int, [_vp, ctypes.c_int32, _i32p]),
            "blest_msbfs": (ctypes.c_int, [_vp, _i32p, ctypes.c_int32, _i32p]),
            "blest_bfs_parents": (ctypes.c_int, [_vp, ctypes.c_int32, _i32p, _i32p]),
            "blest_bfs_multiroot": (ctypes.c_int, [_vp, _i32p, ctypes.c_int32, _i32p]),
            "blest_batch_bfs": (ctypes.c_int, [_vp, _i32p, _i32p]),
            "blest_batch_graph_capture": (ctypes.c_int, [_vp, _vp]),
            "blest_batch_graph_launch": (ctypes.c_int, [_vp, _i32p, _vp]),
            "blest_bfs_device": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp]),
            "blest_msbfs_device": (ctypes.c_int, [_vp, _i32p, ctypes.c_int32, _vp, _vp]),
            "blest_bfs_multiroot_device": (ctypes.c_int, [_vp, _i32p, ctypes.c_int32, _vp, _vp]),
            "blest_sync": (ctypes.c_int, [_vp]),
            "blest_get_run_info": (ctypes.c_int, [_vp, ctypes.POINTER(RunInfo), _i32p, ctypes.c_int32]),
            "blest_autotune": (ctypes.c_int, [_vp, _i32p, ctypes.c_int32, ctypes.POINTER(TuneResult)]),
            "blest_autotune_msbfs": (ctypes.c_int, [_vp, _i32p, ctypes.c_int32, ctypes.POINTER(MsTuneResult)]),
            "blest_autotune_multiroot": (ctypes.c_int, [_vp, _i32p, ctypes.c_int32, ctypes.POINTER(TuneResult)]),
            "blest_shard_begin": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp, _vp]),
            "blest_shard_pull": (ctypes.c_int, [_vp, _vp, _vp]),
            "blest_shard_merge": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, ctypes.c_int32, _vp]),
            "blest_shard_finish": (ctypes.c_int, [_vp, _vp, _i32p, _vp]),
            "blest_shard_sweep": (ctypes.c_int, [_vp, _vp, _vp]),
            "blest_shard_more": (ctypes.c_int, [_vp, _i32p]),
            "blest_get_level_times": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int32]),
            "blest_get_level_arrivals": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64),
                                                        ctypes.POINTER(ctypes.c_uint64), ctypes.c_int32]),
            "blest_graph_save": (ctypes.c_int, [_vp, ctypes.c_char_p]),
            "blest_graph_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(_vp)]),
            "blest_distance_stats": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                                    ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                                    ctypes.POINTER(ctypes.c_int32)]),
            "blest_export_size": (ctypes.c_int64, [_vp, ctypes.c_int32]),
            "blest_export": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, ctypes.c_int64]),
            "blest_compute_order": (ctypes.c_int, [ctypes.c_int32, _i32p, _i32p, ctypes.c_int,
                                                   ctypes.POINTER(CreateParams), _i32p]),
            "blest_is_social": (ctypes.c_int32, [ctypes.c_int32, _i32p, _i32p]),
            "blest_debug_pull": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, ctypes.c_int32, _vp]),
            "blest_bfs_static_scratch": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, _vp, _vp, _vp, _vp,
                                                        ctypes.c_int32, _vp, ctypes.c_int32, _vp]),
            "blest_server_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int32, ctypes.POINTER(ServerParams),
                                                   ctypes.POINTER(_vp)]),
            "blest_server_submit": (ctypes.c_int, [_vp, ctypes.c_int32, _i32p, ctypes.c_int32, _vp,
                                                   ctypes.POINTER(ctypes.c_uint64)]),
            "blest_server_wait": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
            "blest_server_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(ServerStats)]),
            "blest_server_pause": (ctypes.c_int, [_vp, ctypes.c_int32]),
            "blest_server_destroy": (None, [_vp]),
            "blest_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "blest_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def _check(status: int, where: str) -> None:
    if status != BLEST_OK:
        msg = lib().blest_last_error()
        raise BlestError(status, where, msg.decode() if msg else "")


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_i32p)


PREPASS = {"hub": 0, "gorder": 1}


def _params(window=None, threads=None, skip_symmetry_check=False, prepass="hub"):
    if window is None and threads is None and not skip_symmetry_check and prepass == "hub":
        return None
    return CreateParams(int(window or 0), int(threads or 0), 1 if skip_symmetry_check else 0, PREPASS[prepass])


def _dev_ptr(x) -> int:
    """Device address of a CUDA tensor (or an int already holding one)."""
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError("expected a CUDA tensor")
        if not x.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return int(x.data_ptr())
    raise TypeError("expected a CUDA tensor or a device pointer")


CUDA_STREAM_LEGACY = 1   # cudaStreamLegacy


def _stream_ptr(stream) -> int | None:
    """cudaStream_t of a torch stream.  torch's default stream is the legacy
    NULL stream; NULL means "the handle's own stream" to the C ABI, so it is
    passed as cudaStreamLegacy instead."""
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    p = int(stream.cuda_stream)
    return p if p != 0 else CUDA_STREAM_LEGACY


# ------------------------------------------------------------------- graphs

def blest_graph_create(n: int, row_ptr, col_idx, order: int = BLEST_ORDER_NONE) -> int:
    rp, ci = _i32(row_ptr), _i32(col_idx)
    h = _vp()
    _check(lib().blest_graph_create(int(n), _ptr(rp), _ptr(ci), int(order), ctypes.byref(h)), "blest_graph_create")
    return h.value


def blest_graph_create_ex(n: int, row_ptr, col_idx, order: int = BLEST_ORDER_NONE, window=None, threads=None,
                          skip_symmetry_check=False, prepass: str = "hub") -> int:
    rp, ci = _i32(row_ptr), _i32(col_idx)
    h = _vp()
    p = _params(window, threads, skip_symmetry_check, prepass)
    _check(lib().blest_graph_create_ex(int(n), _ptr(rp), _ptr(ci), int(order), ctypes.byref(p) if p else None,
                                       ctypes.byref(h)), "blest_graph_create_ex")
    return h.value


def blest_batch_create(graphs, orders, window=None, threads=None) -> int:
    """graphs: sequence of (n, row_ptr, col_idx) in local ids."""
    G = len(graphs)
    ns = _i32([g[0] for g in graphs])
    keep = [(_i32(g[1]), _i32(g[2])) for g in graphs]
    rps = (_i32p * max(G, 1))(*[_ptr(k[0]) for k in keep])
    cis = (_i32p * max(G, 1))(*[_ptr(k[1]) for k in keep])
    od = _i32(orders)
    h = _vp()
    p = _params(window, threads)
    _check(lib().blest_batch_create(G, _ptr(ns), rps, cis, _ptr(od), ctypes.byref(p) if p else None,
                                    ctypes.byref(h)), "blest_batch_create")
    return h.value


def blest_destroy(h: int | None) -> None:
    if h:
        lib().blest_destroy(h)


def blest_set_option(h: int, key: int, value: int) -> None:
    _check(lib().blest_set_option(h, int(key), int(value)), "blest_set_option")


def blest_get_stats(h: int) -> dict:
    s = Stats()
    _check(lib().blest_get_stats(h, ctypes.byref(s)), "blest_get_stats")
    return s.as_dict()


# --------------------------------------------------------------- traversal

def _n_of(h: int) -> int:
    return int(blest_get_stats(h)["n"])


def blest_bfs(h: int, src: int, levels: np.ndarray | None = None) -> np.ndarray:
    n = _n_of(h)
    out = np.empty(n, np.int32) if levels is None else levels
    if out.dtype != np.int32 or not out.flags.c_contiguous or out.size != n:
        raise ValueError("levels must be a contiguous int32 array of n entries")
    _check(lib().blest_bfs(h, int(src), _ptr(out)), "blest_bfs")
    return out


def blest_bfs_parents(h: int, src: int) -> tuple[np.ndarray, np.ndarray]:
    n = _n_of(h)
    lv = np.empty(n, np.int32)
    par = np.empty(n, np.int32)
    _check(lib().blest_bfs_parents(h, int(src), _ptr(lv), _ptr(par)), "blest_bfs_parents")
    return lv, par


def blest_msbfs(h: int, srcs, levels: np.ndarray | None = None) -> np.ndarray:
    s = _i32(srcs)
    n = _n_of(h)
    out = np.empty((len(s), n), np.int32) if levels is None else levels
    if out.dtype != np.int32 or not out.flags.c_contiguous or out.size != len(s) * n:
        raise ValueError("levels must be a contiguous int32 array of k*n entries")
    _check(lib().blest_msbfs(h, _ptr(s), len(s), _ptr(out)), "blest_msbfs")
    return out


def blest_bfs_multiroot(h: int, srcs, levels: np.ndarray | None = None) -> np.ndarray:
    s = _i32(srcs)
    n = _n_of(h)
    out = np.empty(n, np.int32) if levels is None else levels
    _check(lib().blest_bfs_multiroot(h, _ptr(s), len(s), _ptr(out)), "blest_bfs_multiroot")
    return out


def blest_batch_bfs(h: int, srcs_local, levels: np.ndarray | None = None) -> np.ndarray:
    s = _i32(srcs_local)
    n = _n_of(h)
    out = np.empty(n, np.int32) if levels is None else levels
    _check(lib().blest_batch_bfs(h, _ptr(s), _ptr(out)), "blest_batch_bfs")
    return out


def blest_batch_graph_capture(h: int, d_levels) -> None:
    _check(lib().blest_batch_graph_capture(h, _dev_ptr(d_levels)), "blest_batch_graph_capture")


def blest_batch_graph_launch(h: int, srcs_local, stream=None) -> None:
    s = _i32(srcs_local)
    _check(lib().blest_batch_graph_launch(h, _ptr(s), _stream_ptr(stream)), "blest_batch_graph_launch")


def blest_bfs_device(h: int, src: int, d_levels, stream=None) -> None:
    _check(lib().blest_bfs_device(h, int(src), _dev_ptr(d_levels), _stream_ptr(stream)), "blest_bfs_device")


def blest_msbfs_device(h: int, srcs, d_levels, stream=None) -> None:
    s = _i32(srcs)
    _check(lib().blest_msbfs_device(h, _ptr(s), len(s), _dev_ptr(d_levels), _stream_ptr(stream)),
           "blest_msbfs_device")


def blest_bfs_multiroot_device(h: int, srcs, d_levels, stream=None) -> None:
    s = _i32(srcs)
    _check(lib().blest_bfs_multiroot_device(h, _ptr(s), len(s), _dev_ptr(d_levels), _stream_ptr(stream)),
           "blest_bfs_multiroot_device")


def blest_sync(h: int) -> None:
    _check(lib().blest_sync(h), "blest_sync")


def blest_get_run_info(h: int, cap: int = 0) -> tuple[dict, np.ndarray]:
    info = RunInfo()
    buf = np.zeros(max(cap, 1), np.int32)
    _check(lib().blest_get_run_info(h, ctypes.byref(info), _ptr(buf), int(cap)), "blest_get_run_info")
    d = {f: getattr(info, f) for f, _ in info._fields_}
    return d, buf[:max(0, min(cap, d["recorded"]))].copy()


def blest_autotune(h: int, srcs) -> dict:
    s = _i32(srcs)
    r = TuneResult()
    _check(lib().blest_autotune(h, _ptr(s), len(s), ctypes.byref(r)), "blest_autotune")
    return {f: getattr(r, f) for f, _ in r._fields_}


def blest_shard_begin(h: int, rank: int, world: int, src: int, d_levels, stream=None) -> None:
    _check(lib().blest_shard_begin(h, int(rank), int(world), int(src), _dev_ptr(d_levels), _stream_ptr(stream)),
           "blest_shard_begin")


def blest_shard_pull(h: int, d_words, stream=None) -> None:
    _check(lib().blest_shard_pull(h, _dev_ptr(d_words), _stream_ptr(stream)), "blest_shard_pull")


def blest_shard_merge(d_dst, d_src, words: int, count: int, stream=None) -> None:
    _check(lib().blest_shard_merge(_dev_ptr(d_dst), _dev_ptr(d_src), int(words), int(count), _stream_ptr(stream)),
           "blest_shard_merge")


def blest_shard_finish(h: int, d_merged, stream=None) -> bool:
    more = ctypes.c_int32(0)
    _check(lib().blest_shard_finish(h, _dev_ptr(d_merged), ctypes.byref(more), _stream_ptr(stream)),
           "blest_shard_finish")
    return bool(more.value)


def blest_shard_sweep(h: int, d_merged, stream=None) -> None:
    _check(lib().blest_shard_sweep(h, _dev_ptr(d_merged), _stream_ptr(stream)), "blest_shard_sweep")


def blest_shard_more(h: int) -> bool:
    more = ctypes.c_int32(0)
    _check(lib().blest_shard_more(h, ctypes.byref(more)), "blest_shard_more")
    return bool(more.value)


def blest_autotune_multiroot(h: int, srcs) -> dict:
    s = _i32(srcs)
    r = TuneResult()
    _check(lib().blest_autotune_multiroot(h, _ptr(s), len(s), ctypes.byref(r)), "blest_autotune_multiroot")
    return {f: getattr(r, f) for f, _ in r._fields_}


def blest_autotune_msbfs(h: int, srcs) -> dict:
    s = _i32(srcs)
    r = MsTuneResult()
    _check(lib().blest_autotune_msbfs(h, _ptr(s), len(s), ctypes.byref(r)), "blest_autotune_msbfs")
    return {f: getattr(r, f) for f, _ in r._fields_}


def blest_get_level_times(h: int, cap: int = 1 << 17) -> np.ndarray:
    out = np.zeros(cap, np.uint64)
    _check(lib().blest_get_level_times(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), int(cap)),
           "blest_get_level_times")
    return out


def blest_get_level_arrivals(h: int, cap: int, phase: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """(first, last) globaltimer stamps at which blocks finished each level's
    stage 1 (phase 0) or finalisation sweep (phase 1)."""
    first = np.zeros(cap, np.uint64)
    last = np.zeros(cap, np.uint64)
    p = ctypes.POINTER(ctypes.c_uint64)
    _check(lib().blest_get_level_arrivals(h, int(phase), first.ctypes.data_as(p), last.ctypes.data_as(p), int(cap)),
           "blest_get_level_arrivals")
    return first, last


def blest_graph_save(h: int, path: str) -> None:
    _check(lib().blest_graph_save(h, os.fsencode(path)), "blest_graph_save")


def blest_graph_load(path: str) -> int:
    out = _vp()
    _check(lib().blest_graph_load(os.fsencode(path), ctypes.byref(out)), "blest_graph_load")
    return out.value


def blest_distance_stats(h: int, srcs) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(reached, sum of distances, eccentricity) per source, each of len(srcs)."""
    s = _i32(srcs)
    k = len(s)
    reached = np.zeros(k, np.int64)
    total = np.zeros(k, np.int64)
    ecc = np.zeros(k, np.int32)
    p64 = ctypes.POINTER(ctypes.c_int64)
    _check(lib().blest_distance_stats(h, s.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), k,
                                      reached.ctypes.data_as(p64), total.ctypes.data_as(p64),
                                      ecc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "blest_distance_stats")
    return reached, total, ecc


# ------------------------------------------------------------------ export

_EXPORT_DTYPES = {BLEST_ARRAY_MASKS: np.uint32, BLEST_ARRAY_COMPACT_MASKS: np.uint32}


def blest_export_size(h: int, which: int) -> int:
    return int(lib().blest_export_size(h, int(which)))


def blest_export(h: int, which: int) -> np.ndarray:
    nbytes = blest_export_size(h, which)
    if nbytes < 0:
        raise BlestError(1, "blest_export", "unknown array")
    out = np.empty(nbytes // 4, _EXPORT_DTYPES.get(which, np.int32))
    _check(lib().blest_export(h, int(which), out.ctypes.data_as(_vp), nbytes), "blest_export")
    return out


# --------------------------------------------------------------- host only

def blest_compute_order(n: int, row_ptr, col_idx, order: int, window=None, threads=None,
                        prepass: str = "hub") -> np.ndarray:
    rp, ci = _i32(row_ptr), _i32(col_idx)
    out = np.empty(max(n, 1), np.int32)
    p = _params(window, threads, prepass=prepass)
    _check(lib().blest_compute_order(int(n), _ptr(rp), _ptr(ci), int(order), ctypes.byref(p) if p else None,
                                     _ptr(out)), "blest_compute_order")
    return out[:n]


def blest_is_social(n: int, row_ptr, col_idx) -> bool:
    rp, ci = _i32(row_ptr), _i32(col_idx)
    r = lib().blest_is_social(int(n), _ptr(rp), _ptr(ci))
    if r < 0:
        _check(-r, "blest_is_social")
    return bool(r)


def blest_debug_pull(d_masks, d_alpha, tiles: int, pull: int, d_hits) -> None:
    _check(lib().blest_debug_pull(_dev_ptr(d_masks), _dev_ptr(d_alpha), int(tiles), int(pull), _dev_ptr(d_hits)),
           "blest_debug_pull")


def blest_bfs_static_scratch(n: int, num_vss: int, d_real_ptrs, d_row_ids, d_masks, d_new_id, src_bvss: int,
                             d_levels, update: int = BLEST_UPDATE_LAZY, stream=None) -> None:
    """Allocation-free single-source traversal (see include/blest.h); device
    arguments are CUDA tensors or raw pointers, d_new_id may be None."""
    _check(lib().blest_bfs_static_scratch(int(n), int(num_vss), _dev_ptr(d_real_ptrs), _dev_ptr(d_row_ids),
                                          _dev_ptr(d_masks), None if d_new_id is None else _dev_ptr(d_new_id),
                                          int(src_bvss), _dev_ptr(d_levels), int(update), _stream_ptr(stream)),
           "blest_bfs_static_scratch")


def blest_server_create(handles, memory_cap_bytes=0, max_batch_sources=0, max_inflight=0, blocks_per_sm=0,
                        max_queries_per_launch=0, narrow_sms=0, narrow_levels=0, long_slots=0) -> int:
    arr = (_vp * len(handles))(*handles)
    p = ServerParams(int(memory_cap_bytes), int(max_batch_sources), int(max_inflight), int(blocks_per_sm),
                     int(max_queries_per_launch), int(narrow_sms), int(narrow_levels), int(long_slots))
    s = _vp()
    _check(lib().blest_server_create(arr, len(handles), ctypes.byref(p), ctypes.byref(s)), "blest_server_create")
    return s.value


def blest_server_submit(server: int, graph: int, srcs, levels=None) -> int:
    """levels: None, a numpy int32 array (host) or a CUDA tensor / device pointer of k*n int32."""
    s = _i32(srcs)
    if levels is None:
        ptr = None
    elif isinstance(levels, np.ndarray):
        if levels.dtype != np.int32 or not levels.flags.c_contiguous:
            raise ValueError("levels must be a contiguous int32 array")
        ptr = levels.ctypes.data
    else:
        ptr = _dev_ptr(levels)
    t = ctypes.c_uint64()
    _check(lib().blest_server_submit(server, int(graph), _ptr(s), len(s), ptr, ctypes.byref(t)), "blest_server_submit")
    return t.value


def blest_server_wait(server: int, ticket: int, timeout_s: float = -1.0) -> float:
    lat = ctypes.c_double()
    _check(lib().blest_server_wait(server, ctypes.c_uint64(ticket), float(timeout_s), ctypes.byref(lat)),
           "blest_server_wait")
    return lat.value


def blest_server_pause(server: int, paused: bool) -> None:
    _check(lib().blest_server_pause(server, 1 if paused else 0), "blest_server_pause")


def blest_server_get_stats(server: int) -> dict:
    st = ServerStats()
    _check(lib().blest_server_get_stats(server, ctypes.byref(st)), "blest_server_get_stats")
    return {f: getattr(st, f) for f, _ in st._fields_}


def blest_server_destroy(server: int | None) -> None:
    if server:
        lib().blest_server_destroy(server)


class BlestGraph:
    """Owning wrapper: ``with BlestGraph(n, rp, ci, order) as g: g.bfs(src)``."""

    def __init__(self, n, row_ptr, col_idx, order=BLEST_ORDER_NONE, **kw):
        self.h = blest_graph_create_ex(n, row_ptr, col_idx, order, **kw) if kw else \
            blest_graph_create(n, row_ptr, col_idx, order)

    def close(self):
        blest_destroy(self.h)
        self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.close()
        except Exception:
            pass

    def bfs(self, src):
        return blest_bfs(self.h, src)

    def msbfs(self, srcs):
        return blest_msbfs(self.h, srcs)

    def stats(self):
        return blest_get_stats(self.h)

    def set_option(self, key, value):
        blest_set_option(self.h, key, value)
