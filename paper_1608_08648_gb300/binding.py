"""ctypes binding of the C ABI in include/ossort.h (argument marshalling only).

Every function here has the name and the arguments of its C counterpart; all
sorting work runs in libossort.so's CUDA kernels.  If the library is missing
the first call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

OS_I32, OS_U64, OS_F64, OS_S32 = 0, 1, 2, 3
OS_DET, OS_RAN = 0, 1
OS_OK, OS_ERR_ARG, OS_ERR_WS, OS_ERR_UNSUPPORTED, OS_ERR_CUDA, OS_ERR_DEVICE = range(6)
OS_STABLE = 1
OS_REQ_HOST_INPUT = 1
OS_DET_MERGE = 2
OS_MAX_N = 1 << 31
OS_MAX_P = 4096
OS_MAX_PS = 1 << 24
OS_NOALLOC_SCRATCH_BYTES = 64 << 20
OS_SEG_MAX_CLASSES = 32
OS_SEG_MAX_PS = 4096
OS_SEG_MAX_NSEG = 1 << 26

_u32, _u64, _i32, _vp, _sz = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t


class os_params(ctypes.Structure):
    _fields_ = [("split", _i32), ("p", _u32), ("s", _u32), ("flags", _u32), ("seed", _u64)]


class os_stats(ctypes.Structure):
    _fields_ = [("p_used", _u32), ("depth", _u32), ("max_bucket", _u64), ("repart_keys", _u64),
                ("splitter_keys", _vp), ("splitter_tags", _vp), ("bucket_sizes", _vp)]


class os_counters(ctypes.Structure):
    _fields_ = [("errors", _u32), ("depth", _u32), ("repart_keys", _u64), ("bad_site", _u32),
                ("bad_index", _u32), ("split_keys", _u64)]


class os_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", _u64), ("total_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double)]


class os_seg_class(ctypes.Structure):
    _fields_ = [("max_len", _u64), ("p", _u32), ("s", _u32), ("tile", _u32), ("reserved", _u32)]


class os_seg_stats(ctypes.Structure):
    _fields_ = [("bucket_base", _vp), ("bucket_sizes", _vp), ("splitter_keys", _vp), ("splitter_tags", _vp),
                ("bucket_cap", _u64)]


class os_server_config(ctypes.Structure):
    _fields_ = [("d_arena", _vp), ("arena_bytes", _sz), ("streams", _u32), ("max_inflight", _u32)]


class os_request(ctypes.Structure):
    _fields_ = [("key_type", _i32), ("flags", _u32), ("d_keys_in", _vp), ("n", _u64), ("prm", os_params)]


class os_result(ctypes.Structure):
    _fields_ = [("ticket", _u64), ("status", _i32), ("stream", _u32), ("d_keys_out", _vp), ("n", _u64),
                ("bytes", _u64), ("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double),
                ("done_s", ctypes.c_double)]


class os_server_stats(ctypes.Structure):
    _fields_ = [("submitted", _u64), ("admitted", _u64), ("completed", _u64), ("released", _u64),
                ("queued", _u32), ("inflight", _u32), ("arena_in_use", _u64), ("arena_peak", _u64),
                ("arena_bytes", _u64), ("max_inflight_seen", _u32)]


_lib = None


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """The loaded libossort.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with paper_1608_08648_gb300.build.build() "
                              "(requires nvcc); there is no CPU fallback")
        L = ctypes.CDLL(path)
        L.os_version.restype = ctypes.c_int
        L.os_version.argtypes = []
        L.os_last_cuda_error.restype = ctypes.c_int
        L.os_last_cuda_error.argtypes = []
        L.os_strerror.restype = ctypes.c_char_p
        L.os_strerror.argtypes = [ctypes.c_int]
        L.os_workspace_size.restype = ctypes.c_int
        L.os_workspace_size.argtypes = [ctypes.c_int, _u64, ctypes.c_int, ctypes.POINTER(os_params),
                                        ctypes.POINTER(_sz)]
        L.os_workspace_size_host.restype = ctypes.c_int
        L.os_workspace_size_host.argtypes = L.os_workspace_size.argtypes
        L.os_sort.restype = ctypes.c_int
        L.os_sort.argtypes = [ctypes.c_int, _vp, _vp, _vp, _vp, _u64, ctypes.POINTER(os_params), _vp, _sz, _vp,
                              ctypes.POINTER(os_stats)]
        L.os_sort_host.restype = ctypes.c_int
        L.os_sort_host.argtypes = [ctypes.c_int, _vp, _vp, _vp, _vp, _u64, ctypes.POINTER(os_params), _vp, _sz,
                                   _vp]
        L.os_sort_noalloc.restype = ctypes.c_int
        L.os_sort_noalloc.argtypes = [ctypes.c_int, _vp, _vp, _vp, _vp, _u64, ctypes.POINTER(os_params), _vp,
                                      ctypes.POINTER(os_stats)]
        L.os_launch_count.restype = _u64
        L.os_launch_count.argtypes = []
        L.os_profile_start.restype = ctypes.c_int
        L.os_profile_start.argtypes = []
        L.os_profile_stop.restype = ctypes.c_int
        L.os_profile_stop.argtypes = [ctypes.POINTER(os_kernel_time), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.os_check.restype = ctypes.c_int
        L.os_check.argtypes = [_vp, _vp, ctypes.POINTER(_u32)]
        L.os_server_create.restype = ctypes.c_int
        L.os_server_create.argtypes = [ctypes.POINTER(os_server_config), ctypes.POINTER(_vp)]
        L.os_server_submit.restype = ctypes.c_int
        L.os_server_submit.argtypes = [_vp, ctypes.POINTER(os_request), ctypes.POINTER(_u64)]
        L.os_server_poll.restype = ctypes.c_int
        L.os_server_poll.argtypes = [_vp, ctypes.POINTER(os_result), _u32, ctypes.c_int64, ctypes.POINTER(_u32)]
        L.os_server_release.restype = ctypes.c_int
        L.os_server_release.argtypes = [_vp, _u64]
        L.os_server_get_stats.restype = ctypes.c_int
        L.os_server_get_stats.argtypes = [_vp, ctypes.POINTER(os_server_stats)]
        L.os_server_replay.restype = ctypes.c_int
        L.os_server_replay.argtypes = [_vp, ctypes.POINTER(os_request), ctypes.POINTER(ctypes.c_double), _u32,
                                       ctypes.POINTER(os_result)]
        L.os_server_destroy.restype = ctypes.c_int
        L.os_server_destroy.argtypes = [_vp]
        L.os_read_counters.restype = ctypes.c_int
        L.os_read_counters.argtypes = [_vp, _vp, ctypes.POINTER(os_counters)]
        cls_p = ctypes.POINTER(os_seg_class)
        L.os_workspace_size_segmented.restype = ctypes.c_int
        L.os_workspace_size_segmented.argtypes = [ctypes.c_int, _u64, _u32, ctypes.c_int, cls_p, _u32,
                                                  ctypes.POINTER(_sz)]
        L.os_sort_segmented.restype = ctypes.c_int
        L.os_sort_segmented.argtypes = [ctypes.c_int, _vp, _vp, _vp, _vp, _u64, _vp, _u32, cls_p, _u32, _u64,
                                        _vp, _sz, _vp, ctypes.POINTER(os_seg_stats)]
        L.os_graph_capture_segmented.restype = ctypes.c_int
        L.os_graph_capture_segmented.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, _vp, _vp, _vp, _vp, _u64, _vp,
                                                 _u32, cls_p, _u32, _u64, _vp, _sz, ctypes.POINTER(os_seg_stats)]
        L.os_graph_launch.restype = ctypes.c_int
        L.os_graph_launch.argtypes = [_vp, _vp]
        L.os_graph_kernels.restype = _u64
        L.os_graph_kernels.argtypes = [_vp]
        L.os_graph_destroy.restype = ctypes.c_int
        L.os_graph_destroy.argtypes = [_vp]
        L.os_seg_default_classes.restype = ctypes.c_int
        L.os_seg_default_classes.argtypes = [ctypes.c_int, _u64, cls_p, _u32, ctypes.POINTER(_u32)]
        L.os_tune_segmented.restype = ctypes.c_int
        L.os_tune_segmented.argtypes = [ctypes.c_int, _vp, _vp, _vp, _vp, _u64, _vp, _vp, _u32, _u64, _vp, _sz,
                                        _vp, _u32, cls_p, _u32, ctypes.POINTER(_u32), ctypes.POINTER(ctypes.c_float)]
        _lib = L
    return _lib


def os_version() -> int:
    return lib().os_version()


def os_last_cuda_error() -> int:
    return lib().os_last_cuda_error()


def os_strerror(status: int) -> str:
    return lib().os_strerror(status).decode()


def os_workspace_size(key_type: int, n: int, has_vals: bool, prm: os_params) -> tuple[int, int]:
    b = _sz(0)
    rc = lib().os_workspace_size(key_type, n, int(bool(has_vals)), ctypes.byref(prm), ctypes.byref(b))
    return rc, int(b.value)


def os_workspace_size_host(key_type: int, n: int, has_vals: bool, prm: os_params) -> tuple[int, int]:
    b = _sz(0)
    rc = lib().os_workspace_size_host(key_type, n, int(bool(has_vals)), ctypes.byref(prm), ctypes.byref(b))
    return rc, int(b.value)


def os_sort(key_type: int, d_keys_in: int, d_keys_out: int, d_vals_in: int | None, d_vals_out: int | None,
            n: int, prm: os_params, d_ws: int, ws_bytes: int, stream: int | None,
            stats: os_stats | None = None) -> int:
    return lib().os_sort(key_type, d_keys_in, d_keys_out, d_vals_in, d_vals_out, n, ctypes.byref(prm), d_ws,
                         ws_bytes, stream, ctypes.byref(stats) if stats is not None else None)


def os_sort_host(key_type: int, h_keys_in: int, h_keys_out: int, h_vals_in: int | None, h_vals_out: int | None,
                 n: int, prm: os_params, d_ws: int, ws_bytes: int, stream: int | None) -> int:
    return lib().os_sort_host(key_type, h_keys_in, h_keys_out, h_vals_in, h_vals_out, n, ctypes.byref(prm), d_ws,
                              ws_bytes, stream)


def os_sort_noalloc(key_type: int, d_keys_in: int, d_keys_out: int, d_vals_in: int | None,
                    d_vals_out: int | None, n: int, prm: os_params, stream: int | None,
                    stats: "os_stats | None" = None) -> int:
    return lib().os_sort_noalloc(key_type, d_keys_in, d_keys_out, d_vals_in, d_vals_out, n, ctypes.byref(prm),
                                 stream, ctypes.byref(stats) if stats is not None else None)


def os_check(d_ws: int, stream: int | None) -> tuple[int, int]:
    bits = _u32(0)
    rc = lib().os_check(d_ws, stream, ctypes.byref(bits))
    return rc, int(bits.value)


def os_read_counters(d_ws: int, stream: int | None) -> tuple[int, dict]:
    c = os_counters()
    rc = lib().os_read_counters(d_ws, stream, ctypes.byref(c))
    return rc, {"errors": int(c.errors), "depth": int(c.depth), "repart_keys": int(c.repart_keys),
                "bad_site": int(c.bad_site), "bad_index": int(c.bad_index), "split_keys": int(c.split_keys)}


def os_launch_count() -> int:
    return int(lib().os_launch_count())


def os_profile_start() -> int:
    return lib().os_profile_start()


def os_profile_stop(max_entries: int = 64) -> tuple[int, list[dict]]:
    arr = (os_kernel_time * max_entries)()
    cnt = ctypes.c_int(0)
    rc = lib().os_profile_stop(arr, max_entries, ctypes.byref(cnt))
    out = [{"name": arr[i].name.decode(), "launches": int(arr[i].launches), "total_ms": float(arr[i].total_ms),
            "max_ms": float(arr[i].max_ms)} for i in range(min(cnt.value, max_entries))]
    return rc, out


def _class_array(classes) -> tuple[ctypes.Array, int]:
    """classes: a sequence of os_seg_class or of (max_len, p, s, tile) tuples."""
    arr = (os_seg_class * max(1, len(classes)))()
    for i, c in enumerate(classes):
        arr[i] = c if isinstance(c, os_seg_class) else os_seg_class(int(c[0]), int(c[1]), int(c[2]), int(c[3]), 0)
    return arr, len(classes)


def os_workspace_size_segmented(key_type: int, n: int, nseg: int, has_vals: bool, classes) -> tuple[int, int]:
    """classes None: the bound covering every table os_tune_segmented may return."""
    b = _sz(0)
    if classes is None:
        rc = lib().os_workspace_size_segmented(key_type, n, nseg, int(bool(has_vals)), None, 0, ctypes.byref(b))
    else:
        arr, k = _class_array(classes)
        rc = lib().os_workspace_size_segmented(key_type, n, nseg, int(bool(has_vals)), arr, k, ctypes.byref(b))
    return rc, int(b.value)


def os_sort_segmented(key_type: int, d_keys_in: int, d_keys_out: int, d_vals_in: int | None,
                      d_vals_out: int | None, n: int, d_seg_offsets: int, nseg: int, classes, seed: int,
                      d_ws: int, ws_bytes: int, stream: int | None, stats: os_seg_stats | None = None) -> int:
    arr, k = _class_array(classes)
    return lib().os_sort_segmented(key_type, d_keys_in, d_keys_out, d_vals_in, d_vals_out, n, d_seg_offsets, nseg,
                                   arr, k, seed & ((1 << 64) - 1), d_ws, ws_bytes, stream,
                                   ctypes.byref(stats) if stats is not None else None)


def os_graph_capture_segmented(key_type: int, d_keys_in: int, d_keys_out: int, d_vals_in: int | None,
                               d_vals_out: int | None, n: int, d_seg_offsets: int, nseg: int, classes, seed: int,
                               d_ws: int, ws_bytes: int, stats: os_seg_stats | None = None) -> tuple[int, int]:
    """Returns (status, graph handle)."""
    h = _vp(None)
    arr, k = _class_array(classes)
    rc = lib().os_graph_capture_segmented(ctypes.byref(h), key_type, d_keys_in, d_keys_out, d_vals_in, d_vals_out,
                                          n, d_seg_offsets, nseg, arr, k, seed & ((1 << 64) - 1), d_ws, ws_bytes,
                                          ctypes.byref(stats) if stats is not None else None)
    return rc, (h.value or 0)


def os_graph_launch(graph: int, stream: int | None) -> int:
    return lib().os_graph_launch(graph, stream)


def os_graph_kernels(graph: int) -> int:
    return int(lib().os_graph_kernels(graph))


def os_graph_destroy(graph: int) -> int:
    return lib().os_graph_destroy(graph)


def os_seg_default_classes(key_type: int, max_len: int, max_classes: int = OS_SEG_MAX_CLASSES):
    """Returns (status, [os_seg_class, ...])."""
    arr = (os_seg_class * max_classes)()
    k = _u32(0)
    rc = lib().os_seg_default_classes(key_type, max_len, arr, max_classes, ctypes.byref(k))
    return rc, [arr[i] for i in range(k.value)]


def os_tune_segmented(key_type: int, d_keys_in: int, d_keys_out: int, d_vals_in: int | None,
                      d_vals_out: int | None, n: int, d_seg_offsets: int, h_seg_offsets: int, nseg: int, seed: int,
                      d_ws: int, ws_bytes: int, stream: int | None, reps: int = 3,
                      max_classes: int = OS_SEG_MAX_CLASSES):
    """Returns (status, [os_seg_class, ...], best_ms)."""
    arr = (os_seg_class * max_classes)()
    k = _u32(0)
    ms = ctypes.c_float(0.0)
    rc = lib().os_tune_segmented(key_type, d_keys_in, d_keys_out, d_vals_in, d_vals_out, n, d_seg_offsets,
                                 h_seg_offsets, nseg, seed & ((1 << 64) - 1), d_ws, ws_bytes, stream, reps, arr,
                                 max_classes, ctypes.byref(k), ctypes.byref(ms))
    return rc, [arr[i] for i in range(k.value)], float(ms.value)


def os_server_create(d_arena: int, arena_bytes: int, streams: int, max_inflight: int) -> tuple[int, int]:
    """Returns (status, server handle)."""
    cfg = os_server_config(d_arena, arena_bytes, streams, max_inflight)
    h = _vp(None)
    rc = lib().os_server_create(ctypes.byref(cfg), ctypes.byref(h))
    return rc, (h.value or 0)


def os_server_submit(server: int, req: os_request) -> tuple[int, int]:
    """Returns (status, ticket)."""
    t = _u64(0)
    rc = lib().os_server_submit(server, ctypes.byref(req), ctypes.byref(t))
    return rc, int(t.value)


def os_server_poll(server: int, max_results: int = 64, timeout_us: int = 0) -> tuple[int, list]:
    arr = (os_result * max(1, max_results))()
    k = _u32(0)
    rc = lib().os_server_poll(server, arr, max_results, timeout_us, ctypes.byref(k))
    return rc, [arr[i] for i in range(k.value)]


def os_server_release(server: int, ticket: int) -> int:
    return lib().os_server_release(server, ticket)


def os_server_get_stats(server: int) -> tuple[int, os_server_stats]:
    st = os_server_stats()
    rc = lib().os_server_get_stats(server, ctypes.byref(st))
    return rc, st


def os_server_replay(server: int, reqs, arrival_s) -> tuple[int, list]:
    """reqs: a sequence of os_request; arrival_s: non-decreasing seconds."""
    n = len(reqs)
    ra = (os_request * max(1, n))(*reqs)
    ta = (ctypes.c_double * max(1, n))(*arrival_s)
    res = (os_result * max(1, n))()
    rc = lib().os_server_replay(server, ra, ta, n, res)
    return rc, [res[i] for i in range(n)]


def os_server_destroy(server: int) -> int:
    return lib().os_server_destroy(server)
