"""ctypes binding of the C ABI in include/ossort.h (argument marshalling only).

Every function here has the name and the arguments of its C counterpart; all
sorting work runs in libossort.so's CUDA kernels.  If the library is missing
the first call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

OS_I32, OS_U64, OS_F64 = 0, 1, 2
OS_DET, OS_RAN = 0, 1
OS_OK, OS_ERR_ARG, OS_ERR_WS, OS_ERR_UNSUPPORTED, OS_ERR_CUDA, OS_ERR_DEVICE = range(6)
OS_STABLE = 1
OS_MAX_N = 1 << 31
OS_MAX_P = 4096
OS_MAX_PS = 1 << 24
OS_NOALLOC_SCRATCH_BYTES = 64 << 20

_u32, _u64, _i32, _vp, _sz = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t


class os_params(ctypes.Structure):
    _fields_ = [("split", _i32), ("p", _u32), ("s", _u32), ("flags", _u32), ("seed", _u64)]


class os_stats(ctypes.Structure):
    _fields_ = [("p_used", _u32), ("depth", _u32), ("max_bucket", _u64), ("repart_keys", _u64),
                ("splitter_keys", _vp), ("splitter_tags", _vp), ("bucket_sizes", _vp)]


class os_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", _u64), ("total_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double)]


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
        L.os_sort_noalloc.argtypes = [ctypes.c_int, _vp, _vp, _vp, _vp, _u64, ctypes.POINTER(os_params), _vp]
        L.os_launch_count.restype = _u64
        L.os_launch_count.argtypes = []
        L.os_profile_start.restype = ctypes.c_int
        L.os_profile_start.argtypes = []
        L.os_profile_stop.restype = ctypes.c_int
        L.os_profile_stop.argtypes = [ctypes.POINTER(os_kernel_time), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.os_check.restype = ctypes.c_int
        L.os_check.argtypes = [_vp, _vp, ctypes.POINTER(_u32)]
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
                    d_vals_out: int | None, n: int, prm: os_params, stream: int | None) -> int:
    return lib().os_sort_noalloc(key_type, d_keys_in, d_keys_out, d_vals_in, d_vals_out, n, ctypes.byref(prm),
                                 stream)


def os_check(d_ws: int, stream: int | None) -> tuple[int, int]:
    bits = _u32(0)
    rc = lib().os_check(d_ws, stream, ctypes.byref(bits))
    return rc, int(bits.value)


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
