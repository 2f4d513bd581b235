"""GB300-native oversampling sample sort (SqDet / SqRan of Gerbessiotis, arXiv 1608.08648).

The sort runs in libossort.so (hand-written CUDA for sm_103a behind the C ABI of
include/ossort.h).  PyTorch only provides device memory and streams here.

    import paper_1608_08648_gb300 as oss
    out = oss.sort(keys_cuda_tensor, split="ran", p=1024, s=16, seed=1)
"""
from __future__ import annotations

import ctypes

from .binding import (OS_DET, OS_F64, OS_I32, OS_OK, OS_RAN, OS_STABLE, OS_U64, os_check,  # noqa: F401
                      os_kernel_time, os_last_cuda_error, os_launch_count, os_params, os_profile_start,
                      os_profile_stop, os_sort, os_sort_host, os_stats, os_strerror, os_version, os_workspace_size,
                      os_workspace_size_host)

KEY_TYPES = {"i32": OS_I32, "u64": OS_U64, "f64": OS_F64}
SPLITS = {"det": OS_DET, "ran": OS_RAN}


class OssortError(RuntimeError):
    def __init__(self, status: int, what: str = "os_sort"):
        from .binding import os_last_cuda_error as _lce
        super().__init__(f"{what} failed: status {status} ({os_strerror(status)}), cuda error {_lce()}")
        self.status = status


def _key_type(t, key_type):
    import torch
    if key_type is not None:
        return KEY_TYPES[key_type] if isinstance(key_type, str) else int(key_type)
    if t.dtype == torch.int32:
        return OS_I32
    if t.dtype == torch.float64:
        return OS_F64
    if t.dtype in (torch.int64,) + ((torch.uint64,) if hasattr(torch, "uint64") else ()):
        return OS_U64
    raise TypeError(f"unsupported key dtype {t.dtype}: int32, float64 or (u)int64")


def params(split="ran", p=1024, s=16, seed=0, flags=OS_STABLE) -> os_params:
    return os_params(SPLITS[split] if isinstance(split, str) else int(split), int(p), int(s), int(flags),
                     int(seed) & ((1 << 64) - 1))


def workspace_bytes(n, key_type="i32", has_vals=False, split="ran", p=1024, s=16) -> int:
    kt = KEY_TYPES[key_type] if isinstance(key_type, str) else int(key_type)
    rc, b = os_workspace_size(kt, int(n), has_vals, params(split, p, s))
    if rc != OS_OK:
        raise OssortError(rc, "os_workspace_size")
    return b


def sort(keys, values=None, *, split="ran", p=1024, s=16, seed=0, out=None, values_out=None, workspace=None,
         stream=None, key_type=None, stats=False):
    """Sort a 1-D CUDA tensor of keys (int32, float64 or 64-bit unsigned held in int64/uint64),
    optionally carrying an int32/uint32 payload, stably.  Returns (keys_out, values_out, stats)."""
    import torch
    assert keys.is_cuda and keys.dim() == 1 and keys.is_contiguous()
    kt = _key_type(keys, key_type)
    n = keys.numel()
    prm = params(split, p, s, seed)
    hv = values is not None
    if out is None:
        out = torch.empty_like(keys)
    if hv:
        assert values.is_cuda and values.numel() == n and values.element_size() == 4
        if values_out is None:
            values_out = torch.empty_like(values)
    rc, need = os_workspace_size(kt, n, hv, prm)
    if rc != OS_OK:
        raise OssortError(rc, "os_workspace_size")
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=keys.device)
    st = stream if stream is not None else torch.cuda.current_stream(keys.device)
    st_handle = st.cuda_stream if hasattr(st, "cuda_stream") else int(st)
    info = None
    st_struct = None
    if stats:
        import numpy as np
        kb = 4 if kt == OS_I32 else 8
        spl_k = np.zeros(max(p - 1, 1) * kb, dtype=np.uint8)
        spl_t = np.zeros(max(p - 1, 1), dtype=np.uint64)
        sizes = np.zeros(p, dtype=np.uint64)
        st_struct = os_stats(0, 0, 0, 0, spl_k.ctypes.data_as(ctypes.c_void_p),
                             spl_t.ctypes.data_as(ctypes.c_void_p), sizes.ctypes.data_as(ctypes.c_void_p))
    rc = os_sort(kt, keys.data_ptr(), out.data_ptr(), values.data_ptr() if hv else None,
                 values_out.data_ptr() if hv else None, n, prm, workspace.data_ptr(), workspace.numel(),
                 st_handle, st_struct)
    if rc != OS_OK:
        raise OssortError(rc)
    if stats:
        dt = {OS_I32: np.int32, OS_U64: np.uint64, OS_F64: np.float64}[kt]
        pu = int(st_struct.p_used)
        info = {"p_used": pu, "depth": int(st_struct.depth), "max_bucket": int(st_struct.max_bucket),
                "repart_keys": int(st_struct.repart_keys),
                "spl_keys": spl_k.view(dt)[: (p - 1 if pu > 1 else 0)], "spl_tags": spl_t[: (p - 1 if pu > 1 else 0)],
                "bucket_sizes": sizes}
    return out, values_out, info
