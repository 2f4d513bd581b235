"""GB300-native oversampling sample sort (SqDet / SqRan of Gerbessiotis, arXiv 1608.08648).

The sort runs in libossort.so (hand-written CUDA for sm_103a behind the C ABI of
include/ossort.h).  PyTorch only provides device memory and streams here.

    import paper_1608_08648_gb300 as oss
    out = oss.sort(keys_cuda_tensor, split="ran", p=1024, s=16, seed=1)
"""
from __future__ import annotations

import ctypes

from .binding import (OS_DET, OS_F64, OS_I32, OS_OK, OS_RAN, OS_S32, OS_STABLE, OS_U64, os_check,  # noqa: F401
                      os_graph_capture_segmented, os_graph_destroy, os_graph_kernels, os_graph_launch,
                      os_kernel_time, os_last_cuda_error, os_launch_count, os_params, os_profile_start,
                      os_profile_stop, os_read_counters, os_seg_class, os_seg_default_classes, os_seg_stats,
                      os_sort, os_sort_host,
                      os_sort_segmented, os_stats, os_strerror, os_tune_segmented, os_version, os_workspace_size,
                      os_workspace_size_host, os_workspace_size_segmented)

KEY_TYPES = {"i32": OS_I32, "u64": OS_U64, "f64": OS_F64, "s32": OS_S32}
SPLITS = {"det": OS_DET, "ran": OS_RAN}


class OssortError(RuntimeError):
    def __init__(self, status: int, what: str = "os_sort"):
        from .binding import os_last_cuda_error as _lce
        super().__init__(f"{what} failed: status {status} ({os_strerror(status)}), cuda error {_lce()}")
        self.status = status


def _key_type_host(t, key_type):
    import torch
    if key_type is not None:
        return KEY_TYPES[key_type] if isinstance(key_type, str) else int(key_type)
    return {torch.int32: OS_I32, torch.float64: OS_F64, torch.int64: OS_U64}[t.dtype]


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
    if t.dtype == torch.uint8:
        return OS_S32
    raise TypeError(f"unsupported key dtype {t.dtype}: int32, float64, (u)int64 or uint8 (32-byte strings)")


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
         stream=None, key_type=None, stats=False, det_merge=False):
    """Sort a CUDA tensor of keys (1-D int32, float64 or 64-bit unsigned held in int64/uint64;
    or uint8 of shape (n, 32): 32-byte strings in memcmp order), optionally carrying an
    int32/uint32 payload, stably.  det_merge (SqDet only): steps 4-5 as in Algorithm 1 (split the
    sorted sequences, merge every bucket's pieces).  Returns (keys_out, values_out, stats)."""
    import torch
    assert keys.is_cuda and keys.is_contiguous()
    kt = _key_type(keys, key_type)
    if kt == OS_S32:
        assert keys.dtype == torch.uint8 and keys.numel() % 32 == 0
        n = keys.numel() // 32
    else:
        assert keys.dim() == 1
        n = keys.numel()
    prm = params(split, p, s, seed, OS_STABLE | (2 if det_merge else 0))
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
        kb = {OS_I32: 4, OS_S32: 32}.get(kt, 8)
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
        dt = {OS_I32: np.int32, OS_U64: np.uint64, OS_F64: np.float64, OS_S32: np.uint8}[kt]
        pu = int(st_struct.p_used)
        sk = spl_k.view(dt).reshape(-1, 32) if kt == OS_S32 else spl_k.view(dt)
        info = {"p_used": pu, "depth": int(st_struct.depth), "max_bucket": int(st_struct.max_bucket),
                "repart_keys": int(st_struct.repart_keys),
                "spl_keys": sk[: (p - 1 if pu > 1 else 0)], "spl_tags": spl_t[: (p - 1 if pu > 1 else 0)],
                "bucket_sizes": sizes}
    return out, values_out, info


# ---- batched segmented sort ---------------------------------------------------

def default_classes(key_type, max_len):
    """The library's starting class table for segments up to max_len, as
    (max_len, p, s, tile) tuples."""
    kt = KEY_TYPES[key_type] if isinstance(key_type, str) else int(key_type)
    rc, cl = os_seg_default_classes(kt, int(max_len))
    if rc != OS_OK:
        raise OssortError(rc, "os_seg_default_classes")
    return [(c.max_len, c.p, c.s, c.tile) for c in cl]


def _seg_common(keys, offsets, values, key_type):
    import torch
    assert keys.is_cuda and keys.dim() == 1 and keys.is_contiguous()
    assert offsets.is_cuda and offsets.dtype == torch.int64 and offsets.dim() == 1 and offsets.is_contiguous()
    kt = _key_type(keys, key_type)
    if values is not None:
        assert values.is_cuda and values.numel() == keys.numel() and values.element_size() == 4
    return kt, keys.numel(), offsets.numel() - 1


def segmented_workspace_bytes(n, nseg, key_type="f64", has_vals=False, classes=None) -> int:
    """Workspace of os_sort_segmented (classes None: any table the tuner may return)."""
    kt = KEY_TYPES[key_type] if isinstance(key_type, str) else int(key_type)
    rc, b = os_workspace_size_segmented(kt, int(n), int(nseg), has_vals, classes)
    if rc != OS_OK:
        raise OssortError(rc, "os_workspace_size_segmented")
    return b


def sort_segmented(keys, offsets, values=None, *, classes=None, seed=0, out=None, values_out=None,
                   workspace=None, stream=None, key_type=None, stats=False):
    """Sort every segment [offsets[g], offsets[g+1]) of a 1-D CUDA tensor on its own
    (os_sort_segmented).  offsets: CUDA int64 tensor of nseg + 1 entries.  classes:
    (max_len, p, s, tile) tuples; None takes default_classes for the longest segment
    (which reads the offsets back to the host).  Returns (keys_out, values_out, stats),
    stats a dict of CUDA tensors (bucket_base, bucket_sizes, splitter_keys,
    splitter_tags) when requested."""
    import torch
    kt, n, nseg = _seg_common(keys, offsets, values, key_type)
    if classes is None:
        max_len = int((offsets[1:] - offsets[:-1]).max().item()) if nseg > 0 else 0
        classes = default_classes(kt, max_len)
    if out is None:
        out = torch.empty_like(keys)
    hv = values is not None
    if hv and values_out is None:
        values_out = torch.empty_like(values)
    rc, need = os_workspace_size_segmented(kt, n, nseg, hv, classes)
    if rc != OS_OK:
        raise OssortError(rc, "os_workspace_size_segmented")
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=keys.device)
    st = stream if stream is not None else torch.cuda.current_stream(keys.device)
    st_handle = st.cuda_stream if hasattr(st, "cuda_stream") else int(st)
    info, so = None, None
    if stats:
        cap = nseg * max(int(c[1]) for c in classes) + 1
        info = {"bucket_base": torch.zeros(nseg + 1, dtype=torch.int32, device=keys.device),
                "bucket_sizes": torch.zeros(cap, dtype=torch.int32, device=keys.device),
                "splitter_keys": torch.zeros(cap, dtype=keys.dtype, device=keys.device),
                "splitter_tags": torch.zeros(cap, dtype=torch.int32, device=keys.device)}
        so = os_seg_stats(info["bucket_base"].data_ptr(), info["bucket_sizes"].data_ptr(),
                          info["splitter_keys"].data_ptr(), info["splitter_tags"].data_ptr(), cap)
    rc = os_sort_segmented(kt, keys.data_ptr(), out.data_ptr(), values.data_ptr() if hv else None,
                           values_out.data_ptr() if hv else None, n, offsets.data_ptr(), nseg, classes, seed,
                           workspace.data_ptr(), workspace.numel(), st_handle, so)
    if rc != OS_OK:
        raise OssortError(rc, "os_sort_segmented")
    return out, values_out, info


class SegmentedGraph:
    """A CUDA graph of one os_sort_segmented call on fixed buffers
    (os_graph_capture_segmented); launch() replays the whole batched sort on a
    stream.  The keys, payloads and offsets may be rewritten in place between
    launches."""

    def __init__(self, keys, offsets, out, values=None, values_out=None, *, classes, seed=0, workspace=None,
                 key_type=None):
        import torch
        kt, n, nseg = _seg_common(keys, offsets, values, key_type)
        hv = values is not None
        rc, need = os_workspace_size_segmented(kt, n, nseg, hv, classes)
        if rc != OS_OK:
            raise OssortError(rc, "os_workspace_size_segmented")
        if workspace is None or workspace.numel() < need:
            workspace = torch.empty(need, dtype=torch.uint8, device=keys.device)
        self._keep = (keys, offsets, out, values, values_out, workspace)
        rc, self.handle = os_graph_capture_segmented(kt, keys.data_ptr(), out.data_ptr(),
                                                     values.data_ptr() if hv else None,
                                                     values_out.data_ptr() if hv else None, n, offsets.data_ptr(),
                                                     nseg, classes, seed, workspace.data_ptr(), workspace.numel())
        if rc != OS_OK:
            raise OssortError(rc, "os_graph_capture_segmented")
        self.kernels = os_graph_kernels(self.handle)
        self.workspace = workspace

    def launch(self, stream=None):
        import torch
        st = stream if stream is not None else torch.cuda.current_stream()
        rc = os_graph_launch(self.handle, st.cuda_stream if hasattr(st, "cuda_stream") else int(st))
        if rc != OS_OK:
            raise OssortError(rc, "os_graph_launch")

    def close(self):
        if getattr(self, "handle", 0):
            os_graph_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tune_segmented(keys, offsets, values=None, *, seed=0, reps=3, workspace=None, stream=None, key_type=None):
    """os_tune_segmented on the caller's batch: returns (classes, best_ms), classes as
    (max_len, p, s, tile) tuples."""
    import numpy as np
    import torch
    kt, n, nseg = _seg_common(keys, offsets, values, key_type)
    hv = values is not None
    rc, need = os_workspace_size_segmented(kt, n, nseg, hv, None)
    if rc != OS_OK:
        raise OssortError(rc, "os_workspace_size_segmented")
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=keys.device)
    h_off = np.ascontiguousarray(offsets.cpu().numpy().astype(np.uint64))
    out = torch.empty_like(keys)
    vout = torch.empty_like(values) if hv else None
    st = stream if stream is not None else torch.cuda.current_stream(keys.device)
    rc, cl, ms = os_tune_segmented(kt, keys.data_ptr(), out.data_ptr(), values.data_ptr() if hv else None,
                                   vout.data_ptr() if hv else None, n, offsets.data_ptr(), h_off.ctypes.data, nseg,
                                   seed, workspace.data_ptr(), workspace.numel(), st.cuda_stream, reps)
    if rc != OS_OK:
        raise OssortError(rc, "os_tune_segmented")
    return [(c.max_len, c.p, c.s, c.tile) for c in cl], ms


# ---- serving loop -----------------------------------------------------------------

class Server:
    """A sort server over one device arena (os_server_*).  submit() takes a resident
    CUDA tensor of keys; poll() returns finished requests with their sorted keys as a
    tensor view into the arena, valid until release(ticket)."""

    def __init__(self, arena_bytes, streams=8, max_inflight=64, device=None):
        import torch
        from . import binding as _b
        self._b = _b
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=device or "cuda")
        rc, self.handle = _b.os_server_create(self.arena.data_ptr(), self.arena.numel(), streams, max_inflight)
        if rc != OS_OK:
            raise OssortError(rc, "os_server_create")
        self._inputs = {}      # ticket -> (input tensor, dtype): kept alive while the request may read it

    def request(self, keys, split="ran", p=1024, s=16, seed=0, key_type=None):
        """An os_request for keys resident on the device, or (a CPU tensor, best
        pinned) keys the server copies in itself when it admits the request."""
        kt = _key_type(keys, key_type) if keys.is_cuda else _key_type_host(keys, key_type)
        flags = 0 if keys.is_cuda else self._b.OS_REQ_HOST_INPUT
        return self._b.os_request(kt, flags, keys.data_ptr(), keys.numel(), params(split, p, s, seed))

    def submit(self, keys, split="ran", p=1024, s=16, seed=0, key_type=None):
        assert keys.dim() == 1 and keys.is_contiguous()
        rc, t = self._b.os_server_submit(self.handle, self.request(keys, split, p, s, seed, key_type))
        if rc != OS_OK:
            raise OssortError(rc, "os_server_submit")
        self._inputs[t] = (keys, keys.dtype)
        return t

    def poll(self, max_results=64, timeout_us=0):
        """[(ticket, status, output tensor, record)] of newly finished requests."""
        rc, res = self._b.os_server_poll(self.handle, max_results, timeout_us)
        if rc != OS_OK:
            raise OssortError(rc, "os_server_poll")
        out = []
        for r in res:
            keys, dt = self._inputs.pop(r.ticket, (None, None))
            view = None
            if keys is not None and r.status == OS_OK:
                off = r.d_keys_out - self.arena.data_ptr()
                view = self.arena[off:off + r.n * keys.element_size()].view(dt)
            out.append((r.ticket, r.status, view, r))
        return out

    def release(self, ticket):
        rc = self._b.os_server_release(self.handle, ticket)
        if rc != OS_OK:
            raise OssortError(rc, "os_server_release")

    def stats(self):
        rc, st = self._b.os_server_get_stats(self.handle)
        return {f: getattr(st, f) for f, _ in st._fields_}

    def replay(self, requests, arrival_s):
        """Open-loop replay (os_server_replay): request i is submitted arrival_s[i]
        seconds after the start; returns the os_result records in request order."""
        rc, res = self._b.os_server_replay(self.handle, requests, arrival_s)
        if rc != OS_OK:
            raise OssortError(rc, "os_server_replay")
        return res

    def close(self):
        if getattr(self, "handle", 0):
            self._b.os_server_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
