"""Python access to the CPU oracle (plain C, ``oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``.  The library never imports it.

The oracle follows SqDet (Algorithm 1) and SqRan (Algorithm 2) step by step, with
the tagged duplicate handling of Section 2.2; see ``oracle.c`` for the readings of
the paper it takes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

KT = {"i32": 0, "u64": 1, "f64": 2, "s32": 3}
NP_DT = {"i32": np.int32, "u64": np.uint64, "f64": np.float64, "s32": np.uint8}
SPLIT = {"det": 0, "ran": 1}

_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C11, -O2) if it is missing or stale."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stale = force or not os.path.exists(_LIB) or any(
        os.path.getmtime(f) > os.path.getmtime(_LIB) for f in (_SRC, _HDR))
    if stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-Wall", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u64, u32, i32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p
        lib.oracle_splitmix64_raw.restype = u64
        lib.oracle_splitmix64_raw.argtypes = [u64, u64]
        lib.oracle_splitmix64.restype = u64
        lib.oracle_splitmix64.argtypes = [u64, u64, u64]
        lib.oracle_ran_index.restype = u64
        lib.oracle_ran_index.argtypes = [u64, u64, u64]
        lib.oracle_key_cmp.restype = i32
        lib.oracle_key_cmp.argtypes = [i32, u64, u64]
        lib.oracle_str_cmp.restype = i32
        lib.oracle_str_cmp.argtypes = [ctypes.c_char_p, ctypes.c_char_p]
        lib.oracle_sort.restype = i32
        lib.oracle_sort.argtypes = [i32, vp, vp, u64, i32, u32, u32, u64,
                                    vp, vp, vp, vp, vp, vp]
        lib.oracle_sort_mc.restype = i32
        lib.oracle_sort_mc.argtypes = [i32, vp, vp, u64, i32, u32, u32, u64,
                                       vp, vp, vp, vp, vp, vp, u32, i32]
        lib.oracle_some_sort.restype = i32
        lib.oracle_some_sort.argtypes = [i32, vp, vp, u64, vp, vp]
        _lib = lib
    return _lib


def splitmix64_raw(state: int, i: int) -> int:
    return int(_load().oracle_splitmix64_raw(state, i))


def splitmix64(seed: int, stream: int, i: int) -> int:
    return int(_load().oracle_splitmix64(seed, stream, i))


def ran_index(seed: int, j: int, n: int) -> int:
    return int(_load().oracle_ran_index(seed, j, n))


def key_cmp(kt: str, a_bits: int, b_bits: int) -> int:
    return int(_load().oracle_key_cmp(KT[kt], a_bits, b_bits))


def str_cmp(a: bytes, b: bytes) -> int:
    assert len(a) == 32 and len(b) == 32
    return int(_load().oracle_str_cmp(a, b))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def sort(keys: np.ndarray, kt: str, split: str, p: int, s: int, seed: int = 0,
         vals: np.ndarray | None = None, merge: bool = True, threads: int = 1,
         par_step5: bool = False) -> dict:
    """Run SqDet / SqRan on the CPU.

    Returns a dict with ``keys`` / ``vals`` (the output Y, when ``merge``),
    ``spl_keys`` and ``spl_tags`` (the p-1 tagged splitters), ``bucket_sizes``
    (p entries) and ``p_used`` (p, or 1 when the input is too small to sample).
    ``threads`` > 1 runs the multi-core form of Section 2.4 (McDet / McRan: step 1
    over that many threads, and step 5 too when ``par_step5``)."""
    lib = _load()
    keys = np.ascontiguousarray(keys, dtype=NP_DT[kt])
    if kt == "s32":
        keys = keys.reshape(-1, 32)     # n records of 32 bytes
    n = keys.shape[0]
    if vals is not None:
        vals = np.ascontiguousarray(vals, dtype=np.uint32)
        assert vals.shape[0] == n
    shape = (n, 32) if kt == "s32" else (n,)
    out_k = np.empty(shape, dtype=NP_DT[kt]) if merge else None
    out_v = np.empty(n, dtype=np.uint32) if (merge and vals is not None) else None
    spl_k = np.zeros((max(p - 1, 0), 32) if kt == "s32" else max(p - 1, 0), dtype=NP_DT[kt])
    spl_t = np.zeros(max(p - 1, 0), dtype=np.uint64)
    sizes = np.zeros(p, dtype=np.uint64)
    p_used = ctypes.c_uint32(0)
    args = (KT[kt], _ptr(keys), _ptr(vals), n, SPLIT[split], p, s, seed,
            _ptr(out_k), _ptr(out_v), _ptr(spl_k), _ptr(spl_t), _ptr(sizes), ctypes.byref(p_used))
    if threads > 1:
        rc = lib.oracle_sort_mc(*args, threads, 1 if par_step5 else 0)
    else:
        rc = lib.oracle_sort(*args)
    if rc != 0:
        raise RuntimeError(f"oracle_sort failed with code {rc}")
    pu = int(p_used.value)
    if pu == 1:
        spl_k = spl_k[:0]
        spl_t = spl_t[:0]
    return {"keys": out_k, "vals": out_v, "spl_keys": spl_k, "spl_tags": spl_t,
            "bucket_sizes": sizes, "p_used": pu}


def some_sort(keys: np.ndarray, kt: str, vals: np.ndarray | None = None) -> dict:
    """SomeSort (the oracle's stable merge sort) on the whole input: the
    stand-alone sort the paper's tables compare against."""
    lib = _load()
    keys = np.ascontiguousarray(keys, dtype=NP_DT[kt])
    if kt == "s32":
        keys = keys.reshape(-1, 32)
    n = keys.shape[0]
    if vals is not None:
        vals = np.ascontiguousarray(vals, dtype=np.uint32)
    out_k = np.empty(keys.shape, dtype=NP_DT[kt])
    out_v = np.empty(n, dtype=np.uint32) if vals is not None else None
    rc = lib.oracle_some_sort(KT[kt], _ptr(keys), _ptr(vals), n, _ptr(out_k), _ptr(out_v))
    if rc != 0:
        raise RuntimeError(f"oracle_some_sort failed with code {rc}")
    return {"keys": out_k, "vals": out_v}
