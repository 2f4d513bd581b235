"""Host-side parts of the serving loop: the arena allocator (against a
brute-force model), argument checks of the server ABI and the request trace
of the serving workload (no GPU)."""
import math
import os
import shutil
import subprocess

import pytest

from paper_1608_08648_gb300 import binding as B
from paper_1608_08648_gb300 import build as _build
from paper_1608_08648_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def test_arena_allocator_against_model(tmp_path):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "alloc_check")
    subprocess.check_call([gxx, "-std=c++17", "-O2", "-Wall", "-o", exe,
                           os.path.join(HERE, "native", "alloc_check.cpp")])
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout[-2000:]
    assert "allocator consistent" in r.stdout


def test_server_argument_checks_without_gpu():
    _build.build()
    assert B.os_server_create(None, 1 << 20, 2, 4)[0] == B.OS_ERR_ARG
    assert B.os_server_create(4096, 1 << 20, 0, 4)[0] == B.OS_ERR_ARG
    assert B.os_server_create(4096, 1 << 20, 65, 4)[0] == B.OS_ERR_ARG
    assert B.os_server_create(4096, 1 << 20, 2, 0)[0] == B.OS_ERR_ARG
    assert B.os_server_create(4096, 16, 2, 4)[0] == B.OS_ERR_ARG
    req = B.os_request(B.OS_I32, 0, 4096, 10, B.os_params(B.OS_RAN, 4, 4, 0, 1))
    assert B.os_server_submit(None, req)[0] == B.OS_ERR_ARG
    assert B.os_server_poll(None)[0] == B.OS_ERR_ARG
    assert B.os_server_release(None, 1) == B.OS_ERR_ARG
    assert B.os_server_destroy(None) == B.OS_ERR_ARG


def test_serving_trace_shape():
    t = inputs.serving_trace(20000, rate=2000.0, lo=4096, hi=1 << 26, seed=5)
    n = t["n"]
    assert len(n) == 20000 and min(n) >= 4096 and max(n) < 1 << 26
    arr = t["arrival_s"]
    assert all(b >= a for a, b in zip(arr, arr[1:]))
    assert abs(arr[-1] - 10.0) < 0.5                       # 20,000 arrivals at 2,000 per second
    assert abs(sum(d == "f64" for d in t["dtype"]) / 20000 - 0.5) < 0.02
    assert abs(sum(d == "dup" for d in t["dist"]) / 20000 - 0.5) < 0.02
    mean = (2 ** 26 - 4096) / math.log(2 ** 26 / 4096)     # mean of the log-uniform length
    assert abs(sum(n) / 20000 / mean - 1) < 0.05
    assert all(0 <= o <= (1 << 26) - m for o, m in zip(t["offset"], n))
