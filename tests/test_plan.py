"""The workspace the planner measures equals the workspace a real sort takes,
for every key type, payload choice, splitter choice and a grid of n, p, s
(host-only build of the orchestration code; no kernel is launched)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_measured_plan_matches_live_plan(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "plan_check")
    subprocess.check_call([nvcc, "-std=c++17", "-O1", "-DOSSORT_NO_LAUNCH",
                           "-gencode=arch=compute_103a,code=compute_103a", "--expt-relaxed-constexpr",
                           "-o", exe, os.path.join(HERE, "native", "plan_check.cu")])
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout[-4000:]
    assert "consistent" in r.stdout
