"""The C ABI library builds, loads without a GPU and exports every declared entry
point; argument checks and workspace planning work on the host."""
import os
import re

import pytest

from paper_1608_08648_gb300 import binding as B
from paper_1608_08648_gb300 import build as _build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ossort.h")


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return B.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*|size_t|uint64_t)\s+(os_\w+)\s*\(", text, flags=re.M)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 11
    for name in names:
        assert hasattr(lib, name), name


def test_version_and_strerror(lib):
    assert B.os_version() == 10000
    assert B.os_strerror(B.OS_OK) == "ok"
    assert "workspace" in B.os_strerror(B.OS_ERR_WS)


def test_argument_checks_without_gpu(lib):
    prm = B.os_params(B.OS_RAN, 1024, 16, 0, 1)
    assert B.os_workspace_size(7, 10, False, prm)[0] == B.OS_ERR_ARG
    assert B.os_workspace_size(B.OS_I32, 10, False, B.os_params(B.OS_RAN, 0, 16, 0, 1))[0] == B.OS_ERR_ARG
    assert B.os_workspace_size(B.OS_I32, 10, False, B.os_params(B.OS_RAN, 4, 0, 0, 1))[0] == B.OS_ERR_ARG
    assert B.os_workspace_size(B.OS_I32, 10, False, B.os_params(5, 4, 1, 0, 1))[0] == B.OS_ERR_ARG
    assert B.os_workspace_size(B.OS_I32, 10, False, B.os_params(B.OS_RAN, 4, 1, 8, 0))[0] == B.OS_ERR_ARG
    assert B.os_workspace_size(B.OS_I32, 10, False, B.os_params(B.OS_RAN, 8192, 1, 0, 1))[0] == \
        B.OS_ERR_UNSUPPORTED
    assert B.os_workspace_size(B.OS_I32, (1 << 31) + 1, False, prm)[0] == B.OS_ERR_UNSUPPORTED
    # null keys, payload given on one side only, and a missing workspace are refused
    assert B.os_sort(B.OS_I32, None, None, None, None, 10, prm, None, 0, None) == B.OS_ERR_ARG
    assert B.os_sort(B.OS_I32, 16, 16, 16, None, 10, prm, None, 0, None) == B.OS_ERR_ARG
    assert B.os_sort(B.OS_I32, 16, 16, None, None, 10, prm, None, 0, None) == B.OS_ERR_WS


def test_workspace_grows_with_n_and_payload(lib):
    for kt in (B.OS_I32, B.OS_U64, B.OS_F64):
        for split in (B.OS_DET, B.OS_RAN):
            prm = B.os_params(split, 64, 8, 0, 1)
            sizes = [B.os_workspace_size(kt, n, False, prm)[1] for n in (0, 1000, 1 << 20, 1 << 24)]
            assert sizes == sorted(sizes) and sizes[-1] > (1 << 24)
            rc, a = B.os_workspace_size(kt, 1 << 20, False, prm)
            rc2, b = B.os_workspace_size(kt, 1 << 20, True, prm)
            assert rc == rc2 == B.OS_OK and b > a
            rc3, h = B.os_workspace_size_host(kt, 1 << 20, True, prm)
            assert rc3 == B.OS_OK and h > b
