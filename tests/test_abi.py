"""The C-ABI library builds, loads and exports every call of include/vd.h;
host-side argument checks work without a GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "vd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|size_t|const char\*)\s+(vd_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_06408_gb300 import build, vd

    build.build()
    return vd.load_library(build_if_missing=False)


def test_header_declares_the_boundary():
    fns = header_functions()
    for f in ("vd_create", "vd_destroy", "vd_build", "vd_build_batched", "vd_backward", "vd_get_status",
              "vd_error_string", "vd_workspace_bytes"):
        assert f in fns


def test_library_exports_every_declared_symbol(lib):
    from paper_2605_06408_gb300 import vd

    for f in header_functions():
        assert hasattr(lib, f), f
    assert set(header_functions()) == set(vd.ABI_FUNCTIONS)


def test_error_strings_and_null_arguments(lib):
    from paper_2605_06408_gb300 import vd

    for code in range(0, -7, -1):
        assert len(lib.vd_error_string(code)) > 0
    assert lib.vd_build(None, None, None, 10, vd.VdBox(), None, None) == vd.VD_ERR_INVALID_ARG
    assert lib.vd_backward(None, None, None, None, None, 1, None) == vd.VD_ERR_INVALID_ARG
    assert lib.vd_create(None, 0, None) == vd.VD_ERR_INVALID_ARG
    assert lib.vd_get_status(None, None) == vd.VD_ERR_INVALID_ARG
    cfg = vd.VdConfig()
    assert lib.vd_default_config(ctypes.byref(cfg)) == vd.VD_OK
    assert cfg.leaf_size == 16 and cfg.cull_mode == 0


def test_workspace_bytes_grows_with_n(lib):
    a, b = lib.vd_workspace_bytes(10_000, 0), lib.vd_workspace_bytes(1_000_000, 1)
    assert 0 < a < b
    # ~0.5 KB per site: 20M sites fit easily in the GPU's memory
    assert lib.vd_workspace_bytes(20_000_000, 0) < 16 * 2**30
