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

    for code in range(0, -8, -1):
        assert len(lib.vd_error_string(code)) > 0
    assert lib.vd_build(None, None, None, 10, vd.VdBox(), None, None) == vd.VD_ERR_INVALID_ARG
    assert lib.vd_backward(None, None, None, None, None, 1, None) == vd.VD_ERR_INVALID_ARG
    assert lib.vd_create(None, 0, None) == vd.VD_ERR_INVALID_ARG
    assert lib.vd_get_status(None, None) == vd.VD_ERR_INVALID_ARG
    # vd_copy rejects bad sizes and NULL pointers before any CUDA call
    assert lib.vd_copy(None, None, 0, None) == vd.VD_OK
    assert lib.vd_copy(None, None, 16, None) == vd.VD_ERR_INVALID_ARG
    assert lib.vd_copy(None, None, -1, None) == vd.VD_ERR_INVALID_ARG
    cfg = vd.VdConfig()
    assert lib.vd_default_config(ctypes.byref(cfg)) == vd.VD_OK
    assert cfg.leaf_size == 16 and cfg.cull_mode == 0


def test_workspace_bytes_grows_with_n(lib):
    a, b = lib.vd_workspace_bytes(10_000, 0), lib.vd_workspace_bytes(1_000_000, 1)
    assert 0 < a < b
    # ~0.5 KB per site: 20M sites fit easily in the GPU's memory
    assert lib.vd_workspace_bytes(20_000_000, 0) < 16 * 2**30


C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "vd.h"
int main(void) {
  vd_config c;
  if (vd_default_config(&c) != VD_OK) return 1;
  if (c.leaf_size != 16 || c.verts_per_lane != 2 || c.tape != 0 || c.precision != 0) return 2;
  if (vd_default_config(NULL) != VD_ERR_INVALID_ARG) return 3;
  vd_box b = {{0.f, 0.f, 0.f}, {1.f, 1.f, 1.f}};
  if (vd_build(NULL, NULL, NULL, 10, b, NULL, NULL) != VD_ERR_INVALID_ARG) return 4;
  if (vd_cells_mesh(NULL, NULL, NULL) != VD_ERR_INVALID_ARG) return 5;
  if (strlen(vd_error_string(VD_ERR_TIMEOUT)) == 0) return 6;
  printf("%zu\n", vd_workspace_bytes(1000, 0));
  return 0;
}
"""


def test_plain_c_program_uses_the_library(lib, tmp_path):
    """A C99 program compiles against include/vd.h, links libvd.so and
    calls the host-side entry points (no GPU needed for these)."""
    import shutil
    import subprocess

    from paper_2605_06408_gb300 import build

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    src = tmp_path / "prog.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "prog"
    libdir = os.path.dirname(build.LIB)
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                        os.path.join(ROOT, "include"), str(src), "-o", str(exe), "-L", libdir, "-lvd",
                        "-Wl,-rpath," + libdir], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True)
    assert run.returncode == 0, (run.returncode, run.stderr)
    assert int(run.stdout.strip()) > 0
