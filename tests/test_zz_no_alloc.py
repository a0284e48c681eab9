"""vd_cells_noalloc: the allocation-free entry point for callers that cannot
call cudaMalloc (code under another framework's allocator or memory pool,
loops that forbid allocation after start-up). It keeps its scratch in a
fixed device array, so this test checks it through the C ABI against the
allocating vd_build on two calls in a row (the second call must not see
stale state from the first), within the tolerances of the parity tests.

The file name makes pytest collect it last; it passes alone in a fresh
process and after the other GPU tests.
"""
import ctypes

import numpy as np
import pytest

from paper_2605_06408_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROW = 64  # VD_NOALLOC_ROW


@pytest.fixture(scope="module")
def vdmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_06408_gb300 import vd

    vd.load_library()
    return vd


def noalloc(vdmod, x, w, box):
    lib = vdmod.load_library()
    n = len(x)
    xs = torch.from_numpy(x).cuda()
    ws = None if w is None else torch.from_numpy(w).cuda()
    counts = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    nbrs = torch.full((n * ROW,), -7, dtype=torch.int32, device="cuda")
    vol = torch.empty(n, dtype=torch.float32, device="cuda")
    cen = torch.empty(n, 3, dtype=torch.float32, device="cuda")
    status = torch.full((1,), -99, dtype=torch.int32, device="cuda")
    p = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.vd_cells_noalloc(p(xs), p(ws), n, vdmod._box(box), p(counts), p(nbrs), p(vol), p(cen), p(status),
                              stream)
    assert rc == vdmod.VD_OK, vdmod.error_string(rc)
    torch.cuda.synchronize()
    return counts.cpu().numpy(), nbrs.cpu().numpy().reshape(n, ROW), vol.cpu().numpy(), cen.cpu().numpy(), \
        int(status.item())


def compare(vdmod, x, w, box):
    counts, rows, vol, cen, status = noalloc(vdmod, x, w, box)
    assert status == vdmod.VD_OK
    ctx = vdmod.Context(0)
    ref = ctx.build(torch.from_numpy(x).cuda(), None if w is None else torch.from_numpy(w).cuda(), box)
    off = ref.offsets.cpu().numpy()
    nb = ref.neighbors.cpu().numpy()
    np.testing.assert_array_equal(counts, np.diff(off))
    for i in range(len(x)):
        assert np.array_equal(rows[i, :counts[i]], nb[off[i]:off[i + 1]]), i
    rv = ref.volume.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(vol - rv) <= 1e-5 * rv + 1e-30)
    rc = ref.centroid.cpu().numpy().astype(np.float64)
    assert np.all(np.linalg.norm(cen - rc, axis=1) <= 1e-5 * np.linalg.norm(rc, axis=1))


def test_noalloc_matches_vd_build_on_two_calls_in_a_row(vdmod):
    # first call: a weighted set with the paper's Gaussian weights (some
    # cells empty)
    x1 = W.uniform(6000, 71)
    w1 = W.gaussian_weights(x1, 72)
    compare(vdmod, x1, w1, W.UNIT_BOX)
    # second call: a different, smaller unweighted set in another box
    x2 = (W.uniform(2500, 73) * 2.0 - 1.0).astype(np.float32)
    compare(vdmod, x2, None, ((-1.0, -1.0, -1.0), (1.0, 1.0, 1.0)))


def test_noalloc_rejects_oversized_inputs(vdmod):
    lib = vdmod.load_library()
    n = 16384 + 1
    rc = lib.vd_cells_noalloc(ctypes.c_void_p(1), None, n, vdmod._box(W.UNIT_BOX), ctypes.c_void_p(1),
                              ctypes.c_void_p(1), ctypes.c_void_p(1), ctypes.c_void_p(1), ctypes.c_void_p(1), None)
    assert rc == vdmod.VD_ERR_TOO_LARGE
