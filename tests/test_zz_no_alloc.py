"""vd_cells_noalloc: the entry point for callers that cannot call cudaMalloc
(code running under another framework's allocator or memory pool, loops
that forbid allocation once started, callers that must not create a
context workspace). Its scratch is one fixed device array inside the
library, so this file checks, through the C ABI:
  - two calls in a row (the second must not see the first's state) against
    the allocating vd_build and against the FP64 oracle, within the parity
    tests' tolerances;
  - duplicate sites, sites outside the box and a dominant weight;
  - the overflow row (count -1, NaN volume and centroid, status word);
  - that a call allocates no device memory.

The file name makes pytest collect it last; it passes alone in a fresh
process and after the other GPU tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2605_06408_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROW = 64  # VD_NOALLOC_ROW
VOL_RTOL = CEN_RTOL = 1e-5


@pytest.fixture(scope="module")
def vdmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_06408_gb300 import vd

    vd.load_library()
    return vd


class NoAlloc:
    """Device inputs and outputs of one vd_cells_noalloc call."""

    def __init__(self, vdmod, x, w, box):
        self.lib = vdmod.load_library()
        self.vd = vdmod
        n = len(x)
        self.n, self.box = n, box
        self.xs = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        self.ws = None if w is None else torch.from_numpy(np.ascontiguousarray(w)).cuda()
        self.counts = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        self.nbrs = torch.full((n * ROW,), -7, dtype=torch.int32, device="cuda")
        self.vol = torch.empty(n, dtype=torch.float32, device="cuda")
        self.cen = torch.empty(n, 3, dtype=torch.float32, device="cuda")
        self.status = torch.full((1,), -99, dtype=torch.int32, device="cuda")

    def call(self):
        p = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        rc = self.lib.vd_cells_noalloc(p(self.xs), p(self.ws), self.n, self.vd._box(self.box), p(self.counts),
                                       p(self.nbrs), p(self.vol), p(self.cen), p(self.status), stream)
        assert rc == self.vd.VD_OK, self.vd.error_string(rc)
        torch.cuda.synchronize()

    def result(self):
        return (self.counts.cpu().numpy(), self.nbrs.cpu().numpy().reshape(self.n, ROW), self.vol.cpu().numpy(),
                self.cen.cpu().numpy(), int(self.status.item()))


def noalloc(vdmod, x, w, box):
    c = NoAlloc(vdmod, x, w, box)
    c.call()
    return c.result()


def check_against(counts, rows, vol, cen, offsets, nbrs, rvol, rcen, cells):
    """Rows, volumes and centroids of `cells` against a reference CSR."""
    for i in cells:
        assert counts[i] == offsets[i + 1] - offsets[i], i
        assert np.array_equal(rows[i, :counts[i]], nbrs[offsets[i]:offsets[i + 1]]), i
    rv = np.asarray(rvol, np.float64)[cells]
    assert np.all(np.abs(vol[cells] - rv) <= VOL_RTOL * rv + 1e-30)
    rc = np.asarray(rcen, np.float64)[cells]
    assert np.all(np.linalg.norm(cen[cells] - rc, axis=1) <= CEN_RTOL * np.linalg.norm(rc, axis=1))


def compare(vdmod, x, w, box, cells=None):
    """vd_cells_noalloc against vd_build and the FP64 oracle."""
    counts, rows, vol, cen, status = noalloc(vdmod, x, w, box)
    cells = np.arange(len(x)) if cells is None else cells
    ref = oracle.cells(x, w, box)
    assert ref["stats"]["ambiguous"] == 0 and ref["stats"]["degenerate"] == 0
    check_against(counts, rows, vol, cen, ref["offsets"], ref["indices"], ref["vol"], ref["cen"], cells)
    ctx = vdmod.Context(0)
    b = ctx.build(torch.from_numpy(x).cuda(), None if w is None else torch.from_numpy(w).cuda(), box)
    check_against(counts, rows, vol, cen, b.offsets.cpu().numpy().astype(np.int64), b.neighbors.cpu().numpy(),
                  b.volume.cpu().numpy(), b.centroid.cpu().numpy(), cells)
    return status


def test_noalloc_matches_vd_build_and_oracle_on_two_calls_in_a_row(vdmod):
    # first call: a weighted set with the paper's Gaussian weights (some
    # cells empty)
    x1 = W.uniform(6000, 71)
    w1 = W.gaussian_weights(x1, 72)
    assert compare(vdmod, x1, w1, W.UNIT_BOX) == vdmod.VD_OK
    # second call: a different, smaller unweighted set in another box
    x2 = (W.uniform(2500, 73) * 2.0 - 1.0).astype(np.float32)
    assert compare(vdmod, x2, None, ((-1.0, -1.0, -1.0), (1.0, 1.0, 1.0))) == vdmod.VD_OK


def test_noalloc_duplicates_outside_sites_and_dominant_weight(vdmod):
    x = np.array([[0.21, 0.23, 0.19], [0.81, 0.52, 0.47], [0.21, 0.23, 0.19], [0.53, 0.91, 0.12],
                  [-0.27, 0.56, 0.44], [1.71, 0.42, 0.61]], np.float32)
    for w in (None, np.array([0.0, 0.0, 0.01, 0.0, 0.003, 2.0], np.float32)):
        assert compare(vdmod, x, w, W.UNIT_BOX) == vdmod.VD_OK
    x = W.uniform(500, 5)
    w = np.zeros(500, np.float32)
    w[17] = 10.0  # owns the whole box: every other cell is empty
    assert compare(vdmod, x, w, W.UNIT_BOX) == vdmod.VD_OK
    counts, _, vol, _, _ = noalloc(vdmod, x, w, W.UNIT_BOX)
    assert counts[17] == 0 and vol[17] == pytest.approx(1.0, rel=1e-6)
    assert np.count_nonzero(vol) == 1


def test_noalloc_overflow_row_and_status(vdmod):
    """A site surrounded by 150 others on a sphere has a 150-face cell, more
    than this entry point holds: its row says -1, its volume and centroid are
    NaN, the status word says VD_ERR_CELL_OVERFLOW; the other cells are
    still right."""
    k = 150
    i = np.arange(k) + 0.5
    phi = np.arccos(1 - 2 * i / k)
    th = np.pi * (1 + 5 ** 0.5) * i
    s = np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)
    s = s * (0.2 + 0.002 * W.rng_for(3).random((k, 1)))
    bg = W.uniform(2000, 4)
    bg = bg[np.linalg.norm(bg - 0.5, axis=1) > 0.3]
    x = np.concatenate([[[0.5, 0.5, 0.5]], 0.5 + s, bg]).astype(np.float32)
    counts, rows, vol, cen, status = noalloc(vdmod, x, None, W.UNIT_BOX)
    assert status == vdmod.VD_ERR_CELL_OVERFLOW
    assert counts[0] == -1 and np.isnan(vol[0]) and np.all(np.isnan(cen[0]))
    ok = np.flatnonzero(counts >= 0)
    assert len(ok) >= len(x) - 5
    ref = oracle.cells(x, None, W.UNIT_BOX)
    check_against(counts, rows, vol, cen, ref["offsets"], ref["indices"], ref["vol"], ref["cen"], ok)


def test_noalloc_allocates_no_device_memory(vdmod):
    """After a first call (which looks up the scratch array's address), a
    second call leaves the device's free memory unchanged."""
    x = W.uniform(8000, 75)
    w = W.gaussian_weights(x, 76)
    c = NoAlloc(vdmod, x, w, W.UNIT_BOX)
    c.call()
    first = c.result()
    assert first[4] == vdmod.VD_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    c.call()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    second = c.result()
    assert second[4] == vdmod.VD_OK
    for a, b in zip(first[:4], second[:4]):
        assert np.array_equal(a, b)


def test_noalloc_rejects_oversized_inputs(vdmod):
    lib = vdmod.load_library()
    n = 16384 + 1
    rc = lib.vd_cells_noalloc(ctypes.c_void_p(1), None, n, vdmod._box(W.UNIT_BOX), ctypes.c_void_p(1),
                              ctypes.c_void_p(1), ctypes.c_void_p(1), ctypes.c_void_p(1), ctypes.c_void_p(1), None)
    assert rc == vdmod.VD_ERR_TOO_LARGE
