"""Explicit mesh output (vd_cells_mesh) and vertex gradients
(vd_backward_mesh) through the C ABI against the FP64 oracle: the vertices of
sampled cells (matched by their defining sites) and the site / weight
gradients of a loss on the vertices of a subset of cells."""
import numpy as np
import pytest

import oracle
from paper_2605_06408_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BOX = W.UNIT_BOX


@pytest.fixture(scope="module")
def vdmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_06408_gb300 import vd

    vd.load_library()
    return vd


def dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()


def key_grad(i, t):
    a, b, c = sorted(t)
    return np.array([np.sin(0.37 * i + 0.11 * a + 0.05 * b + 0.02 * c),
                     np.cos(0.29 * i - 0.07 * a + 0.13 * b - 0.03 * c),
                     np.sin(0.19 * i + 0.17 * a - 0.09 * b + 0.23 * c)])


def workload(weighted):
    x = W.mixture(20_000, 91)
    w = W.power_weights(x, 92) if weighted else None
    return x, w


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("tape", [0, 1])
def test_mesh_matches_oracle_vertices(vdmod, weighted, tape):
    x, w = workload(weighted)
    ctx = vdmod.Context(0, {"tape": tape})
    res = ctx.build(dev(x), dev(w), BOX)
    off, verts, sites = ctx.mesh()
    off = off.cpu().numpy().astype(np.int64)
    verts = verts.cpu().numpy().astype(np.float64)
    sites = sites.cpu().numpy()
    assert off[-1] == len(verts)
    vol = res.volume.cpu().numpy()
    assert np.all((np.diff(off) == 0) == (vol == 0))  # empty cells have no vertices
    for i in np.sort(W.rng_for(93).choice(len(x), 120, replace=False)):
        pos, tri = oracle.cell_vertices(x, w, BOX, int(i))
        want = {tuple(sorted(t)): x[i].astype(np.float64) + p for p, t in zip(pos, tri)}
        got = {tuple(sorted(s)): v for s, v in zip(sites[off[i]:off[i + 1]], verts[off[i]:off[i + 1]])}
        assert set(got) == set(want), i
        scale = max(1e-12, np.abs(pos).max()) if len(pos) else 1.0
        for k, v in want.items():
            assert np.abs(got[k] - v).max() <= 1e-5 * scale + 1e-7, (i, k)


@pytest.mark.parametrize("weighted", [False, True])
def test_vertex_gradient_matches_oracle(vdmod, weighted):
    x, w = workload(weighted)
    ctx = vdmod.Context(0, {"tape": 1})
    ctx.build(dev(x), dev(w), BOX)
    off_t, verts, sites = ctx.mesh()
    off = off_t.cpu().numpy().astype(np.int64)
    sites = sites.cpu().numpy()
    S = np.sort(W.rng_for(94).choice(len(x), 60, replace=False))
    g = np.zeros((len(verts), 3), np.float32)
    for i in S:
        for r in range(off[i], off[i + 1]):
            g[r] = key_grad(int(i), tuple(int(s) for s in sites[r]))
    gp, gw = ctx.backward(None, None, want_weights=weighted, grad_vertices=dev(g), vertex_offsets=off_t)
    gpo, gwo = oracle.vertex_grad(x, w, BOX, S, key_grad)
    gp = gp.cpu().numpy().astype(np.float64)
    touched = np.abs(gpo).max(1) > 0
    err = np.abs(gp - gpo).max(1)[touched] / np.abs(gpo).max(1)[touched]
    # about 10x the measured errors (Voronoi: max 4.4e-6, p99 2.4e-6; power:
    # max 1.1e-5, p99 2.6e-6; power weights: p99 2.0e-6)
    assert np.quantile(err, 0.99) < 3e-5 and err.max() < 1.2e-4, (np.quantile(err, 0.99), err.max())
    assert np.abs(gp[~touched]).max() == 0.0
    if weighted:
        gw = gw.cpu().numpy().astype(np.float64)
        tw = np.abs(gwo) > 0
        ew = np.abs(gw - gwo)[tw] / np.maximum(np.abs(gwo)[tw], 1e-3 * np.abs(gwo).max())
        assert np.quantile(ew, 0.99) < 3e-5 and ew.max() < 1.2e-4, (np.quantile(ew, 0.99), ew.max())


def test_mesh_autograd_function(vdmod):
    """mesh_cells: the gradient of a loss on volumes, centroids and vertices
    equals the direct call of the adjoint."""
    x, w = workload(True)
    xs = dev(x).requires_grad_(True)
    ws = dev(w).requires_grad_(True)
    vol, cen, verts, off, nb, voff, vsites = vdmod.mesh_cells(xs, ws, BOX)
    L = 3.0 * vol.sum() + (cen * cen).sum() + (verts * verts).sum()
    L.backward()
    ctx = vdmod.Context(0, {"tape": 1})
    ctx.build(dev(x), dev(w), BOX)
    voff2, verts2, _ = ctx.mesh()
    gv = torch.full_like(vol, 3.0)
    gp, gw = ctx.backward(gv, 2.0 * cen.detach(), grad_vertices=2.0 * verts2, vertex_offsets=voff2)
    assert torch.allclose(xs.grad, gp, rtol=1e-4, atol=1e-6 * gp.abs().max().item())
    assert torch.allclose(ws.grad, gw, rtol=1e-4, atol=1e-6 * gw.abs().max().item())


def test_mesh_capacity_paths(vdmod):
    """A too-small vertex buffer reports VD_ERR_CAPACITY with the size to
    allocate (the wrapper retries); capacity 0 gives counts and offsets only."""
    import ctypes

    x, w = workload(False)
    ctx = vdmod.Context(0)
    ctx.build(dev(x), None, BOX)
    off_full, verts_full, sites_full = ctx.mesh()
    off_small, verts_small, sites_small = ctx.mesh(capacity=10)  # retried at the reported size
    assert torch.equal(off_small, off_full) and torch.equal(sites_small, sites_full)
    assert torch.equal(verts_small, verts_full)
    n = len(x)
    off = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    nv = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    m = vdmod.VdMesh(off.data_ptr(), None, None, 0, nv.data_ptr(), st.data_ptr())
    lib = vdmod.load_library()
    assert lib.vd_cells_mesh(ctx._h, ctypes.byref(m), None) == vdmod.VD_OK
    torch.cuda.synchronize()
    assert int(st.item()) == vdmod.VD_OK and int(nv.item()) == len(verts_full)
    assert torch.equal(off, off_full)
    verts = torch.empty(5, 3, dtype=torch.float32, device="cuda")
    sites = torch.empty(5, 3, dtype=torch.int32, device="cuda")
    m = vdmod.VdMesh(off.data_ptr(), verts.data_ptr(), sites.data_ptr(), 5, nv.data_ptr(), st.data_ptr())
    assert lib.vd_cells_mesh(ctx._h, ctypes.byref(m), None) == vdmod.VD_OK
    torch.cuda.synchronize()
    assert int(st.item()) == vdmod.VD_ERR_CAPACITY and int(nv.item()) == len(verts_full)
