"""The partition of one diagram's cells (vd_set_partition) through the C
ABI: three parts, each a context holding the whole LBVH that builds one
contiguous Morton-order range of the cells, merged as the ranks of a
multi-GPU job would merge them (paper_2605_06408_gb300.partition), give the
cells of one whole build and of the FP64 oracle; their adjoints sum to the
whole adjoint. Run here on one GPU, one part after another."""
import numpy as np
import pytest

import oracle
from paper_2605_06408_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def vdmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_06408_gb300 import vd

    vd.load_library()
    return vd


def dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("weighted", [False, True])
def test_three_parts_merge_into_the_whole_diagram(vdmod, weighted):
    from paper_2605_06408_gb300 import partition

    n, nparts = 200_000, 3
    x = W.mixture(n, 81)
    w = W.power_weights(x, 82) if weighted else None
    xs, ws = dev(x), dev(w)
    whole = vdmod.Context(0, {"tape": 1})
    full = whole.build(xs, ws, W.UNIT_BOX)
    parts, ctxs = [], []
    for p in range(nparts):
        c = vdmod.Context(0, {"tape": 1})
        c.set_partition(p, nparts)
        r = c.build(xs, ws, W.UNIT_BOX)
        assert c.status()["error"] == 0
        parts.append(r)
        ctxs.append(c)
    # the parts' non-empty rows are disjoint, cover the whole diagram's, and
    # each part holds at most its range's share of the cells
    owned = [torch.diff(r.offsets) > 0 for r in parts]
    cover = sum(o.int() for o in owned)
    assert int(cover.max().item()) <= 1
    assert torch.equal(cover.bool(), torch.diff(full.offsets) > 0)
    assert all(int(o.sum().item()) <= n // nparts + 1 for o in owned)
    off, nb = partition.merge_parts([r.offsets for r in parts], [r.neighbors for r in parts])
    vol = sum(r.volume for r in parts)
    cen = sum(r.centroid for r in parts)
    assert torch.equal(off, full.offsets) and torch.equal(nb, full.neighbors)
    assert torch.equal(vol, full.volume) and torch.equal(cen, full.centroid)
    # against the oracle on sampled cells
    cells = np.sort(W.rng_for(83).choice(n, 1500, replace=False))
    ref = oracle.cells(x, w, W.UNIT_BOX, cells=cells)
    assert ref["stats"]["ambiguous"] == 0 and ref["stats"]["degenerate"] == 0
    o, b = off.cpu().numpy().astype(np.int64), nb.cpu().numpy()
    for q, i in enumerate(cells):
        assert np.array_equal(b[o[i]:o[i + 1]], ref["nbrs"][q]), i
    v = vol.cpu().numpy().astype(np.float64)[cells]
    assert np.all(np.abs(v - ref["vol"]) <= 1e-5 * ref["vol"] + 1e-30)
    # adjoint: the parts' gradients sum to the whole gradient
    c, d = W.loss_coefficients(n, 84)
    gv, gc = dev(c.astype(np.float32)), dev(d.astype(np.float32))
    gp_full, gw_full = whole.backward(gv, gc, want_weights=weighted)
    gp = torch.zeros_like(gp_full)
    gw = torch.zeros_like(gw_full) if weighted else None
    for ctx in ctxs:
        a, b2 = ctx.backward(gv, gc, want_weights=weighted)
        gp += a
        if weighted:
            gw += b2
    scale = gp_full.abs().max().item()
    assert torch.allclose(gp, gp_full, rtol=1e-5, atol=1e-6 * scale)
    if weighted:
        assert torch.allclose(gw, gw_full, rtol=1e-5, atol=1e-6 * gw_full.abs().max().item())


def test_partition_arguments(vdmod):
    c = vdmod.Context(0)
    for part, nparts in ((1, 1), (-1, 2), (0, 0), (3, 3)):
        with pytest.raises(vdmod.VdError):
            c.set_partition(part, nparts)
    c.set_partition(0, 1)
