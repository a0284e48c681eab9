"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Neighbour lists must be identical; volumes within 1e-5 relative and
centroids within 1e-5 of |g| (the FP32 tolerance of the target), on seeded
inputs shaped like the paper's workloads, on edge cases, and on every
configuration knob (leaf size, capacities, culling/traversal ablations).
"""
import numpy as np
import pytest

import oracle
from paper_2605_06408_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

VOL_RTOL = 1e-5
CEN_RTOL = 1e-5


@pytest.fixture(scope="module")
def vdmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_06408_gb300 import vd

    vd.load_library()
    return vd


@pytest.fixture(scope="module")
def ctx(vdmod):
    return vdmod.Context(0)


def dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rows(res):
    off = res.offsets.cpu().numpy().astype(np.int64)
    nb = res.neighbors.cpu().numpy()
    return off, nb


def assert_parity(res, ref, cells=None, what=""):
    off, nb = rows(res)
    vol = res.volume.cpu().numpy().astype(np.float64)
    cen = res.centroid.cpu().numpy().astype(np.float64)
    idx = np.arange(len(vol)) if cells is None else np.asarray(cells)
    bad = []
    for q, i in enumerate(idx):
        g = nb[off[i]:off[i + 1]]
        if not np.array_equal(g, ref["nbrs"][q]):
            bad.append(int(i))
    assert not bad, f"{what}: {len(bad)} neighbour lists differ, first cells {bad[:5]}"
    rv = ref["vol"]
    dv = np.abs(vol[idx] - rv)
    assert np.all(dv <= VOL_RTOL * rv + 1e-30), f"{what}: max rel vol err {np.max(dv / np.maximum(rv, 1e-300)):.3g}"
    empty = rv == 0
    assert np.all(vol[idx][empty] == 0.0)
    dc = np.linalg.norm(cen[idx] - ref["cen"], axis=1)
    gn = np.linalg.norm(ref["cen"], axis=1)
    assert np.all(dc <= CEN_RTOL * gn), f"{what}: max centroid err {np.max(dc / gn):.3g}"


def build(ctx, x, w=None, box=W.UNIT_BOX, **kw):
    return ctx.build(dev(x), dev(w), box, **kw)


# ------------------------------------------------------------------ workloads

def test_uniform_10k_full(ctx):
    x, _, box = W.config("uniform10k")
    res = build(ctx, x, None, box)
    ref = oracle.cells(x, None, box)
    assert_parity(res, ref, what="uniform10k")
    st = ctx.status()
    assert st["error"] == 0 and st["failed_cells"] == 0 and st["fp64_ambiguous"] == 0


@pytest.mark.parametrize("kind", ["mixture", "power", "surfaces", "gradient", "gaussian_w", "clustered"])
def test_workloads_100k_full(ctx, kind):
    n = 100_000
    w = None
    if kind in ("mixture", "power"):
        x = W.mixture(n, 11)
        if kind == "power":
            w = W.power_weights(x, 12)
    elif kind == "surfaces":
        x = W.surfaces(n, 13)
    elif kind == "gradient":
        x = W.gradient(n, 14)
    elif kind == "clustered":  # the paper's K=10 case: many sites clamped onto the box faces
        x = W.clustered(n, 10, 17)
    else:
        x = W.uniform(n, 15)
        w = W.gaussian_weights(x, 16)
    res = build(ctx, x, w)
    ref = oracle.cells(x, w, max_nbrs=8192)
    assert ref["stats"]["ambiguous"] == 0 and ref["stats"]["degenerate"] == 0
    assert_parity(res, ref, what=kind)
    st = ctx.status()
    assert st["error"] == 0 and st["fp64_ambiguous"] == 0


def test_configs_at_full_size_sampled(ctx):
    """1M mixture (Voronoi and power) at full size: 3000 sampled cells, and
    every cell whose build took an FP64 sign still inside its FP64 error
    bound, against the oracle (whose every sign is exact)."""
    x = W.mixture(1_000_000, 1)
    rng = W.rng_for(99)
    sample = np.sort(rng.choice(len(x), 3000, replace=False))
    sess = oracle.Session(x, None)
    for w in (None, W.power_weights(x, 2)):
        if w is not None:
            sess = oracle.Session(x, w)
        res = build(ctx, x, w)
        what = "1M" + (" power" if w is not None else "")
        ref = sess.cells(sample)
        assert ref["stats"]["ambiguous"] == 0 and ref["stats"]["degenerate"] == 0
        assert_parity(res, ref, cells=sample, what=what)
        flagged = ctx.ambiguous_cells()
        assert len(flagged) <= ctx.status()["ambiguous_cells"]
        if len(flagged):
            rf = sess.cells(flagged)
            assert rf["stats"]["ambiguous"] == 0 and rf["stats"]["degenerate"] == 0
            assert_parity(res, rf, cells=flagged, what=what + " FP64-ambiguous cells")
        # properties that hold at any size: volumes partition the box,
        # adjacency is symmetric
        vol = res.volume.double().sum().item()
        assert vol == pytest.approx(1.0, rel=2e-5)
        off, nb = rows(res)
        src = np.repeat(np.arange(len(x)), np.diff(off))
        fwd = src.astype(np.int64) * len(x) + nb
        bwd = nb.astype(np.int64) * len(x) + src
        assert np.array_equal(np.sort(fwd), np.sort(bwd))


# ------------------------------------------------------------------ knobs

@pytest.fixture(scope="module")
def knob_inputs():
    """A clustered Voronoi set and a power set with empty cells, with the
    oracle's cells of both."""
    x = W.mixture(6000, 21)
    out = {}
    for name, w in (("voronoi", None), ("power", W.power_weights(x, 22))):
        ref = oracle.cells(x, w, max_nbrs=8192)
        assert ref["stats"]["ambiguous"] == 0 and ref["stats"]["degenerate"] == 0
        out[name] = (w, ref)
    assert np.count_nonzero(out["power"][1]["vol"] == 0) > 100
    return x, out


@pytest.mark.parametrize("cfg", [
    {}, {"cull_mode": 2}, {"cull_mode": 1}, {"traversal": 1}, {"leaf_size": 1}, {"leaf_size": 32},
    {"verts_per_lane": 4, "queue_per_lane": 1}, {"verts_per_lane": 2, "queue_per_lane": 1},
    {"warps_per_block": 8, "blocks_per_sm": 2}, {"warm_start": 1}, {"warm_start": 1, "verts_per_lane": 4},
    {"warm_start": 2}, {"warm_start": 2, "leaf_size": 8}, {"warm_start": 2, "traversal": 1},
    {"warm_start": 2, "cull_mode": 1},
    {"cell_mode": 1}, {"cell_mode": 1, "cull_mode": 1}, {"cell_mode": 1, "traversal": 1},
    {"cell_mode": 1, "leaf_size": 8}, {"cull_mode": 1, "traversal": 1},
])
def test_configuration_knobs_match_oracle(vdmod, knob_inputs, cfg):
    """Every knob (warm start, the ablations of Sec. 5: isotropic culling,
    no culling, depth-first traversal; capacities, block shapes, the thread
    form) builds the oracle's cells, Voronoi and power (with empty cells)."""
    x, refs = knob_inputs
    ctx = vdmod.Context(0, cfg)
    for name, (w, ref) in refs.items():
        res = build(ctx, x, w)
        assert_parity(res, ref, what=f"{name} {cfg}")
        st = ctx.status()
        assert st["error"] == 0 and st["failed_cells"] == 0


# ------------------------------------------------------------------ edge cases

def test_single_site_and_tiny_sets(ctx):
    box = ((-1.0, 0.0, -0.5), (2.0, 0.75, 1.5))
    for n in (1, 2, 3, 7, 16, 17, 33):
        x = W.uniform(n, 40 + n) * np.array([3.0, 0.75, 2.0], np.float32) + np.array([-1.0, 0.0, -0.5], np.float32)
        x = x.astype(np.float32)
        res = build(ctx, x, None, box)
        ref = oracle.cells(x, None, box)
        assert_parity(res, ref, what=f"n={n}")


def test_duplicates_outside_sites_and_dominant_weight(ctx):
    x = np.array([[0.21, 0.23, 0.19], [0.81, 0.52, 0.47], [0.21, 0.23, 0.19], [0.53, 0.91, 0.12],
                  [-0.27, 0.56, 0.44], [1.71, 0.42, 0.61]], np.float32)
    for w in (None, np.array([0.0, 0.0, 0.01, 0.0, 0.003, 2.0], np.float32)):
        res = build(ctx, x, w)
        ref = oracle.cells(x, w)
        assert_parity(res, ref, what="duplicates")
    x = W.uniform(500, 5)
    w = np.zeros(500, np.float32)
    w[17] = 10.0
    res = build(ctx, x, w)
    ref = oracle.cells(x, w)
    assert_parity(res, ref, what="dominant")
    assert ctx.status()["empty_cells"] == 499


def test_large_cell_uses_the_large_capacity_pass(ctx):
    """A site surrounded by 150 others on a sphere has a 150-face cell, more
    than the register-resident capacity holds."""
    k = 150
    i = np.arange(k) + 0.5
    phi = np.arccos(1 - 2 * i / k)
    th = np.pi * (1 + 5 ** 0.5) * i
    s = np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)
    rng = W.rng_for(3)
    s = s * (0.2 + 0.002 * rng.random((k, 1)))
    bg = W.uniform(2000, 4)
    bg = bg[np.linalg.norm(bg - 0.5, axis=1) > 0.3]
    x = np.concatenate([[[0.5, 0.5, 0.5]], 0.5 + s, bg]).astype(np.float32)
    res = build(ctx, x)
    ref = oracle.cells(x)
    assert ref["counts"][0] >= 140
    assert_parity(res, ref, what="large cell")
    st = ctx.status()
    assert st["overflow_cells"] >= 1 and st["failed_cells"] == 0


def test_capacity_retry_and_invalid_input(vdmod, ctx):
    x = W.uniform(5000, 8)
    res = build(ctx, x, nnz_capacity=100)  # too small: re-copied through vd_copy_neighbors
    ref = oracle.cells(x)
    assert_parity(res, ref, what="capacity retry")
    bad = x.copy()
    bad[10, 1] = np.nan
    with pytest.raises(vdmod.VdError) as e:
        build(ctx, bad)
    assert e.value.code == vdmod.VD_ERR_INVALID_ARG


# ------------------------------------------------------------------ batched

def test_batched_matches_per_set_oracle(ctx):
    rng = W.rng_for(31)
    sizes = [1, 5, 17, 300, 2000, 9000, 40, 12000]
    xs, ws, flags, boxes = [], [], [], []
    for k, m in enumerate(sizes):
        lo = rng.uniform(-2, 0, 3)
        hi = lo + rng.uniform(0.5, 2, 3)
        p = (lo + (hi - lo) * W.uniform(m, 100 + k)).astype(np.float32)
        xs.append(p)
        weighted = k % 2 == 1
        ws.append(W.power_weights(p, 200 + k) if (weighted and m > 1) else np.zeros(m, np.float32))
        flags.append(1 if weighted else 0)
        boxes.append((lo.astype(np.float32), hi.astype(np.float32)))
    offs = np.concatenate([[0], np.cumsum(sizes)])
    X, Wt = np.concatenate(xs), np.concatenate(ws)
    res = ctx.build_batched(dev(X), dev(Wt), offs, boxes, flags)
    off, nb = rows(res)
    vol = res.volume.cpu().numpy()
    for k, m in enumerate(sizes):
        ref = oracle.cells(xs[k], ws[k] if flags[k] else None, boxes[k])
        for q in range(m):
            i = offs[k] + q
            assert np.array_equal(nb[off[i]:off[i + 1]], ref["nbrs"][q]), (k, q)
        np.testing.assert_allclose(vol[offs[k]:offs[k + 1]], ref["vol"], rtol=VOL_RTOL, atol=1e-30)


# ------------------------------------------------------------------ backward

@pytest.mark.parametrize("weighted", [False, True])
def test_backward_matches_oracle_gradient(ctx, weighted):
    n = 4000
    x = W.mixture(n, 61)
    w = W.power_weights(x, 62) if weighted else None
    c, d = W.loss_coefficients(n, 63)
    res = build(ctx, x, w)
    gp, gw = ctx.backward(dev(c.astype(np.float32)), dev(d.astype(np.float32)), want_weights=weighted)
    ogp, ogw, _ = oracle.grad(x, w, W.UNIT_BOX, c, d)
    gp = gp.cpu().numpy().astype(np.float64)
    # FP32 adjoint vs FP64 analytic gradient: per-site error relative to the
    # site's own gradient scale (terms scale like 1/V for the centroid part).
    # Bounds are about 10x the measured errors (Voronoi: max 1.3e-5, p99
    # 2.0e-6; power: max 8.3e-4 on a sliver cell of volume ~1e-12, p99 4.3e-6;
    # power weights: max 5.9e-4, p99 1.2e-5)
    scale = np.maximum(np.abs(ogp).max(1), 1e-3 * np.abs(ogp).max())
    err = np.abs(gp - ogp).max(1) / scale
    emax, ep99 = (8e-3, 4e-5) if weighted else (1.3e-4, 2e-5)
    assert np.quantile(err, 0.99) < ep99 and err.max() < emax, (np.quantile(err, 0.99), err.max())
    if weighted:
        gw = gw.cpu().numpy().astype(np.float64)
        sw = np.maximum(np.abs(ogw), 1e-3 * np.abs(ogw).max())
        ew = np.abs(gw - ogw) / sw
        assert np.quantile(ew, 0.99) < 1.2e-4 and ew.max() < 6e-3, (np.quantile(ew, 0.99), ew.max())


def test_autograd_function(vdmod):
    from paper_2605_06408_gb300.vd import cells

    x = W.uniform(2000, 71)
    sites = dev(x).requires_grad_(True)
    ctx = vdmod.Context(0)
    vol, cen, off, nb = cells(sites, None, W.UNIT_BOX, ctx)
    (vol.sum() * 0 + (cen * cen).sum()).backward()
    c = np.zeros(2000)
    d = 2 * cen.detach().cpu().numpy().astype(np.float64)
    ogp, _, _ = oracle.grad(x, None, W.UNIT_BOX, c, d)
    np.testing.assert_allclose(sites.grad.cpu().numpy(), ogp, rtol=1e-3, atol=1e-3 * np.abs(ogp).max())


@pytest.mark.parametrize("weighted", [False, True])
def test_backward_tape_equals_recompute(vdmod, weighted):
    """The adjoint from the forward's tape and from re-clipped cells: both
    match the oracle's analytic gradient on a subset, and each other up to
    FP32 rounding of the vertices (ill-conditioned power cells amplify it)."""
    x = W.mixture(50_000, 61)
    w = W.power_weights(x, 62) if weighted else None
    c, d = W.loss_coefficients(len(x), 63)
    gv, gc = dev(c.astype(np.float32)), dev(d.astype(np.float32))
    ctx = vdmod.Context(0, {"tape": 1})
    res = build(ctx, x, w)
    gp_t, gw_t = ctx.backward(gv, gc, want_weights=weighted)
    st = ctx.status()
    # the large cells' polytopes came from the large-cell tape: every record
    # the forward wrote was read back
    assert st["large_tape_records"] > 0 and st["large_tape_restored"] == st["large_tape_records"]
    gp_r, gw_r = ctx.backward(gv, gc, want_weights=weighted, recompute=True)
    assert ctx.status()["large_tape_restored"] == 0
    # both against the oracle on 150 cells and their neighbours
    off = res.offsets.cpu().numpy().astype(np.int64)
    nb = res.neighbors.cpu().numpy()
    K = np.sort(W.rng_for(64).choice(len(x), 150, replace=False))
    K = K[np.diff(off)[K] > 0]
    cells = np.unique(np.concatenate([K] + [nb[off[q]:off[q + 1]] for q in K]))
    ogp, _, _ = oracle.grad(x, w, W.UNIT_BOX, c, d, cells=cells)
    # bounds about 10x the measured errors against the oracle (Voronoi: max
    # 2.2e-6, p99 1.6e-6; power: max 1.2e-4, p99 2.8e-5)
    emax, ep99 = (1.2e-3, 3e-4) if weighted else (2.2e-5, 1.6e-5)
    for g in (gp_t, gp_r):
        gg = g.cpu().numpy()[K].astype(np.float64)
        err = np.abs(gg - ogp[K]).max(1) / np.maximum(np.abs(ogp[K]).max(1), 1e-30)
        assert np.quantile(err, 0.99) < ep99 and err.max() < emax, (np.quantile(err, 0.99), err.max())
    # tape vs recompute on every site: FP32 rounding of the vertices, which
    # sliver power cells amplify (measured: Voronoi max 1.1e-5, p999 3.3e-6;
    # power max 1.4e-2 on one sliver cell, p999 6.2e-5; weights p99 1.0e-5)
    scale = gp_r.abs().max(dim=1).values.clamp_min(1e-30)
    rel = (gp_t - gp_r).abs().max(dim=1).values / scale
    rmax, r999 = (0.05, 6e-4) if weighted else (1.1e-4, 3.3e-5)
    assert rel.quantile(0.999).item() < r999 and rel.max().item() < rmax, (rel.quantile(0.999).item(),
                                                                            rel.max().item())
    if weighted:
        sw = gw_r.abs().clamp_min(1e-3 * gw_r.abs().max().item())
        assert ((gw_t - gw_r).abs() / sw).quantile(0.99).item() < 1e-4
    # a context without a tape re-clips: the same as recompute
    nt = vdmod.Context(0, {"tape": 0})
    build(nt, x, w)
    gp_n, _ = nt.backward(gv, gc, want_weights=weighted)
    assert torch.allclose(gp_n, gp_r, rtol=1e-5, atol=1e-6 * gp_r.abs().max().item())
