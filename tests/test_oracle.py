"""Pins for the FP64 CPU oracle against facts that do not come from the
oracle itself: closed forms, library cross-checks (Qhull via scipy),
exact-integer certificates, invariants of Eq. 1 and finite differences.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2605_06408_gb300 import workloads as W

BOX = ((0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def edges(nbrs):
    return {(i, int(j)) for i, nb in enumerate(nbrs) for j in nb}


# ---------------------------------------------------------------- closed forms

def test_single_site_is_the_box():
    x = np.array([[0.3, 0.6, 0.2]], np.float32)
    box = ((-1.0, 0.0, 0.5 - 1.0), (2.0, 0.75, 1.5))
    r = oracle.cells(x, bbox=box)
    assert r["counts"][0] == 0
    assert r["vol"][0] == pytest.approx(3.0 * 0.75 * 2.0, rel=1e-14)
    np.testing.assert_allclose(r["cen"][0], [0.5, 0.375, 0.5], rtol=0, atol=1e-14)


def test_two_site_closed_forms():
    """Golden two-site cells (tests/golden/closed_forms.json, Sec. 3 Eq. 1)."""
    with open(os.path.join(GOLDEN, "closed_forms.json")) as f:
        g = json.load(f)
    for case in g["cases"]:
        x = np.array(case["xyz"], np.float32)
        w = np.array(case["w"], np.float32)
        r = oracle.cells(x, w, bbox=g["box"], mode="brute")
        for i in range(2):
            assert r["vol"][i] == pytest.approx(case["vol"][i], rel=1e-11, abs=1e-14)
            if case["vol"][i] > 0 and case["vol"][1 - i] > 0:
                assert list(r["nbrs"][i]) == [1 - i]
        if case["kind"] == "slab":
            for i in range(2):
                if case["vol"][i] > 1e-9:
                    np.testing.assert_allclose(r["cen"][i], case["cen"][i], rtol=0, atol=1e-11)


def test_dominant_weight_owns_the_box():
    x = W.uniform(200, 5)
    w = np.zeros(200, np.float32)
    w[17] = 10.0  # > squared box diagonal: pow(x, 17) < pow(x, j) everywhere
    r = oracle.cells(x, w)
    assert r["vol"][17] == pytest.approx(1.0, rel=1e-13)
    assert r["counts"][17] == 0
    others = np.arange(200) != 17
    assert np.all(r["vol"][others] == 0.0) and np.all(r["counts"][others] == 0)
    np.testing.assert_array_equal(r["cen"][others], x[others].astype(np.float64))
    assert r["stats"]["empty"] == 199


def test_bcc_truncated_octahedra():
    """Interior cells of a (slightly jittered) BCC lattice with cube side a
    are truncated octahedra: 14 neighbours, V = a^3/2, centroid = site."""
    x, a = W.bcc_lattice(k=3, jitter=1e-7)
    r = oracle.cells(x)
    interior = np.all((x > 1.5 * a) & (x < 1.0 - 1.5 * a), axis=1)
    assert interior.sum() > 50
    assert np.all(r["counts"][interior] == 14)
    assert np.all(r["nverts"][interior] == 24)
    np.testing.assert_allclose(r["vol"][interior], a ** 3 / 2, rtol=1e-5)
    np.testing.assert_allclose(r["cen"][interior], x[interior], rtol=0, atol=1e-6 * a)
    # the 14 are the 8 body-diagonal and 6 axis lattice neighbours
    for i in np.nonzero(interior)[0][:20]:
        d = np.linalg.norm(x[r["nbrs"][i]] - x[i], axis=1) / a
        assert np.sum(np.abs(d - np.sqrt(3) / 2) < 1e-3) == 8
        assert np.sum(np.abs(d - 1.0) < 1e-3) == 6


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("kind", ["uniform", "mixture", "power"])
def test_partition_invariants(kind):
    n = 3000
    if kind == "uniform":
        x, w = W.uniform(n, 0), None
    else:
        x = W.mixture(n, 1)
        w = W.power_weights(x, 2) if kind == "power" else None
    r = oracle.cells(x, w)
    assert r["stats"]["ambiguous"] == 0
    assert r["stats"]["topo_fail"] == 0 and r["stats"]["facewalk_fail"] == 0
    # cells partition the box: volumes and first moments add up
    assert r["vol"].sum() == pytest.approx(1.0, rel=1e-12)
    mom = (r["vol"][:, None] * r["cen"]).sum(0)
    np.testing.assert_allclose(mom, [0.5, 0.5, 0.5], rtol=1e-12)
    assert np.all(r["vol"] >= 0)
    # adjacency is symmetric
    E = edges(r["nbrs"])
    assert all((j, i) in E for (i, j) in E)
    assert len(E) % 2 == 0
    # simple polytopes: every vertex has degree 3, so F = V/2 + 2
    ne = r["nverts"] > 0
    np.testing.assert_array_equal(r["nfaces"][ne], r["nverts"][ne] // 2 + 2)
    assert np.all(r["nverts"][ne] % 2 == 0)
    if kind == "power":
        assert r["stats"]["empty"] > 0  # weights large enough to hide sites
        empty = r["vol"] == 0
        np.testing.assert_array_equal(r["cen"][empty], x[empty].astype(np.float64))


def test_equal_weights_reproduce_voronoi():
    x = W.mixture(2000, 3)
    v = oracle.cells(x)
    for c in (0.0, 0.25, -3.0):
        p = oracle.cells(x, np.full(2000, c, np.float32))
        assert all(np.array_equal(a, b) for a, b in zip(v["nbrs"], p["nbrs"]))
        np.testing.assert_allclose(p["vol"], v["vol"], rtol=1e-9, atol=1e-15)


def test_weight_shift_and_scaling_invariance():
    x = W.uniform(1500, 9)
    w = W.power_weights(x, 4)
    base = oracle.cells(x, w)
    # adding a constant (a power of two keeps float32 exact) changes nothing
    shifted = oracle.cells(x, (w.astype(np.float64) + 0.5).astype(np.float32))
    same = sum(np.array_equal(a, b) for a, b in zip(base["nbrs"], shifted["nbrs"]))
    assert same == len(x)
    # scaling positions by 2 and weights by 4 scales volumes by 8
    scaled = oracle.cells(2 * x, 4 * w, bbox=((0, 0, 0), (2, 2, 2)))
    assert all(np.array_equal(a, b) for a, b in zip(base["nbrs"], scaled["nbrs"]))
    np.testing.assert_allclose(scaled["vol"], 8 * base["vol"], rtol=1e-10, atol=1e-18)


def test_duplicates_and_outside_sites():
    x = np.array([[0.2, 0.2, 0.2], [0.8, 0.5, 0.5], [0.2, 0.2, 0.2], [0.5, 0.9, 0.1]], np.float32)
    r = oracle.cells(x)
    assert r["vol"][2] == 0.0 and r["counts"][2] == 0  # equal weight: lower index wins
    assert r["vol"][0] > 0
    assert np.all(np.isfinite(r["vol"])) and r["vol"].sum() == pytest.approx(1.0, rel=1e-12)
    assert all(2 not in nb for nb in r["nbrs"])  # the loser is nobody's neighbour
    assert r["stats"]["ambiguous"] == 0
    w = np.array([0.0, 0.0, 0.01, 0.0], np.float32)
    r = oracle.cells(x, w)
    assert r["vol"][0] == 0.0 and r["vol"][2] > 0  # larger weight wins
    assert r["vol"].sum() == pytest.approx(1.0, rel=1e-12)
    # a site outside the box still owns the part of the box nearest to it
    y = np.array([[-0.25, 0.5, 0.5], [0.75, 0.5, 0.5]], np.float32)
    r = oracle.cells(y)
    assert r["vol"][0] == pytest.approx(0.25, rel=1e-13)  # bisector x = 0.25
    assert list(r["nbrs"][0]) == [1]
    y = np.array([[-0.5, 0.5, 0.5], [0.5, 0.5, 0.5]], np.float32)
    assert oracle.cells(y)["vol"][0] == 0.0  # bisector on the box face


# ---------------------------------------------------------------- brute force vs k-d stream

def test_brute_equals_kd_on_uniform_10k():
    x, _, box = W.config("uniform10k")
    a = oracle.cells(x, bbox=box, mode="kd")
    b = oracle.cells(x, bbox=box, mode="brute")
    assert all(np.array_equal(p, q) for p, q in zip(a["nbrs"], b["nbrs"]))
    np.testing.assert_allclose(a["vol"], b["vol"], rtol=1e-12)
    assert a["stats"]["ambiguous"] == 0 and b["stats"]["ambiguous"] == 0


def test_brute_equals_kd_on_weighted_subset():
    x = W.mixture(6000, 12)
    w = W.power_weights(x, 13)
    a = oracle.cells(x, w, mode="kd")
    b = oracle.cells(x, w, mode="brute")
    assert all(np.array_equal(p, q) for p, q in zip(a["nbrs"], b["nbrs"]))
    np.testing.assert_allclose(a["vol"], b["vol"], rtol=1e-11, atol=1e-18)


# ---------------------------------------------------------------- exact arithmetic

@pytest.mark.parametrize("weighted", [False, True])
def test_exact_predicates_agree_and_certify(weighted):
    x = W.snap_to_grid(W.mixture(1500, 21))
    w = W.snap_weights(W.power_weights(x, 22)) if weighted else None
    e = oracle.cells(x, w, exact=True)
    f = oracle.cells(x, w, exact=False)
    assert e["stats"]["degenerate"] == 0 and e["stats"]["orient_fail"] == 0
    assert f["stats"]["ambiguous"] == 0
    assert all(np.array_equal(p, q) for p, q in zip(e["nbrs"], f["nbrs"]))
    # empty-sphere certificate in exact integer arithmetic: no final vertex
    # of cell i has smaller power distance to any other site
    viol, st = oracle.certify(x, w, exact=True)
    assert viol.sum() == 0 and st["degenerate"] == 0


def _rational_side(x, w, box, i, ids):
    """Sign of pow(v, i) - pow(v, h) (Eq. 1: positive means v lies outside
    the half-space of h) for the vertex v where the three planes of ids[:3]
    meet, all in exact rational arithmetic from the float32 inputs; box face
    f bounds the cell by the box side it names."""
    from fractions import Fraction as F

    P = [[F(float(c)) for c in x[k]] for k in range(len(x))]
    Wt = [F(float(c)) for c in (w if w is not None else np.zeros(len(x)))]
    lo = [F(float(c)) for c in box[0]]
    hi = [F(float(c)) for c in box[1]]

    def row(j):  # a . X = r in world coordinates X
        if j >= 0:
            a = [2 * (P[j][k] - P[i][k]) for k in range(3)]
            r = sum(P[j][k] ** 2 - P[i][k] ** 2 for k in range(3)) + Wt[i] - Wt[j]
            return a, r
        f = -1 - j
        ax = f >> 1
        a = [F(0)] * 3
        a[ax] = F(-1) if f & 1 else F(1)
        return a, (-lo[ax] if f & 1 else hi[ax])

    A, r = zip(*[row(j) for j in ids[:3]])

    def det(m):
        return (m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
                + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]))

    D = det(A)
    if D == 0:
        return 0
    X = []
    for k in range(3):
        m = [list(a) for a in A]
        for q in range(3):
            m[q][k] = r[q]
        X.append(det(m) / D)
    h = ids[3]
    if h >= 0:
        pi = sum((X[k] - P[i][k]) ** 2 for k in range(3)) - Wt[i]
        ph = sum((X[k] - P[h][k]) ** 2 for k in range(3)) - Wt[h]
        d = pi - ph
    else:
        f = -1 - h
        ax = f >> 1
        d = (lo[ax] - X[ax]) if f & 1 else (X[ax] - hi[ax])
    return (d > 0) - (d < 0)


def test_exact_side_matches_rational_arithmetic():
    """The expansion arithmetic behind the oracle's exact fallback against
    exact rationals (Python fractions) on random, exactly degenerate and
    near-degenerate configurations, Voronoi and power, with box faces."""
    rng = W.rng_for(5)
    box = ((0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    counts = {-1: 0, 0: 0, 1: 0}
    for t in range(320):
        kind = t % 4 if t < 240 else 4 + t % 2
        if kind == 0:  # generic
            x = rng.random((5, 3)).astype(np.float32)
        elif kind >= 4:
            # five sites at sign / permutation images of one offset d about a
            # centre c (all at |d| from c), d with 21 random bits per axis:
            # exactly degenerate, but the determinants' products need more
            # than 53 bits (kind 5: the last site one ulp off the sphere)
            d = (rng.integers(2 ** 20, 2 ** 21, 3) * 2.0 ** -24).astype(np.float64)
            imgs = [(0, 1, 2, 1, 1, 1), (1, 2, 0, -1, 1, 1), (2, 0, 1, 1, -1, 1), (0, 2, 1, 1, 1, -1),
                    (2, 1, 0, -1, -1, 1)]
            x = np.array([[0.5 + sx * d[a], 0.5 + sy * d[b], 0.5 + sz * d[c_]] for a, b, c_, sx, sy, sz in imgs],
                         np.float64)
            assert np.all(x.astype(np.float32).astype(np.float64) == x)
            x = x.astype(np.float32)
            if kind == 5:
                k = int(rng.integers(0, 3))
                x[4, k] = np.nextafter(x[4, k], np.float32(2.0 if t % 4 == 1 else -2.0))
        elif kind == 1:  # five sites on one sphere: exactly degenerate
            c = rng.integers(8, 24, 3)
            pts = [c + np.array(v) for v in ((3, 0, 0), (-3, 0, 0), (0, 3, 0), (0, 0, -3), (0, -3, 0))]
            x = (np.array(pts, np.float64) / 32.0).astype(np.float32)
        else:  # one site moved by one float32 ulp off a common sphere
            c = rng.integers(8, 24, 3)
            pts = [c + np.array(v) for v in ((3, 0, 0), (-3, 0, 0), (0, 3, 0), (0, 0, -3), (0, -3, 0))]
            x = (np.array(pts, np.float64) / 32.0).astype(np.float32)
            k = int(rng.integers(0, 3))
            x[4, k] = np.nextafter(x[4, k], np.float32(2.0 if kind == 2 else -2.0))
        w = None
        if t % 8 >= 4:  # power: equal weights keep the sphere; others perturb it
            w = np.full(5, 0.001, np.float32) if kind in (1, 4) else (rng.random(5) * 1e-3).astype(np.float32)
        ids = [1, 2, 3, 4]
        if t % 5 == 0 and kind < 4:
            ids = [1, 2, -1 - int(rng.integers(0, 6)), 4]  # a box face among the three planes
        got = oracle.exact_side(x, w, box, 0, ids)
        want = _rational_side(x, w, box, 0, ids)
        assert got == want, (t, got, want)
        counts[want] += 1
    assert counts[0] >= 40 and counts[1] >= 20 and counts[-1] >= 20


@pytest.mark.parametrize("weighted", [False, True])
def test_fp64_with_exact_fallback_equals_integer_mode_on_degenerate_lattices(weighted):
    """On a cubic and a BCC lattice (five or more cospherical sites
    everywhere: many predicates exactly 0) the FP64 filter cannot decide;
    its exact fallback must take exactly the decisions of the integer mode,
    so every cell is the same."""
    # spacing: 17 random bits on the 2^-20 grid, so that the integer mode
    # applies and the FP64 determinants round (their products pass 53 bits)
    a = int(W.rng_for(8).integers(2 ** 16, 2 ** 17)) * 2.0 ** -20
    k = np.stack(np.meshgrid(*[np.arange(6)] * 3, indexing="ij"), -1).reshape(-1, 3).astype(np.float64)
    cube = 0.25 + k * a
    bcc = np.concatenate([cube, 0.25 + (k[:125] + 0.5) * a])
    assert np.all(np.round(bcc * 2 ** 20) == bcc * 2 ** 20)
    for pts in (cube, bcc):
        x = pts.astype(np.float32)
        w = np.full(len(x), 2.0 ** -10, np.float32) if weighted else None
        e = oracle.cells(x, w, exact=True)
        f = oracle.cells(x, w, exact=False)
        assert e["stats"]["degenerate"] > 0
        assert f["stats"]["exact_resolved"] > 0 and f["stats"]["ambiguous"] == 0
        assert f["stats"]["degenerate"] == e["stats"]["degenerate"]
        assert all(np.array_equal(p, q) for p, q in zip(e["nbrs"], f["nbrs"]))
        np.testing.assert_allclose(f["vol"], e["vol"], rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------- library cross-checks

def test_voronoi_neighbours_equal_qhull_delaunay_edges():
    from scipy.spatial import Delaunay

    x = W.uniform(400, 31)
    big = ((-1e5,) * 3, (1e5,) * 3)
    r = oracle.cells(x, bbox=big)
    tri = Delaunay(x.astype(np.float64))
    E = {(int(s[a]), int(s[b])) for s in tri.simplices for a in range(4) for b in range(4) if a != b}
    assert edges(r["nbrs"]) == E


def test_power_neighbours_equal_lifted_lower_hull_edges():
    from scipy.spatial import ConvexHull

    x = W.uniform(300, 32)
    w = W.power_weights(x, 33, scale=0.5)
    big = ((-1e4,) * 3, (1e4,) * 3)
    r = oracle.cells(x, w, bbox=big)
    p = x.astype(np.float64)
    lift = np.concatenate([p, (p * p).sum(1, keepdims=True) - w.astype(np.float64)[:, None]], 1)
    hull = ConvexHull(lift)
    E = set()
    for s, eq in zip(hull.simplices, hull.equations):
        if eq[3] < 0:  # facet of the lower hull (outward normal points down)
            E |= {(int(s[a]), int(s[b])) for a in range(4) for b in range(4) if a != b}
    assert edges(r["nbrs"]) == E


def test_poisson_voronoi_meijering_means():
    """Mean faces 48 pi^2/35 + 2 = 15.54 and vertices 96 pi^2/35 = 27.07 per
    interior Poisson-Voronoi cell (Meijering 1953)."""
    x, _, box = W.config("uniform10k")
    r = oracle.cells(x, bbox=box)
    h = 2.5 * (1.0 / 10_000) ** (1 / 3)
    interior = np.all((x > h) & (x < 1 - h), axis=1)
    assert interior.sum() > 4000
    assert r["nfaces"][interior].mean() == pytest.approx(48 * np.pi ** 2 / 35 + 2, abs=0.15)
    assert r["nverts"][interior].mean() == pytest.approx(96 * np.pi ** 2 / 35, abs=0.3)


# ---------------------------------------------------------------- gradients

def _loss(x, w, c, d):
    r = oracle.cells(x, w)
    return float((c * r["vol"]).sum() + (d * r["cen"]).sum()), r["nbrs"]


@pytest.mark.parametrize("weighted", [False, True])
def test_gradient_matches_central_differences(weighted):
    n = 120
    x = W.uniform(n, 41)
    w = W.power_weights(x, 42, scale=0.5) if weighted else None
    c, d = W.loss_coefficients(n, 43)
    gp, gw, st = oracle.grad(x, w, BOX, c, d)
    rng = W.rng_for(44)
    _, nb0 = _loss(x, w, c, d)
    for k in rng.choice(n, 6, replace=False):
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[k, a] = np.float32(x[k, a] + 2.0 ** -16)
            xm[k, a] = np.float32(x[k, a] - 2.0 ** -16)
            Lp, nbp = _loss(xp, w, c, d)
            Lm, nbm = _loss(xm, w, c, d)
            if not all(np.array_equal(u, v) for u, v in zip(nbp, nbm)):
                continue  # combinatorics changed within +-h: outside the contract
            fd = (Lp - Lm) / (float(xp[k, a]) - float(xm[k, a]))
            assert fd == pytest.approx(gp[k, a], rel=2e-5, abs=2e-6)
        if weighted:
            wp, wm = w.copy(), w.copy()
            hw = max(2.0 ** -30, 64 * float(np.spacing(w[k])))
            wp[k] = np.float32(w[k] + hw)
            wm[k] = np.float32(w[k] - hw)
            fd = (_loss(x, wp, c, d)[0] - _loss(x, wm, c, d)[0]) / (float(wp[k]) - float(wm[k]))
            assert fd == pytest.approx(gw[k], rel=2e-5, abs=2e-6)


def test_total_volume_gradient_vanishes():
    """sum_i V_i = vol(box) for every configuration, so its gradient is 0."""
    n = 500
    x = W.mixture(n, 51)
    w = W.power_weights(x, 52)
    gp, gw, _ = oracle.grad(x, w, BOX, np.ones(n), np.zeros((n, 3)))
    r = oracle.cells(x, w)
    scale = np.mean(r["vol"] ** (2.0 / 3.0))  # typical face area
    assert np.abs(gp).max() < 1e-9 * scale
    assert np.abs(gw).max() < 1e-9 * scale / np.median(r["vol"][r["vol"] > 0] ** (1 / 3))


def test_gradient_subset_matches_full():
    n = 400
    x = W.uniform(n, 61)
    c, d = W.loss_coefficients(n, 62)
    gp, gw, _ = oracle.grad(x, None, BOX, c, d)
    r = oracle.cells(x)
    k = 123
    sub = np.unique(np.concatenate([[k], r["nbrs"][k]])).astype(np.int64)
    gps, gws, _ = oracle.grad(x, None, BOX, c, d, cells=sub)
    np.testing.assert_allclose(gps[k], gp[k], rtol=1e-12, atol=1e-15)
    assert gws[k] == pytest.approx(gw[k], rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("weighted", [False, True])
def test_fd_grad_matches_analytic_and_full_rebuild(weighted):
    """oracle.fd_grad (central differences in FP64, each affected cell
    rebuilt from its neighbour row) agrees with the Reynolds-transport
    gradient and with differences of full rebuilds (float32 steps)."""
    n = 150
    x = W.uniform(n, 71)
    w = W.power_weights(x, 72, scale=0.5) if weighted else None
    c, d = W.loss_coefficients(n, 73)
    r = oracle.cells(x, w)
    off = np.concatenate([[0], np.cumsum([len(v) for v in r["nbrs"]])]).astype(np.int64)
    nb = np.concatenate(r["nbrs"]).astype(np.int32)
    sites = np.arange(n, dtype=np.int64)
    gp_fd, gw_fd = oracle.fd_grad(x, w, BOX, off, nb, c, d, sites, hx=1e-7, hw=1e-9)
    gp, gw, _ = oracle.grad(x, w, BOX, c, d)
    scale = np.abs(gp).max()
    np.testing.assert_allclose(gp_fd, gp, rtol=1e-6, atol=1e-7 * scale)
    if weighted:
        np.testing.assert_allclose(gw_fd, gw, rtol=1e-5, atol=1e-6 * np.abs(gw).max())
    # against full rebuilds with float32 steps where the combinatorics hold
    # (non-empty cells: an empty cell reports its site as centroid)
    for k in [q for q in range(n) if r["vol"][q] > 0][:3]:
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[k, a] = np.float32(x[k, a] + 2.0 ** -16)
            xm[k, a] = np.float32(x[k, a] - 2.0 ** -16)
            Lp, nbp = _loss(xp, w, c, d)
            Lm, nbm = _loss(xm, w, c, d)
            if not all(np.array_equal(u, v) for u, v in zip(nbp, nbm)):
                continue
            fd = (Lp - Lm) / (float(xp[k, a]) - float(xm[k, a]))
            assert fd == pytest.approx(gp_fd[k, a], rel=2e-5, abs=2e-6)


def _vertex_key_grad(i, t):
    # a fixed pseudo-random gradient per (cell, defining sites)
    a, b, c = sorted(t)
    return np.array([np.sin(0.37 * i + 0.11 * a + 0.05 * b + 0.02 * c),
                     np.cos(0.29 * i - 0.07 * a + 0.13 * b - 0.03 * c),
                     np.sin(0.19 * i + 0.17 * a - 0.09 * b + 0.23 * c)])


@pytest.mark.parametrize("weighted", [False, True])
def test_vertex_grad_matches_central_differences(weighted):
    """oracle.vertex_grad (implicit differentiation of each vertex's 3x3
    system) against differences of the vertices rebuilt around a perturbed
    site, vertices matched by their defining sites."""
    n = 60
    x = W.uniform(n, 81)
    w = W.power_weights(x, 82, scale=0.5) if weighted else None
    cells = np.arange(n)
    gp, gw = oracle.vertex_grad(x, w, BOX, cells, _vertex_key_grad)

    def loss(xx, ww):
        L, keys = 0.0, []
        for i in cells:
            pos, tri = oracle.cell_vertices(xx, ww, BOX, int(i))
            for v, t in zip(pos, tri):
                L += float(_vertex_key_grad(int(i), tuple(t)) @ (xx[i].astype(np.float64) + v))
                keys.append((int(i),) + tuple(sorted(t)))
        return L, sorted(keys)

    checked = 0
    for k in (5, 17, 33):
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[k, a] = np.float32(x[k, a] + 2.0 ** -14)
            xm[k, a] = np.float32(x[k, a] - 2.0 ** -14)
            Lp, kp = loss(xp, w)
            Lm, km = loss(xm, w)
            if kp != km:
                continue  # combinatorics changed within +-h
            fd = (Lp - Lm) / (float(xp[k, a]) - float(xm[k, a]))
            assert fd == pytest.approx(gp[k, a], rel=1e-4, abs=1e-5)
            checked += 1
        if weighted:
            wp, wm = w.copy(), w.copy()
            hw = max(2.0 ** -26, 64 * float(np.spacing(w[k])))
            wp[k] = np.float32(w[k] + hw)
            wm[k] = np.float32(w[k] - hw)
            Lp, kp = loss(x, wp)
            Lm, km = loss(x, wm)
            if kp == km:
                fd = (Lp - Lm) / (float(wp[k]) - float(wm[k]))
                assert fd == pytest.approx(gw[k], rel=1e-4, abs=1e-4)
    assert checked >= 6
