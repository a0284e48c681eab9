"""Seeded synthetic point sets shaped like the paper's workloads.

This module holds input generators only: no clipping, culling or any other
arithmetic of the method. Both the CUDA path's tests/benchmark and the
oracle's tests draw their inputs from here.

Every generator uses ``numpy.random.Generator(PCG64(seed))`` and returns
float32 arrays. Exact duplicate positions (after rounding to float32) are
removed, and draws that fall outside the box are redrawn (truncated
distributions), so that inputs are in generic position.

Workloads (box = unit cube unless stated):
  uniform      -- white noise, Sec. 5.1 "Synthetic test cases", Eq. 3
                  (the paper's [-10,10]^3 rescaled to [0,1]^3).
  mixture      -- 64 anisotropic Gaussian clusters (per-axis sigma
                  log-uniform in [1e-3, 1e-1]) + 10% uniform background: a
                  heavier-tailed version of the clustered set of Sec. 5.1.
  power_weights-- w_i = r_i^2, r_i = 0.2 * nn_i * exp(N(0,1)) with nn_i the
                  site's own nearest-neighbour distance (stands in for the
                  weighted sets of Sec. 5.1 "Power diagrams"; produces
                  empty cells).
  gaussian_weights -- the paper's own weights w ~ N(0, (d_nn^2/3)^2).
  gradient     -- linear density gradient along x (Sec. 5.1, third set).
  batched      -- 256 independent sets, sizes log-uniform in [1e3, 2e5].
  surfaces     -- nested Gaussian shells (sigma 1e-2 .. 1e-5) around 32
                  random smooth surfaces + 1% background: density spanning
                  more than four orders of magnitude, standing in for the
                  Radiant Foam scenes (Sec. 5.1 "Real-world test cases"),
                  whose checkpoints are not available here.
"""
from __future__ import annotations

import numpy as np

UNIT_BOX = ((0.0, 0.0, 0.0), (1.0, 1.0, 1.0))


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def dedupe(x: np.ndarray) -> np.ndarray:
    """Drop exact duplicate rows (float32 bit patterns), keeping the first
    occurrence and the original order."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    if x.shape[0] < 2:
        return x
    b = x.view(np.uint32).reshape(-1, 3)
    k1 = (b[:, 0].astype(np.uint64) << np.uint64(32)) | b[:, 1].astype(np.uint64)
    k2 = b[:, 2]
    order = np.lexsort((np.arange(x.shape[0]), k2, k1))
    s1, s2 = k1[order], k2[order]
    dup = np.zeros(x.shape[0], bool)
    dup[1:] = (s1[1:] == s1[:-1]) & (s2[1:] == s2[:-1])
    keep = np.ones(x.shape[0], bool)
    keep[order[dup]] = False
    return x[keep]


def _in_box(p: np.ndarray) -> np.ndarray:
    return np.all((p >= 0.0) & (p <= 1.0), axis=1)


def uniform(n: int, seed: int = 0) -> np.ndarray:
    """n sites uniform in [0,1)^3."""
    rng = rng_for(seed)
    out = np.zeros((0, 3), np.float32)
    while out.shape[0] < n:
        m = n - out.shape[0]
        draw = rng.random((m + m // 100 + 16, 3), dtype=np.float32)
        out = dedupe(np.concatenate([out, draw]))
    return np.ascontiguousarray(out[:n])


def _gauss_truncated(rng, centre, sigma, m):
    """m draws of N(centre, diag(sigma^2)) redrawn until inside the box."""
    pts = np.zeros((0, 3), np.float64)
    while pts.shape[0] < m:
        k = m - pts.shape[0]
        d = centre + rng.standard_normal((2 * k + 16, 3)) * sigma
        d = d[_in_box(d)]
        pts = np.concatenate([pts, d[:k]])
    return pts


def mixture(n: int, seed: int = 1, clusters: int = 64, background: float = 0.10) -> np.ndarray:
    """Anisotropic Gaussian mixture + uniform background, float32, deduped."""
    rng = rng_for(seed)
    centres = rng.random((clusters, 3))
    sigmas = 10.0 ** rng.uniform(-3.0, -1.0, size=(clusters, 3))

    def draw(m):
        n_bg = int(round(background * m))
        n_cl = m - n_bg
        per = np.full(clusters, n_cl // clusters)
        per[: n_cl - per.sum()] += 1
        parts = [_gauss_truncated(rng, centres[c], sigmas[c], int(per[c])) for c in range(clusters)]
        parts.append(rng.random((n_bg, 3)))
        return np.concatenate(parts).astype(np.float32)

    out = dedupe(draw(n))
    while out.shape[0] < n:
        out = dedupe(np.concatenate([out, draw(n - out.shape[0] + 16)]))
    out = out[:n]
    return np.ascontiguousarray(out[rng.permutation(n)])


def clustered(n: int, clusters: int, seed: int = 6, sigma: float = 0.005) -> np.ndarray:
    """The paper's clustered test case (Sec. 5.1) scaled to the unit box:
    `clusters` centres uniform in the box, sites split evenly among them,
    isotropic Gaussian with sigma = 0.1 / 20 (0.1 in the paper's [-10, 10]^3),
    clamped to the box; float32, deduped."""
    rng = rng_for(seed)
    centres = rng.random((clusters, 3))

    def draw(m):
        per = np.full(clusters, m // clusters)
        per[: m - per.sum()] += 1
        lab = np.repeat(np.arange(clusters), per)
        p = centres[lab] + sigma * rng.standard_normal((m, 3))
        return np.clip(p, 0.0, 1.0).astype(np.float32)

    out = dedupe(draw(n))
    while out.shape[0] < n:
        out = dedupe(np.concatenate([out, draw(n - out.shape[0] + 16)]))
    out = out[:n]
    return np.ascontiguousarray(out[rng.permutation(n)])


def nearest_neighbour_distance(x: np.ndarray) -> np.ndarray:
    """Each site's distance to its nearest other site (float64)."""
    from scipy.spatial import cKDTree

    p = np.asarray(x, dtype=np.float64)
    d, _ = cKDTree(p).query(p, k=2)
    return d[:, 1]


def power_weights(x: np.ndarray, seed: int = 2, scale: float = 0.2, sigma: float = 1.0) -> np.ndarray:
    """w_i = r_i^2 with r_i = scale * nn_i * exp(sigma * N(0,1))."""
    rng = rng_for(seed)
    nn = nearest_neighbour_distance(x)
    r = scale * nn * np.exp(sigma * rng.standard_normal(x.shape[0]))
    return (r * r).astype(np.float32)


def gaussian_weights(x: np.ndarray, seed: int = 2, ratio: float = 1.0 / 3.0) -> np.ndarray:
    """The paper's power-diagram weights: w ~ N(0, (r d_nn^2)^2), d_nn the
    median nearest-neighbour distance, r = 1/3 in its main runs (Sec. 5.1)
    and swept in its weight-distribution ablation."""
    rng = rng_for(seed)
    dnn = float(np.median(nearest_neighbour_distance(x)))
    return (rng.standard_normal(x.shape[0]) * (ratio * dnn * dnn)).astype(np.float32)


def gradient(n: int, seed: int = 5) -> np.ndarray:
    """Density growing linearly along x: x = sqrt(u), y, z uniform."""
    rng = rng_for(seed)
    out = np.zeros((0, 3), np.float32)
    while out.shape[0] < n:
        m = n - out.shape[0] + 16
        p = np.empty((m, 3))
        p[:, 0] = np.sqrt(rng.random(m))
        p[:, 1:] = rng.random((m, 2))
        out = dedupe(np.concatenate([out, p.astype(np.float32)]))
    return np.ascontiguousarray(out[:n])


def batched(seed: int = 3, nsets: int = 256, lo: float = 1e3, hi: float = 2e5):
    """256 independent sets. Returns (xyz float32[N,3], weights float32[N]
    (zeros for Voronoi sets), offsets int64[nsets+1], weighted uint8[nsets])."""
    rng = rng_for(seed)
    sizes = np.rint(10.0 ** rng.uniform(np.log10(lo), np.log10(hi), size=nsets)).astype(np.int64)
    kinds = rng.random(nsets)
    xs, ws, flags = [], [], []
    for s in range(nsets):
        sub_seed = int(rng.integers(0, 2**31 - 1))
        m = int(sizes[s])
        pts = uniform(m, sub_seed) if kinds[s] < 0.5 else mixture(m, sub_seed)
        weighted = s % 2 == 1
        w = power_weights(pts, sub_seed + 1) if weighted else np.zeros(m, np.float32)
        xs.append(pts)
        ws.append(w)
        flags.append(1 if weighted else 0)
    offsets = np.zeros(nsets + 1, np.int64)
    offsets[1:] = np.cumsum(sizes)
    return (np.ascontiguousarray(np.concatenate(xs)), np.ascontiguousarray(np.concatenate(ws)),
            offsets, np.asarray(flags, np.uint8))


def _random_rotation(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    return q * np.sign(np.diag(r))


def _surface_points(rng, kind, prm, m):
    """m points on a surface with unit normals."""
    if kind == 0:  # sphere
        c, R = prm
        u = rng.standard_normal((m, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        return c + R * u, u
    if kind == 1:  # torus
        c, R, r, Q = prm
        a = rng.random(m) * 2 * np.pi
        b = rng.random(m) * 2 * np.pi
        ring = np.stack([np.cos(a), np.sin(a), np.zeros(m)], 1)
        nrm = np.cos(b)[:, None] * ring + np.sin(b)[:, None] * np.array([0.0, 0.0, 1.0])
        p = R * ring + r * nrm
        return c + p @ Q.T, nrm @ Q.T
    # height field z = z0 + sum_k a_k sin(f_k . (x, y) + phi_k), along axis ax
    z0, amp, freq, phase, ax = prm
    uv = rng.random((m, 2))
    arg = uv @ freq.T + phase
    h = z0 + np.sin(arg) @ amp
    dh = (np.cos(arg) * amp) @ freq  # gradient of h
    nrm = np.concatenate([-dh, np.ones((m, 1))], 1)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    p = np.concatenate([uv, h[:, None]], 1)
    perm = [(1, 2, 0), (2, 0, 1), (0, 1, 2)][ax]
    inv = np.argsort(perm)
    return p[:, inv], nrm[:, inv]


def surfaces(n: int, seed: int = 4, nsurf: int = 32, sigmas=(1e-2, 1e-3, 1e-4, 1e-5),
             background: float = 0.01) -> np.ndarray:
    """Nested Gaussian shells around random smooth surfaces + background."""
    rng = rng_for(seed)
    surf = []
    for s in range(nsurf):
        kind = s % 3
        if kind == 0:
            surf.append((0, (rng.uniform(0.2, 0.8, 3), rng.uniform(0.05, 0.3))))
        elif kind == 1:
            R = rng.uniform(0.1, 0.25)
            surf.append((1, (rng.uniform(0.3, 0.7, 3), R, R * rng.uniform(0.15, 0.5), _random_rotation(rng))))
        else:
            k = 4
            surf.append((2, (rng.uniform(0.3, 0.7), rng.uniform(0.01, 0.05, k),
                             rng.uniform(2, 12, (k, 2)) * rng.choice([-1, 1], (k, 2)),
                             rng.uniform(0, 2 * np.pi, k), int(rng.integers(0, 3)))))

    def draw(m):
        n_bg = int(round(background * m))
        n_sh = m - n_bg
        per = np.full(nsurf * len(sigmas), n_sh // (nsurf * len(sigmas)))
        per[: n_sh - per.sum()] += 1
        parts = [rng.random((n_bg, 3))]
        q = 0
        for kind, prm in surf:
            for sg in sigmas:
                k = int(per[q])
                q += 1
                got = np.zeros((0, 3))
                while got.shape[0] < k:
                    t = k - got.shape[0]
                    p, nrm = _surface_points(rng, kind, prm, 2 * t + 16)
                    p = p + nrm * (sg * rng.standard_normal((p.shape[0], 1)))
                    p = p[_in_box(p)]
                    got = np.concatenate([got, p[:t]])
                parts.append(got)
        return np.concatenate(parts).astype(np.float32)

    out = dedupe(draw(n))
    while out.shape[0] < n:
        out = dedupe(np.concatenate([out, draw(max(n - out.shape[0], 1024))]))
    out = out[:n]
    return np.ascontiguousarray(out[rng.permutation(n)])


def loss_coefficients(n: int, seed: int = 4):
    """Seeded c_i ~ N(0,1), d_i ~ N(0, I_3) for L = sum c_i V_i + d_i . g_i."""
    rng = rng_for(seed + 1000)
    return rng.standard_normal(n), rng.standard_normal((n, 3))


def snap_to_grid(x: np.ndarray, bits: int = 20) -> np.ndarray:
    """Round coordinates down to the 2^-bits grid (exactly representable)."""
    s = float(2 ** bits)
    return dedupe((np.floor(np.asarray(x, np.float64) * s) / s).astype(np.float32))


def snap_weights(w: np.ndarray, bits: int = 40) -> np.ndarray:
    s = float(2 ** bits)
    return (np.round(np.asarray(w, np.float64) * s) / s).astype(np.float32)


def bcc_lattice(k: int = 3, seed: int = 7, jitter: float = 0.0):
    """Body-centred cubic lattice with cube side a = 2^-k inside the unit
    box, offset from the box faces, with optional uniform jitter (fraction
    of a). Returns (xyz float32, a)."""
    a = 2.0 ** -k
    m = int(round(1.0 / a))
    g = (np.arange(m) + 0.25) * a
    c = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    b = c + 0.5 * a
    b = b[np.all(b < 1.0, axis=1)]
    p = np.concatenate([c, b])
    if jitter:
        rng = rng_for(seed)
        p = p + rng.uniform(-jitter * a, jitter * a, p.shape)
    return p.astype(np.float32), a


def config(name: str):
    """The benchmark configurations by name: (xyz, weights or None, box)."""
    if name == "uniform10k":
        return uniform(10_000, 0), None, UNIT_BOX
    if name == "mixture1M":
        return mixture(1_000_000, 1), None, UNIT_BOX
    if name == "power1M":
        x = mixture(1_000_000, 1)
        return x, power_weights(x, 2), UNIT_BOX
    if name == "surfaces20M":
        return surfaces(20_000_000, 4), None, UNIT_BOX
    raise KeyError(name)
