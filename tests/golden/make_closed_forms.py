"""Write closed_forms.json: two-site power cells in the unit box whose
volume (and, for axis-aligned splits, centroid) have closed forms.

Two sites split the box by the single radical plane of Eq. 1 (Sec. 3):
    2 (p1 - p0) . x <= |p1|^2 - |p0|^2 + w0 - w1      (cell of site 0).
Volume of the unit cube cut by a . x <= b with every a_k > 0 (after
reflecting coordinates with a_k < 0) is the inclusion-exclusion sum over
cube corners v:  V = sum_v (-1)^{|v|} max(0, b - a.v)^3 / (6 a_1 a_2 a_3).
This script uses only that formula; it calls neither the oracle nor the
CUDA path.
"""
import itertools
import json
import os

import numpy as np


def cube_halfspace_volume(a, b):
    a = np.asarray(a, np.float64).copy()
    b = float(b)
    for k in range(3):
        if a[k] < 0:  # x_k -> 1 - x_k
            b -= a[k]
            a[k] = -a[k]
    tot = 0.0
    for v in itertools.product((0, 1), repeat=3):
        t = b - float(np.dot(a, v))
        if t > 0:
            tot += (-1) ** sum(v) * t ** 3
    return tot / (6.0 * a[0] * a[1] * a[2])


def main():
    rng = np.random.Generator(np.random.PCG64(11))
    cases = []
    # general planes: random site pairs and weights
    for _ in range(24):
        p = rng.random((2, 3)).astype(np.float32)
        w = (rng.standard_normal(2) * 0.01).astype(np.float32)
        p64, w64 = p.astype(np.float64), w.astype(np.float64)
        a = 2.0 * (p64[1] - p64[0])
        b = float(p64[1] @ p64[1] - p64[0] @ p64[0] + w64[0] - w64[1])
        v0 = cube_halfspace_volume(a, b)
        cases.append({"kind": "plane", "xyz": p.tolist(), "w": w.tolist(), "vol": [v0, 1.0 - v0]})
    # axis-aligned: sites differ only along one axis -> slab cells
    for _ in range(8):
        ax = int(rng.integers(0, 3))
        base = rng.random(3).astype(np.float32)
        p = np.stack([base, base]).astype(np.float32)
        p[0, ax], p[1, ax] = np.sort(rng.random(2)).astype(np.float32)
        w = (rng.standard_normal(2) * 0.01).astype(np.float32)
        p64, w64 = p.astype(np.float64), w.astype(np.float64)
        xm = 0.5 * (p64[0, ax] + p64[1, ax]) + (w64[0] - w64[1]) / (2.0 * (p64[1, ax] - p64[0, ax]))
        xm = min(max(xm, 0.0), 1.0)
        c0 = [0.5, 0.5, 0.5]
        c1 = [0.5, 0.5, 0.5]
        c0[ax] = xm / 2.0
        c1[ax] = (1.0 + xm) / 2.0
        cases.append({"kind": "slab", "xyz": p.tolist(), "w": w.tolist(), "vol": [xm, 1.0 - xm],
                      "cen": [c0, c1]})
    out = {
        "source": "closed forms of the two-site power cell, Sec. 3 Eq. 1; written by make_closed_forms.py",
        "box": [[0, 0, 0], [1, 1, 1]],
        "cases": cases,
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "closed_forms.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
