"""FP64 CPU oracle for 3D Voronoi / power cells (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It shares no code with the CUDA path.

The arithmetic lives in ``vd_oracle.c`` (plain C, FP64, OpenMP over cells);
this module compiles it with gcc and marshals numpy arrays through ctypes.
What it computes is the cell of Eq. 1 (Sec. 3) clipped to a box, following
the clipping procedure of App. B; see the header of ``vd_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

STAT_NAMES = ("ambiguous", "degenerate", "orient_fail", "topo_fail", "clips", "tests", "empty", "facewalk_fail",
              "exact_resolved")

ERRORS = {
    -1: "invalid argument",
    -2: "inconsistent cell topology",
    -3: "neighbour capacity exceeded",
    -4: "exact mode needs coordinates on the 2^-20 grid and weights on the 2^-40 grid",
    -5: "out of memory",
}


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-fopenmp", "-std=gnu11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            I32 = ctypes.c_int32
            C = ctypes.c_int
            lib.oracle_cells.argtypes = [P, P, I64, P, P, P, I64, C, C, P, P, P, I64, P, P, P, P, P, C]
            lib.oracle_cells.restype = C
            lib.oracle_grad.argtypes = [P, P, I64, P, P, P, I64, P, P, P, P, P, C]
            lib.oracle_grad.restype = C
            lib.oracle_certify.argtypes = [P, P, I64, P, P, P, I64, C, P, P, C]
            lib.oracle_certify.restype = C
            lib.oracle_cell_vertices.argtypes = [P, P, I64, P, P, I64, C, C, P, P, I32]
            lib.oracle_cell_vertices.restype = C
            lib.oracle_stat_count.restype = C
            lib.oracle_exact_side.argtypes = [P, P, I64, P, P, I64, P]
            lib.oracle_exact_side.restype = C
            lib.oracle_session_open.argtypes = [P, P, I64, P, P, C, C, P]
            lib.oracle_session_open.restype = P
            lib.oracle_session_cells.argtypes = [P, P, I64, P, P, P, I64, P, P, P, P, P, C]
            lib.oracle_session_cells.restype = C
            lib.oracle_session_close.argtypes = [P]
            lib.oracle_session_close.restype = None
            lib.oracle_fd_grad.argtypes = [P, P, I64, P, P, P, P, P, P, P, I64, P, P, P, P, C]
            lib.oracle_fd_grad.restype = C
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _prep(xyz, w, bbox):
    xyz = np.ascontiguousarray(np.asarray(xyz, dtype=np.float32).reshape(-1, 3))
    w = None if w is None else np.ascontiguousarray(np.asarray(w, dtype=np.float32).reshape(-1))
    if w is not None and w.shape[0] != xyz.shape[0]:
        raise ValueError("weights must have one entry per site")
    lo = np.ascontiguousarray(np.asarray(bbox[0], dtype=np.float32).reshape(3))
    hi = np.ascontiguousarray(np.asarray(bbox[1], dtype=np.float32).reshape(3))
    return xyz, w, lo, hi


def _check(rc):
    if rc != 0:
        raise RuntimeError(f"oracle error {rc}: {ERRORS.get(rc, 'unknown')}")


def _threads(threads):
    return int(threads) if threads else (os.cpu_count() or 1)


def cells(xyz, w=None, bbox=((0, 0, 0), (1, 1, 1)), cells=None, mode="kd", exact=False,
          threads=None, max_nbrs=None):
    """Cells of the listed sites (all if ``cells`` is None).

    Returns a dict: ``counts`` int32[m], ``nbrs`` list of ascending int32
    arrays, ``offsets``/``indices`` (CSR), ``vol`` float64[m], ``cen``
    float64[m,3], ``nverts``/``nfaces`` int32[m] and ``stats`` (dict).
    """
    del max_nbrs  # neighbour lists are unbounded (kept for call compatibility)
    lib = _load()
    xyz, w, lo, hi = _prep(xyz, w, bbox)
    n = xyz.shape[0]
    idx = None if cells is None else np.ascontiguousarray(np.asarray(cells, dtype=np.int64).reshape(-1))
    m = n if idx is None else idx.shape[0]
    cap = 20 * m + 1024
    while True:
        counts = np.zeros(m, np.int32)
        offsets = np.zeros(m + 1, np.int64)
        nb = np.zeros(cap, np.int32)
        vol = np.zeros(m, np.float64)
        cen = np.zeros((m, 3), np.float64)
        nv = np.zeros(m, np.int32)
        nf = np.zeros(m, np.int32)
        st = np.zeros(lib.oracle_stat_count() + 1, np.int64)
        rc = lib.oracle_cells(_ptr(xyz), _ptr(w), n, _ptr(lo), _ptr(hi), _ptr(idx), m,
                              0 if mode == "brute" else 1, 1 if exact else 0, _ptr(counts), _ptr(offsets),
                              _ptr(nb), cap, _ptr(vol), _ptr(cen), _ptr(nv), _ptr(nf), _ptr(st),
                              _threads(threads))
        if rc == -3 and st[-1] > cap:
            cap = int(st[-1])
            continue
        _check(rc)
        break
    return _cells_result(offsets, nb, counts, vol, cen, nv, nf, st)


def _cells_result(offsets, nb, counts, vol, cen, nv, nf, st):
    indices = nb[: offsets[-1]].copy()
    return {
        "counts": counts,
        "offsets": offsets,
        "indices": indices,
        "nbrs": np.split(indices, offsets[1:-1]) if counts.shape[0] else [],
        "vol": vol,
        "cen": cen,
        "nverts": nv,
        "nfaces": nf,
        "stats": dict(zip(STAT_NAMES, st[:-1].tolist())),
    }


class Session:
    """One point set kept set up (duplicate marks, k-d tree) across calls:
    ``Session(xyz, w, bbox).cells(cells)`` returns what ``cells(xyz, w,
    bbox, cells=cells)`` returns, with the same arithmetic, without building
    the tree again for every sample of cells."""

    def __init__(self, xyz, w=None, bbox=((0, 0, 0), (1, 1, 1)), mode="kd", exact=False):
        self._lib = _load()
        self.xyz, self.w, self.lo, self.hi = _prep(xyz, w, bbox)
        rc = ctypes.c_int(0)
        self._h = self._lib.oracle_session_open(_ptr(self.xyz), _ptr(self.w), self.xyz.shape[0], _ptr(self.lo),
                                                _ptr(self.hi), 0 if mode == "brute" else 1, 1 if exact else 0,
                                                ctypes.byref(rc))
        if not self._h:
            _check(rc.value or -5)

    def cells(self, cells=None, threads=None):
        lib = self._lib
        n = self.xyz.shape[0]
        idx = None if cells is None else np.ascontiguousarray(np.asarray(cells, dtype=np.int64).reshape(-1))
        m = n if idx is None else idx.shape[0]
        cap = 20 * m + 1024
        while True:
            counts = np.zeros(m, np.int32)
            offsets = np.zeros(m + 1, np.int64)
            nb = np.zeros(cap, np.int32)
            vol = np.zeros(m, np.float64)
            cen = np.zeros((m, 3), np.float64)
            nv = np.zeros(m, np.int32)
            nf = np.zeros(m, np.int32)
            st = np.zeros(lib.oracle_stat_count() + 1, np.int64)
            rc = lib.oracle_session_cells(self._h, _ptr(idx), m, _ptr(counts), _ptr(offsets), _ptr(nb), cap,
                                          _ptr(vol), _ptr(cen), _ptr(nv), _ptr(nf), _ptr(st), _threads(threads))
            if rc == -3 and st[-1] > cap:
                cap = int(st[-1])
                continue
            _check(rc)
            return _cells_result(offsets, nb, counts, vol, cen, nv, nf, st)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.oracle_session_close(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def grad(xyz, w, bbox, c, d, cells=None, threads=None):
    """Gradient of L = sum_i c_i V_i + d_i . g_i over the listed cells.

    Returns ``(gp float64[n,3], gw float64[n], stats)``.
    """
    lib = _load()
    xyz, w, lo, hi = _prep(xyz, w, bbox)
    n = xyz.shape[0]
    c = np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(n))
    d = np.ascontiguousarray(np.asarray(d, dtype=np.float64).reshape(n, 3))
    idx = None if cells is None else np.ascontiguousarray(np.asarray(cells, dtype=np.int64).reshape(-1))
    m = n if idx is None else idx.shape[0]
    gp = np.zeros((n, 3), np.float64)
    gw = np.zeros(n, np.float64)
    st = np.zeros(lib.oracle_stat_count(), np.int64)
    rc = lib.oracle_grad(_ptr(xyz), _ptr(w), n, _ptr(lo), _ptr(hi), _ptr(idx), m, _ptr(c), _ptr(d),
                         _ptr(gp), _ptr(gw), _ptr(st), _threads(threads))
    _check(rc)
    return gp, gw, dict(zip(STAT_NAMES, st.tolist()))


def fd_grad(xyz, w, bbox, offsets, nbrs, c, d, sites, hx, hw=None, threads=None):
    """Central finite differences in FP64 of L = sum_i c_i V_i + d_i . g_i
    with respect to the positions (and weights) of `sites`, holding the cell
    combinatorics of the diagram (CSR offsets[n+1], nbrs) fixed; hx / hw are
    per-site steps. Returns (gp float64[m,3], gw float64[m] or None)."""
    lib = _load()
    xyz, w, lo, hi = _prep(xyz, w, bbox)
    n = xyz.shape[0]
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64).reshape(n + 1))
    nb = np.ascontiguousarray(np.asarray(nbrs, dtype=np.int32).reshape(-1))
    c = np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(n))
    d = np.ascontiguousarray(np.asarray(d, dtype=np.float64).reshape(n, 3))
    idx = np.ascontiguousarray(np.asarray(sites, dtype=np.int64).reshape(-1))
    m = idx.shape[0]
    hx = np.ascontiguousarray(np.broadcast_to(np.asarray(hx, dtype=np.float64), (m,)))
    hwa = None if w is None else np.ascontiguousarray(np.broadcast_to(np.asarray(hw, dtype=np.float64), (m,)))
    gp = np.zeros((m, 3), np.float64)
    gw = None if w is None else np.zeros(m, np.float64)
    rc = lib.oracle_fd_grad(_ptr(xyz), _ptr(w), n, _ptr(lo), _ptr(hi), _ptr(off), _ptr(nb), _ptr(c), _ptr(d),
                            _ptr(idx), m, _ptr(hx), _ptr(hwa), _ptr(gp), _ptr(gw), _threads(threads))
    _check(rc)
    return gp, gw


def exact_side(xyz, w, bbox, i, planes):
    """Exact sign (+1 / -1 / 0) of n_h . v - b_h, where v is the vertex of
    the planes of planes[0..2] in the frame of site i and h the plane of
    planes[3] (site indices, or -1-f for box face f), from the oracle's
    expansion arithmetic."""
    lib = _load()
    xyz, w, lo, hi = _prep(xyz, w, bbox)
    ids = np.ascontiguousarray(np.asarray(planes, dtype=np.int64).reshape(4))
    r = lib.oracle_exact_side(_ptr(xyz), _ptr(w), xyz.shape[0], _ptr(lo), _ptr(hi), int(i), _ptr(ids))
    if r not in (-1, 0, 1):
        raise RuntimeError(f"oracle_exact_side returned {r}")
    return r


def certify(xyz, w=None, bbox=((0, 0, 0), (1, 1, 1)), cells=None, exact=False, threads=None):
    """Per-cell count of (final vertex, other site) pairs violating the
    empty-sphere condition pow(v, i) <= pow(v, m)."""
    lib = _load()
    xyz, w, lo, hi = _prep(xyz, w, bbox)
    n = xyz.shape[0]
    idx = None if cells is None else np.ascontiguousarray(np.asarray(cells, dtype=np.int64).reshape(-1))
    m = n if idx is None else idx.shape[0]
    viol = np.zeros(m, np.int64)
    st = np.zeros(lib.oracle_stat_count(), np.int64)
    rc = lib.oracle_certify(_ptr(xyz), _ptr(w), n, _ptr(lo), _ptr(hi), _ptr(idx), m, 1 if exact else 0,
                            _ptr(viol), _ptr(st), _threads(threads))
    _check(rc)
    return viol, dict(zip(STAT_NAMES, st.tolist()))


def cell_vertices(xyz, w, bbox, i, mode="kd", exact=False, cap=4096):
    """Final vertices of one cell: (positions float64[k,3] in coordinates
    relative to the site, defining sites int64[k,3]; box faces are -1-f)."""
    lib = _load()
    xyz, w, lo, hi = _prep(xyz, w, bbox)
    pos = np.zeros((cap, 3), np.float64)
    tri = np.zeros((cap, 3), np.int64)
    k = lib.oracle_cell_vertices(_ptr(xyz), _ptr(w), xyz.shape[0], _ptr(lo), _ptr(hi), int(i),
                                 0 if mode == "brute" else 1, 1 if exact else 0, _ptr(pos), _ptr(tri), cap)
    if k < 0:
        _check(k)
    return pos[:k].copy(), tri[:k].copy()


def vertex_grad(xyz, w, bbox, cells, gfun, threads=None):
    """Gradient, with respect to the site positions and weights, of
    L = sum over the listed cells i and their vertices x of gfun(i, sites) . x,
    the cell combinatorics held fixed. `sites` is the vertex's triple of
    other defining sites (-1-f for box face f, as cell_vertices gives them);
    gfun returns a float64[3]. Each vertex solves A x = r with the rows
    2 (p_j - p_i) . x = |p_j|^2 - |p_i|^2 + w_i - w_j of its site planes and
    +-x_axis = bound of its box faces; with lambda = A^-T g, implicit
    differentiation gives dL/dp_j = 2 lambda_j (p_j - x), dL/dw_j = -lambda_j,
    dL/dp_i += 2 lambda_j (x - p_i), dL/dw_i += lambda_j. Plain FP64 numpy
    over the oracle's own vertices. Returns (gp float64[n,3], gw float64[n])."""
    x = np.asarray(xyz, dtype=np.float32).reshape(-1, 3)
    wt = None if w is None else np.asarray(w, dtype=np.float32).reshape(-1)
    n = x.shape[0]
    gp = np.zeros((n, 3), np.float64)
    gw = np.zeros(n, np.float64)
    P = x.astype(np.float64)
    for i in np.asarray(cells, dtype=np.int64).reshape(-1):
        pos, tri = cell_vertices(x, wt, bbox, int(i))
        pi = P[i]
        for v, t in zip(pos, tri):
            X = pi + v
            g = np.asarray(gfun(int(i), tuple(int(s) for s in t)), dtype=np.float64)
            A = np.zeros((3, 3))
            for k, s in enumerate(t):
                if s >= 0:
                    A[k] = 2.0 * (P[s] - pi)
                else:
                    f = -1 - s
                    A[k, f >> 1] = -1.0 if (f & 1) else 1.0
            lam = np.linalg.solve(A.T, g)
            for k, s in enumerate(t):
                if s < 0:
                    continue
                gp[s] += 2.0 * lam[k] * (P[s] - X)
                gp[i] += 2.0 * lam[k] * (X - pi)
                gw[s] -= lam[k]
                gw[i] += lam[k]
    return gp, gw
