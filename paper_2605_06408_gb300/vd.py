"""Thin binding of libvd's C ABI (include/vd.h).

Argument marshalling only: PyTorch provides device memory and streams, and
every step of a build runs in libvd's kernels. There is no CPU fallback: if
libvd.so is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass
from typing import Optional, Sequence

import torch

from . import build as _build

VD_OK = 0
VD_ERR_INVALID_ARG = -1
VD_ERR_CUDA = -2
VD_ERR_CAPACITY = -3
VD_ERR_CELL_OVERFLOW = -4
VD_ERR_NO_FORWARD = -5
VD_ERR_TOO_LARGE = -6
VD_ERR_TIMEOUT = -7

ABI_FUNCTIONS = (
    "vd_default_config", "vd_create", "vd_destroy", "vd_set_config", "vd_reserve", "vd_workspace_bytes",
    "vd_build", "vd_copy_neighbors", "vd_build_batched", "vd_backward", "vd_get_timings", "vd_get_status",
    "vd_error_string", "vd_cells_noalloc", "vd_autotune", "vd_autotune_batched", "vd_cells_mesh",
    "vd_backward_mesh", "vd_ambiguous_cells", "vd_set_partition", "vd_copy",
)
VD_TUNE_FORCE = 1


class VdBox(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_float * 3), ("hi", ctypes.c_float * 3)]


class VdOut(ctypes.Structure):
    _fields_ = [
        ("offsets", ctypes.c_void_p),
        ("neighbors", ctypes.c_void_p),
        ("nnz_capacity", ctypes.c_int64),
        ("nnz_out", ctypes.c_void_p),
        ("volume", ctypes.c_void_p),
        ("centroid", ctypes.c_void_p),
        ("status", ctypes.c_void_p),
    ]


class VdMesh(ctypes.Structure):
    _fields_ = [
        ("vertex_offsets", ctypes.c_void_p),
        ("vertices", ctypes.c_void_p),
        ("vertex_sites", ctypes.c_void_p),
        ("capacity", ctypes.c_int64),
        ("nverts_out", ctypes.c_void_p),
        ("status", ctypes.c_void_p),
    ]


class VdConfig(ctypes.Structure):
    _fields_ = [
        ("leaf_size", ctypes.c_int32),
        ("verts_per_lane", ctypes.c_int32),
        ("queue_per_lane", ctypes.c_int32),
        ("cull_mode", ctypes.c_int32),
        ("traversal", ctypes.c_int32),
        ("warps_per_block", ctypes.c_int32),
        ("blocks_per_sm", ctypes.c_int32),
        ("counters", ctypes.c_int32),
        ("timing", ctypes.c_int32),
        ("warm_start", ctypes.c_int32),
        ("cell_mode", ctypes.c_int32),
        ("tape", ctypes.c_int32),
        ("precision", ctypes.c_int32),
    ]


class VdTimings(ctypes.Structure):
    _fields_ = [(k, ctypes.c_float) for k in ("pack_ms", "sort_ms", "bvh_ms", "cells_ms", "overflow_ms", "csr_ms",
                                              "backward_ms", "total_ms")] + [
        ("launches", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class VdStatus(ctypes.Structure):
    _fields_ = [("error", ctypes.c_int32), ("reserved", ctypes.c_int32)] + [
        (k, ctypes.c_int64)
        for k in ("nnz", "empty_cells", "overflow_cells", "failed_cells", "fp64_fallbacks", "fp64_ambiguous",
                  "candidates", "clips", "nodes", "vertex_tests", "new_vertices", "refined_vertices",
                  "refined_volumes")
    ] + [("overflow_reason", ctypes.c_int64 * 4)] + [
        (k, ctypes.c_int64)
        for k in ("large_candidates", "large_clips", "large_nodes", "large_vertex_tests", "large_new_vertices",
                  "large_tape_records", "large_tape_restored", "ambiguous_cells")
    ]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load libvd.so (building it first if missing and nvcc is present)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"libvd.so not found at {path}; run paper_2605_06408_gb300/build.py")
            _build.build()
        lib = ctypes.CDLL(path)
        P, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        lib.vd_default_config.argtypes = [ctypes.POINTER(VdConfig)]
        lib.vd_create.argtypes = [ctypes.POINTER(P), I, ctypes.POINTER(VdConfig)]
        lib.vd_destroy.argtypes = [P]
        lib.vd_set_config.argtypes = [P, ctypes.POINTER(VdConfig)]
        lib.vd_reserve.argtypes = [P, I64, I]
        lib.vd_workspace_bytes.argtypes = [I64, I]
        lib.vd_workspace_bytes.restype = ctypes.c_size_t
        lib.vd_build.argtypes = [P, P, P, I64, VdBox, ctypes.POINTER(VdOut), P]
        lib.vd_copy_neighbors.argtypes = [P, ctypes.POINTER(VdOut), P]
        lib.vd_build_batched.argtypes = [P, P, P, P, P, P, ctypes.c_int32, ctypes.POINTER(VdOut), P]
        lib.vd_backward.argtypes = [P, P, P, P, P, I, P]
        lib.vd_get_status.argtypes = [P, ctypes.POINTER(VdStatus)]
        lib.vd_get_timings.argtypes = [P, ctypes.POINTER(VdTimings)]
        lib.vd_cells_noalloc.argtypes = [P, P, I64, VdBox, P, P, P, P, P, P]
        lib.vd_autotune.argtypes = [P, P, P, I64, VdBox, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(VdConfig), P]
        lib.vd_cells_mesh.argtypes = [P, ctypes.POINTER(VdMesh), P]
        lib.vd_backward_mesh.argtypes = [P, P, P, P, P, P, P, P]
        lib.vd_autotune_batched.argtypes = [P, P, P, P, P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.POINTER(VdConfig), P]
        lib.vd_ambiguous_cells.argtypes = [P, P, I64, P]
        lib.vd_set_partition.argtypes = [P, ctypes.c_int32, ctypes.c_int32]
        lib.vd_copy.argtypes = [P, P, I64, P]
        lib.vd_error_string.argtypes = [I]
        lib.vd_error_string.restype = ctypes.c_char_p
        for f in ABI_FUNCTIONS:
            if f not in ("vd_workspace_bytes", "vd_error_string"):
                getattr(lib, f).restype = I
        _lib = lib
        return lib


def error_string(code: int) -> str:
    return load_library().vd_error_string(int(code)).decode()


class VdError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {error_string(code)} ({code})" if what else f"{error_string(code)} ({code})")


def _check(code: int, what: str):
    if code != VD_OK:
        raise VdError(code, what)


def default_config() -> dict:
    c = VdConfig()
    _check(load_library().vd_default_config(ctypes.byref(c)), "vd_default_config")
    return {k: getattr(c, k) for k, _ in VdConfig._fields_}


def _config_struct(cfg: Optional[dict]) -> VdConfig:
    c = VdConfig()
    load_library().vd_default_config(ctypes.byref(c))
    for k, v in (cfg or {}).items():
        setattr(c, k, int(v))
    return c


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_ptr(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def copy_(dst: torch.Tensor, src: torch.Tensor) -> torch.Tensor:
    """dst[...] = src through vd_copy: the library's SM copy between device
    memory and page-locked host memory (either side; a CUDA tensor or a
    pinned CPU tensor), on the current stream of the CUDA side's device.
    Both tensors contiguous, of the same dtype and number of elements."""
    if dst.dtype != src.dtype or dst.numel() != src.numel():
        raise ValueError("copy_: dst and src differ in dtype or size")
    if not (dst.is_contiguous() and src.is_contiguous()):
        raise ValueError("copy_: tensors must be contiguous")
    dev = dst.device if dst.is_cuda else src.device
    if not dev.type == "cuda":
        raise ValueError("copy_: one side must be a CUDA tensor")
    for t in (dst, src):
        if not t.is_cuda and not t.is_pinned():
            raise ValueError("copy_: a CPU tensor must be pinned (page-locked)")
    nbytes = dst.numel() * dst.element_size()
    with torch.cuda.device(dev):
        _check(load_library().vd_copy(_ptr(dst), _ptr(src), nbytes, _stream_ptr(dev)), "vd_copy")
    return dst


def _box(bbox) -> VdBox:
    b = VdBox()
    lo, hi = bbox
    for k in range(3):
        b.lo[k] = float(lo[k])
        b.hi[k] = float(hi[k])
    return b


@dataclass
class Cells:
    """Result of a build: CSR neighbour lists, volumes and centroids."""
    offsets: torch.Tensor     # int32 [n+1]
    neighbors: torch.Tensor   # int32 [nnz]
    volume: torch.Tensor      # float32 [n]
    centroid: torch.Tensor    # float32 [n, 3]
    status: int
    nnz: int


class Context:
    """A libvd context on one CUDA device (owns the workspace)."""

    def __init__(self, device: int = 0, config: Optional[dict] = None):
        self._lib = load_library()
        self.device = torch.device("cuda", device)
        self._h = ctypes.c_void_p()
        cs = _config_struct(config)
        _check(self._lib.vd_create(ctypes.byref(self._h), device, ctypes.byref(cs)), "vd_create")
        self.config = {k: getattr(cs, k) for k, _ in VdConfig._fields_}
        self._builds = 0
        self._last_n = 0
        self._nnz_hint = 0

    def close(self):
        if self._h:
            self._lib.vd_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_config(self, **cfg):
        merged = dict(self.config)
        merged.update(cfg)
        cs = _config_struct(merged)
        _check(self._lib.vd_set_config(self._h, ctypes.byref(cs)), "vd_set_config")
        self.config = merged

    # ------------------------------------------------------------ autotuner
    def autotune(self, sites: torch.Tensor, weights: Optional[torch.Tensor] = None, bbox=((0, 0, 0), (1, 1, 1)),
                 max_trials: int = 0, force: bool = False) -> dict:
        """Time candidate configurations of build() on this input (vd_autotune)
        and keep the fastest; returns it. Synchronises; tune before capturing
        a graph. A following backward() needs a new build()."""
        sites = sites.contiguous()
        weights = None if weights is None else weights.contiguous()
        best = VdConfig()
        rc = self._lib.vd_autotune(self._h, _ptr(sites), _ptr(weights), sites.shape[0], _box(bbox), int(max_trials),
                                   VD_TUNE_FORCE if force else 0, ctypes.byref(best), _stream_ptr(self.device))
        _check(rc, "vd_autotune")
        self.config = {k: getattr(best, k) for k, _ in VdConfig._fields_}
        return dict(self.config)

    def autotune_batched(self, sites: torch.Tensor, weights: Optional[torch.Tensor], set_offsets: Sequence[int],
                         boxes, weighted: Optional[Sequence[int]] = None, max_trials: int = 0,
                         force: bool = False) -> dict:
        """vd_autotune_batched: as autotune() for build_batched()."""
        import numpy as np

        sites = sites.contiguous()
        offs = np.ascontiguousarray(np.asarray(set_offsets, dtype=np.int64))
        nsets = offs.shape[0] - 1
        bx = (VdBox * nsets)()
        for k, b in enumerate(boxes):
            bx[k] = _box(b)
        wf = None if weighted is None else np.ascontiguousarray(np.asarray(weighted, dtype=np.uint8))
        best = VdConfig()
        rc = self._lib.vd_autotune_batched(self._h, _ptr(sites), _ptr(weights), offs.ctypes.data_as(ctypes.c_void_p),
                                           ctypes.cast(bx, ctypes.c_void_p),
                                           None if wf is None else wf.ctypes.data_as(ctypes.c_void_p), nsets,
                                           int(max_trials), VD_TUNE_FORCE if force else 0, ctypes.byref(best),
                                           _stream_ptr(self.device))
        _check(rc, "vd_autotune_batched")
        self.config = {k: getattr(best, k) for k, _ in VdConfig._fields_}
        return dict(self.config)

    def set_partition(self, part: int, nparts: int):
        """Build only part `part` of `nparts` contiguous Morton-order ranges
        of the cells from now on (vd_set_partition); (0, 1) builds all."""
        _check(self._lib.vd_set_partition(self._h, int(part), int(nparts)), "vd_set_partition")
        self.partition = (int(part), int(nparts))

    def reserve(self, n: int, weighted: bool = False):
        _check(self._lib.vd_reserve(self._h, int(n), int(weighted)), "vd_reserve")

    @staticmethod
    def workspace_bytes(n: int, weighted: bool = False) -> int:
        return int(load_library().vd_workspace_bytes(int(n), int(weighted)))

    # ------------------------------------------------------------ forward
    def _alloc_out(self, n: int, cap: int):
        dev = self.device
        out = {
            "offsets": torch.empty(n + 1, dtype=torch.int32, device=dev),
            "neighbors": torch.empty(max(cap, 1), dtype=torch.int32, device=dev),
            "nnz": torch.zeros(1, dtype=torch.int64, device=dev),
            "volume": torch.empty(n, dtype=torch.float32, device=dev),
            "centroid": torch.empty(n, 3, dtype=torch.float32, device=dev),
            "status": torch.zeros(1, dtype=torch.int32, device=dev),
        }
        s = VdOut()
        s.offsets = out["offsets"].data_ptr()
        s.neighbors = out["neighbors"].data_ptr()
        s.nnz_capacity = cap
        s.nnz_out = out["nnz"].data_ptr()
        s.volume = out["volume"].data_ptr()
        s.centroid = out["centroid"].data_ptr()
        s.status = out["status"].data_ptr()
        return out, s

    def _finish(self, out, s, n: int, sync: bool) -> Cells:
        if not sync:
            return Cells(out["offsets"], out["neighbors"], out["volume"], out["centroid"], 0, -1)
        st = int(out["status"].item())
        nnz = int(out["nnz"].item())
        if st == VD_ERR_CAPACITY:
            out2, s2 = self._alloc_out(n, nnz)
            out2["volume"], out2["centroid"] = out["volume"], out["centroid"]
            _check(self._lib.vd_copy_neighbors(self._h, ctypes.byref(s2), _stream_ptr(self.device)),
                   "vd_copy_neighbors")
            st = int(out2["status"].item())
            out = out2
        if st != VD_OK:
            raise VdError(st, "device status")
        self._nnz_hint = nnz
        return Cells(out["offsets"], out["neighbors"][:nnz], out["volume"], out["centroid"], st, nnz)

    def build(self, sites: torch.Tensor, weights: Optional[torch.Tensor] = None, bbox=((0, 0, 0), (1, 1, 1)),
              nnz_capacity: Optional[int] = None, sync: bool = True) -> Cells:
        """Cells of `sites` (float32 [n,3] on this device) clipped to `bbox`."""
        sites = sites.contiguous()
        assert sites.dtype == torch.float32 and sites.is_cuda and sites.dim() == 2 and sites.shape[1] == 3
        n = sites.shape[0]
        if weights is not None:
            weights = weights.contiguous()
            assert weights.dtype == torch.float32 and weights.is_cuda and weights.shape == (n,)
        cap = int(nnz_capacity) if nnz_capacity is not None else max(24 * n, self._nnz_hint + n)
        out, s = self._alloc_out(n, cap)
        rc = self._lib.vd_build(self._h, _ptr(sites), _ptr(weights), n, _box(bbox), ctypes.byref(s),
                                _stream_ptr(self.device))
        _check(rc, "vd_build")
        self._builds += 1
        self._last_n = n
        return self._finish(out, s, n, sync)

    def build_batched(self, sites: torch.Tensor, weights: Optional[torch.Tensor], set_offsets: Sequence[int],
                      boxes, weighted: Optional[Sequence[int]] = None, nnz_capacity: Optional[int] = None,
                      sync: bool = True) -> Cells:
        """Independent cells of many sets in one launch; neighbour indices
        are local to each row's set, offsets global."""
        import numpy as np

        sites = sites.contiguous()
        n = sites.shape[0]
        offs = np.ascontiguousarray(np.asarray(set_offsets, dtype=np.int64))
        nsets = offs.shape[0] - 1
        bx = (VdBox * nsets)()
        for k, b in enumerate(boxes):
            bx[k] = _box(b)
        wf = None
        if weighted is not None:
            wf = np.ascontiguousarray(np.asarray(weighted, dtype=np.uint8))
        cap = int(nnz_capacity) if nnz_capacity is not None else 24 * n
        out, s = self._alloc_out(n, cap)
        rc = self._lib.vd_build_batched(self._h, _ptr(sites), _ptr(weights), offs.ctypes.data_as(ctypes.c_void_p),
                                        ctypes.cast(bx, ctypes.c_void_p),
                                        None if wf is None else wf.ctypes.data_as(ctypes.c_void_p), nsets,
                                        ctypes.byref(s), _stream_ptr(self.device))
        _check(rc, "vd_build_batched")
        self._builds += 1
        self._last_n = n
        return self._finish(out, s, n, sync)

    # ------------------------------------------------------------ backward
    def mesh(self, capacity: Optional[int] = None):
        """The vertices of every cell of the last build (vd_cells_mesh):
        (vertex_offsets int32 [n+1], vertices float32 [V,3] world positions,
        vertex_sites int32 [V,3] the other defining sites or -1-f for box
        faces). The order is the one backward(grad_vertices=...) expects."""
        n = self._last_n
        dev = self.device
        off = torch.empty(n + 1, dtype=torch.int32, device=dev)
        nv = torch.zeros(1, dtype=torch.int64, device=dev)
        st = torch.zeros(1, dtype=torch.int32, device=dev)
        cap = int(capacity) if capacity is not None else 64 * n

        def run(cap):
            verts = torch.empty(max(cap, 1), 3, dtype=torch.float32, device=dev)
            sites = torch.empty(max(cap, 1), 3, dtype=torch.int32, device=dev)
            m = VdMesh(off.data_ptr(), verts.data_ptr(), sites.data_ptr(), cap, nv.data_ptr(), st.data_ptr())
            _check(self._lib.vd_cells_mesh(self._h, ctypes.byref(m), _stream_ptr(dev)), "vd_cells_mesh")
            torch.cuda.synchronize(dev)
            return verts, sites

        verts, sites = run(cap)
        total = int(nv.item())
        if int(st.item()) == VD_ERR_CAPACITY or total > cap:
            verts, sites = run(total)
        elif int(st.item()) != VD_OK:
            raise VdError(int(st.item()), "vd_cells_mesh")
        return off, verts[:total], sites[:total]

    def backward(self, grad_volume: Optional[torch.Tensor], grad_centroid: Optional[torch.Tensor],
                 want_weights: bool = True, recompute: bool = False,
                 grad_vertices: Optional[torch.Tensor] = None, vertex_offsets: Optional[torch.Tensor] = None):
        """Gradients (float32 [n,3], float32 [n] or None) of
        sum gv_i V_i + gc_i . g_i for the last build of this context."""
        n = self._last_n
        gp = torch.empty(n, 3, dtype=torch.float32, device=self.device)
        gw = torch.empty(n, dtype=torch.float32, device=self.device) if want_weights else None
        gv = None if grad_volume is None else grad_volume.contiguous().float()
        gc = None if grad_centroid is None else grad_centroid.contiguous().float()
        if grad_vertices is not None:
            if recompute or vertex_offsets is None:
                raise ValueError("vertex gradients need the mesh's vertex_offsets and recompute=False")
            gvx = grad_vertices.contiguous().float()
            rc = self._lib.vd_backward_mesh(self._h, _ptr(gv), _ptr(gc), _ptr(gvx), _ptr(vertex_offsets.contiguous()),
                                            _ptr(gp), _ptr(gw), _stream_ptr(self.device))
            _check(rc, "vd_backward_mesh")
            return gp, gw
        rc = self._lib.vd_backward(self._h, _ptr(gv), _ptr(gc), _ptr(gp), _ptr(gw), 1 if recompute else 0,
                                   _stream_ptr(self.device))
        _check(rc, "vd_backward")
        return gp, gw

    def timings(self) -> dict:
        t = VdTimings()
        _check(self._lib.vd_get_timings(self._h, ctypes.byref(t)), "vd_get_timings")
        return {k: getattr(t, k) for k, _ in VdTimings._fields_ if k != "reserved"}

    def ambiguous_cells(self):
        """Original indices (int64 numpy array, sorted, unique) of the cells
        of the last forward build that took an FP64 sign test still inside
        its FP64 error bound (vd_ambiguous_cells)."""
        import numpy as np

        cnt = ctypes.c_int64()
        _check(self._lib.vd_ambiguous_cells(self._h, None, 0, ctypes.byref(cnt)), "vd_ambiguous_cells")
        buf = np.zeros(max(int(cnt.value), 1), np.int64)
        _check(self._lib.vd_ambiguous_cells(self._h, buf.ctypes.data_as(ctypes.c_void_p), buf.shape[0],
                                            ctypes.byref(cnt)), "vd_ambiguous_cells")
        return np.unique(buf[:min(int(cnt.value), buf.shape[0])])

    def status(self) -> dict:
        st = VdStatus()
        _check(self._lib.vd_get_status(self._h, ctypes.byref(st)), "vd_get_status")
        d = {k: getattr(st, k) for k, _ in VdStatus._fields_ if k not in ("reserved", "overflow_reason")}
        d["overflow_reason"] = dict(zip(("queue", "vertices", "planes", "neighbors"), list(st.overflow_reason)))
        return d


class _CellsFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, sites, weights, context, bbox):
        res = context.build(sites.detach(), None if weights is None else weights.detach(), bbox)
        fctx.context = context
        fctx.build_id = context._builds
        fctx.has_w = weights is not None
        fctx.mark_non_differentiable(res.offsets, res.neighbors)
        return res.volume, res.centroid, res.offsets, res.neighbors

    @staticmethod
    def backward(fctx, gvol, gcen, _go, _gn):
        if fctx.context._builds != fctx.build_id:
            raise RuntimeError("the context was rebuilt after this forward; backward needs its own context")
        gp, gw = fctx.context.backward(gvol, gcen, want_weights=fctx.has_w)
        return gp, (gw if fctx.has_w else None), None, None


def cells(sites: torch.Tensor, weights: Optional[torch.Tensor] = None, bbox=((0, 0, 0), (1, 1, 1)),
          context: Optional[Context] = None):
    """Differentiable build: returns (volume, centroid, offsets, neighbors).
    Gradients flow from volume and centroid to sites and weights with the
    cell combinatorics held fixed."""
    if context is None:
        # a backward is planned when any input needs a gradient: keep the tape
        grad = sites.requires_grad or (weights is not None and weights.requires_grad)
        context = Context(sites.device.index or 0, {"tape": 1} if grad else None)
    return _CellsFn.apply(sites, weights, context, bbox)


class _MeshCellsFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, sites, weights, context, bbox):
        res = context.build(sites.detach(), None if weights is None else weights.detach(), bbox)
        voff, verts, vsites = context.mesh()
        fctx.context = context
        fctx.build_id = context._builds
        fctx.has_w = weights is not None
        fctx.voff = voff
        fctx.mark_non_differentiable(res.offsets, res.neighbors, voff, vsites)
        return res.volume, res.centroid, verts, res.offsets, res.neighbors, voff, vsites

    @staticmethod
    def backward(fctx, gvol, gcen, gverts, _go, _gn, _gvo, _gvs):
        if fctx.context._builds != fctx.build_id:
            raise RuntimeError("the context was rebuilt after this forward; backward needs its own context")
        gp, gw = fctx.context.backward(gvol, gcen, want_weights=fctx.has_w, grad_vertices=gverts,
                                       vertex_offsets=fctx.voff)
        return gp, (gw if fctx.has_w else None), None, None


def mesh_cells(sites: torch.Tensor, weights: Optional[torch.Tensor] = None, bbox=((0, 0, 0), (1, 1, 1)),
               context: Optional[Context] = None):
    """Differentiable build with the explicit mesh: returns (volume,
    centroid, vertices [V,3], offsets, neighbors, vertex_offsets,
    vertex_sites). Gradients flow from volume, centroid and the vertex
    positions to sites and weights, the cell combinatorics held fixed."""
    if context is None:
        context = Context(sites.device.index or 0, {"tape": 1})
    return _MeshCellsFn.apply(sites, weights, context, bbox)
