"""GB300 narrow-band signed distance fields of closed triangle meshes
(Characteristic/Scan Conversion method, arXiv:1903.00353).

Thin Python binding of the C ABI declared in include/sdf.h: it marshals torch
tensors (device memory, the current CUDA stream) into the library's calls and
does no computation of its own.  Every step of the method runs in the CUDA
kernels of csrc/.  There is no CPU fallback: without the compiled library or a
CUDA device the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Sequence

import torch

from . import _buildlib

__all__ = ["Grid", "Features", "sdf_build_features", "sdf_narrow_band", "sdf_narrow_band_backward",
           "SDFFunction", "Batch", "sdf_batch_create", "band_l2_loss", "load_library", "kernel_launches", "SDFError",
           "memory_stats",
           "BandList", "sdf_narrow_band_list", "sdf_narrow_band_lists", "sdf_narrow_band_sparse", "band_list_backward", "band_list_l2",
           "FLAG_DISABLE_SADDLE", "FLAG_NO_SYNC", "FLAG_TIMING", "FLAG_AUTOTUNE", "FLAG_FILL_SIGN",
           "FLAG_CELL_LOOP", "FLAG_VERTEX_CONE", "FLAG_VERTEX_HEMISPHERE", "FLAG_GRAD_F64"]

FLAG_DISABLE_SADDLE = 0x1
FLAG_NO_SYNC = 0x2
FLAG_TIMING = 0x4
FLAG_AUTOTUNE = 0x8
FLAG_FILL_SIGN = 0x10
FLAG_CELL_LOOP = 0x20
FLAG_VERTEX_CONE = 0x40
FLAG_VERTEX_HEMISPHERE = 0x80
FLAG_GRAD_F64 = 0x100


_STATUS_KEYS = ("candidates", "band_points", "fp64_points", "pairs", "rows", "rows_hit")
ERR_LIST_OVERFLOW = 9


class SDFError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {load_library().sdf_status_string(code).decode()} (status {code})")


class _CGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("origin", ctypes.c_float * 3), ("h", ctypes.c_float), ("k0", ctypes.c_int32)]


_lib = None


def load_library(path: str | None = None):
    """Load the compiled library (build it first with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _buildlib.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    P, I64, I32, U32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
    L.sdf_build_features.argtypes = [P, I64, U32, P, ctypes.POINTER(P)]
    L.sdf_features_update_positions.argtypes = [P, P, P]
    L.sdf_narrow_band.argtypes = [ctypes.POINTER(P), ctypes.POINTER(_CGrid), ctypes.POINTER(ctypes.c_float), I32,
                                  ctypes.POINTER(P), ctypes.POINTER(P), U32, P]
    L.sdf_narrow_band_backward.argtypes = [ctypes.POINTER(P), ctypes.POINTER(_CGrid), ctypes.POINTER(ctypes.c_float),
                                           I32, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), U32, P]
    L.sdf_features_info.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I64)]
    L.sdf_features_vertex_map.argtypes = [P, P, P]
    L.sdf_narrow_band_static.argtypes = [P, ctypes.POINTER(_CGrid), ctypes.c_float, P, P, P]
    L.sdf_narrow_band_static.restype = ctypes.c_int
    L.sdf_features_face_map.argtypes = [P, P, P]
    L.sdf_features_face_map.restype = ctypes.c_int
    L.sdf_features_vertices.argtypes = [P, P, P]
    L.sdf_features_edges.argtypes = [P, P, P]
    L.sdf_features_edges.restype = ctypes.c_int
    L.sdf_features_error_bound.argtypes = [P, ctypes.POINTER(_CGrid), ctypes.c_float, ctypes.POINTER(ctypes.c_double), P]
    L.sdf_features_error_bound.restype = ctypes.c_int
    L.sdf_features_status.argtypes = [P, ctypes.POINTER(I64), P]
    L.sdf_features_destroy.argtypes = [P]
    L.sdf_features_destroy.restype = None
    L.sdf_features_timing.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I64), ctypes.c_int]
    L.sdf_features_timing.restype = ctypes.c_int
    L.sdf_kernel_launches.argtypes = []
    L.sdf_kernel_launches.restype = I64
    L.sdf_memory_stats.argtypes = [ctypes.POINTER(I64)]
    L.sdf_memory_stats.restype = ctypes.c_int
    L.sdf_probe_rate.argtypes = [I32, P, I64, I64, ctypes.POINTER(I64), P]
    L.sdf_probe_rate.restype = ctypes.c_int
    L.sdf_status_string.argtypes = [ctypes.c_int]
    L.sdf_status_string.restype = ctypes.c_char_p
    L.sdf_batch_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(_CGrid), ctypes.POINTER(ctypes.c_float), I32,
                                   ctypes.POINTER(P), ctypes.POINTER(P), U32, P, ctypes.POINTER(P)]
    L.sdf_batch_run.argtypes = [P, P]
    L.sdf_batch_status.argtypes = [P, ctypes.POINTER(I64), P]
    L.sdf_batch_info.argtypes = [P, ctypes.POINTER(I32), ctypes.POINTER(ctypes.c_double)]
    L.sdf_batch_timing.argtypes = [P, ctypes.POINTER(ctypes.c_float)]
    L.sdf_band_l2_loss.argtypes = [P, P, I64, P, P, P, P]
    L.sdf_narrow_band_list.argtypes = [P, ctypes.POINTER(_CGrid), ctypes.c_float, P, P, P, I64, P, U32, P]
    L.sdf_narrow_band_sparse.argtypes = [P, ctypes.POINTER(_CGrid), ctypes.c_float, P, P, I64, P, U32, P]
    L.sdf_narrow_band_sparse.restype = ctypes.c_int
    L.sdf_narrow_band_lists.argtypes = [ctypes.POINTER(P), ctypes.POINTER(_CGrid), ctypes.POINTER(ctypes.c_float), I32,
                                        ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(I64),
                                        ctypes.POINTER(P), U32, P]
    L.sdf_band_list_backward.argtypes = [P, ctypes.POINTER(_CGrid), P, I64, P, P, P, U32, P]
    L.sdf_band_list_l2.argtypes = [P, ctypes.POINTER(_CGrid), P, I64, P, P, P, P, P, P, U32, P]
    L.sdf_batch_destroy.argtypes = [P]
    L.sdf_batch_destroy.restype = None
    for name in ("sdf_build_features", "sdf_features_update_positions", "sdf_narrow_band",
                 "sdf_narrow_band_backward", "sdf_features_info", "sdf_features_vertex_map",
                 "sdf_features_vertices", "sdf_features_status", "sdf_batch_create", "sdf_batch_run",
                 "sdf_batch_status", "sdf_batch_info", "sdf_batch_timing", "sdf_band_l2_loss",
                 "sdf_narrow_band_list", "sdf_narrow_band_lists", "sdf_band_list_backward", "sdf_band_list_l2"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def kernel_launches() -> int:
    """Process-wide number of kernels the library has launched."""
    return int(load_library().sdf_kernel_launches())


def memory_stats() -> dict:
    """Memory the library has taken: device pool allocations made (process-wide), bytes in use and
    reserved in the current device's pool, pinned host allocations made."""
    out = (ctypes.c_int64 * 4)()
    _check(load_library().sdf_memory_stats(out), "sdf_memory_stats")
    return {"pool_allocs": int(out[0]), "pool_used": int(out[1]), "pool_reserved": int(out[2]),
            "host_allocs": int(out[3])}


PROBE_SMEM_ATOMIC_MIN, PROBE_GLOBAL_ATOMIC_MIN, PROBE_FP64_FMA = 0, 1, 2


def probe_rate(kind: int, buf: torch.Tensor, iters: int, stream=None) -> int:
    """One launch of a rate probe (sdf_probe_rate) on `buf` (a CUDA tensor of 8-byte words); returns
    the launch's operation count, which the caller divides by the launch's event-timed duration."""
    if not buf.is_cuda or buf.element_size() != 8 or not buf.is_contiguous():
        raise ValueError("buf must be a contiguous CUDA tensor of 8-byte elements")
    ops = ctypes.c_int64(0)
    _check(load_library().sdf_probe_rate(int(kind), ctypes.c_void_p(buf.data_ptr()), buf.numel(), int(iters),
                                         ctypes.byref(ops), _stream(stream)), "sdf_probe_rate")
    return int(ops.value)


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _check(code: int, what: str):
    if code != 0:
        raise SDFError(code, what)


def _dev_f32(t: torch.Tensor, name: str) -> torch.Tensor:
    if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    return t


def _grad_vertices(gv: torch.Tensor | None, n_vert: int) -> tuple[torch.Tensor, int]:
    """The vertex-gradient accumulator: a new float32 [V, 3] zero tensor, or the caller's float32
    or float64 one (float64 sets FLAG_GRAD_F64: the sums are taken in FP64)."""
    if gv is None:
        return torch.zeros(n_vert, 3, dtype=torch.float32, device="cuda"), 0
    if not gv.is_cuda or gv.dtype not in (torch.float32, torch.float64) or not gv.is_contiguous() \
            or tuple(gv.shape) != (n_vert, 3):
        raise ValueError("grad_vertices must be a contiguous float32 or float64 CUDA tensor [V, 3]")
    return gv, FLAG_GRAD_F64 if gv.dtype == torch.float64 else 0


@dataclass(frozen=True)
class Grid:
    """Cell-centred grid: point (i,j,k) at origin + (i+1/2, j+1/2, k0+k+1/2) h, stored x fastest
    (k0 > 0: the z-slab of layers k0 .. k0+nz-1 of a larger grid with the same origin and h)."""
    nx: int
    ny: int
    nz: int
    origin: tuple = (0.0, 0.0, 0.0)
    h: float = 1.0
    k0: int = 0

    @staticmethod
    def cube(n: int, lo: float = 0.0, hi: float = 1.0) -> "Grid":
        return Grid(n, n, n, (lo, lo, lo), (hi - lo) / n)

    def c(self) -> _CGrid:
        g = _CGrid()
        g.nx, g.ny, g.nz = self.nx, self.ny, self.nz
        for k in range(3):
            g.origin[k] = float(self.origin[k])
        g.h = float(self.h)
        g.k0 = int(self.k0)
        return g

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


class Features:
    """Library-owned feature records of one closed mesh (sdf_build_features)."""

    def __init__(self, handle: int, n_tri: int):
        self._h = ctypes.c_void_p(handle)
        self.n_tri = n_tri
        n = ctypes.c_int64()
        c = (ctypes.c_int64 * 8)()
        _check(load_library().sdf_features_info(self._h, ctypes.byref(n), c), "sdf_features_info")
        self.counts = [int(x) for x in c]
        self.n_vert, self.n_edge = self.counts[0], self.counts[1]

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise RuntimeError("features destroyed")
        return self._h

    def vertex_map(self) -> torch.Tensor:
        out = torch.empty(3 * self.n_tri, dtype=torch.int32, device="cuda")
        _check(load_library().sdf_features_vertex_map(self.handle, out.data_ptr(), _stream()), "vertex_map")
        return out

    def face_map(self) -> torch.Tensor:
        """Soup triangle index of every library face id (faces are stored in a spatial order)."""
        out = torch.empty(self.n_tri, dtype=torch.int32, device="cuda")
        _check(load_library().sdf_features_face_map(self.handle, out.data_ptr(), _stream()), "face_map")
        return out

    def edges(self) -> torch.Tensor:
        """Edge table int32 [E, 4]: (va, vb, f1, f2) per library edge id (end points va < vb, f1 the
        face holding va -> vb, f2 the face holding vb -> va)."""
        out = torch.empty(self.n_edge, 4, dtype=torch.int32, device="cuda")
        _check(load_library().sdf_features_edges(self.handle, out.data_ptr(), _stream()), "edges")
        return out

    def error_bound(self, grid: "Grid", w: float) -> dict:
        """The FP32 error windows of the narrow band on this grid and band (synchronises):
        delta (bound on the FP32 distance error), eps (inclusion tolerance), ds (sign window) and
        the largest pseudonormal term of the sign window."""
        b = (ctypes.c_double * 4)()
        cg = grid.c()
        _check(load_library().sdf_features_error_bound(self.handle, ctypes.byref(cg), float(w), b, _stream()),
               "sdf_features_error_bound")
        return {"delta": b[0], "eps": b[1], "ds": b[2], "ds_normal": b[3]}

    def vertices(self) -> torch.Tensor:
        out = torch.empty(self.n_vert, 3, dtype=torch.float32, device="cuda")
        _check(load_library().sdf_features_vertices(self.handle, out.data_ptr(), _stream()), "vertices")
        return out

    def update_positions(self, vertices: torch.Tensor):
        v = _dev_f32(vertices, "vertices")
        if v.shape != (self.n_vert, 3):
            raise ValueError("vertices must be [V, 3]")
        _check(load_library().sdf_features_update_positions(self.handle, v.data_ptr(), _stream()),
               "sdf_features_update_positions")

    def status(self):
        st = (ctypes.c_int64 * 6)()
        code = load_library().sdf_features_status(self.handle, st, _stream())
        _check(code, "sdf_features_status")
        return dict(zip(_STATUS_KEYS, [int(x) for x in st]))

    def timing(self, reset: bool = False):
        """Accumulated stage times (ms) of calls made with FLAG_TIMING: bin, tile, fp64, adjoint."""
        ms = (ctypes.c_double * 4)()
        calls = (ctypes.c_int64 * 4)()
        _check(load_library().sdf_features_timing(self.handle, ms, calls, int(reset)), "sdf_features_timing")
        names = ("bin", "tile", "fp64", "adjoint")
        return {n: (float(ms[i]), int(calls[i])) for i, n in enumerate(names)}

    def destroy(self):
        if self._h is not None and _lib is not None:
            _lib.sdf_features_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def sdf_build_features(soup: torch.Tensor, flags: int = 0, stream=None) -> Features:
    """Weld, pair and build feature records from a float32 CUDA soup [T, 3, 3]."""
    s = _dev_f32(soup, "soup")
    if s.dim() != 3 or s.shape[1:] != (3, 3):
        raise ValueError("soup must be [T, 3, 3]")
    h = ctypes.c_void_p()
    _check(load_library().sdf_build_features(s.data_ptr(), s.shape[0], flags, _stream(stream), ctypes.byref(h)),
           "sdf_build_features")
    return Features(h.value, s.shape[0])


def _ptr_array(tensors):
    arr = (ctypes.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        arr[i] = None if t is None else t.data_ptr()
    return arr


def sdf_narrow_band(features: Features | Sequence[Features], grid: Grid | Sequence[Grid], w,
                    out: torch.Tensor | Sequence[torch.Tensor] | None = None, winner: bool | Sequence = False,
                    flags: int = 0, stream=None):
    """Narrow-band SDF on one grid (or a batch when lists are given).

    Returns dist [nz, ny, nx] (and winner ids when winner=True); lists for a batch."""
    batch = isinstance(features, (list, tuple))
    feats = list(features) if batch else [features]
    grids = list(grid) if batch else [grid]
    ws = list(w) if batch else [w]
    n = len(feats)
    if not (len(grids) == len(ws) == n):
        raise ValueError("features, grid and w must have the same length")
    if out is None:
        outs = [torch.empty(g.shape, dtype=torch.float32, device="cuda") for g in grids]
    else:
        outs = list(out) if batch else [out]
        for o, g in zip(outs, grids):
            _dev_f32(o, "out")
            if o.numel() != g.nx * g.ny * g.nz:
                raise ValueError("out has the wrong size")
    if isinstance(winner, (list, tuple)):
        wins = list(winner)
    elif isinstance(winner, torch.Tensor):
        if batch:
            raise ValueError("a batch takes a list of winner tensors")
        if not winner.is_cuda or winner.dtype != torch.int32 or not winner.is_contiguous():
            raise ValueError("winner must be a contiguous int32 CUDA tensor")
        wins = [winner]
    elif winner:
        wins = [torch.empty(g.shape, dtype=torch.int32, device="cuda") for g in grids]
    else:
        wins = [None] * n
    fa = (ctypes.c_void_p * n)(*[f.handle.value for f in feats])
    ga = (_CGrid * n)(*[g.c() for g in grids])
    wa = (ctypes.c_float * n)(*[float(x) for x in ws])
    _check(load_library().sdf_narrow_band(fa, ga, wa, n, _ptr_array(outs), _ptr_array(wins), flags,
                                          _stream(stream)), "sdf_narrow_band")
    res = [(o, wn) if wn is not None else o for o, wn in zip(outs, wins)]
    return res if batch else res[0]


class Batch:
    """A fixed batch of (mesh, grid, output) problems whose run() is a replayable launch sequence
    (no allocation, no synchronisation), suitable for CUDA-graph capture."""

    def __init__(self, handle: int, feats, outs, wins):
        self._h = ctypes.c_void_p(handle)
        self.features, self.outs, self.winners = list(feats), outs, wins

    def run(self, stream=None):
        _check(load_library().sdf_batch_run(self._h, _stream(stream)), "sdf_batch_run")

    def status(self, stream=None):
        st = (ctypes.c_int64 * 6)()
        _check(load_library().sdf_batch_status(self._h, st, _stream(stream)), "sdf_batch_status")
        return dict(zip(_STATUS_KEYS, [int(x) for x in st]))

    def info(self):
        shape = (ctypes.c_int32 * 3)()
        ms = ctypes.c_double()
        _check(load_library().sdf_batch_info(self._h, shape, ctypes.byref(ms)), "sdf_batch_info")
        return {"tile": tuple(int(x) for x in shape), "tuned_ms": float(ms.value)}

    def timing(self):
        """Stage times (ms) of the last run of a batch created with timing=True: bin, tile, fp64."""
        ms = (ctypes.c_float * 3)()
        _check(load_library().sdf_batch_timing(self._h, ms), "sdf_batch_timing")
        return {"bin": float(ms[0]), "tile": float(ms[1]), "fp64": float(ms[2])}

    def destroy(self):
        if self._h is not None and self._h.value:
            load_library().sdf_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def sdf_batch_create(features: Sequence[Features], grids: Sequence[Grid], w: Sequence[float],
                     out: Sequence[torch.Tensor] | None = None, winner: bool | Sequence = False,
                     autotune: bool = False, timing: bool = False, fill_sign: bool = False,
                     stream=None) -> Batch:
    """Create a batch; its outputs hold the result on return.  Keep the Features alive meanwhile."""
    feats, grids, ws = list(features), list(grids), list(w)
    n = len(feats)
    if not (len(grids) == len(ws) == n) or n < 1:
        raise ValueError("features, grids and w must be non-empty and of the same length")
    if out is None:
        outs = [torch.empty(g.shape, dtype=torch.float32, device="cuda") for g in grids]
    else:
        outs = list(out)
        for o, g in zip(outs, grids):
            _dev_f32(o, "out")
            if o.numel() != g.nx * g.ny * g.nz:
                raise ValueError("out has the wrong size")
    if isinstance(winner, (list, tuple)):
        wins = list(winner)
    elif winner:
        wins = [torch.empty(g.shape, dtype=torch.int32, device="cuda") for g in grids]
    else:
        wins = [None] * n
    fa = (ctypes.c_void_p * n)(*[f.handle.value for f in feats])
    ga = (_CGrid * n)(*[g.c() for g in grids])
    wa = (ctypes.c_float * n)(*[float(x) for x in ws])
    h = ctypes.c_void_p()
    _check(load_library().sdf_batch_create(fa, ga, wa, n, _ptr_array(outs), _ptr_array(wins),
                                           (FLAG_AUTOTUNE if autotune else 0) | (FLAG_TIMING if timing else 0) |
                                           (FLAG_FILL_SIGN if fill_sign else 0),
                                           _stream(stream), ctypes.byref(h)),
           "sdf_batch_create")
    return Batch(h.value, feats, outs, wins)


def sdf_narrow_band_backward(features: Features, grid: Grid, w: float, grad_dist: torch.Tensor,
                             winner: torch.Tensor | None = None, grad_vertices: torch.Tensor | None = None,
                             flags: int = 0, stream=None) -> torch.Tensor:
    """dL/d(welded vertices) [V, 3] for upstream dL/dd on the grid; accumulates into grad_vertices."""
    g = _dev_f32(grad_dist, "grad_dist")
    grad_vertices, f64 = _grad_vertices(grad_vertices, features.n_vert)
    flags |= f64
    fa = (ctypes.c_void_p * 1)(features.handle.value)
    ga = (_CGrid * 1)(grid.c())
    wa = (ctypes.c_float * 1)(float(w))
    _check(load_library().sdf_narrow_band_backward(fa, ga, wa, 1, _ptr_array([g]),
                                                   _ptr_array([winner]) if winner is not None else None,
                                                   _ptr_array([grad_vertices]), flags, _stream(stream)),
           "sdf_narrow_band_backward")
    return grad_vertices


def band_l2_loss(dist: torch.Tensor, target: torch.Tensor, grad: torch.Tensor | None = None, stream=None):
    """L = sum over the band (finite dist) of (dist - target)^2 and dL/d dist (0 outside the band),
    in one pass; returns (loss as a 0-d float64 CUDA tensor, grad, band point count as a 0-d int64
    CUDA tensor)."""
    d, t = _dev_f32(dist, "dist"), _dev_f32(target, "target")
    if d.numel() != t.numel():
        raise ValueError("dist and target differ in size")
    if grad is None:
        grad = torch.empty_like(d)
    else:
        _dev_f32(grad, "grad")
    loss = torch.empty((), dtype=torch.float64, device=d.device)
    band = torch.empty((), dtype=torch.int64, device=d.device)
    _check(load_library().sdf_band_l2_loss(d.data_ptr(), t.data_ptr(), d.numel(), grad.data_ptr(),
                                           loss.data_ptr(), band.data_ptr(), _stream(stream)), "sdf_band_l2_loss")
    return loss, grad, band


class BandList:
    """Compact band list on the device: entries int32 [capacity, 2] = (point index, winner feature),
    written by sdf_narrow_band_list, and its length as a device int64 [1] (count, which may exceed
    the capacity after an overflow).  Reading len() synchronises; the list calls do not."""

    def __init__(self, capacity: int, device="cuda"):
        self.entries = torch.empty((max(int(capacity), 1), 2), dtype=torch.int32, device=device)
        self.count = torch.zeros(1, dtype=torch.int64, device=device)
        self.dist = None  # float32 [capacity] signed distances, written by the sparse forward

    @property
    def capacity(self) -> int:
        return self.entries.shape[0]

    def __len__(self) -> int:
        return min(int(self.count.item()), self.capacity)

    def indices(self) -> torch.Tensor:
        return self.entries[: len(self), 0]

    def winners(self) -> torch.Tensor:
        return self.entries[: len(self), 1]

    @staticmethod
    def default_capacity(grid: "Grid") -> int:
        """An eighth of the grid points (at least 2^16, at most all): the band is a thin shell."""
        n = grid.nx * grid.ny * grid.nz
        return min(n, max(1 << 16, n // 8))


def sdf_narrow_band_list(features: Features, grid: Grid, w: float, out: torch.Tensor | None = None,
                         band_list: BandList | None = None, winner: bool | torch.Tensor = False, flags: int = 0,
                         stream=None):
    """The narrow band of one problem and its band as a compact list: returns (dist, band_list) or
    (dist, band_list, winner).  A list that turns out too short is grown to the band's length and
    the call repeated (synchronous calls only; with FLAG_NO_SYNC the overflow is reported by
    features.status())."""
    if out is None:
        out = torch.empty(grid.shape, dtype=torch.float32, device="cuda")
    else:
        _dev_f32(out, "out")
        if out.numel() != grid.nx * grid.ny * grid.nz:
            raise ValueError("out has the wrong size")
    if isinstance(winner, torch.Tensor):
        if not winner.is_cuda or winner.dtype != torch.int32 or not winner.is_contiguous():
            raise ValueError("winner must be a contiguous int32 CUDA tensor")
        win = winner
    else:
        win = torch.empty(grid.shape, dtype=torch.int32, device="cuda") if winner else None
    if band_list is None:
        band_list = BandList(BandList.default_capacity(grid))
    ga = (_CGrid * 1)(grid.c())
    for attempt in range(2):
        code = load_library().sdf_narrow_band_list(
            features.handle, ga, float(w), out.data_ptr(), win.data_ptr() if win is not None else None,
            band_list.entries.data_ptr(), band_list.capacity, band_list.count.data_ptr(), flags, _stream(stream))
        if code == ERR_LIST_OVERFLOW and attempt == 0:
            need = int(band_list.count.item())
            band_list.entries = torch.empty((need + need // 4 + 1024, 2), dtype=torch.int32, device="cuda")
            continue
        _check(code, "sdf_narrow_band_list")
        break
    return (out, band_list, win) if win is not None else (out, band_list)


def sdf_narrow_band_sparse(features: Features, grid: Grid, w: float, band_list: BandList | None = None,
                           flags: int = 0, stream=None) -> BandList:
    """The narrow band of one problem as a band list with distances and no dense field: returns the
    BandList, whose `dist` tensor (float32 [capacity]) holds the signed distance of each entry.  A
    list that turns out too short is grown to the band's length and the call repeated (synchronous
    calls only)."""
    if band_list is None:
        band_list = BandList(BandList.default_capacity(grid))
    ga = (_CGrid * 1)(grid.c())
    for attempt in range(2):
        if band_list.dist is None or band_list.dist.numel() < band_list.capacity:
            band_list.dist = torch.empty(band_list.capacity, dtype=torch.float32, device=band_list.entries.device)
        code = load_library().sdf_narrow_band_sparse(
            features.handle, ga, float(w), band_list.entries.data_ptr(), band_list.dist.data_ptr(),
            band_list.capacity, band_list.count.data_ptr(), flags, _stream(stream))
        if code == ERR_LIST_OVERFLOW and attempt == 0:
            need = int(band_list.count.item())
            band_list.entries = torch.empty((need + need // 4 + 1024, 2), dtype=torch.int32, device="cuda")
            continue
        _check(code, "sdf_narrow_band_sparse")
        break
    return band_list


def sdf_narrow_band_lists(features: Sequence[Features], grids: Sequence[Grid], ws: Sequence[float],
                          outs: Sequence[torch.Tensor] | None = None,
                          band_lists: Sequence[BandList] | None = None, stream=None):
    """The narrow bands of a batch of problems in one launch sequence, each with its band list:
    returns (dists, band_lists).  Lists that turn out too short are grown to their band's length
    and the call repeated once."""
    feats, grids, ws = list(features), list(grids), list(ws)
    n = len(feats)
    if not (len(grids) == len(ws) == n) or n == 0:
        raise ValueError("features, grids and ws must have the same, non-zero length")
    if outs is None:
        outs = [torch.empty(g.shape, dtype=torch.float32, device="cuda") for g in grids]
    else:
        outs = list(outs)
        for o, g in zip(outs, grids):
            _dev_f32(o, "out")
            if o.numel() != g.nx * g.ny * g.nz:
                raise ValueError("out has the wrong size")
    lists = list(band_lists) if band_lists is not None else [BandList(BandList.default_capacity(g)) for g in grids]
    if len(lists) != n:
        raise ValueError("one band list per problem")
    fa = (ctypes.c_void_p * n)(*[f.handle.value for f in feats])
    ga = (_CGrid * n)(*[g.c() for g in grids])
    wa = (ctypes.c_float * n)(*[float(x) for x in ws])
    for attempt in range(2):
        caps = (ctypes.c_int64 * n)(*[bl.capacity for bl in lists])
        code = load_library().sdf_narrow_band_lists(
            fa, ga, wa, n, _ptr_array(outs), None, _ptr_array([bl.entries for bl in lists]), caps,
            _ptr_array([bl.count for bl in lists]), 0, _stream(stream))
        if code == ERR_LIST_OVERFLOW and attempt == 0:
            for bl in lists:
                need = int(bl.count.item())
                if need > bl.capacity:
                    bl.entries = torch.empty((need + need // 4 + 1024, 2), dtype=torch.int32, device="cuda")
            continue
        _check(code, "sdf_narrow_band_lists")
        break
    return outs, lists


def band_list_backward(features: Features, grid: Grid, band_list: BandList, grad_dist: torch.Tensor,
                       grad_vertices: torch.Tensor | None = None, flags: int = 0, stream=None) -> torch.Tensor:
    """dL/d(welded vertices) [V, 3] for upstream dL/dd, summed over the listed band points only;
    accumulates into grad_vertices."""
    g = _dev_f32(grad_dist, "grad_dist")
    if g.numel() != grid.nx * grid.ny * grid.nz:
        raise ValueError("grad_dist has the wrong size")
    grad_vertices, f64 = _grad_vertices(grad_vertices, features.n_vert)
    ga = (_CGrid * 1)(grid.c())
    _check(load_library().sdf_band_list_backward(features.handle, ga, band_list.entries.data_ptr(),
                                                 band_list.capacity, band_list.count.data_ptr(), g.data_ptr(),
                                                 grad_vertices.data_ptr(), flags | f64, _stream(stream)),
           "sdf_band_list_backward")
    return grad_vertices


def band_list_l2(features: Features, grid: Grid, band_list: BandList, dist: torch.Tensor, target: torch.Tensor,
                 grad_vertices: torch.Tensor | None = None, flags: int = 0, stream=None):
    """L = sum over the listed band points of (dist - target)^2 and dL/d(welded vertices), fused in
    one pass over the list (no dense gradient); accumulates into grad_vertices.  Returns (loss as a
    0-d float64 CUDA tensor, grad_vertices, band point count as a 0-d int64 CUDA tensor)."""
    d, t = _dev_f32(dist, "dist"), _dev_f32(target, "target")
    n = grid.nx * grid.ny * grid.nz
    if d.numel() != n or t.numel() != n:
        raise ValueError("dist and target must have the grid's size")
    grad_vertices, f64 = _grad_vertices(grad_vertices, features.n_vert)
    loss = torch.empty((), dtype=torch.float64, device=d.device)
    band = torch.empty((), dtype=torch.int64, device=d.device)
    ga = (_CGrid * 1)(grid.c())
    _check(load_library().sdf_band_list_l2(features.handle, ga, band_list.entries.data_ptr(), band_list.capacity,
                                           band_list.count.data_ptr(), d.data_ptr(), t.data_ptr(),
                                           grad_vertices.data_ptr(), loss.data_ptr(), band.data_ptr(), flags | f64,
                                           _stream(stream)), "sdf_band_list_l2")
    return loss, grad_vertices, band


class SDFFunction(torch.autograd.Function):
    """dist = SDFFunction.apply(vertices [V,3], features, grid, w): the narrow band of the mesh with
    the features' connectivity at the given welded vertex positions; differentiable in vertices."""

    @staticmethod
    def forward(ctx, vertices, features: Features, grid: Grid, w: float):
        features.update_positions(vertices.detach().contiguous())
        dist, win = sdf_narrow_band(features, grid, w, winner=True)
        ctx.features, ctx.grid, ctx.w = features, grid, w
        ctx.save_for_backward(win)
        return dist

    @staticmethod
    def backward(ctx, grad_dist):
        (win,) = ctx.saved_tensors
        gv = sdf_narrow_band_backward(ctx.features, ctx.grid, ctx.w, grad_dist.contiguous(), winner=win)
        return gv, None, None, None
