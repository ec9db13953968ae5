"""ctypes binding of the FP64 CPU oracle (oracle/oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's CPU
baseline / reference leg use it.  The product path never imports this module.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_ERRORS = {2: "non-manifold or non-oriented mesh", 3: "degenerate triangle", 4: "non-finite coordinate",
           6: "out of memory"}


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (plain C, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
            L.om_build_soup.argtypes = [P, I64, ctypes.POINTER(P)]
            L.om_build_indexed.argtypes = [P, I64, P, I64, ctypes.POINTER(P)]
            L.om_free.argtypes = [P]
            L.om_counts.argtypes = [P, P]
            for f in ("om_vertices", "om_triangles", "om_soup_vid", "om_vclass", "om_pseudonormals"):
                getattr(L, f).argtypes = [P, P]
            L.om_sdf_points.argtypes = [P, P, I64, ctypes.c_int, P, P, P]
            L.om_band_points.argtypes = [P, P, P, D, D, P, I64, ctypes.c_int, P, P, P]
            L.om_narrow_band.argtypes = [P, P, P, D, D, ctypes.c_int, P, P]
            L.om_adjoint_points.argtypes = [P, P, P, I64, D, P]
            L.om_adjoint_features.argtypes = [P, P, P, P, P, I64, P, P]
            L.om_set_num_threads.argtypes = [ctypes.c_int]
            L.om_set_num_threads.restype = None
            L.om_num_threads.restype = ctypes.c_int
            _lib = L
        return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleMesh:
    """Welded mesh with FP64 pseudonormals, built from an FP32 soup or an indexed mesh."""

    def __init__(self, handle):
        self._h = handle
        c = np.zeros(8, dtype=np.int64)
        lib().om_counts(self._h, _ptr(c))
        self.V, self.E = int(c[0]), int(c[1])
        self.n_convex, self.n_concave, self.n_flat, self.n_saddle = (int(x) for x in c[2:6])
        self.n_convex_edges, self.n_concave_edges = int(c[6]), int(c[7])

    @classmethod
    def from_soup(cls, soup: np.ndarray) -> "OracleMesh":
        s = np.ascontiguousarray(soup, dtype=np.float32).reshape(-1, 9)
        h = ctypes.c_void_p()
        st = lib().om_build_soup(_ptr(s), s.shape[0], ctypes.byref(h))
        if st:
            raise ValueError(f"oracle: {_ERRORS.get(st, st)}")
        m = cls(h)
        m.T = s.shape[0]
        return m

    @classmethod
    def from_indexed(cls, X: np.ndarray, tri: np.ndarray) -> "OracleMesh":
        X = np.ascontiguousarray(X, dtype=np.float64)
        tri = np.ascontiguousarray(tri, dtype=np.int32)
        h = ctypes.c_void_p()
        st = lib().om_build_indexed(_ptr(X), X.shape[0], _ptr(tri), tri.shape[0], ctypes.byref(h))
        if st:
            raise ValueError(f"oracle: {_ERRORS.get(st, st)}")
        m = cls(h)
        m.T = tri.shape[0]
        return m

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.om_free(self._h)
            self._h = None

    # ------------------------------------------------------------------ accessors
    def vertices(self) -> np.ndarray:
        out = np.empty((self.V, 3), dtype=np.float64)
        lib().om_vertices(self._h, _ptr(out))
        return out

    def triangles(self) -> np.ndarray:
        out = np.empty((self.T, 3), dtype=np.int32)
        lib().om_triangles(self._h, _ptr(out))
        return out

    def soup_vid(self) -> np.ndarray:
        out = np.empty(3 * self.T, dtype=np.int32)
        lib().om_soup_vid(self._h, _ptr(out))
        return out

    def vertex_classes(self) -> np.ndarray:
        out = np.empty(self.V, dtype=np.int8)
        lib().om_vclass(self._h, _ptr(out))
        return out

    def pseudonormals(self) -> np.ndarray:
        out = np.empty((self.V, 3), dtype=np.float64)
        lib().om_pseudonormals(self._h, _ptr(out))
        return out

    # ------------------------------------------------------------------ queries
    def sdf_points(self, pts: np.ndarray, pruned: bool = True):
        """Signed distance (no band) at arbitrary points; returns (d, triangle, region)."""
        p = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        n = p.shape[0]
        d = np.empty(n)
        t = np.empty(n, dtype=np.int32)
        r = np.empty(n, dtype=np.int32)
        lib().om_sdf_points(self._h, _ptr(p), n, int(pruned), _ptr(d), _ptr(t), _ptr(r))
        return d, t, r

    def band_points(self, dims, origin, h: float, w: float, idx: np.ndarray, pruned: bool = True):
        """Narrow-band value (+inf outside) at grid points given by linear index (x fastest)."""
        dims = np.ascontiguousarray(dims, dtype=np.int32)
        origin = np.ascontiguousarray(origin, dtype=np.float64)
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        n = idx.shape[0]
        d = np.empty(n)
        t = np.empty(n, dtype=np.int32)
        r = np.empty(n, dtype=np.int32)
        lib().om_band_points(self._h, _ptr(dims), _ptr(origin), float(h), float(w), _ptr(idx), n, int(pruned),
                             _ptr(d), _ptr(t), _ptr(r))
        return d, t, r

    def narrow_band(self, dims, origin, h: float, w: float, pruned: bool = True, winners: bool = False):
        """Dense narrow band [nz, ny, nx] (float64, +inf outside) and optionally winning triangles."""
        dims = np.ascontiguousarray(dims, dtype=np.int32)
        origin = np.ascontiguousarray(origin, dtype=np.float64)
        nx, ny, nz = (int(x) for x in dims)
        out = np.empty((nz, ny, nx))
        tri = np.empty((nz, ny, nx), dtype=np.int32) if winners else None
        lib().om_narrow_band(self._h, _ptr(dims), _ptr(origin), float(h), float(w), int(pruned), _ptr(out),
                             _ptr(tri) if winners else None)
        return (out, tri) if winners else out

    def adjoint_points(self, pts: np.ndarray, g: np.ndarray, w: float) -> np.ndarray:
        """d(sum_p g_p d(p)) / d(welded vertices) [V,3] (band membership found here)."""
        p = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        g = np.ascontiguousarray(g, dtype=np.float64)
        out = np.empty((self.V, 3))
        lib().om_adjoint_points(self._h, _ptr(p), _ptr(g), p.shape[0], float(w), _ptr(out))
        return out

    def adjoint_features(self, pts: np.ndarray, g: np.ndarray, tri: np.ndarray, region: np.ndarray):
        """The adjoint of sum_p g_p d_F(p) [V,3] with each point's feature F GIVEN as (triangle,
        region label: 0 face, 1+k edge from corner k to k+1, 4+k corner k), and the signed
        distances d_F(p) [n]; no band test."""
        p = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        g = np.ascontiguousarray(g, dtype=np.float64)
        tri = np.ascontiguousarray(tri, dtype=np.int32)
        region = np.ascontiguousarray(region, dtype=np.int32)
        n = p.shape[0]
        assert g.shape == (n,) and tri.shape == (n,) and region.shape == (n,)
        if n and (tri.min() < 0 or tri.max() >= self.T or region.min() < 0 or region.max() > 6):
            raise ValueError("feature out of range")
        out = np.empty((self.V, 3))
        d = np.empty(n)
        lib().om_adjoint_features(self._h, _ptr(p), _ptr(g), _ptr(tri), _ptr(region), n, _ptr(out), _ptr(d))
        return out, d


def num_threads() -> int:
    return int(lib().om_num_threads())


_DEFAULT_THREADS = None


def num_threads_default() -> int:
    """The thread count the oracle started with (before any set_num_threads)."""
    return _DEFAULT_THREADS if _DEFAULT_THREADS else num_threads()


def set_num_threads(n: int) -> None:
    """OpenMP threads of the following oracle calls (1: sums in one fixed order)."""
    global _DEFAULT_THREADS
    if _DEFAULT_THREADS is None:
        _DEFAULT_THREADS = num_threads()
    lib().om_set_num_threads(int(n))


def grid_points(dims, origin, h: float, idx: np.ndarray) -> np.ndarray:
    """Cell-centre coordinates (float64) of linear grid indices (x fastest)."""
    nx, ny, _ = (int(x) for x in dims)
    idx = np.asarray(idx, dtype=np.int64)
    i, j, k = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    o = np.asarray(origin, dtype=np.float64)
    return np.stack([o[0] + (i + 0.5) * h, o[1] + (j + 0.5) * h, o[2] + (k + 0.5) * h], axis=1)
