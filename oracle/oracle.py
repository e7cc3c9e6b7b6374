"""ctypes binding of the dSASA oracle (``dsasa_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py``; the product path never imports it.

The oracle computes, on the CPU in FP64 with exact predicates, the regular triangulation
of the probe-inflated atoms (paper Step 1), its alpha = 0 dual complex (Step 2) and the
per-atom inclusion-exclusion areas with their gradient (Step 3, Eqs. sainexclu/inexclu).
``gauss_bonnet`` is an unrelated exact per-sphere area (arc arrangement on each sphere)
used to pin the whole chain.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, f) for f in ("dsasa_oracle.cpp", "exact.hpp", "dual.hpp")]
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

PROBE = 1.4


def build(force: bool = False) -> str:
    """Compile the oracle (g++, plain C++17) in-tree; returns the shared-library path."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SRC)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp, _SRC[0]]
        try:   # OpenMP only serves the timing of the area stage on all cores
            subprocess.check_call(cmd[:1] + ["-fopenmp"] + cmd[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            lp = ctypes.POINTER(ctypes.c_long)
            lib.oracle_build.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_char_p, ctypes.c_int]
            lib.oracle_build.restype = ctypes.c_void_p
            lib.oracle_free.argtypes = [ctypes.c_void_p]
            lib.oracle_counts.argtypes = [ctypes.c_void_p, lp]
            lib.oracle_times.argtypes = [ctypes.c_void_p, dp]
            lib.oracle_term_counts.argtypes = [ctypes.c_void_p, lp]
            lib.oracle_simplices.argtypes = [ctypes.c_void_p, ctypes.c_int, ip]
            lib.oracle_redundant.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_ubyte)]
            lib.oracle_areas.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
            lib.oracle_areas.restype = ctypes.c_long
            lib.oracle_areas_parallel.argtypes = [ctypes.c_void_p, dp, dp, dp, dp, ctypes.c_int, ip]
            lib.oracle_areas_parallel.restype = ctypes.c_long
            lib.oracle_volumes.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
            lib.oracle_volumes.restype = ctypes.c_long
            lib.oracle_gauss_bonnet.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, dp]
            lib.oracle_gauss_bonnet.restype = ctypes.c_int
            lib.oracle_tri_term.argtypes = [dp, dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp]
            lib.oracle_tri_term.restype = ctypes.c_int
            lib.oracle_predicate.argtypes = [ctypes.c_int, ctypes.c_int, dp, ip]
            lib.oracle_predicate.restype = ctypes.c_int
            _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


COUNT_KEYS = ("rt_tets", "rt_tets_total", "K0", "K1", "K2", "K3", "redundant", "rt_tris", "rt_edges",
              "power_tests", "sos", "alpha_tests", "orient_tests", "degenerate_insertions")


class Oracle:
    """Triangulation + dual complex of one molecule; areas/gradients on demand."""

    def __init__(self, coords, radii, probe: float = PROBE):
        lib = _load()
        self.coords = np.ascontiguousarray(coords, dtype=np.float64).reshape(-1, 3)
        self.radii = np.ascontiguousarray(radii, dtype=np.float64).reshape(-1)
        self.probe = float(probe)
        self.n = self.coords.shape[0]
        err = ctypes.create_string_buffer(512)
        h = lib.oracle_build(self.n, _d(self.coords), _d(self.radii), self.probe, err, 512)
        if not h:
            raise RuntimeError("oracle build failed: " + err.value.decode())
        self._h = ctypes.c_void_p(h)
        self._lib = lib

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and self._lib is not None:
            self._lib.oracle_free(h)
            self._h = None

    def counts(self) -> dict:
        out = (ctypes.c_long * 14)()
        self._lib.oracle_counts(self._h, out)
        return dict(zip(COUNT_KEYS, list(out)))

    def times(self) -> dict:
        out = (ctypes.c_double * 2)()
        self._lib.oracle_times(self._h, out)
        return {"triangulation_s": out[0], "alpha_s": out[1]}

    TERM_KEYS = ("vertex_constants", "solid_angles", "dihedrals", "edge_caps", "triangles")

    def term_counts(self) -> dict:
        """Numbers of the terms of Eq. (sainexclu) the area computation evaluates."""
        out = (ctypes.c_long * 5)()
        self._lib.oracle_term_counts(self._h, out)
        return dict(zip(self.TERM_KEYS, list(out)))

    def simplices(self, dim: int) -> np.ndarray:
        """dim 0..3: the dual complex C (sorted tuples); dim 4: all triangulation tetrahedra."""
        c = self.counts()
        m = {0: c["K0"], 1: c["K1"], 2: c["K2"], 3: c["K3"], 4: c["rt_tets"]}[dim]
        w = {0: 1, 1: 2, 2: 3, 3: 4, 4: 4}[dim]
        out = np.zeros(max(m * w, 1), dtype=np.int32)
        self._lib.oracle_simplices(self._h, dim, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return out[: m * w].reshape(m, w) if w > 1 else out[:m]

    def redundant(self) -> np.ndarray:
        out = np.zeros(max(self.n, 1), dtype=np.uint8)
        self._lib.oracle_redundant(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
        return out[: self.n].astype(bool)

    def areas(self, weights=None, grad: bool = True):
        """Per-atom SASA, total, and d(sum_i w_i A_i)/dx (n, 3) (None if grad=False)."""
        a = np.zeros(max(self.n, 1))
        g = np.zeros((max(self.n, 1), 3)) if grad else None
        tot = ctypes.c_double(0)
        w = None
        if weights is not None:
            w = np.ascontiguousarray(weights, dtype=np.float64).reshape(-1)
        bad = self._lib.oracle_areas(self._h, _d(w) if w is not None else None, _d(a),
                                     _d(g) if g is not None else None, ctypes.byref(tot))
        if bad:
            raise RuntimeError(f"{bad} triangles of C without a triple point")
        return a[: self.n], tot.value, (g[: self.n] if g is not None else None)


    def areas_parallel(self, threads: int, grad: bool = True):
        """areas() with the term loops on `threads` OpenMP threads (for timing the area and
        gradient stage on all cores); returns (areas, total, grad, threads used)."""
        a = np.zeros(max(self.n, 1))
        g = np.zeros((max(self.n, 1), 3)) if grad else None
        tot = ctypes.c_double(0)
        used = ctypes.c_int(1)
        bad = self._lib.oracle_areas_parallel(self._h, None, _d(a), _d(g) if g is not None else None,
                                              ctypes.byref(tot), int(threads), ctypes.byref(used))
        if bad:
            raise RuntimeError(f"{bad} triangles of C without a triple point")
        return a[: self.n], tot.value, (g[: self.n] if g is not None else None), used.value

    def volumes(self, grad: bool = True, weights=None):
        """Per-atom volumes vol(B_i cap L_i), their total (the union volume) and
        d(sum_i w_i V_i)/dx (n, 3) (None if grad=False; weights None = ones, the gradient of
        the union volume)."""
        v = np.zeros(max(self.n, 1))
        g = np.zeros((max(self.n, 1), 3)) if grad else None
        tot = ctypes.c_double(0)
        w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64).reshape(-1)
        bad = self._lib.oracle_volumes(self._h, _d(w) if w is not None else None, _d(v),
                                       _d(g) if g is not None else None, ctypes.byref(tot))
        if bad:
            raise RuntimeError(f"{bad} triangles of C without a triple point")
        return v[: self.n], tot.value, (g[: self.n] if g is not None else None)


def sasa(coords, radii, probe: float = PROBE, weights=None, grad: bool = True):
    """One-shot: (areas, total, grad)."""
    return Oracle(coords, radii, probe).areas(weights, grad)


def gauss_bonnet(coords, radii, probe: float = PROBE):
    """Independent exact per-sphere exposed areas; returns (areas, n_nongeneric)."""
    lib = _load()
    xyz = np.ascontiguousarray(coords, dtype=np.float64).reshape(-1, 3)
    r = np.ascontiguousarray(radii, dtype=np.float64).reshape(-1)
    out = np.zeros(max(xyz.shape[0], 1))
    bad = lib.oracle_gauss_bonnet(xyz.shape[0], _d(xyz), _d(r), float(probe), _d(out))
    return out[: xyz.shape[0]], bad


def tri_term(p1, p2, p3, R1, R2, R3):
    """S_123^(1) of Eq. (trianglev) (radii include the probe) and its 3x3 gradient."""
    lib = _load()
    ps = [np.ascontiguousarray(p, dtype=np.float64) for p in (p1, p2, p3)]
    v = ctypes.c_double(0)
    g = np.zeros(9)
    ok = lib.oracle_tri_term(_d(ps[0]), _d(ps[1]), _d(ps[2]), R1, R2, R3, ctypes.byref(v), _d(g))
    return (v.value if ok else None), g.reshape(3, 3)


def predicate(kind: int, pts_xyzR, ids) -> int:
    """Exact sign predicates: 0 orient, 1 conflict (-1 = conflict), 2 tet psi, 3 tri psi, 4 edge psi,
    5/6/7 attachment of a triangle / edge / vertex by the last point (1 = attached)."""
    lib = _load()
    a = np.ascontiguousarray(pts_xyzR, dtype=np.float64).reshape(-1, 4)
    idx = np.ascontiguousarray(ids, dtype=np.int32)
    return lib.oracle_predicate(kind, a.shape[0], _d(a), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))


def local_patch(coords, radii, centre_ids, probe: float = PROBE, cutoff: float = None):
    """Indices of the atoms within `cutoff` of any centre atom (sorted).

    A_i and the gradient entry g_i of atom i depend only on the atoms whose balls overlap
    B_i: every simplex of the dual complex that contains i lies in B_i, where a ball that
    misses B_i never has the smaller power.  A patch of radius R_i + R_max around i therefore
    reproduces atom i's outputs exactly; the default 4 R_max + 1 A keeps a margin.  Pinned
    against the whole-molecule oracle in tests/test_oracle_local_patch.py."""
    coords = np.asarray(coords)
    rmax = float(np.max(radii)) + probe
    if cutoff is None:
        cutoff = 4.0 * rmax + 1.0
    c = coords[np.asarray(centre_ids)]
    d2 = ((coords[None, :, :] - c[:, None, :]) ** 2).sum(-1).min(0)
    return np.nonzero(d2 <= cutoff * cutoff)[0]
