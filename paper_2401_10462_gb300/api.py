"""Thin ctypes binding of libdsasa.so (include/dsasa.h): argument marshalling only.

Every step of the computation runs in the CUDA library; this module passes device
pointers of torch CUDA tensors (or host numpy buffers for ``dsasa_compute_host``) and the
current torch stream.  There is no CPU fallback: if the library is missing, importing
this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = _build.LIB

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")

_lib = ctypes.CDLL(LIB_PATH)

DSASA_OK = 0
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_CAPACITY", 4: "ERR_UNRESOLVED", 5: "ERR_CUDA",
                6: "ERR_UNIMPLEMENTED", 7: "ERR_DEGENERATE", 8: "ERR_INPUT", 9: "ERR_CHECK"}
DSASA_MIXED, DSASA_FP64 = 0, 1
PROBE = 1.4


class dsasa_config(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("skin", ctypes.c_double), ("max_atoms", ctypes.c_int64),
                ("max_cells", ctypes.c_int64), ("carry", ctypes.c_int)]


_vp, _dp, _i64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64
_lib.dsasa_default_config.argtypes = [ctypes.POINTER(dsasa_config)]
_lib.dsasa_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, _vp, ctypes.POINTER(dsasa_config)]
_lib.dsasa_set_stream.argtypes = [_vp, _vp]
_lib.dsasa_set_precision.argtypes = [_vp, ctypes.c_int]
_lib.dsasa_compute.argtypes = [_vp, _vp, _vp, ctypes.c_double, _i64, _vp, _vp]
_lib.dsasa_compute_vjp.argtypes = [_vp, _vp, _vp, ctypes.c_double, _i64, _vp, _vp, _vp]
_lib.dsasa_compute_volume.argtypes = [_vp, _vp, _vp, ctypes.c_double, _i64, _vp, _vp, _vp, _vp]
_lib.dsasa_compute_volume_vjp.argtypes = [_vp, _vp, _vp, ctypes.c_double, _i64, _vp, _vp, _vp, _vp]
_lib.dsasa_compute_sr.argtypes = [_vp, _vp, _vp, ctypes.c_double, _i64, _vp, ctypes.c_int, _vp, _vp]
_lib.dsasa_sr_tests.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64)]
_lib.dsasa_lists_reused.argtypes = [_vp, ctypes.POINTER(ctypes.c_int)]
_lib.dsasa_cells_carried.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64)]
_lib.dsasa_compute_batch.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), _vp, _vp, ctypes.c_double,
                                     _vp, _vp, _vp]
_lib.dsasa_arena_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, _i64]
_lib.dsasa_arena_invalidate.argtypes = [_vp, _i64, _i64, _vp]
_lib.dsasa_arena_destroy.argtypes = [_vp]
_lib.dsasa_compute_batch_resident.argtypes = [_vp, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                              ctypes.POINTER(ctypes.c_int64), _vp, _vp, ctypes.c_double, _vp, _vp,
                                              _vp, _vp]
_lib.dsasa_batch_reused.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int32)]
_lib.dsasa_compute_host.argtypes = [_vp, _vp, _vp, ctypes.c_double, _i64, _vp, _vp, _vp]
_lib.dsasa_status_sync.argtypes = [_vp]
_lib.dsasa_deferred_count.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64)]
_lib.dsasa_set_timing.argtypes = [_vp, ctypes.c_int]
_lib.dsasa_kernel_times.argtypes = [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
_lib.dsasa_export_complex.argtypes = [_vp, _vp, _vp, ctypes.c_double, _i64, _vp, _i64, ctypes.POINTER(ctypes.c_int64)]
_lib.dsasa_last_error.argtypes = [_vp]
_lib.dsasa_debug_fail_allocations.argtypes = [ctypes.c_int]
_lib.dsasa_kernel_launches.argtypes = []
_lib.dsasa_kernel_launches.restype = ctypes.c_int64
_lib.dsasa_last_error.restype = ctypes.c_char_p
_lib.dsasa_destroy.argtypes = [_vp]
_lib.dsasa_version.restype = ctypes.c_char_p
for _f in ("dsasa_create", "dsasa_set_stream", "dsasa_set_precision", "dsasa_compute", "dsasa_compute_vjp",
           "dsasa_compute_batch", "dsasa_compute_host", "dsasa_status_sync", "dsasa_export_complex",
           "dsasa_deferred_count", "dsasa_set_timing", "dsasa_kernel_times", "dsasa_compute_volume",
           "dsasa_compute_volume_vjp", "dsasa_compute_sr", "dsasa_arena_create", "dsasa_arena_invalidate",
           "dsasa_compute_batch_resident", "dsasa_batch_reused",
           "dsasa_sr_tests", "dsasa_lists_reused"):
    getattr(_lib, _f).restype = ctypes.c_int

EXPORTED = ("dsasa_default_config", "dsasa_create", "dsasa_set_stream", "dsasa_set_precision", "dsasa_compute",
            "dsasa_compute_vjp", "dsasa_compute_batch", "dsasa_compute_host", "dsasa_status_sync",
            "dsasa_export_complex", "dsasa_last_error", "dsasa_destroy", "dsasa_version", "dsasa_deferred_count",
            "dsasa_set_timing", "dsasa_kernel_times", "dsasa_compute_volume",
            "dsasa_compute_volume_vjp", "dsasa_arena_create", "dsasa_arena_invalidate", "dsasa_arena_destroy",
            "dsasa_compute_batch_resident", "dsasa_batch_reused",
            "dsasa_compute_sr", "dsasa_sr_tests", "dsasa_lists_reused", "dsasa_cells_carried", "dsasa_kernel_launches",
            "dsasa_debug_fail_allocations")


class DSASAError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dsasa {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def version() -> str:
    return _lib.dsasa_version().decode()


def kernel_launches() -> int:
    """CUDA kernels launched by the library since it was loaded (all contexts)."""
    return int(_lib.dsasa_kernel_launches())


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(t.ctypes.data)


def _check_tensor(t, name, n, width=None):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    shape = (n,) if width is None else (n, width)
    if tuple(t.shape) != shape:
        raise ValueError(f"{name} must have shape {shape}, got {tuple(t.shape)}")


class Context:
    """One dsasa_ctx bound to a device and a stream (default: torch's current stream)."""

    def __init__(self, device: int = 0, stream=None, precision: str | int = "mixed", skin: float = 0.0,
                 max_atoms: int = 0, max_cells: int = 0, carry: int = 1):
        cfg = dsasa_config()
        _lib.dsasa_default_config(ctypes.byref(cfg))
        cfg.precision = precision if isinstance(precision, int) else {"mixed": DSASA_MIXED, "fp64": DSASA_FP64}[precision]
        cfg.skin = float(skin)
        cfg.max_atoms = int(max_atoms)
        cfg.max_cells = int(max_cells)
        cfg.carry = int(carry)   # 0 off, 1 beyond one wave of the fused cell kernel, 2 always
        self.device = device
        h = _vp()
        st = _lib.dsasa_create(ctypes.byref(h), device, _vp(self._stream_handle(stream)), ctypes.byref(cfg))
        if st != DSASA_OK:
            raise DSASAError(st, "dsasa_create failed")
        self._h = h
        self._stream = stream

    @staticmethod
    def _stream_handle(stream):
        if stream is None:
            import torch
            return torch.cuda.current_stream().cuda_stream
        if isinstance(stream, int):
            return stream
        return stream.cuda_stream

    def _sync_stream(self):
        if self._stream is None:
            _lib.dsasa_set_stream(self._h, _vp(self._stream_handle(None)))

    def _raise(self, st):
        if st != DSASA_OK:
            raise DSASAError(st, _lib.dsasa_last_error(self._h).decode())

    def set_precision(self, precision):
        p = precision if isinstance(precision, int) else {"mixed": DSASA_MIXED, "fp64": DSASA_FP64}[precision]
        self._raise(_lib.dsasa_set_precision(self._h, p))

    def compute(self, coords, radii, areas_out, grad_out=None, weights=None, probe: float = PROBE):
        """dsasa_compute_vjp on device tensors (asynchronous on the stream)."""
        n = int(coords.shape[0])
        _check_tensor(coords, "coords", n, 3)
        _check_tensor(radii, "radii", n)
        _check_tensor(areas_out, "areas_out", n)
        if grad_out is not None:
            _check_tensor(grad_out, "grad_out", n, 3)
        if weights is not None:
            _check_tensor(weights, "weights", n)
        self._sync_stream()
        self._raise(_lib.dsasa_compute_vjp(self._h, _ptr(coords), _ptr(radii), float(probe), n, _ptr(weights),
                                           _ptr(areas_out), _ptr(grad_out)))

    def compute_volume(self, coords, radii, areas_out, volumes_out, grad_out=None, vol_grad_out=None,
                       probe: float = PROBE):
        """dsasa_compute_volume: areas, per-atom power-cell volumes (sum = union volume) and
        optionally d(area sum)/dx and d(union volume)/dx, on device tensors."""
        n = int(coords.shape[0])
        _check_tensor(coords, "coords", n, 3)
        _check_tensor(radii, "radii", n)
        _check_tensor(areas_out, "areas_out", n)
        _check_tensor(volumes_out, "volumes_out", n)
        if grad_out is not None:
            _check_tensor(grad_out, "grad_out", n, 3)
        if vol_grad_out is not None:
            _check_tensor(vol_grad_out, "vol_grad_out", n, 3)
        self._sync_stream()
        self._raise(_lib.dsasa_compute_volume(self._h, _ptr(coords), _ptr(radii), float(probe), n, _ptr(areas_out),
                                              _ptr(grad_out), _ptr(volumes_out), _ptr(vol_grad_out)))

    def compute_volume_vjp(self, coords, radii, weights, areas_out, volumes_out, vol_grad_out,
                           probe: float = PROBE):
        """dsasa_compute_volume_vjp: areas, per-atom volumes and d(sum_i w_i V_i)/dx for volume
        weights w (device tensor, or None for ones)."""
        n = int(coords.shape[0])
        _check_tensor(coords, "coords", n, 3)
        _check_tensor(radii, "radii", n)
        _check_tensor(areas_out, "areas_out", n)
        _check_tensor(volumes_out, "volumes_out", n)
        _check_tensor(vol_grad_out, "vol_grad_out", n, 3)
        if weights is not None:
            _check_tensor(weights, "weights", n)
        self._sync_stream()
        self._raise(_lib.dsasa_compute_volume_vjp(self._h, _ptr(coords), _ptr(radii), float(probe), n, _ptr(weights),
                                                  _ptr(areas_out), _ptr(volumes_out), _ptr(vol_grad_out)))

    def compute_sr(self, coords, radii, unit_points, areas_out, exposed_out=None, probe: float = PROBE):
        """dsasa_compute_sr: Shrake-Rupley areas on the m float32 unit vectors unit_points
        (device tensor (m, 3)); optional int32 exposed-point counts."""
        n = int(coords.shape[0])
        _check_tensor(coords, "coords", n, 3)
        _check_tensor(radii, "radii", n)
        _check_tensor(areas_out, "areas_out", n)
        import torch
        if unit_points.dtype != torch.float32 or not unit_points.is_cuda or not unit_points.is_contiguous():
            raise ValueError("unit_points must be a contiguous float32 CUDA tensor (m, 3)")
        if exposed_out is not None and (exposed_out.dtype != torch.int32 or exposed_out.numel() != n):
            raise ValueError("exposed_out must be int32 with n entries")
        self._sync_stream()
        self._raise(_lib.dsasa_compute_sr(self._h, _ptr(coords), _ptr(radii), float(probe), n, _ptr(unit_points),
                                          int(unit_points.shape[0]), _ptr(areas_out), _ptr(exposed_out)))

    def lists_reused(self) -> bool:
        """Whether the last call reused the Verlet lists (contexts with skin > 0)."""
        r = ctypes.c_int(0)
        self._raise(_lib.dsasa_lists_reused(self._h, ctypes.byref(r)))
        return bool(r.value)

    def cells_carried(self) -> int:
        """Atoms whose cell the last call carried from the previous call (skin > 0, carry on)."""
        t = ctypes.c_int64(0)
        self._raise(_lib.dsasa_cells_carried(self._h, ctypes.byref(t)))
        return int(t.value)

    def sr_tests(self) -> int:
        """Point-neighbour tests of the last compute_sr call."""
        t = ctypes.c_int64(0)
        self._raise(_lib.dsasa_sr_tests(self._h, ctypes.byref(t)))
        return int(t.value)

    def compute_batch(self, offsets, coords, radii, areas_out, grad_out=None, weights=None, probe: float = PROBE):
        """dsasa_compute_batch: molecule m owns atoms [offsets[m], offsets[m+1])."""
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        n = int(off[-1])
        _check_tensor(coords, "coords", n, 3)
        _check_tensor(radii, "radii", n)
        _check_tensor(areas_out, "areas_out", n)
        self._sync_stream()
        self._raise(_lib.dsasa_compute_batch(self._h, len(off) - 1, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                             _ptr(coords), _ptr(radii), float(probe), _ptr(weights), _ptr(areas_out),
                                             _ptr(grad_out)))

    def compute_batch_resident(self, offsets, coords, radii, areas_out, grad_out=None, arena=None,
                               arena_base=None, mol_ready=None, weights=None, probe: float = PROBE):
        """dsasa_compute_batch_resident: a batch with optional resident lists (arena: an Arena,
        arena_base: slot of each molecule or -1) and per-molecule ready flags (mol_ready:
        int32 tensor of n_mol zeros, device or pinned host).  The output tensors may be
        pinned host tensors (zero-copy)."""
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        n_mol = len(off) - 1
        base = None
        if arena is not None:
            base = np.ascontiguousarray(arena_base, dtype=np.int64)
            if base.shape != (n_mol,):
                raise ValueError("arena_base needs one entry per molecule")
        self._sync_stream()
        p64 = ctypes.POINTER(ctypes.c_int64)
        self._raise(_lib.dsasa_compute_batch_resident(
            self._h, arena._h if arena is not None else None, n_mol, off.ctypes.data_as(p64),
            base.ctypes.data_as(p64) if base is not None else None, _ptr(coords), _ptr(radii), float(probe),
            _ptr(weights), _ptr(areas_out), _ptr(grad_out), _ptr(mol_ready)))

    def batch_reused(self, n_mol: int) -> np.ndarray:
        """Per molecule of the last resident batch: whether its lists were reused."""
        out = np.zeros(max(n_mol, 1), dtype=np.int32)
        self._raise(_lib.dsasa_batch_reused(self._h, n_mol, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
        return out[:n_mol].astype(bool)

    def compute_host(self, coords, radii, weights=None, grad: bool = True, probe: float = PROBE, out=None):
        """dsasa_compute_host on numpy buffers, synchronised.  Buffers in pinned memory (e.g.
        numpy views of torch tensors made with pin_memory=True) are read and written in place
        by the kernels; pageable ones are copied through device staging buffers."""
        xyz = np.ascontiguousarray(coords, dtype=np.float64)
        r = np.ascontiguousarray(radii, dtype=np.float64)
        n = xyz.shape[0]
        w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
        if out is None:
            a = np.empty(n)
            g = np.empty((n, 3)) if grad else None
        else:
            a, g = out
            for arr, shape in ((a, (n,)), (g, (n, 3))):
                if arr is not None and (arr.dtype != np.float64 or arr.shape != shape or not arr.flags.c_contiguous
                                        or not arr.flags.writeable):
                    raise ValueError(f"out arrays must be writeable C-contiguous float64 of shape {shape}")
        self._sync_stream()
        dp = lambda x: None if x is None else x.ctypes.data   # the address (cheaper than data_as)
        self._raise(_lib.dsasa_compute_host(self._h, dp(xyz), dp(r), float(probe), n, dp(w), dp(a), dp(g)))
        return a, g

    def status_sync(self):
        """Synchronise and raise if a device-side error was recorded since the last call."""
        self._raise(_lib.dsasa_status_sync(self._h))

    PHASES = ("cell_list", "cell", "classify", "terms", "large")

    def set_timing(self, enable: bool = True):
        """Record CUDA events around each kernel phase of every compute call (diagnostics)."""
        self._raise(_lib.dsasa_set_timing(self._h, int(bool(enable))))

    def kernel_times(self):
        """({phase: summed device ms}, calls) since the last read; resets the sums."""
        ms = (ctypes.c_double * len(self.PHASES))()
        calls = ctypes.c_int64(0)
        self._raise(_lib.dsasa_kernel_times(self._h, ms, ctypes.byref(calls)))
        return {p: float(ms[k]) for k, p in enumerate(self.PHASES)}, int(calls.value)

    def deferred_count(self) -> int:
        """Atoms of the last call whose cell went to the large-capacity pass."""
        d = ctypes.c_int64(0)
        self._raise(_lib.dsasa_deferred_count(self._h, ctypes.byref(d)))
        return int(d.value)

    def status_code(self) -> int:
        return _lib.dsasa_status_sync(self._h)

    def export_complex(self, coords, radii, probe: float = PROBE, max_records: int = None):
        """Records (owner, v0, v1, v2, v3) of every simplex of C seen by every atom's cell."""
        import torch
        n = int(coords.shape[0])
        cap = max_records or 64 * n + 64
        rec = torch.empty((cap, 5), dtype=torch.int32, device=coords.device)
        cnt = ctypes.c_int64(0)
        self._sync_stream()
        st = _lib.dsasa_export_complex(self._h, _ptr(coords), _ptr(radii), float(probe), n, _ptr(rec), cap,
                                       ctypes.byref(cnt))
        self._raise(st)
        return rec[: cnt.value]

    def close(self):
        if getattr(self, "_h", None):
            _lib.dsasa_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Arena:
    """A dsasa_arena: resident Verlet lists of molecules kept on one device across calls."""

    def __init__(self, capacity_atoms: int, device: int = 0):
        h = _vp()
        st = _lib.dsasa_arena_create(ctypes.byref(h), device, int(capacity_atoms))
        if st != DSASA_OK:
            raise DSASAError(st, "dsasa_arena_create failed")
        self._h = h
        self.capacity = int(capacity_atoms)

    def invalidate(self, base: int, n: int, stream=None):
        s = Context._stream_handle(stream)
        st = _lib.dsasa_arena_invalidate(self._h, int(base), int(n), _vp(s))
        if st != DSASA_OK:
            raise DSASAError(st, "dsasa_arena_invalidate failed")

    def close(self):
        if getattr(self, "_h", None):
            _lib.dsasa_arena_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default_ctx = {}


def default_context(device: int = 0, precision: str = "mixed") -> Context:
    key = (device, precision)
    if key not in _default_ctx:
        _default_ctx[key] = Context(device=device, precision=precision)
    return _default_ctx[key]


def sasa(coords, radii, probe: float = PROBE, weights=None, grad: bool = True, precision: str = "mixed",
         check: bool = True):
    """SASA per atom (and d(sum w_i A_i)/dx) for CUDA float64 tensors; returns (areas, grad)."""
    import torch
    ctx = default_context(coords.device.index or 0, precision)
    n = coords.shape[0]
    areas = torch.empty(n, dtype=torch.float64, device=coords.device)
    g = torch.empty((n, 3), dtype=torch.float64, device=coords.device) if grad else None
    ctx.compute(coords.contiguous(), radii.contiguous(), areas, g, weights, probe)
    if check:
        ctx.status_sync()
    return areas, g
