"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds no surface-area arithmetic: it only places atoms and draws radii
(the C core is ``gen/molgen.c``).  The shapes stand in for the paper's workloads
(mini-proteins, RNA hairpins, large assemblies; Sec. "Simulated protein systems, RNA
systems" and "Speed Comparison"), whose structures are not available here.

Recipe (every draw comes from a xoshiro256** stream seeded by splitmix64(seed)):

* ``globule(n, seed)`` - self-avoiding chain, bond 1.53 A, non-bonded minimum 2.6 A
  (|i-j| >= 3; 2.2 A for |i-j| = 2), confined in a sphere whose radius starts at
  (3n / (4 pi 0.1))^(1/3) (0.1 atoms/A^3) and grows by 2 % whenever the walk keeps
  failing; radii H 1.2 (50 %), C 1.7 (30 %), N 1.55 (9 %), O 1.52 (10 %), S 1.8 (1 %).
* ``rna(n, seed)`` - two helical strands, helix radius 20 A, rise 3.4 A, 10 nt/turn,
  strand 2 phase-shifted by 180 degrees; per nucleotide one P (1.9 A) on the backbone
  plus 31 atoms grown inward (H/C/N/O 40/30/12/16).
* ``shell(n, seed)`` - chains of 300 atoms filling a 30 A thick spherical shell; the outer
  radius starts at 150 A and grows by 2 % (refill) until n atoms fit.

Every coordinate then receives a uniform jitter in (-1e-6, 1e-6) A, which makes the
inputs generic (no exact co-spherical or co-planar subsets).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

PROBE = 1.4
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen", "molgen.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libmolgen.so")
_lock = threading.Lock()
_lib = None


def build_generators(force: bool = False) -> str:
    """Compile the generator core (plain C, no CUDA) in-tree and return the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_generators())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.molgen_globule.argtypes = [ctypes.c_int, ctypes.c_uint64, dp, dp]
            lib.molgen_globule.restype = ctypes.c_double
            lib.molgen_rna.argtypes = [ctypes.c_int, ctypes.c_uint64, dp, dp]
            lib.molgen_rna.restype = ctypes.c_double
            lib.molgen_shell.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int, dp, dp]
            lib.molgen_shell.restype = ctypes.c_double
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Molecule:
    """coords (n, 3) float64 [A], radii (n,) float64 [A] (unprobed), plus metadata."""

    def __init__(self, kind, coords, radii, seed, extent):
        self.kind = kind
        self.coords = coords
        self.radii = radii
        self.seed = seed
        self.extent = extent

    @property
    def n(self) -> int:
        return int(self.coords.shape[0])

    def density(self) -> float:
        """Atoms per A^3 of the confining volume (the generator's achieved packing)."""
        if self.kind == "globule":
            return self.n / (4.0 / 3.0 * math.pi * self.extent ** 3)
        if self.kind == "shell":
            ro, ri = self.extent, self.extent - 30.0
            return self.n / (4.0 / 3.0 * math.pi * (ro ** 3 - ri ** 3))
        return float("nan")

    def __repr__(self):
        return f"Molecule({self.kind}, n={self.n}, seed={self.seed}, extent={self.extent:.2f})"


def globule(n: int, seed: int = 0) -> Molecule:
    xyz = np.zeros((max(n, 1), 3), dtype=np.float64)
    rad = np.zeros(max(n, 1), dtype=np.float64)
    rc = _load().molgen_globule(int(n), int(seed) & (2 ** 64 - 1), _ptr(xyz), _ptr(rad))
    if rc < 0:
        raise RuntimeError(f"globule generator failed (n={n}, seed={seed})")
    return Molecule("globule", xyz[:n].copy(), rad[:n].copy(), seed, rc)


def rna(n: int, seed: int = 0) -> Molecule:
    xyz = np.zeros((max(n, 1), 3), dtype=np.float64)
    rad = np.zeros(max(n, 1), dtype=np.float64)
    r = _load().molgen_rna(int(n), int(seed) & (2 ** 64 - 1), _ptr(xyz), _ptr(rad))
    if r < 0:
        raise RuntimeError(f"rna generator failed (n={n}, seed={seed})")
    return Molecule("rna", xyz[:n].copy(), rad[:n].copy(), seed, r)


def shell(n: int, seed: int = 0, r_out: float = 150.0, thickness: float = 30.0, chain: int = 300) -> Molecule:
    xyz = np.zeros((max(n, 1), 3), dtype=np.float64)
    rad = np.zeros(max(n, 1), dtype=np.float64)
    ro = _load().molgen_shell(int(n), int(seed) & (2 ** 64 - 1), float(r_out), float(thickness), int(chain),
                              _ptr(xyz), _ptr(rad))
    if ro < 0:
        raise RuntimeError(f"shell generator failed (n={n}, seed={seed})")
    return Molecule("shell", xyz[:n].copy(), rad[:n].copy(), seed, ro)


def serving_requests(count: int = 4096, seed: int = 0, lo: int = 300, hi: int = 50000, rna_frac: float = 0.3):
    """The request mix of the serving stream: (kind, n_atoms, seed) triples.

    Sizes are log-uniform over [lo, hi]; 70 % globules, 30 % RNA mimics."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.exp(rng.uniform(math.log(lo), math.log(hi), size=count)).astype(np.int64)
    kinds = np.where(rng.uniform(size=count) < rna_frac, "rna", "globule")
    seeds = rng.integers(0, 2 ** 31 - 1, size=count)
    return [(str(k), int(s), int(sd)) for k, s, sd in zip(kinds, sizes, seeds)]


def _cache_dir():
    import tempfile
    return os.environ.get("DSASA_INPUT_CACHE", os.path.join(tempfile.gettempdir(), "dsasa_inputs"))


def make(kind: str, n: int, seed: int, cache: bool = True) -> Molecule:
    """Generate (or load from the on-disk cache, for n >= 10,000) one molecule."""
    gen = {"globule": globule, "rna": rna, "shell": shell}[kind]
    if not cache or n < 10000:
        return gen(n, seed)
    path = os.path.join(_cache_dir(), f"{kind}_{n}_{seed}.npz")
    if os.path.exists(path):
        try:
            d = np.load(path)
            return Molecule(kind, d["coords"], d["radii"], seed, float(d["extent"]))
        except Exception:
            pass
    m = gen(n, seed)
    try:
        os.makedirs(_cache_dir(), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}.npz"
        np.savez(tmp, coords=m.coords, radii=m.radii, extent=m.extent)
        os.replace(tmp, path)
    except OSError:
        pass
    return m


def sphere_points(m: int) -> np.ndarray:
    """m float32 unit vectors on the golden-angle spiral (the point set of the Shrake-Rupley
    cross-check): z_k = 1 - (2k + 1)/m, phi_k = k pi (3 - sqrt 5), computed in float64 and
    rounded once."""
    k = np.arange(m, dtype=np.float64)
    z = 1.0 - (2.0 * k + 1.0) / m
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = k * np.pi * (3.0 - np.sqrt(5.0))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], 1).astype(np.float32)


def poisson_arrivals(count: int, rate_per_s: float, seed: int = 0) -> np.ndarray:
    """Arrival times (s) of a Poisson stream at the given rate."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))
