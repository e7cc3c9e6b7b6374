"""Shrake-Rupley numerical SASA, plain numpy: the oracle of the GPU cross-check.

TEST INFRASTRUCTURE ONLY (tests/ and bench.py's CPU legs import it).

Definition (Shrake & Rupley 1973; the numerical comparator the paper's accuracy study
uses, Sec. "Accuracy"): m points are placed on each probe-inflated sphere; a point is
exposed when it lies strictly outside every other ball that overlaps the sphere; the area
of atom i is 4 pi R_i^2 (exposed points) / m.

The decision for each point is taken in float32 with the arithmetic the GPU kernel uses,
so that the exposed counts can be compared exactly:
    x = R_i * s_k                       (R_i = float32(r_i + probe), s_k float32 unit vectors)
    q = float32(p_j - p_i)              (difference in float64, then rounded)
    d = x - q;  d2 = (d_x d_x + d_y d_y) + d_z d_z    (each operation rounded to float32)
    covered by j  <=>  d2 <= float32(R_j) * float32(R_j)
The overlapping neighbours are those with |p_i - p_j|^2 < (R_i + R_j)^2 in float64.
"""
from __future__ import annotations

import numpy as np

# the point set is an input of the method (shared with the GPU path by the input module)
from paper_2401_10462_gb300.inputs import sphere_points  # noqa: F401

PROBE = 1.4


def exposed_counts(coords, radii, points, probe: float = PROBE) -> np.ndarray:
    """Number of exposed points of every atom (int64[n])."""
    xyz = np.asarray(coords, dtype=np.float64)
    R = np.asarray(radii, dtype=np.float64) + probe
    Rf = R.astype(np.float32)
    R2f = Rf * Rf
    pts = np.asarray(points, dtype=np.float32)
    n = len(R)
    out = np.zeros(n, dtype=np.int64)
    for i in range(n):
        dd = ((xyz - xyz[i]) ** 2).sum(1)
        nb = np.nonzero((dd < (R + R[i]) ** 2) & (np.arange(n) != i))[0]
        x = pts * Rf[i]                                   # (m, 3) float32
        if len(nb) == 0:
            out[i] = len(pts)
            continue
        q = (xyz[nb] - xyz[i]).astype(np.float32)         # (k, 3)
        d = x[:, None, :] - q[None, :, :]                 # float32
        d2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
        covered = (d2 <= R2f[nb][None, :]).any(1)
        out[i] = int((~covered).sum())
    return out


def areas(coords, radii, m: int = 960, probe: float = PROBE) -> np.ndarray:
    pts = sphere_points(m)
    R = np.asarray(radii, dtype=np.float64) + probe
    return 4.0 * np.pi * R * R * exposed_counts(coords, radii, pts, probe) / m
