"""Shrake-Rupley numerical SASA, plain numpy: the oracle of the GPU cross-check.

TEST INFRASTRUCTURE ONLY (tests/ and bench.py's CPU legs import it).

Definition (Shrake & Rupley 1973; the numerical comparator of the paper's accuracy study,
Sec. "Accuracy"): m sample points are placed on each probe-inflated sphere,
x_k = p_i + R_i s_k with R_i = fl64(r_i + probe) and s_k the given (float32) unit vectors
taken as exact numbers; a point is exposed when it lies strictly outside every other ball,
|x_k - p_j|^2 > R_j^2 for all j != i; the area of atom i is 4 pi R_i^2 (exposed points) / m.

Every decision is taken on the real numbers: the margin |x_k - p_j|^2 - R_j^2 is evaluated
in float64, and where its magnitude is below the float64 evaluation error (a near-tie) it
is evaluated again exactly in rational arithmetic.  Only balls with |p_i - p_j| <= R_i + R_j
can hold a point of sphere i, so only those are tested.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

# the point set is an input of the method (shared with the GPU path by the input module)
from paper_2401_10462_gb300.inputs import sphere_points  # noqa: F401

PROBE = 1.4


def neighbours(coords, R, i: int) -> np.ndarray:
    """Indices j != i whose balls can hold a point of sphere i (|p_i - p_j| <= R_i + R_j)."""
    d2 = ((coords - coords[i]) ** 2).sum(1)
    ok = d2 <= (R + R[i]) ** 2 * (1.0 + 1e-12)
    ok[i] = False
    return np.nonzero(ok)[0]


def point_margins(coords, radii, points, i: int, probe: float = PROBE):
    """For atom i: (nb, D, margin) with nb its neighbour indices (k,), D[k_pt, j] the vector
    x_k - p_j (m, k, 3) and margin[k_pt, j] = |x_k - p_j|^2 - R_j^2 (m, k), all in float64.
    Their float64 error is below 1e-13 of (|D|^2 + R_j^2)."""
    xyz = np.asarray(coords, dtype=np.float64)
    R = np.asarray(radii, dtype=np.float64) + probe
    s = np.asarray(points, dtype=np.float32).astype(np.float64)
    nb = neighbours(xyz, R, i)
    x = R[i] * s                                       # (m, 3), relative to p_i
    Q = xyz[nb] - xyz[i]                               # (k, 3)
    D = x[:, None, :] - Q[None, :, :]
    margin = (D * D).sum(-1) - R[nb][None, :] ** 2
    return nb, D, margin


def _exact_margin_sign(p_i, p_j, r_i, r_j, s, probe) -> int:
    """Sign of |p_i + R_i s - p_j|^2 - R_j^2 in rational arithmetic (R = fl64(r + probe))."""
    Ri, Rj = Fraction(float(r_i + probe)), Fraction(float(r_j + probe))
    acc = Fraction(0)
    for c in range(3):
        d = Fraction(float(p_i[c])) + Ri * Fraction(float(s[c])) - Fraction(float(p_j[c]))
        acc += d * d
    v = acc - Rj * Rj
    return (v > 0) - (v < 0)


def exposed_mask(coords, radii, points, i: int, probe: float = PROBE) -> np.ndarray:
    """Exposed sample points of atom i (bool, m) by the definition."""
    xyz = np.asarray(coords, dtype=np.float64)
    r = np.asarray(radii, dtype=np.float64)
    s = np.asarray(points, dtype=np.float32)
    nb, D, margin = point_margins(xyz, r, s, i, probe)
    if len(nb) == 0:
        return np.ones(len(s), dtype=bool)
    scale = (D * D).sum(-1) + (r[nb] + probe)[None, :] ** 2
    sign = np.sign(margin)
    near = np.abs(margin) <= 1e-13 * scale
    for kp, kj in zip(*np.nonzero(near)):
        j = nb[kj]
        sign[kp, kj] = _exact_margin_sign(xyz[i], xyz[j], r[i], r[j], s[kp], probe)
    return (sign > 0).all(1)


def exposed_counts(coords, radii, points, probe: float = PROBE) -> np.ndarray:
    """Number of exposed points of every atom (int64[n]) by the definition."""
    n = len(radii)
    return np.array([int(exposed_mask(coords, radii, points, i, probe).sum()) for i in range(n)], dtype=np.int64)


def areas(coords, radii, m: int = 960, probe: float = PROBE) -> np.ndarray:
    pts = sphere_points(m)
    R = np.asarray(radii, dtype=np.float64) + probe
    return 4.0 * np.pi * R * R * exposed_counts(coords, radii, pts, probe) / m
