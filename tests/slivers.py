"""Inputs with sliver atoms (test helper): an atom whose exposed area is driven down to
about 1e-5 A^2, so that its area and its neighbours' gradient entries come from terms that
cancel about a million-fold.  The oracle decides the geometry (bisection on the position of
one neighbour moved towards the atom), so no value here comes from the CUDA path."""
import numpy as np

P = 1.4


def sliver(m, orc, target=1e-5, seed=0, max_tries=40):
    """(coords, radii, i) for molecule m with one atom i of exposed area in
    [target / 2, 2 target]: a small exposed atom, one of its neighbours moved along the line
    to it until the exposed area is that small."""
    xyz, r = m.coords.copy(), m.radii
    a, _, _ = orc.sasa(xyz, r, grad=False)
    R = r + P
    rng = np.random.default_rng(seed)
    cand = np.nonzero((a > 0.05) & (a < 3.0))[0]
    for i in rng.permutation(cand)[:max_tries]:
        d = np.linalg.norm(xyz - xyz[i], axis=1)
        nb = np.nonzero((d < R + R[i]) & (np.arange(len(r)) != i))[0]
        for j in nb[np.argsort(d[nb])]:
            u = (xyz[i] - xyz[j]) / d[j]
            patch = orc.local_patch(xyz, r, [i])
            k_i, k_j = np.searchsorted(patch, i), np.searchsorted(patch, j)
            if patch[k_j] != j:
                continue
            px = xyz[patch].copy()

            def area(t):
                q = px.copy()
                q[k_j] = xyz[j] + t * u
                return orc.sasa(q, r[patch], grad=False)[0][k_i]

            hi = min(d[j] - 0.5, 2.0)
            if area(hi) > 0:
                continue
            lo = 0.0
            for _ in range(60):
                mid = 0.5 * (lo + hi)
                v = area(mid)
                if target / 2 <= v <= 2 * target:
                    out = xyz.copy()
                    out[j] = xyz[j] + mid * u
                    return out, r.copy(), int(i)
                if v > target:
                    lo = mid
                else:
                    hi = mid
    raise RuntimeError("no sliver atom found")
