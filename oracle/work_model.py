"""Algorithmic work of the hot path on one workload, counted by the oracle.

TEST AND MEASUREMENT INFRASTRUCTURE: run by hand to write the work-model record that
bench.py divides by its kernel times (python -m oracle.work_model); it calls the oracle only.

The model (one certification per star tetrahedron, plus the cost of every term of
Eq. (sainexclu) over the boundary of the dual complex, the gradient three times the forward
terms) prices each item by the operations its formula needs, counted from the formulas:

  certification of a tetrahedron (i, a, b, c) of atom i's star: its orientation determinant
      (about 20 flop) and the power test of the opposite atom across each of its 4 faces
      (about 125 flop each): 520 flop
  solid angle omega (Eq. vertex, Van Oosterom-Strackee form): 40 flop, atan2 + 3 sqrt
  dihedral angle phi with its cap factor (Eqs. phiedge, edge): 35 + 15 flop, atan2 + 2 rsqrt
      + sqrt + division
  edge cap 2 pi R h (Eq. edge): 15 flop, sqrt + division
  triangle term S_ijk^(i) (Eq. trianglev: triple point, two dihedrals, one solid angle):
      180 flop, 4 special functions
  vertex constant 4 pi R^2: 3 flop

The counts (star tetrahedra from the triangulation, terms from the area computation) are
per atom of the workload; special-function operations are counted apart from flop.
"""
from __future__ import annotations

import json
import os
import sys

FLOP = {"certification": 520.0, "vertex_constants": 3.0, "solid_angles": 40.0, "dihedrals": 50.0,
        "edge_caps": 15.0, "triangles": 180.0}
SFU = {"certification": 0.0, "vertex_constants": 0.0, "solid_angles": 4.0, "dihedrals": 5.0,
       "edge_caps": 2.0, "triangles": 4.0}
GRAD_FACTOR = 3.0   # backward of every term, relative to its forward cost


def model(coords, radii, probe: float = 1.4) -> dict:
    from oracle import oracle
    o = oracle.Oracle(coords, radii, probe)
    n = o.n
    c = o.counts()
    t = o.term_counts()
    star = 4.0 * c["rt_tets"] / n          # tetrahedra of the triangulation around each atom
    per = {k: v / n for k, v in t.items()}
    fwd = sum(FLOP[k] * per[k] for k in per)
    fwd_sfu = sum(SFU[k] * per[k] for k in per)
    return {
        "n_atoms": n,
        "star_tets_per_atom": star,
        "terms_per_atom": per,
        "flop_table": FLOP, "sfu_table": SFU, "grad_factor": GRAD_FACTOR,
        "cell_flop_per_atom": FLOP["certification"] * star,
        "terms_flop_per_atom": fwd * (1.0 + GRAD_FACTOR),
        "terms_sfu_per_atom": fwd_sfu * (1.0 + GRAD_FACTOR),
        "dual_complex": {k: c[k] for k in ("K0", "K1", "K2", "K3")},
    }


def main():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from paper_2401_10462_gb300 import inputs
    m = inputs.globule(5000, 0)
    out = {"workload": "globule-5000, seed 0, probe 1.4 A", **model(m.coords, m.radii),
           "written_by": "python -m oracle.work_model (oracle counts only)"}
    path = os.path.join(root, "profiles", "work_model_globule5000.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
