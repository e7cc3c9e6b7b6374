"""CPU unit tests of the CUDA path's arithmetic header (csrc/dsasa_math.cuh, compiled for
the host by g++): every predicate tier against the oracle's exact rational signs, and the
hand-derived dihedral / triangle-term gradients against the oracle's dual numbers and
finite differences."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "mathcheck.cpp")
HDR = os.path.join(ROOT, "paper_2401_10462_gb300", "csrc", "dsasa_math.cuh")
SO = os.path.join(ROOT, "paper_2401_10462_gb300", "_build", "libmathcheck.so")
P = 1.4


@pytest.fixture(scope="module")
def mc():
    os.makedirs(os.path.dirname(SO), exist_ok=True)
    if not os.path.exists(SO) or os.path.getmtime(SO) < max(os.path.getmtime(SRC), os.path.getmtime(HDR)):
        tmp = SO + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, SRC])
        os.replace(tmp, SO)
    lib = ctypes.CDLL(SO)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.mc_pred.argtypes = [ctypes.c_int, ctypes.c_int, dp]
    lib.mc_xp_len.argtypes = [ctypes.c_int, dp]
    lib.mc_sos_clip.argtypes = [dp, ctypes.POINTER(ctypes.c_int)]
    lib.mc_lens_grad_f32.argtypes = [dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, ctypes.c_int]
    lib.mc_dihedral_grad.argtypes = [dp, dp, ctypes.c_int]
    lib.mc_dihedral_grad.restype = ctypes.c_double
    lib.mc_solid_angle.argtypes = [dp, dp, dp]
    lib.mc_solid_angle.restype = ctypes.c_double
    lib.mc_tri_term_grad.argtypes = [dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, ctypes.c_int]
    lib.mc_tri_term_grad.restype = ctypes.c_double
    lib.mc_tri_term.argtypes = [dp, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    lib.mc_tri_term.restype = ctypes.c_double
    lib.mc_tri_mixed.argtypes = [dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, ctypes.c_int]
    lib.mc_tri_mixed.restype = ctypes.c_double
    lib.mc_tri_ff.argtypes = [dp, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    lib.mc_tri_ff.restype = ctypes.c_double
    lib.mc_ff_op.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
    lib.mc_ff_op.restype = ctypes.c_double
    lib.mc_dihedral_grad_s.argtypes = [dp, ctypes.c_double, dp]
    lib.mc_dihedral_grad_s.restype = ctypes.c_double
    lib.mc_cap64.argtypes = [ctypes.c_double] * 3
    lib.mc_cap64.restype = ctypes.c_double
    return lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _oracle_sign(orc, kind, pts):
    """The oracle's exact answer for the CUDA predicate `kind` on rows pts (row 0 = atom i)."""
    n = len(pts)
    if kind == 0:   # clip: vertex (1,2,3) beyond plane 4 <=> 4 conflicts with tet (0,1,2,3)
        o = orc.predicate(0, pts, [0, 1, 2, 3])
        order = [0, 1, 2, 3] if o > 0 else [0, 2, 1, 3]
        return -orc.predicate(1, pts, order + [4]), o
    if kind == 1:
        return orc.predicate(2, pts, [0, 1, 2, 3]), None
    if kind == 2:
        return orc.predicate(3, pts, [0, 1, 2]), None
    if kind == 3:
        return (1 if orc.predicate(5, pts, [0, 1, 2, 3]) else -1), None
    if kind == 4:
        return orc.predicate(4, pts, [0, 1]), None
    if kind == 5:
        return (1 if orc.predicate(6, pts, [0, 1, 2]) else -1), None
    return (-1 if orc.predicate(7, pts, [0, 1]) else 1), None


def _random_config(rng, kind, near):
    npl = {0: 4, 1: 3, 2: 2, 3: 3, 4: 1, 5: 2, 6: 1}[kind]
    pts = np.zeros((npl + 1, 4))
    pts[:, :3] = rng.normal(scale=2.0, size=(npl + 1, 3)) + np.array([37.1, -12.4, 5.3])
    pts[:, 3] = rng.choice([1.2, 1.52, 1.55, 1.7, 1.8], size=npl + 1) + P
    if near:
        # scale the last radius to bring the predicate near its zero set: bisect on the
        # FP64 value of the defining quantity, the oracle's exact sign deciding
        lo, hi = 0.3, 6.0
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            pts[-1, 3] = mid
            s, _ = _oracle_sign_cache(kind, pts)
            if s > 0:
                hi = mid
            else:
                lo = mid
        pts[-1, 3] = 0.5 * (lo + hi)
    return pts


_ORC = None


def _oracle_sign_cache(kind, pts):
    return _oracle_sign(_ORC, kind, pts)


@pytest.mark.parametrize("kind", range(7))
def test_predicate_tiers_match_exact_oracle(mc, orc, kind):
    global _ORC
    _ORC = orc
    rng = np.random.default_rng(100 + kind)
    decided = [0, 0]
    for t in range(120):
        pts = _random_config(rng, kind, near=(t % 2 == 1))
        ref, o = _oracle_sign(orc, kind, pts)
        if kind == 0 and o == 0:
            continue
        if kind == 0 and o < 0:
            pts = pts[[0, 2, 1, 3, 4]]   # CCW order: D > 0
        sx = mc.mc_pred(kind, 2, _d(pts))
        assert sx != 2, "expansion capacity exceeded"
        assert sx == ref or (ref == 0 and sx == 0) or (kind in (3, 5, 6) and sx <= 0 and ref == -1), (kind, t, sx, ref)
        for tier in (0, 1):
            s = mc.mc_pred(kind, tier, _d(pts))
            if s != 0:
                decided[tier] += 1
                assert s == sx, (kind, tier, t, s, sx)
    assert decided[0] > 30 and decided[1] > 50


def test_exact_tier_on_exact_zero(mc):
    # the bisector passes exactly through p_i when |q|^2 = w_k - w_i (3-4-5 triangle):
    # the filters cannot decide, the exact tier returns 0, as does the oracle's rational
    # evaluation of the same quantity
    pts = np.array([[10.0, -3.0, 2.5, 3.0], [14.0, -3.0, 2.5, 5.0]])
    assert mc.mc_pred(6, 0, _d(pts)) == 0
    assert mc.mc_pred(6, 1, _d(pts)) == 0
    assert mc.mc_pred(6, 2, _d(pts)) == 0


def test_dihedral_gradient_fd(mc):
    rng = np.random.default_rng(0)
    for _ in range(50):
        p = rng.normal(size=(4, 3)) * 2
        g = np.zeros(12)
        th = mc.mc_dihedral_grad(_d(p.reshape(-1)), _d(g), 0)
        g = np.zeros(12)
        buf = np.zeros(12)
        th = mc.mc_dihedral_grad(_d(p.reshape(-1)), buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0)
        h = 1e-6
        for k in range(12):
            pp = p.reshape(-1).copy(); pp[k] += h
            pm = p.reshape(-1).copy(); pm[k] -= h
            d = (mc.mc_dihedral_grad(_d(pp), _d(np.zeros(12)), 0) - mc.mc_dihedral_grad(_d(pm), _d(np.zeros(12)), 0)) / (2 * h)
            assert abs(d - buf[k]) < 1e-6 * max(1, abs(d)), (k, d, buf[k])


def test_solid_angle_matches_excess(mc):
    rng = np.random.default_rng(1)
    for _ in range(50):
        p = rng.normal(size=(4, 3))
        om = mc.mc_solid_angle(_d(p[1] - p[0]), _d(p[2] - p[0]), _d(p[3] - p[0]))
        th = [mc.mc_dihedral_grad(_d(np.stack([p[0], p[a], p[b], p[c]]).reshape(-1)), _d(np.zeros(12)), 0)
              for a, b, c in ((1, 2, 3), (2, 1, 3), (3, 1, 2))]
        assert om == pytest.approx((sum(th) - np.pi) / (4 * np.pi), abs=1e-12)


def test_triangle_term_and_gradient_vs_oracle(mc, orc):
    rng = np.random.default_rng(2)
    n = 0
    while n < 40:
        p = rng.normal(scale=1.8, size=(3, 3))
        R = rng.choice([2.6, 2.92, 2.95, 3.1, 3.2], size=3)
        S_ref, g_ref = orc.tri_term(p[0], p[1], p[2], *R)
        if S_ref is None:
            continue
        n += 1
        g = np.zeros(9)
        gp = g.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        S = mc.mc_tri_term_grad(_d(p.reshape(-1)), *R, gp, 0)
        assert S == pytest.approx(S_ref, rel=1e-9, abs=1e-9)
        assert np.allclose(g.reshape(3, 3), g_ref, rtol=1e-7, atol=1e-8)
        assert mc.mc_tri_term(_d(p.reshape(-1)), *R) == pytest.approx(S_ref, rel=1e-9, abs=1e-9)
        g32 = np.zeros(9)
        S32 = mc.mc_tri_term_grad(_d(p.reshape(-1)), *R, g32.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1)
        assert abs(S32 - S_ref) < 2e-4 * max(1.0, abs(S_ref))
        assert np.abs(g32.reshape(3, 3) - g_ref).max() < 2e-3 * max(1.0, np.abs(g_ref).max())


def test_lens_form_and_closed_gradient_vs_oracle(mc, orc):
    """The triangle term evaluated as in the kernel (FP64 combination of the paper's
    Eq. trianglev) and its closed-form boundary-variation gradient, against the oracle's
    dual-number derivative of Eq. (trianglev)."""
    rng = np.random.default_rng(5)
    n = 0
    while n < 300:
        p = rng.normal(scale=1.8, size=(3, 3))
        R = rng.choice([2.6, 2.92, 2.95, 3.1, 3.2, 3.3], size=3)
        S_ref, g_ref = orc.tri_term(p[0], p[1], p[2], *R)
        if S_ref is None:
            continue
        n += 1
        q = np.concatenate([p[1] - p[0], p[2] - p[0]])
        g = np.zeros(9)
        S = mc.mc_tri_mixed(_d(q), *R, g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0)
        assert S == pytest.approx(S_ref, rel=1e-10, abs=1e-10)
        assert np.allclose(g.reshape(3, 3), g_ref, rtol=1e-8, atol=1e-9)
        g32 = np.zeros(9)
        S32 = mc.mc_tri_mixed(_d(q), *R, g32.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1)
        assert abs(S32 - S_ref) < 1e-4
        assert np.abs(g32.reshape(3, 3) - g_ref).max() < 1e-3 * max(1.0, np.abs(g_ref).max())


def test_float_float_primitives(mc):
    """Two-sum / FMA two-product float-float arithmetic: about 2^-44 relative against double."""
    rng = np.random.default_rng(8)
    for _ in range(2000):
        a, b = rng.uniform(-10, 10, 2) * 10.0 ** rng.integers(-3, 3, 2)
        for op, ref in ((0, a + b), (1, a - b), (2, a * b)):
            r = mc.mc_ff_op(op, a, b)
            scale = abs(a) + abs(b) if op < 2 else abs(a * b)
            assert abs(r - ref) <= 2.0 ** -44 * scale, (op, a, b, r, ref)
        bf = float(np.float32(b))
        assert abs(mc.mc_ff_op(3, a, bf) - a * bf) <= 2.0 ** -44 * abs(a * bf)


def test_triangle_term_float_float(mc, orc):
    """The float-float form of Eq. (trianglev) of the mixed kernel against the oracle: the
    radius quantities carry no float rounding, so the error is that of the float geometry."""
    rng = np.random.default_rng(9)
    n, errs = 0, []
    while n < 300:
        p = rng.normal(scale=1.8, size=(3, 3))
        R = rng.choice([2.6, 2.92, 2.95, 3.1, 3.2, 3.3], size=3)
        S_ref, _ = orc.tri_term(p[0], p[1], p[2], *R)
        if S_ref is None:
            continue
        n += 1
        q = np.concatenate([p[1] - p[0], p[2] - p[0]])
        S = mc.mc_tri_ff(_d(q), *R)
        errs.append(S - S_ref)
        assert abs(S - S_ref) < 1e-4
    # no bias beyond the float geometry's scatter
    errs = np.array(errs)
    assert abs(errs.mean()) < 4 * errs.std() / np.sqrt(len(errs)) + 1e-7


def test_signed_dihedral_gradient_and_cap(mc):
    rng = np.random.default_rng(6)
    for _ in range(50):
        p = rng.normal(size=(4, 3)) * 2
        v6 = np.dot(p[1] - p[0], np.cross(p[2] - p[0], p[3] - p[0]))
        ref = np.zeros(12)
        mc.mc_dihedral_grad(_d(p.reshape(-1)), ref.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0)
        g = np.zeros(12)
        mc.mc_dihedral_grad_s(_d(p.reshape(-1)), float(np.sign(v6)), g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        assert np.allclose(g, ref, rtol=1e-12, atol=1e-12)
    for d, R1, R2 in ((4.0, 3.1, 2.6), (0.7, 3.2, 2.6), (5.6, 2.9, 3.0)):
        t = (d * d + R1 * R1 - R2 * R2) / (2 * d)
        assert mc.mc_cap64(d, R1, R2) == pytest.approx(2 * np.pi * R1 * (R1 - t), rel=1e-13)


def test_clip_ties_broken_as_the_oracle_breaks_them(mc, orc):
    """A cell vertex exactly on a bisector (lattice atoms: the vertex of the three axis
    neighbours lies on the bisector of the body- and face-diagonal ones) is decided by the
    device's Simulation of Simplicity exactly as the oracle's power test decides the same
    tie, for every assignment of atom indices (which decides the perturbation's order)."""
    import itertools
    base = np.array([[0.0, 0.0, 0.0], [2.5, 0.0, 0.0], [0.0, 2.5, 0.0], [0.0, 0.0, 2.5]])
    shifts = (np.array([10.0, -3.0, 7.5]), np.array([-41.5, 12.25, 0.5]))
    ties = 0
    for m in ([2.5, 2.5, 2.5], [2.5, 2.5, 0.0], [0.0, 2.5, 2.5]):
        for radii in ((1.5, 1.5, 1.5, 1.5, 1.5), (1.2, 1.2, 1.2, 1.2, 1.2)):
            for sh in shifts:
                rows = np.zeros((5, 4))
                rows[:4, :3] = base + sh
                rows[4, :3] = np.array(m) + sh
                rows[:, 3] = np.array(radii) + P
                for perm in itertools.permutations(range(5)):
                    g = np.array(perm, dtype=np.int32)          # global index of row k is perm[k]
                    got = mc.mc_sos_clip(_d(rows), g.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
                    assert abs(got) == 10, got                  # an exact tie, broken by the perturbation
                    pts = np.zeros((5, 4))
                    pts[g] = rows                                # the oracle's point k has index k
                    ref = orc.predicate(1, pts, [int(x) for x in g])   # -1: conflict (clipped)
                    assert (got > 0) == (ref == -1), (m, radii, perm, got, ref)
                    ties += 1
    assert ties == 3 * 2 * 2 * 120


def test_lens_gradient_of_near_degenerate_triangles(mc, orc, gen):
    """The float lens gradient of a triangle whose triple points are about to merge (height
    s_t over the plane of the centres small) loses accuracy as 2^-24 R^2 / s_t; with s_t^2 taken
    from the float64 coordinates below 0.01 R^2 (the kernels' rule) every triangle of the
    5,000-atom globule stays within 1e-4 of the float64 gradient, which the plain float
    evaluation misses."""
    m = gen.globule(5000, 2)
    R = m.radii + P
    tris = orc.Oracle(m.coords, m.radii).simplices(2)
    worst_plain = worst_fixed = 0.0
    for t in tris:
        for own in t:
            a, b = [x for x in t if x != own]
            q6 = np.concatenate([m.coords[a] - m.coords[own], m.coords[b] - m.coords[own]])
            q2, q3 = q6[:3], q6[3:]
            # only the near-degenerate ones (the float64 height below R / 3) are of interest
            d2, d3 = np.linalg.norm(q2), np.linalg.norm(q3)
            cr = np.cross(q2, q3)
            b2 = (d2 * d2 - R[a] ** 2 + R[own] ** 2) / 2
            b3 = (d3 * d3 - R[b] ** 2 + R[own] ** 2) / 2
            z = (np.cross(q3, cr) * b2 + np.cross(cr, q2) * b3) / (cr @ cr)
            if R[own] ** 2 - z @ z > R[own] ** 2 / 9:
                continue
            g64, gp, gf = np.zeros(9), np.zeros(9), np.zeros(9)
            mc.mc_tri_mixed(_d(q6), R[own], R[a], R[b], _d(g64), 0)
            mc.mc_lens_grad_f32(_d(q6), R[own], R[a], R[b], _d(gp), 0)
            mc.mc_lens_grad_f32(_d(q6), R[own], R[a], R[b], _d(gf), 1)
            worst_plain = max(worst_plain, np.abs(gp - g64).max())
            worst_fixed = max(worst_fixed, np.abs(gf - g64).max())
    assert worst_fixed < 1e-4 < worst_plain, (worst_fixed, worst_plain)
