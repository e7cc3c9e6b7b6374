// Device (and host-compilable) arithmetic of the dSASA hot path.
//
//  1. Filtered exact predicates.  Every combinatorial decision of the method (which
//     Laguerre-cell vertices exist = which tetrahedra the weighted Delaunay tetrahedrization
//     has, Step 1; which simplices belong to the dual complex C, Step 2) is the sign of a
//     polynomial in the input doubles.  It is evaluated in three tiers:
//       FP32 with a certified error bound  ->  FP64 with a certified error bound  ->
//       exact floating-point expansions (Shewchuk 1997, "Adaptive precision floating-point
//       arithmetic and fast robust geometric predicates": Two-Sum, Two-Product, Grow-,
//       Scale-Expansion and Compress, written from that paper's descriptions).
//     The bound: if every input x~ satisfies |x~ - x| <= u * xbar with xbar >= |x~|, an
//     evaluation whose longest path has `deg` input factors and `depth` roundings errs by at
//     most ((1+u)^(deg+depth) - 1) * Pbar, where Pbar is the same polynomial evaluated on
//     the magnitudes xbar with every sign made positive.  FA<T> carries (value, Pbar).
//  2. The geometric terms of Eqs. (vertex), (phiedge), (edge), (trianglev) and their
//     hand-derived gradients (Eqs. inexclu, triangle), templated on float / double.
//
// Local frame: everything about atom i is expressed relative to its centre p_i.  The power
// bisector of i and a neighbour k is the plane {z : q_k . z = b_k} with
//     q_k = p_k - p_i,   b_k = (|q_k|^2 - w_k + w_i) / 2,   w = R^2,
// and the Laguerre cell L_i is the intersection of the half-spaces q_k . z <= b_k.
#pragma once
#include <math.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define DS_HD __host__ __device__ __forceinline__
#define DS_HDNI __host__ __device__ __noinline__ static
#define DS_HDC __host__ __device__ __noinline__
#else
#define DS_HD inline
#define DS_HDNI static
#define DS_HDC inline
#endif

namespace dsasa {

// ------------------------------------------------------------------ rounding primitives
DS_HD double add_rn(double a, double b) {
#if defined(__CUDA_ARCH__)
    return __dadd_rn(a, b);
#else
    return a + b;
#endif
}
DS_HD double mul_rn(double a, double b) {
#if defined(__CUDA_ARCH__)
    return __dmul_rn(a, b);
#else
    return a * b;
#endif
}
DS_HD double fma_rn(double a, double b, double c) {
#if defined(__CUDA_ARCH__)
    return __fma_rn(a, b, c);
#else
    return fma(a, b, c);
#endif
}
// x + y == a + b exactly, x = fl(a + b)
DS_HD void two_sum(double a, double b, double& x, double& y) {
    x = add_rn(a, b);
    double bv = add_rn(x, -a);
    double av = add_rn(x, -bv);
    y = add_rn(add_rn(a, -av), add_rn(b, -bv));
}
// x + y == a * b exactly, x = fl(a * b)
DS_HD void two_prod(double a, double b, double& x, double& y) {
    x = mul_rn(a, b);
    y = fma_rn(a, b, -x);
}

// ------------------------------------------------------------------ filter numbers
template <class T> struct FA { T v, a; };
template <class T> DS_HD FA<T> operator+(const FA<T>& x, const FA<T>& y) { return {x.v + y.v, x.a + y.a}; }
template <class T> DS_HD FA<T> operator-(const FA<T>& x, const FA<T>& y) { return {x.v - y.v, x.a + y.a}; }
template <class T> DS_HD FA<T> operator*(const FA<T>& x, const FA<T>& y) { return {x.v * y.v, x.a * y.a}; }

// certified sign (+1/-1) or 0 when the bound does not decide
template <class T> DS_HD int fa_sign(const FA<T>& x, T gamma, T tiny) {
    if (!(x.a > tiny)) return 0;
    T lim = gamma * x.a;
    return x.v > lim ? 1 : (x.v < -lim ? -1 : 0);
}
// u = 2^-24 (float), 2^-53 (double).  gamma = 32u covers deg + depth <= 24 with slack;
// the cached clip test (deg 4, depth 9) uses 16u.
constexpr float G32 = 1.9073486328125e-06f;    // 2^-19
constexpr float G32_CLIP = 9.5367431640625e-07f;  // 2^-20
constexpr double G64 = 3.552713678800501e-15;  // 2^-48
constexpr float TINY32 = 1e-30f;
constexpr double TINY64 = 1e-280;

// ------------------------------------------------------------------ expansions
#ifndef DS_XP_N
#define DS_XP_N 32
#endif
// nonoverlapping, increasing magnitude, no zero components; ovf set when a result would
// not fit (the value is then unreliable and the caller reports DSASA_ERR_UNRESOLVED)
struct XP {
    int n;
    int ovf;
    double c[DS_XP_N];
};
DS_HD XP xp_zero() { XP r; r.n = 0; r.ovf = 0; return r; }
DS_HD XP xp_of(double d) { XP r; r.n = 0; r.ovf = 0; if (d != 0.0) { r.c[0] = d; r.n = 1; } return r; }
DS_HD void xp_push(XP& r, double v) {
    if (v == 0.0) return;
    if (r.n < DS_XP_N) r.c[r.n++] = v; else r.ovf = 1;
}
// e <- e + b (Grow-Expansion, zero elimination, in place)
DS_HDNI void xp_compress(XP& e);
DS_HDNI void xp_grow(XP& e, double b) {
    if (e.n >= DS_XP_N) xp_compress(e);   // make room (same value, fewer components)
    double Q = b;
    int m = 0;
    for (int i = 0; i < e.n; ++i) {
        double x, y;
        two_sum(Q, e.c[i], x, y);
        Q = x;
        if (y != 0.0) e.c[m++] = y;
    }
    e.n = m;
    xp_push(e, Q);
}
DS_HDNI void xp_add_to(XP& r, const XP& t) {
    r.ovf |= t.ovf;
    for (int j = 0; j < t.n; ++j) xp_grow(r, t.c[j]);
}
// out <- e * b (Scale-Expansion)
DS_HDNI void xp_scale(const XP& e, double b, XP& out) {
    out.n = 0;
    out.ovf = e.ovf;
    if (e.n == 0 || b == 0.0) return;
    double Q, h;
    two_prod(e.c[0], b, Q, h);
    xp_push(out, h);
    for (int i = 1; i < e.n; ++i) {
        double T, t, Q2;
        two_prod(e.c[i], b, T, t);
        two_sum(Q, t, Q2, h);
        xp_push(out, h);
        two_sum(T, Q2, Q, h);
        xp_push(out, h);
    }
    xp_push(out, Q);
}
// Compress: same value, fewer components
DS_HDNI void xp_compress(XP& e) {
    if (e.n <= 1) return;
    double g[DS_XP_N];
    int bottom = e.n - 1;
    double Q = e.c[e.n - 1];
    for (int i = e.n - 2; i >= 0; --i) {
        double x, q;
        two_sum(Q, e.c[i], x, q);
        if (q != 0.0) { g[bottom--] = x; Q = q; } else Q = x;
    }
    g[bottom] = Q;
    int top = 0;
    for (int i = bottom + 1; i < e.n; ++i) {
        double x, q;
        two_sum(g[i], Q, x, q);
        if (q != 0.0) e.c[top++] = q;
        Q = x;
    }
    if (Q != 0.0) e.c[top++] = Q;
    e.n = top;
}
DS_HDNI void xp_sum(const XP& a, const XP& b, double sb, XP& r) {   // r = a + sb * b, sb = +-1
    r = a;
    r.ovf |= b.ovf;
    for (int j = 0; j < b.n; ++j) xp_grow(r, sb * b.c[j]);
    xp_compress(r);
}
DS_HDNI void xp_prod(const XP& a, const XP& b, XP& r) {
    // scale the longer operand by each component of the shorter one
    const XP& L = a.n >= b.n ? a : b;
    const XP& Sh = a.n >= b.n ? b : a;
    r.n = 0;
    r.ovf = a.ovf | b.ovf;
    XP t;
    for (int j = 0; j < Sh.n; ++j) {
        xp_scale(L, Sh.c[j], t);
        xp_add_to(r, t);
        xp_compress(r);
    }
}
DS_HD XP operator+(const XP& a, const XP& b) { XP r; xp_sum(a, b, 1.0, r); return r; }
DS_HD XP operator-(const XP& a, const XP& b) { XP r; xp_sum(a, b, -1.0, r); return r; }
DS_HD XP operator-(const XP& a) {
    XP r = a;
    for (int i = 0; i < r.n; ++i) r.c[i] = -r.c[i];
    return r;
}
DS_HD XP operator*(const XP& a, const XP& b) { XP r; xp_prod(a, b, r); return r; }
DS_HD XP xp_half(const XP& a) {
    XP r = a;
    for (int i = 0; i < r.n; ++i) r.c[i] *= 0.5;
    return r;
}
DS_HD int xp_sign(const XP& a) { return a.n == 0 ? 0 : (a.c[a.n - 1] > 0 ? 1 : -1); }
DS_HD XP xp_diff(double a, double b) {   // a - b exactly
    double x, y;
    two_sum(a, -b, x, y);
    XP r = xp_zero();
    xp_push(r, y);
    xp_push(r, x);
    return r;
}
DS_HD XP xp_sq(double a) {   // a^2 exactly
    double x, y;
    two_prod(a, a, x, y);
    XP r = xp_zero();
    xp_push(r, y);
    xp_push(r, x);
    return r;
}

// ------------------------------------------------------------------ generic vectors
template <class N> struct V3 { N x, y, z; };
template <class N> DS_HD V3<N> vcross(const V3<N>& a, const V3<N>& b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class N> DS_HD N vdot(const V3<N>& a, const V3<N>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class N> DS_HD V3<N> vmul(const V3<N>& a, const N& s) { return {a.x * s, a.y * s, a.z * s}; }
template <class N> DS_HD V3<N> vadd(const V3<N>& a, const V3<N>& b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }

// a bisector plane {z : q . z = b} in a generic number type
template <class N> struct PlaneN { V3<N> q; N b; };

// ------------------------------------------------------------------ generic predicates
// Cell vertex of planes (A, B, C) in homogeneous form: z = Dv / D (Cramer's rule on
// q_A . z = b_A, q_B . z = b_B, q_C . z = b_C).  D > 0 when (A, B, C) is ordered
// counter-clockwise seen from outside the cell.
template <class N> DS_HD void vertex_hom(const PlaneN<N>& A, const PlaneN<N>& B, const PlaneN<N>& C, V3<N>& Dv, N& D) {
    V3<N> xbc = vcross(B.q, C.q), xca = vcross(C.q, A.q), xab = vcross(A.q, B.q);
    Dv = vadd(vadd(vmul(xbc, A.b), vmul(xca, B.b)), vmul(xab, C.b));
    D = vdot(A.q, xbc);
}
// > 0 : the vertex (A,B,C) lies strictly beyond plane M (pow_M < pow_i there): clipped
template <class N> DS_HD N pred_clip(const PlaneN<N>& A, const PlaneN<N>& B, const PlaneN<N>& C, const PlaneN<N>& M) {
    V3<N> Dv; N D;
    vertex_hom(A, B, C, Dv, D);
    return vdot(M.q, Dv) - M.b * D;
}
// <= 0 : the tetrahedron (i,A,B,C) is in C (orthosphere power psi <= 0): |Dv|^2 - w_i D^2
template <class N> DS_HD N pred_tet_psi(const PlaneN<N>& A, const PlaneN<N>& B, const PlaneN<N>& C, const N& wi) {
    V3<N> Dv; N D;
    vertex_hom(A, B, C, Dv, D);
    return vdot(Dv, Dv) - wi * D * D;
}
// orthocentre of the triangle (i,A,B) in its plane: z = Z / W
template <class N> DS_HD void tri_hom(const PlaneN<N>& A, const PlaneN<N>& B, V3<N>& Z, N& W) {
    V3<N> nn = vcross(A.q, B.q);
    Z = vadd(vmul(vcross(B.q, nn), A.b), vmul(vcross(nn, A.q), B.b));
    W = vdot(nn, nn);
}
// <= 0 : psi of the triangle (i,A,B) is non-positive
template <class N> DS_HD N pred_tri_psi(const PlaneN<N>& A, const PlaneN<N>& B, const N& wi) {
    V3<N> Z; N W;
    tri_hom(A, B, Z, W);
    return vdot(Z, Z) - wi * W * W;
}
// > 0 : the triangle's orthocentre lies strictly beyond plane L (L attaches the triangle)
template <class N> DS_HD N pred_tri_beyond(const PlaneN<N>& A, const PlaneN<N>& B, const PlaneN<N>& L) {
    V3<N> Z; N W;
    tri_hom(A, B, Z, W);
    return vdot(L.q, Z) - L.b * W;
}
// <= 0 : psi of the edge (i,A) non-positive (the balls overlap or touch)
template <class N> DS_HD N pred_edge_psi(const PlaneN<N>& A, const N& wi) {
    return A.b * A.b - wi * vdot(A.q, A.q);
}
// > 0 : the edge's orthocentre z = (b_A / |q_A|^2) q_A lies strictly beyond plane K
template <class N> DS_HD N pred_edge_beyond(const PlaneN<N>& A, const PlaneN<N>& K) {
    return A.b * vdot(K.q, A.q) - K.b * vdot(A.q, A.q);
}

// ------------------------------------------------------------------ plane construction
// Ghost planes bound the initial cell: a cube of half-width h around p_i, h >= R_i * 1.0625
// with at most 24 significant bits so that 2h and 2h^2 are exact doubles (and 2h an exact
// float).  Ghost g in 0..5: +x, -x, +y, -y, +z, -z.
DS_HD double ghost_h(double Ri) {
    double h = Ri * 1.0625 + 0.0625;
    return ceil(h * 1048576.0) / 1048576.0;   // multiple of 2^-20 (< 2^4): <= 24 bits
}
DS_HD void ghost_plane64(int g, double h, double q[3], double& b) {
    q[0] = q[1] = q[2] = 0.0;
    q[g >> 1] = (g & 1) ? -2.0 * h : 2.0 * h;
    b = 2.0 * h * h;
}
// FP64 plane of atom k relative to atom i with its filter magnitudes
DS_HD void plane64(const double pi[3], double Ri, const double pk[3], double Rk, double q[3], double& b, double& babs) {
    q[0] = pk[0] - pi[0];
    q[1] = pk[1] - pi[1];
    q[2] = pk[2] - pi[2];
    double s = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
    double wk = Rk * Rk, wi = Ri * Ri;
    b = 0.5 * ((s - wk) + wi);
    babs = 0.5 * ((s + wk) + wi);
}
DS_HD PlaneN<FA<double>> fa_plane64(const double q[3], double b, double babs, bool exact) {
    PlaneN<FA<double>> P;
    P.q = {{q[0], fabs(q[0])}, {q[1], fabs(q[1])}, {q[2], fabs(q[2])}};
    P.b = {b, exact ? fabs(b) : 8.0 * babs};
    return P;
}
// exact plane of atom k relative to atom i
DS_HD PlaneN<XP> xp_plane(const double pi[3], double Ri, const double pk[3], double Rk) {
    PlaneN<XP> P;
    P.q.x = xp_diff(pk[0], pi[0]);
    P.q.y = xp_diff(pk[1], pi[1]);
    P.q.z = xp_diff(pk[2], pi[2]);
    XP s = P.q.x * P.q.x + P.q.y * P.q.y + P.q.z * P.q.z;
    P.b = xp_half(s - xp_sq(Rk) + xp_sq(Ri));
    return P;
}
DS_HD PlaneN<XP> xp_ghost(int g, double h) {
    double q[3], b;
    ghost_plane64(g, h, q, b);
    PlaneN<XP> P;
    P.q = {xp_of(q[0]), xp_of(q[1]), xp_of(q[2])};
    P.b = xp_of(b);
    return P;
}

// ------------------------------------------------------------------ Simulation of Simplicity
// Ties of the clip test are broken as the regular triangulation breaks ties of its power
// test (Edelsbrunner & Muecke 1990): every atom weight is perturbed, w_k -> w_k + delta_k,
// with infinitesimal delta_k and the delta of a lower atom index dominating every delta of a
// higher one.  With w_i -> w_i + delta_i for the centre atom, an atom plane moves by
// b_k -> b_k + (delta_i - delta_k) / 2; a ghost plane of the initial cube does not move.  The
// clip value P = q_M . Dv - b_M D of vertex (A, B, C) against plane M is linear in the b's:
//     dP/db_A = q_M . (q_B x q_C),  dP/db_B = q_M . (q_C x q_A),  dP/db_C = q_M . (q_A x q_B),
//     dP/db_M = -D,
// so the perturbed sign of an exact zero is the sign of the coefficient of the lowest-indexed
// atom whose coefficient is not zero: -dP/db_k / 2 for a plane atom k, and the sum of the
// atom planes' dP/db_k / 2 for the centre atom i.  (P = -F/2 of the conflict determinant F of
// the tetrahedron (i, A, B, C) against M, so this is the perturbation of that test.)  g[] holds
// the global indices of A, B, C, M (negative for ghost planes) and gi that of atom i.  Returns
// +1 (the vertex is beyond M: clipped) or -1; 0 only if every coefficient vanishes, which
// needs coincident atoms.
DS_HD int sos_clip_sign(const PlaneN<XP>* P, const int* g, int gi) {
    const PlaneN<XP>& A = P[0];
    const PlaneN<XP>& B = P[1];
    const PlaneN<XP>& C = P[2];
    const PlaneN<XP>& M = P[3];
    XP dP[4];
    dP[0] = vdot(M.q, vcross(B.q, C.q));
    dP[1] = vdot(M.q, vcross(C.q, A.q));
    dP[2] = vdot(M.q, vcross(A.q, B.q));
    dP[3] = -vdot(A.q, vcross(B.q, C.q));
    XP ci = xp_zero();
    for (int k = 0; k < 4; ++k)
        if (g[k] >= 0) ci = ci + dP[k];
    // candidates in increasing index: atom i, then the plane atoms
    int best = -1, order_idx = 0x7fffffff;
    int done_mask = 0;
    for (int step = 0; step < 5; ++step) {
        best = -2;
        order_idx = 0x7fffffff;
        if (!(done_mask & 16) && gi < order_idx) { best = 4; order_idx = gi; }
        for (int k = 0; k < 4; ++k)
            if (!(done_mask & (1 << k)) && g[k] >= 0 && g[k] < order_idx) { best = k; order_idx = g[k]; }
        if (best == -2) break;
        done_mask |= 1 << best;
        const int sg = best == 4 ? xp_sign(ci) : -xp_sign(dP[best]);
        if (sg != 0) return sg;
    }
    return 0;
}

// ------------------------------------------------------------------ geometric terms
template <class T> struct P3 { T x, y, z; };
template <class T> DS_HD P3<T> operator+(P3<T> a, P3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T> DS_HD P3<T> operator-(P3<T> a, P3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T> DS_HD P3<T> operator*(P3<T> a, T s) { return {a.x * s, a.y * s, a.z * s}; }
template <class T> DS_HD T dot3(P3<T> a, P3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> DS_HD P3<T> cross3(P3<T> a, P3<T> b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
DS_HD float ds_sqrt(float x) { return sqrtf(x); }
DS_HD double ds_sqrt(double x) { return sqrt(x); }
DS_HD float ds_atan2(float y, float x) { return atan2f(y, x); }
DS_HD double ds_atan2(double y, double x) { return atan2(y, x); }
template <class T> DS_HD T norm3(P3<T> a) { return ds_sqrt(dot3(a, a)); }
template <class T> DS_HD T pi_t() { return (T)3.14159265358979323846; }

// inner dihedral angle (radians) of the tetrahedron (u,v,c,d) along edge (u,v)
template <class T> DS_HD T dihedral(P3<T> u, P3<T> v, P3<T> c, P3<T> d) {
    P3<T> e = v - u, mc = cross3(e, c - u), md = cross3(e, d - u);
    T v6 = dot3(e, cross3(c - u, d - u));
    return ds_atan2(norm3(e) * (v6 < (T)0 ? -v6 : v6), dot3(mc, md));
}
// the same angle and its gradient with respect to u, v, c, d
template <class T> DS_HD T dihedral_grad(P3<T> u, P3<T> v, P3<T> c, P3<T> d, P3<T>& gu, P3<T>& gv, P3<T>& gc, P3<T>& gd) {
    P3<T> e = v - u, ac = c - u, ad = d - u;
    P3<T> mc = cross3(e, ac), md = cross3(e, ad);
    T v6 = dot3(e, cross3(ac, ad));
    T le2 = dot3(e, e), le = ds_sqrt(le2);
    T sg = v6 < (T)0 ? (T)-1 : (T)1;
    T theta = ds_atan2(le * (v6 * sg), dot3(mc, md));
    // moving c (d) along the normal of its face away from the other face opens the angle
    gc = mc * (-sg * le / dot3(mc, mc));
    gd = md * (sg * le / dot3(md, md));
    T ac_ = dot3(ac, e) / le2, ad_ = dot3(ad, e) / le2;
    gv = gc * (-ac_) + gd * (-ad_);
    gu = gc * (ac_ - (T)1) + gd * (ad_ - (T)1);
    return theta;
}
// the same angle with the orientation sign of (u,v,c,d) given (+1 / -1), as it is known
// combinatorially for every tetrahedron the kernel differentiates (no sign error on slivers)
template <class T> DS_HD void dihedral_grad_s(P3<T> u, P3<T> v, P3<T> c, P3<T> d, T sg, P3<T>& gu, P3<T>& gv, P3<T>& gc, P3<T>& gd) {
    P3<T> e = v - u, ac = c - u, ad = d - u;
    P3<T> mc = cross3(e, ac), md = cross3(e, ad);
    T le2 = dot3(e, e), le = ds_sqrt(le2);
    gc = mc * (-sg * le / dot3(mc, mc));
    gd = md * (sg * le / dot3(md, md));
    T ac_ = dot3(ac, e) / le2, ad_ = dot3(ad, e) / le2;
    gv = gc * (-ac_) + gd * (-ad_);
    gu = gc * (ac_ - (T)1) + gd * (ad_ - (T)1);
}
// Van Oosterom-Strackee: atan2(|a.(b x c)|, abc + (a.b)c + (a.c)b + (b.c)a) is half the solid
// angle (steradian) of the cone over a, b, c; the normalised omega of Eq. (vertex) is it / 2 pi
template <class T> DS_HD T solid_angle_half(P3<T> a, P3<T> b, P3<T> c) {
    T la = norm3(a), lb = norm3(b), lc = norm3(c);
    T num = dot3(a, cross3(b, c));
    num = num < (T)0 ? -num : num;
    T den = la * lb * lc + dot3(a, b) * lc + dot3(a, c) * lb + dot3(b, c) * la;
    return ds_atan2(num, den);
}
template <class T> DS_HD T solid_angle(P3<T> a, P3<T> b, P3<T> c) {
    return solid_angle_half(a, b, c) / ((T)2 * pi_t<T>());
}
// cap of sphere 1 inside ball 2 in FP64 with the cancellation-free height
// h1 = R1 - t1 = (R1 + R2 - d)(R2 - R1 + d) / (2d)
DS_HD double cap64(double d, double R1, double R2) {
    return 2.0 * 3.14159265358979323846 * R1 * ((R1 + R2 - d) * (R2 - R1 + d) / (2.0 * d));
}
// distance from the centre of sphere 1 to the plane of the circle where spheres 1, 2 meet
template <class T> DS_HD T t_dist(T d, T R1, T R2) { return (d * d + R1 * R1 - R2 * R2) / ((T)2 * d); }

// one of the two points common to the three sphere surfaces; false if none.  s_ext >= 0
// replaces the height s of the triple points over the plane of the centres (a value computed
// more accurately by the caller)
template <class T> DS_HD bool triple_point(P3<T> p1, P3<T> p2, P3<T> p3, T R1, T R2, T R3, P3<T>& x,
                                           T s_ext = (T)-1) {
    P3<T> q2 = p2 - p1, q3 = p3 - p1;
    T b2 = (dot3(q2, q2) - R2 * R2 + R1 * R1) * (T)0.5;
    T b3 = (dot3(q3, q3) - R3 * R3 + R1 * R1) * (T)0.5;
    P3<T> nn = cross3(q2, q3);
    T W = dot3(nn, nn);
    P3<T> z = (cross3(q3, nn) * b2 + cross3(nn, q2) * b3) * ((T)1 / W);
    T psi = dot3(z, z) - R1 * R1;
    T s = s_ext >= (T)0 ? s_ext : (psi < (T)0 ? ds_sqrt(-psi) : (T)0);
    x = p1 + z + nn * (s / ds_sqrt(W));
    return psi < (T)0;
}

// Squared height s^2 = R1^2 - |z|^2 of the triple points of spheres 1, 2, 3 over the plane of
// their centres (z: the foot of the triple points in that plane, relative to p1; q_k = p_k -
// p1).  Near a degenerate triangle (the triple points about to merge) this difference cancels:
// its error is about u R1^2 for inputs rounded to unit roundoff u, so the height, whose error
// is that over 2 s, is taken from float64 inputs there.
template <class T> DS_HD T triple_height2(P3<T> q2, P3<T> q3, T R1, T R2, T R3) {
    const T b2 = (dot3(q2, q2) - R2 * R2 + R1 * R1) * (T)0.5;
    const T b3 = (dot3(q3, q3) - R3 * R3 + R1 * R1) * (T)0.5;
    const P3<T> nn = cross3(q2, q3);
    const T W = dot3(nn, nn);
    const P3<T> z = (cross3(q3, nn) * b2 + cross3(nn, q2) * b3) * ((T)1 / W);
    return R1 * R1 - dot3(z, z);
}

// S_123^(1): area of sphere 1 inside balls 2 and 3 (Eq. trianglev).  With the spherical
// excess omega_1 = (theta_12 + theta_13 + theta_1x)/(4 pi) - 1/4 of the tetrahedron
// (p1,p2,p3,x), the paper's 1/2 S = Phi_12 S_12 + Phi_13 S_13 - Omega_1 S_1 becomes
//   1/2 S = pi R1^2 - R1 (t12 theta_12 + t13 theta_13) - R1^2 theta_1x.
template <class T> DS_HD T tri_term(P3<T> p1, P3<T> p2, P3<T> p3, T R1, T R2, T R3) {
    P3<T> x;
    triple_point(p1, p2, p3, R1, R2, R3, x);
    T d12 = norm3(p2 - p1), d13 = norm3(p3 - p1);
    T t12 = t_dist(d12, R1, R2), t13 = t_dist(d13, R1, R3);
    T th12 = dihedral(p1, p2, p3, x), th13 = dihedral(p1, p3, p2, x), th1x = dihedral(p1, x, p2, p3);
    return (T)2 * (pi_t<T>() * R1 * R1 - R1 * (t12 * th12 + t13 * th13) - R1 * R1 * th1x);
}
// the same term and its gradient with respect to p1, p2, p3 (Eq. triangle); the triple
// point moves with the centres: (x - p_k) . (dx - dp_k) = 0, so the x-part of the
// gradient is lambda_k (x - p_k) with sum_k lambda_k (x - p_k) = dS/dx.
template <class T> DS_HD T tri_term_grad(P3<T> p1, P3<T> p2, P3<T> p3, T R1, T R2, T R3, P3<T>& g1, P3<T>& g2, P3<T>& g3) {
    P3<T> x;
    triple_point(p1, p2, p3, R1, R2, R3, x);
    P3<T> q2 = p2 - p1, q3 = p3 - p1;
    T d12 = norm3(q2), d13 = norm3(q3);
    T t12 = t_dist(d12, R1, R2), t13 = t_dist(d13, R1, R3);
    T t21 = d12 - t12, t31 = d13 - t13;
    P3<T> a_u, a_v, a_c, a_d, b_u, b_v, b_c, b_d, c_u, c_v, c_c, c_d;
    T th12 = dihedral_grad(p1, p2, p3, x, a_u, a_v, a_c, a_d);
    T th13 = dihedral_grad(p1, p3, p2, x, b_u, b_v, b_c, b_d);
    T th1x = dihedral_grad(p1, x, p2, p3, c_u, c_v, c_c, c_d);
    T half = pi_t<T>() * R1 * R1 - R1 * (t12 * th12 + t13 * th13) - R1 * R1 * th1x;
    P3<T> u12 = q2 * ((T)1 / d12), u13 = q3 * ((T)1 / d13);
    // d t12 / d p2 = (t21 / d12) u12 = - d t12 / d p1
    P3<T> dt12 = u12 * (t21 / d12), dt13 = u13 * (t31 / d13);
    P3<T> h1 = (dt12 * th12 + dt13 * th13) * R1 - (a_u * t12 + b_u * t13) * R1 - c_u * (R1 * R1);
    P3<T> h2 = dt12 * (-R1 * th12) - (a_v * t12 + b_c * t13) * R1 - c_c * (R1 * R1);
    P3<T> h3 = dt13 * (-R1 * th13) - (a_c * t12 + b_v * t13) * R1 - c_d * (R1 * R1);
    P3<T> hx = (a_d * t12 + b_d * t13) * (-R1) - c_v * (R1 * R1);
    P3<T> r1 = x - p1, r2 = x - p2, r3 = x - p3;
    P3<T> s1 = cross3(r2, r3), s2 = cross3(r3, r1), s3 = cross3(r1, r2);
    T idet = (T)1 / dot3(r1, s1);
    T l1 = dot3(hx, s1) * idet, l2 = dot3(hx, s2) * idet, l3 = dot3(hx, s3) * idet;
    g1 = (h1 + r1 * l1) * (T)2;
    g2 = (h2 + r2 * l2) * (T)2;
    g3 = (h3 + r3 * l3) * (T)2;
    return (T)2 * half;
}

// S_123^(1) with the geometry (triple point, dihedral angles) in T and the combination of
// Eq. (trianglev) (spherical-excess form above) in FP64; p1 is the origin
template <class T> DS_HD double tri_term_mixed(P3<T> p2, P3<T> p3, double R1, double R2, double R3) {
    const P3<T> O = {(T)0, (T)0, (T)0};
    P3<T> x;
    triple_point(O, p2, p3, (T)R1, (T)R2, (T)R3, x);
    // t1k = (d1k^2 + R1^2 - Rk^2) / 2 d1k with the radii part in FP64 and the reciprocal of
    // the distance in T (its rounding differs from triangle to triangle: no systematic bias)
    const T e12 = norm3(p2), e13 = norm3(p3);
    const double d12 = (double)e12, d13 = (double)e13;
    double t12 = (d12 * d12 + (R1 - R2) * (R1 + R2)) * (double)((T)0.5 / e12);
    double t13 = (d13 * d13 + (R1 - R3) * (R1 + R3)) * (double)((T)0.5 / e13);
    double th12 = (double)dihedral(O, p2, p3, x), th13 = (double)dihedral(O, p3, p2, x);
    double th1x = (double)dihedral(O, x, p2, p3);
    return 2.0 * (3.14159265358979323846 * R1 * R1 - R1 * (t12 * th12 + t13 * th13) - R1 * R1 * th1x);
}
// Gradient of S_123^(1) (area of sphere 1 inside balls 2 and 3) with respect to p2 and p3,
// p1 at the origin; d/dp1 = -(g2 + g3).  Boundary variation on sphere 1: the lens is bounded
// by an arc of the circle C_12 (angle 2 beta_2, centred on the direction w_2 towards ball 3)
// and an arc of C_13.  Moving p2 changes only C_12 = {u : u.n2 = c2}, and
//   dS = R1^2 [ -2 beta_2 dc2 + 2 s2 sin(beta_2) w_2 . dn2 ],  s2 sin(beta_2) = s_t / R1,
// with s_t the height of the triple points over the plane of the centres; so
//   dS/dp2 = (2 R1 / d2) ( -beta_2 t21 n2 + s_t w_2 ),  w_2 = (n3 - g n2) / sqrt(1 - g^2).
// The half-arc angle is beta_2 = atan2(L, c3 - c2 g), L = (s_t / R1) sqrt(1 - g^2),
// c_k = t1k / R1, g = n2 . n3.  (Same quantity as differentiating Eq. (trianglev).)
template <class T> DS_HD bool lens_grad(P3<T> q2, P3<T> q3, T R1, T R2, T R3, P3<T>& g2, P3<T>& g3,
                                        T st_ext = (T)-1) {
    T d2 = norm3(q2), d3 = norm3(q3);
    T t12 = t_dist(d2, R1, R2), t13 = t_dist(d3, R1, R3);
    T c2 = t12 / R1, c3 = t13 / R1;
    P3<T> cr = cross3(q2, q3);
    T crn = norm3(cr);
    T g = dot3(q2, q3) / (d2 * d3), sg = crn / (d2 * d3);
    T b2 = (d2 * d2 - R2 * R2 + R1 * R1) * (T)0.5, b3 = (d3 * d3 - R3 * R3 + R1 * R1) * (T)0.5;
    P3<T> z = (cross3(q3, cr) * b2 + cross3(cr, q2) * b3) * ((T)1 / (crn * crn));
    T st2 = R1 * R1 - dot3(z, z);
    T st = st_ext >= (T)0 ? st_ext : (st2 > (T)0 ? ds_sqrt(st2) : (T)0);
    T L = (st / R1) * sg;
    T be2 = ds_atan2(L, c3 - c2 * g), be3 = ds_atan2(L, c2 - c3 * g);
    P3<T> n2 = q2 * ((T)1 / d2), n3 = q3 * ((T)1 / d3);
    P3<T> w2 = (n3 - n2 * g) * ((T)1 / sg), w3 = (n2 - n3 * g) * ((T)1 / sg);
    g2 = (n2 * (-be2 * (d2 - t12)) + w2 * st) * ((T)2 * R1 / d2);
    g3 = (n3 * (-be3 * (d3 - t13)) + w3 * st) * ((T)2 * R1 / d3);
    // the gradient is linear in st, whose value here (a difference R1^2 - |z|^2 from rounded
    // inputs) errs by about u R1^2 / st: report when a caller should supply st from more
    // accurate inputs (its square below 0.01 R1^2: measured on the triangles of three
    // 5,000-atom globules, a larger bound no longer lowers the float gradient's worst error,
    // 6e-5, which then comes from elsewhere)
    return st_ext < (T)0 && st2 < (T)0.01 * R1 * R1;
}

// ------------------------------------------------------------------ float-float
// A value carried as an unevaluated sum h + l of two floats (about 48 significant bits),
// used to combine the area terms in FP32 without the systematic rounding of quantities that
// depend only on the radii (R, R^2, R_i +- R_j, pi).  Error-free transformations: Knuth's
// two-sum and the FMA two-product.
struct FF { float h, l; };
DS_HD FF ff_of(double x) {
    float h = (float)x;
    return {h, (float)(x - (double)h)};
}
DS_HD void two_sum_f(float a, float b, float& s, float& e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
DS_HD FF ff_norm(float s, float e) {
    float h = s + e;
    return {h, e - (h - s)};
}
DS_HD FF ff_add(FF a, FF b) {
    float s, e;
    two_sum_f(a.h, b.h, s, e);
    return ff_norm(s, e + (a.l + b.l));
}
DS_HD FF ff_sub(FF a, FF b) { return ff_add(a, FF{-b.h, -b.l}); }
DS_HD FF ff_add_f(FF a, float b) {   // a + b for a plain float b
    float s, e;
    two_sum_f(a.h, b, s, e);
    return ff_norm(s, e + a.l);
}
DS_HD FF ff_mul_f(FF a, float b) {
    float p = a.h * b;
    float e = fmaf(a.h, b, -p);
    return ff_norm(p, fmaf(a.l, b, e));
}
DS_HD FF ff_mul(FF a, FF b) {
    float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    return ff_norm(p, fmaf(a.h, b.l, fmaf(a.l, b.h, e)));
}
DS_HD double ff_to_double(FF a) { return (double)a.h + (double)a.l; }

// S_123^(1) - 2 pi R1^2 (Eq. trianglev in the spherical-excess form, p1 at the origin):
//   -2 R1 (t12 theta_12 + t13 theta_13) - 2 R1^2 theta_1x
// with the geometry in float and the radius quantities R1, R1^2 and R1^2 - Rk^2 in
// float-float; the caller adds c 2 pi R1^2 once per atom in FP64.
DS_HD FF tri_term_ff(P3<float> p2, P3<float> p3, FF R1, FF R2, FF R3, FF R1sq, float s_ext = -1.f) {
    const P3<float> O = {0.f, 0.f, 0.f};
    P3<float> x;
    triple_point(O, p2, p3, R1.h, R2.h, R3.h, x, s_ext);
    const float e12 = norm3(p2), e13 = norm3(p3);
    const FF w12 = ff_mul(ff_sub(R1, R2), ff_add(R1, R2)), w13 = ff_mul(ff_sub(R1, R3), ff_add(R1, R3));
    const float t12 = ((e12 * e12 + w12.h) + w12.l) * (0.5f / e12);
    const float t13 = ((e13 * e13 + w13.h) + w13.l) * (0.5f / e13);
    const float th12 = dihedral(O, p2, p3, x), th13 = dihedral(O, p3, p2, x), th1x = dihedral(O, x, p2, p3);
    const float y = t12 * th12 + t13 * th13;
    return ff_add(ff_mul_f(R1, -2.f * y), ff_mul_f(R1sq, -2.f * th1x));
}

// ------------------------------------------------------------------ volume pieces
// Signed area of the triangle (0, a, b) intersected with the disk |x| <= r in a plane (2-D
// coordinates): the triangle's part inside the circle is bounded by straight pieces of
// the side ab and circular sectors where that side runs outside.
template <class T> DS_HD T tri_disk_area(T ax, T ay, T bx, T by, T r) {
    const T r2 = r * r;
    const T aa = ax * ax + ay * ay, bb = bx * bx + by * by;
    auto crs = [](T ux, T uy, T vx, T vy) { return ux * vy - uy * vx; };
    auto sector = [&](T ux, T uy, T vx, T vy) { return (T)0.5 * r2 * ds_atan2(crs(ux, uy, vx, vy), ux * vx + uy * vy); };
    if (aa <= r2 && bb <= r2) return (T)0.5 * crs(ax, ay, bx, by);
    const T dx = bx - ax, dy = by - ay;
    const T qa = dx * dx + dy * dy, qb = ax * dx + ay * dy, qc = aa - r2;
    const T disc = qb * qb - qa * qc;
    const T sq = disc > (T)0 ? ds_sqrt(disc) : (T)0;
    if (aa <= r2) {   // a inside: the side leaves the circle at t1
        const T t1 = (-qb + sq) / qa;
        const T px = ax + t1 * dx, py = ay + t1 * dy;
        return (T)0.5 * crs(ax, ay, px, py) + sector(px, py, bx, by);
    }
    if (bb <= r2) {   // b inside: the side enters at t0
        const T t0 = (-qb - sq) / qa;
        const T px = ax + t0 * dx, py = ay + t0 * dy;
        return sector(ax, ay, px, py) + (T)0.5 * crs(px, py, bx, by);
    }
    if (qa > (T)0 && disc > (T)0) {   // both outside: the side may cross the disk
        const T t0 = (-qb - sq) / qa, t1 = (-qb + sq) / qa;
        if (t0 > (T)0 && t1 < (T)1) {
            const T px = ax + t0 * dx, py = ay + t0 * dy, qx = ax + t1 * dx, qy = ay + t1 * dy;
            return sector(ax, ay, px, py) + (T)0.5 * crs(px, py, qx, qy) + sector(qx, qy, bx, by);
        }
    }
    return sector(ax, ay, bx, by);
}

// First moment (the integral of the position) of the region tri_disk_area measures, in the
// same 2-D coordinates: a straight piece (0, u, v) contributes its signed area times its
// centroid (u + v) / 3; a circular sector from u to v on the circle |x| = r contributes
// (r^2 / 3) (v_y - u_y, u_x - v_x), i.e. r^3 / 3 times the integral of the unit vector over
// its angle.
template <class T> DS_HD void tri_disk_moment(T ax, T ay, T bx, T by, T r, T& mx, T& my) {
    const T r2 = r * r;
    const T aa = ax * ax + ay * ay, bb = bx * bx + by * by;
    T sx = (T)0, sy = (T)0;
    auto piece = [&](T ux, T uy, T vx, T vy) {
        const T w = (ux * vy - uy * vx) * (T)(1.0 / 6.0);
        sx += w * (ux + vx);
        sy += w * (uy + vy);
    };
    auto arc = [&](T ux, T uy, T vx, T vy) {
        sx += r2 * (T)(1.0 / 3.0) * (vy - uy);
        sy += r2 * (T)(1.0 / 3.0) * (ux - vx);
    };
    if (aa <= r2 && bb <= r2) {
        piece(ax, ay, bx, by);
    } else {
        const T dx = bx - ax, dy = by - ay;
        const T qa = dx * dx + dy * dy, qb = ax * dx + ay * dy, qc = aa - r2;
        const T disc = qb * qb - qa * qc;
        const T sq = disc > (T)0 ? ds_sqrt(disc) : (T)0;
        if (aa <= r2) {
            const T t1 = (-qb + sq) / qa;
            const T px = ax + t1 * dx, py = ay + t1 * dy;
            piece(ax, ay, px, py);
            arc(px, py, bx, by);
        } else if (bb <= r2) {
            const T t0 = (-qb - sq) / qa;
            const T px = ax + t0 * dx, py = ay + t0 * dy;
            arc(ax, ay, px, py);
            piece(px, py, bx, by);
        } else {
            bool crossed = false;
            if (qa > (T)0 && disc > (T)0) {
                const T t0 = (-qb - sq) / qa, t1 = (-qb + sq) / qa;
                if (t0 > (T)0 && t1 < (T)1) {
                    const T px = ax + t0 * dx, py = ay + t0 * dy, qx = ax + t1 * dx, qy = ay + t1 * dy;
                    arc(ax, ay, px, py);
                    piece(px, py, qx, qy);
                    arc(qx, qy, bx, by);
                    crossed = true;
                }
            }
            if (!crossed) arc(ax, ay, bx, by);
        }
    }
    mx = sx;
    my = sy;
}

// ------------------------------------------------------------------ out-of-line forms
// The kernels call the heavy terms through these where code size matters more (one copy of
// each body instead of one per call site); results are returned by value so that no caller
// variable has to live in local memory.  A call inside a hot loop costs more than the code
// (the loop's state is kept across it), so the terms kernel's loops use the inline forms
// (_in) and keep calls for rare paths.
template <class T> struct P3x2 { P3<T> a, b; };
template <class T> DS_HDC T dihedral_ol(P3<T> u, P3<T> v, P3<T> c, P3<T> d) { return dihedral(u, v, c, d); }
// d theta / d u of dihedral_grad_s
template <class T> DS_HD P3<T> dihedral_grad_u_in(P3<T> u, P3<T> v, P3<T> c, P3<T> d, T sg) {
    P3<T> gu, gv, gc, gd;
    dihedral_grad_s(u, v, c, d, sg, gu, gv, gc, gd);
    return gu;
}
template <class T> DS_HDC P3<T> dihedral_grad_u_ol(P3<T> u, P3<T> v, P3<T> c, P3<T> d, T sg) {
    return dihedral_grad_u_in(u, v, c, d, sg);
}
// d theta / d c of dihedral_grad_s
template <class T> DS_HD P3<T> dihedral_grad_c_in(P3<T> u, P3<T> v, P3<T> c, P3<T> d, T sg) {
    P3<T> gu, gv, gc, gd;
    dihedral_grad_s(u, v, c, d, sg, gu, gv, gc, gd);
    return gc;
}
template <class T> DS_HDC double tri_term_mixed_ol(P3<T> p2, P3<T> p3, double R1, double R2, double R3) {
    return tri_term_mixed(p2, p3, R1, R2, R3);
}
template <class T> DS_HDC T tri_disk_area_ol(T ax, T ay, T bx, T by, T r) { return tri_disk_area(ax, ay, bx, by, r); }
template <class T> struct T2 { T x, y; };
template <class T> DS_HDC T2<T> tri_disk_moment_ol(T ax, T ay, T bx, T by, T r) {
    T2<T> m;
    tri_disk_moment(ax, ay, bx, by, r, m.x, m.y);
    return m;
}
template <class T> struct P3x2f { P3<T> a, b; bool refine; };
template <class T> DS_HD P3x2f<T> lens_grad_in(P3<T> q2, P3<T> q3, T R1, T R2, T R3, T st_ext) {
    P3x2f<T> r;
    r.refine = lens_grad(q2, q3, R1, R2, R3, r.a, r.b, st_ext);
    return r;
}
// triple_height2 for float64 inputs in fewer FP64 operations, returned in float: with the
// Gram matrix G of q2, q3 the foot z = a q2 + b q3 solves G (a, b) = (b2, b3), so
// |z|^2 = (b2^2 G33 - 2 b2 b3 G23 + b3^2 G22) / det G and
// s^2 = (R1^2 det G - b2^2 G33 + 2 b2 b3 G23 - b3^2 G22) / det G; the cancellation happens in
// the float64 numerator, and the division is taken in float.
static DS_HD float triple_height2_gram(P3<double> q2, P3<double> q3, double R1, double R2, double R3) {
    const double g22 = dot3(q2, q2), g33 = dot3(q3, q3), g23 = dot3(q2, q3);
    const double R1s = R1 * R1;
    const double b2 = 0.5 * ((g22 - R2 * R2) + R1s), b3 = 0.5 * ((g33 - R3 * R3) + R1s);
    const double det = g22 * g33 - g23 * g23;
    const double num = R1s * det - (b2 * b2 * g33 - 2.0 * b2 * b3 * g23 + b3 * b3 * g22);
    return (float)num / (float)det;
}

}  // namespace dsasa
