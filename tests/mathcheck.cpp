// Host build of the CUDA path's arithmetic header for CPU unit tests.
//
// Compiled by tests/test_device_math.py with g++; exposes the filtered / exact predicates
// and the hand-derived term gradients of csrc/dsasa_math.cuh so that they can be checked
// against the oracle on the CPU before they run on the GPU.  Not part of the product.
#include "../paper_2401_10462_gb300/csrc/dsasa_math.cuh"

#include <algorithm>
#include <cmath>

using namespace dsasa;

namespace {
// plane of point k relative to point i in each tier; xyzR rows are (x, y, z, R)
PlaneN<FA<float>> p32(const double* I, const double* K) {
    double q[3], b, babs;
    plane64(I, I[3], K, K[3], q, b, babs);
    PlaneN<FA<float>> P;
    float qf[3] = {(float)q[0], (float)q[1], (float)q[2]};
    P.q = {{qf[0], fabsf(qf[0])}, {qf[1], fabsf(qf[1])}, {qf[2], fabsf(qf[2])}};
    float bf = (float)b;
    P.b = {bf, fabsf(bf) + (float)(babs * 1.4901161193847656e-08)};   // 2^-26 babs
    return P;
}
PlaneN<FA<double>> p64(const double* I, const double* K) {
    double q[3], b, babs;
    plane64(I, I[3], K, K[3], q, b, babs);
    return fa_plane64(q, b, babs, false);
}
PlaneN<XP> px(const double* I, const double* K) { return xp_plane(I, I[3], K, K[3]); }

template <class N> N eval(int kind, const PlaneN<N>* P, const N& wi) {
    switch (kind) {
        case 0: return pred_clip(P[0], P[1], P[2], P[3]);
        case 1: return pred_tet_psi(P[0], P[1], P[2], wi);
        case 2: return pred_tri_psi(P[0], P[1], wi);
        case 3: return pred_tri_beyond(P[0], P[1], P[2]);
        case 4: return pred_edge_psi(P[0], wi);
        case 5: return pred_edge_beyond(P[0], P[1]);
        default: return P[0].b;   // 6: vertex (origin beyond plane when < 0)
    }
}
int nplanes(int kind) { return kind == 0 ? 4 : kind == 1 ? 3 : kind == 2 ? 2 : kind == 3 ? 3 : kind == 4 ? 1 : kind == 5 ? 2 : 1; }
}  // namespace

extern "C" {

// tier 0 = FP32 filter, 1 = FP64 filter (0 when undecided), 2 = exact expansions
// (returns 2 if the expansion capacity overflowed).  xyzR[0] is atom i, xyzR[1..] the
// planes' atoms in predicate order.
int mc_pred(int kind, int tier, const double* xyzR) {
    const double* I = xyzR;
    int np = nplanes(kind);
    if (tier == 0) {
        PlaneN<FA<float>> P[4];
        for (int k = 0; k < np; ++k) P[k] = p32(I, xyzR + 4 * (k + 1));
        float Rf = (float)I[3];
        FA<float> wi = {Rf * Rf, Rf * Rf};
        return fa_sign(eval(kind, P, wi), G32, TINY32);
    }
    if (tier == 1) {
        PlaneN<FA<double>> P[4];
        for (int k = 0; k < np; ++k) P[k] = p64(I, xyzR + 4 * (k + 1));
        FA<double> wi = {I[3] * I[3], I[3] * I[3]};
        return fa_sign(eval(kind, P, wi), G64, TINY64);
    }
    PlaneN<XP> P[4];
    for (int k = 0; k < np; ++k) P[k] = px(I, xyzR + 4 * (k + 1));
    XP wi = xp_sq(I[3]);
    XP v = eval(kind, P, wi);
    if (v.ovf) return 2;
    return xp_sign(v);
}

// clip test of vertex (A, B, C) against plane M relative to atom i (rows i, A, B, C, M) with
// exact zeros broken by Simulation of Simplicity; g = global indices of i, A, B, C, M
int mc_sos_clip(const double* xyzR, const int* g) {
    const double* I = xyzR;
    PlaneN<XP> P[4];
    for (int k = 0; k < 4; ++k) P[k] = px(I, xyzR + 4 * (k + 1));
    XP v = pred_clip(P[0], P[1], P[2], P[3]);
    if (v.ovf) return 2;
    int s = xp_sign(v);
    if (s != 0) return s;
    int gg[4] = {g[1], g[2], g[3], g[4]};
    return 10 * sos_clip_sign(P, gg, g[0]);   // x10: marks a decision taken by the tie-break
}

int mc_xp_len(int kind, const double* xyzR) {
    const double* I = xyzR;
    PlaneN<XP> P[4];
    for (int k = 0; k < nplanes(kind); ++k) P[k] = px(I, xyzR + 4 * (k + 1));
    XP wi = xp_sq(I[3]);
    return eval(kind, P, wi).n;
}

double mc_dihedral_grad(const double* pts, double* g12, int fp32) {
    if (fp32) {
        P3<float> p[4], g[4];
        for (int k = 0; k < 4; ++k) p[k] = {(float)pts[3 * k], (float)pts[3 * k + 1], (float)pts[3 * k + 2]};
        float th = dihedral_grad(p[0], p[1], p[2], p[3], g[0], g[1], g[2], g[3]);
        for (int k = 0; k < 4; ++k) { g12[3 * k] = g[k].x; g12[3 * k + 1] = g[k].y; g12[3 * k + 2] = g[k].z; }
        return th;
    }
    P3<double> p[4], g[4];
    for (int k = 0; k < 4; ++k) p[k] = {pts[3 * k], pts[3 * k + 1], pts[3 * k + 2]};
    double th = dihedral_grad(p[0], p[1], p[2], p[3], g[0], g[1], g[2], g[3]);
    for (int k = 0; k < 4; ++k) { g12[3 * k] = g[k].x; g12[3 * k + 1] = g[k].y; g12[3 * k + 2] = g[k].z; }
    return th;
}

double mc_solid_angle(const double* a, const double* b, const double* c) {
    return solid_angle(P3<double>{a[0], a[1], a[2]}, P3<double>{b[0], b[1], b[2]}, P3<double>{c[0], c[1], c[2]});
}

double mc_tri_term_grad(const double* p9, double R1, double R2, double R3, double* g9, int fp32) {
    if (fp32) {
        P3<float> p[3], g[3];
        for (int k = 0; k < 3; ++k) p[k] = {(float)p9[3 * k], (float)p9[3 * k + 1], (float)p9[3 * k + 2]};
        float S = tri_term_grad(p[0], p[1], p[2], (float)R1, (float)R2, (float)R3, g[0], g[1], g[2]);
        for (int k = 0; k < 3; ++k) { g9[3 * k] = g[k].x; g9[3 * k + 1] = g[k].y; g9[3 * k + 2] = g[k].z; }
        return S;
    }
    P3<double> p[3], g[3];
    for (int k = 0; k < 3; ++k) p[k] = {p9[3 * k], p9[3 * k + 1], p9[3 * k + 2]};
    double S = tri_term_grad(p[0], p[1], p[2], R1, R2, R3, g[0], g[1], g[2]);
    for (int k = 0; k < 3; ++k) { g9[3 * k] = g[k].x; g9[3 * k + 1] = g[k].y; g9[3 * k + 2] = g[k].z; }
    return S;
}

double mc_tri_term(const double* p9, double R1, double R2, double R3) {
    P3<double> p[3];
    for (int k = 0; k < 3; ++k) p[k] = {p9[3 * k], p9[3 * k + 1], p9[3 * k + 2]};
    return tri_term(p[0], p[1], p[2], R1, R2, R3);
}

// S_123^(1) with p1 at the origin (geometry in float when fp32, combination in FP64) and
// the closed-form lens gradient (g9 = d/dp1, d/dp2, d/dp3)
double mc_tri_mixed(const double* q6, double R1, double R2, double R3, double* g9, int fp32) {
    if (fp32) {
        P3<float> q2 = {(float)q6[0], (float)q6[1], (float)q6[2]}, q3 = {(float)q6[3], (float)q6[4], (float)q6[5]};
        P3<float> g2, g3;
        lens_grad(q2, q3, (float)R1, (float)R2, (float)R3, g2, g3);
        double g[9] = {-(double)(g2.x + g3.x), -(double)(g2.y + g3.y), -(double)(g2.z + g3.z), g2.x, g2.y, g2.z, g3.x, g3.y, g3.z};
        for (int k = 0; k < 9; ++k) g9[k] = g[k];
        return tri_term_mixed(q2, q3, R1, R2, R3);
    }
    P3<double> q2 = {q6[0], q6[1], q6[2]}, q3 = {q6[3], q6[4], q6[5]};
    P3<double> g2, g3;
    lens_grad(q2, q3, R1, R2, R3, g2, g3);
    double g[9] = {-(g2.x + g3.x), -(g2.y + g3.y), -(g2.z + g3.z), g2.x, g2.y, g2.z, g3.x, g3.y, g3.z};
    for (int k = 0; k < 9; ++k) g9[k] = g[k];
    return tri_term_mixed(q2, q3, R1, R2, R3);
}

// the float-float form of S_123^(1) used by the mixed-precision kernel (p1 at the origin)
// the float lens gradient with the triple points' height from the float64 differences when
// lens_grad reports its float value too small to trust (the kernels' rule; fix = 1) or always
// from
// the float geometry (fix = 0); g9 as mc_tri_mixed
void mc_lens_grad_f32(const double* q6, double R1, double R2, double R3, double* g9, int fix) {
    P3<float> q2 = {(float)q6[0], (float)q6[1], (float)q6[2]}, q3 = {(float)q6[3], (float)q6[4], (float)q6[5]};
    P3<float> g2, g3;
    if (lens_grad(q2, q3, (float)R1, (float)R2, (float)R3, g2, g3) && fix) {
        P3<double> d2 = {q6[0], q6[1], q6[2]}, d3 = {q6[3], q6[4], q6[5]};
        const float s2 = triple_height2_gram(d2, d3, R1, R2, R3);
        lens_grad(q2, q3, (float)R1, (float)R2, (float)R3, g2, g3, s2 > 0.f ? std::sqrt(s2) : 0.f);
    }
    double g[9] = {-(double)(g2.x + g3.x), -(double)(g2.y + g3.y), -(double)(g2.z + g3.z), g2.x, g2.y, g2.z, g3.x, g3.y, g3.z};
    for (int k = 0; k < 9; ++k) g9[k] = g[k];
}

double mc_tri_ff(const double* q6, double R1, double R2, double R3) {
    P3<float> q2 = {(float)q6[0], (float)q6[1], (float)q6[2]}, q3 = {(float)q6[3], (float)q6[4], (float)q6[5]};
    FF r1 = ff_of(R1);
    FF v = tri_term_ff(q2, q3, r1, ff_of(R2), ff_of(R3), ff_of(R1 * R1));
    return ff_to_double(v) + 2.0 * 3.14159265358979323846 * R1 * R1;
}
// float-float primitives against double
double mc_ff_op(int op, double a, double b) {
    FF x = ff_of(a), y = ff_of(b);
    FF r = op == 0 ? ff_add(x, y) : (op == 1 ? ff_sub(x, y) : (op == 2 ? ff_mul(x, y) : ff_mul_f(x, (float)b)));
    return ff_to_double(r);
}

double mc_dihedral_grad_s(const double* pts, double sg, double* g12) {
    P3<double> p[4], g[4];
    for (int k = 0; k < 4; ++k) p[k] = {pts[3 * k], pts[3 * k + 1], pts[3 * k + 2]};
    dihedral_grad_s(p[0], p[1], p[2], p[3], sg, g[0], g[1], g[2], g[3]);
    for (int k = 0; k < 4; ++k) { g12[3 * k] = g[k].x; g12[3 * k + 1] = g[k].y; g12[3 * k + 2] = g[k].z; }
    return dihedral(p[0], p[1], p[2], p[3]);
}

double mc_cap64(double d, double R1, double R2) { return cap64(d, R1, R2); }

}  // extern "C"
