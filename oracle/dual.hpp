// Forward-mode dual numbers for the oracle's gradient (test infrastructure only).
//
// A Dual carries a value and its partial derivatives with respect to up to 12 input
// coordinates (the positions of the <= 4 atoms one inclusion-exclusion term involves).
// Differentiating the paper's area formulas this way is independent of the hand-derived
// derivatives the CUDA path uses.
#pragma once
#include <cmath>

namespace oracle {

constexpr int ND = 12;

struct Dual {
    double v = 0.0;
    double d[ND] = {0};
    Dual() = default;
    Dual(double x) : v(x) {}
};

inline Dual operator+(const Dual& a, const Dual& b) { Dual r(a.v + b.v); for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] + b.d[k]; return r; }
inline Dual operator-(const Dual& a, const Dual& b) { Dual r(a.v - b.v); for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] - b.d[k]; return r; }
inline Dual operator-(const Dual& a) { Dual r(-a.v); for (int k = 0; k < ND; ++k) r.d[k] = -a.d[k]; return r; }
inline Dual operator*(const Dual& a, const Dual& b) {
    Dual r(a.v * b.v);
    for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
inline Dual operator/(const Dual& a, const Dual& b) {
    Dual r(a.v / b.v);
    double ib2 = 1.0 / (b.v * b.v);
    for (int k = 0; k < ND; ++k) r.d[k] = (a.d[k] * b.v - a.v * b.d[k]) * ib2;
    return r;
}
inline Dual operator*(const Dual& a, double s) { Dual r(a.v * s); for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] * s; return r; }
inline Dual operator*(double s, const Dual& a) { return a * s; }
inline Dual sqrt(const Dual& a) {
    double s = std::sqrt(a.v);
    Dual r(s);
    double f = s > 0 ? 0.5 / s : 0.0;
    for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] * f;
    return r;
}
inline Dual atan2(const Dual& y, const Dual& x) {
    Dual r(std::atan2(y.v, x.v));
    double den = x.v * x.v + y.v * y.v;
    double f = den > 0 ? 1.0 / den : 0.0;
    for (int k = 0; k < ND; ++k) r.d[k] = (x.v * y.d[k] - y.v * x.d[k]) * f;
    return r;
}
inline Dual fabs(const Dual& a) { return a.v < 0 ? -a : a; }

struct DV { Dual x, y, z; };
inline DV operator+(const DV& a, const DV& b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline DV operator-(const DV& a, const DV& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline DV operator*(const DV& a, const Dual& s) { return {a.x * s, a.y * s, a.z * s}; }
inline DV operator*(const DV& a, double s) { return {a.x * s, a.y * s, a.z * s}; }
inline Dual dot(const DV& a, const DV& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline DV cross(const DV& a, const DV& b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline Dual norm(const DV& a) { return sqrt(dot(a, a)); }

// position of atom with coordinates p whose partials occupy slots [3*slot, 3*slot+3)
inline DV seed_point(const double* p, int slot) {
    DV r;
    r.x = Dual(p[0]); r.y = Dual(p[1]); r.z = Dual(p[2]);
    if (slot >= 0) { r.x.d[3 * slot] = 1.0; r.y.d[3 * slot + 1] = 1.0; r.z.d[3 * slot + 2] = 1.0; }
    return r;
}

}  // namespace oracle
