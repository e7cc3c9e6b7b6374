// Exact dyadic arithmetic for the oracle's geometric predicates.
//
// TEST INFRASTRUCTURE ONLY: the oracle is used by tests/, __graft_entry__.smoke() and
// bench.py's cpu_baseline / reference leg, never by the product path.
//
// Every finite double is m * 2^e with an integer m, so every polynomial predicate of the
// input doubles is a dyadic rational.  A Big holds such a number exactly as
// sign * mag * 2^exp with an arbitrary-length magnitude (little-endian 32-bit limbs).
// Addition aligns exponents by shifting the operand with the larger exponent left;
// multiplication is schoolbook.  Nothing is ever rounded, so the sign of a predicate
// computed this way is its true sign.  This is deliberately simple (and slow); the GPU
// path uses an unrelated scheme (floating-point filters, then floating-point expansions).
#pragma once
#include <cstdint>
#include <cmath>
#include <vector>
#include <algorithm>
#include <stdexcept>

namespace oracle {

struct Big {
    int sign = 0;                 // -1, 0, +1
    std::vector<uint32_t> mag;    // |value| / 2^exp, no leading zero limbs when nonzero
    long exp = 0;
};

namespace detail {
inline void trim(std::vector<uint32_t>& m) { while (!m.empty() && m.back() == 0) m.pop_back(); }

inline std::vector<uint32_t> shl(const std::vector<uint32_t>& a, long bits) {
    if (a.empty()) return {};
    long limbs = bits / 32;
    int b = (int)(bits % 32);
    std::vector<uint32_t> r((size_t)limbs + a.size() + 1, 0);
    for (size_t i = 0; i < a.size(); ++i) {
        uint64_t v = (uint64_t)a[i] << b;
        r[i + limbs] |= (uint32_t)v;
        r[i + limbs + 1] |= (uint32_t)(v >> 32);
    }
    trim(r);
    return r;
}
inline int cmp(const std::vector<uint32_t>& a, const std::vector<uint32_t>& b) {
    if (a.size() != b.size()) return a.size() < b.size() ? -1 : 1;
    for (size_t i = a.size(); i-- > 0;)
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    return 0;
}
inline std::vector<uint32_t> add(const std::vector<uint32_t>& a, const std::vector<uint32_t>& b) {
    std::vector<uint32_t> r(std::max(a.size(), b.size()) + 1, 0);
    uint64_t carry = 0;
    for (size_t i = 0; i < r.size(); ++i) {
        uint64_t s = carry;
        if (i < a.size()) s += a[i];
        if (i < b.size()) s += b[i];
        r[i] = (uint32_t)s;
        carry = s >> 32;
    }
    trim(r);
    return r;
}
// a - b with a >= b
inline std::vector<uint32_t> sub(const std::vector<uint32_t>& a, const std::vector<uint32_t>& b) {
    std::vector<uint32_t> r(a.size(), 0);
    int64_t borrow = 0;
    for (size_t i = 0; i < a.size(); ++i) {
        int64_t s = (int64_t)a[i] - borrow - (i < b.size() ? (int64_t)b[i] : 0);
        borrow = s < 0;
        r[i] = (uint32_t)(s + (borrow << 32));
    }
    trim(r);
    return r;
}
inline std::vector<uint32_t> mul(const std::vector<uint32_t>& a, const std::vector<uint32_t>& b) {
    if (a.empty() || b.empty()) return {};
    std::vector<uint32_t> r(a.size() + b.size(), 0);
    for (size_t i = 0; i < a.size(); ++i) {
        uint64_t carry = 0;
        for (size_t j = 0; j < b.size(); ++j) {
            uint64_t cur = (uint64_t)a[i] * b[j] + r[i + j] + carry;
            r[i + j] = (uint32_t)cur;
            carry = cur >> 32;
        }
        size_t k = i + b.size();
        while (carry) {
            uint64_t cur = (uint64_t)r[k] + carry;
            r[k] = (uint32_t)cur;
            carry = cur >> 32;
            ++k;
        }
    }
    trim(r);
    return r;
}
// divide out trailing zero bits so magnitudes stay short
inline void normalize(Big& x) {
    trim(x.mag);
    if (x.mag.empty()) { x.sign = 0; x.exp = 0; return; }
    size_t z = 0;
    while (x.mag[z] == 0) ++z;
    if (z) { x.mag.erase(x.mag.begin(), x.mag.begin() + (long)z); x.exp += 32 * (long)z; }
    int tz = __builtin_ctz(x.mag[0]);
    if (tz) {
        for (size_t i = 0; i < x.mag.size(); ++i) {
            uint32_t hi = (i + 1 < x.mag.size()) ? x.mag[i + 1] : 0;
            x.mag[i] = (x.mag[i] >> tz) | (uint32_t)((uint64_t)hi << (32 - tz));
        }
        x.exp += tz;
        trim(x.mag);
    }
}
}  // namespace detail

inline Big big(double d) {
    Big r;
    if (d == 0.0) return r;
    if (!std::isfinite(d)) throw std::domain_error("non-finite input to exact arithmetic");
    int e;
    double m = std::frexp(std::fabs(d), &e);          // |d| = m 2^e, m in [0.5, 1)
    uint64_t im = (uint64_t)std::ldexp(m, 53);        // exact: m has <= 53 significant bits
    r.sign = d < 0 ? -1 : 1;
    r.mag = {(uint32_t)im, (uint32_t)(im >> 32)};
    r.exp = (long)e - 53;
    detail::normalize(r);
    return r;
}

inline Big operator-(Big a) { a.sign = -a.sign; return a; }

inline Big operator+(const Big& a, const Big& b) {
    if (a.sign == 0) return b;
    if (b.sign == 0) return a;
    long e = std::min(a.exp, b.exp);
    std::vector<uint32_t> A = detail::shl(a.mag, a.exp - e), B = detail::shl(b.mag, b.exp - e);
    Big r;
    r.exp = e;
    if (a.sign == b.sign) {
        r.mag = detail::add(A, B);
        r.sign = a.sign;
    } else {
        int c = detail::cmp(A, B);
        if (c == 0) return Big{};
        if (c > 0) { r.mag = detail::sub(A, B); r.sign = a.sign; }
        else { r.mag = detail::sub(B, A); r.sign = b.sign; }
    }
    detail::normalize(r);
    return r;
}
inline Big operator-(const Big& a, const Big& b) { return a + (-b); }
inline Big operator*(const Big& a, const Big& b) {
    Big r;
    if (a.sign == 0 || b.sign == 0) return r;
    r.sign = a.sign * b.sign;
    r.mag = detail::mul(a.mag, b.mag);
    r.exp = a.exp + b.exp;
    detail::normalize(r);
    return r;
}
inline int sgn(const Big& a) { return a.sign; }

// approximate value (for diagnostics only; decisions use sgn)
inline double approx(const Big& a) {
    double v = 0.0;
    for (size_t i = a.mag.size(); i-- > 0;) v = v * 4294967296.0 + (double)a.mag[i];
    return a.sign * std::ldexp(v, (int)a.exp);
}

struct BV { Big x, y, z; };
inline BV operator-(const BV& a, const BV& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline BV operator+(const BV& a, const BV& b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline BV operator*(const BV& a, const Big& s) { return {a.x * s, a.y * s, a.z * s}; }
inline Big dot(const BV& a, const BV& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline BV cross(const BV& a, const BV& b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

}  // namespace oracle
