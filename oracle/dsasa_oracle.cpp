// dSASA oracle: a plain, slow CPU implementation of what the method computes.
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
// baseline / reference leg load this library; the product (CUDA) path never does, and the
// two share no code.
//
// Steps, in the paper's order (Sec. "dSASA: an analytical method for SASA"):
//   Step 1  weighted Delaunay tetrahedrization (regular triangulation) of the weighted
//           points p'_i = (p_i, d_i), d_i = (r_i + probe)^2: incremental Bowyer-Watson
//           insertion with exact predicates (exact.hpp) and Simulation of Simplicity on the
//           weights for ties; redundant points (empty Laguerre cell) are left out.
//   Step 2  the dual complex C: the alpha complex at alpha = 0 of the triangulation
//           (reading of "filtered and classified"): a simplex is in C iff it is unattached
//           with non-positive orthosphere power psi, or it is a face of a simplex in C.
//           Equivalently the intersection of the Laguerre-intersection cells
//           LI_i = L_i cap B_i of its vertices is non-empty.
//   Step 3  per-atom inclusion-exclusion, Eq. (sainexclu) with the vertex term Eq. (vertex),
//           the solid angle of the printed Van Oosterom-Strackee form (atan2 reading), the
//           edge term Eqs. (phiedge)/(edge) and the triangle term Eq. (trianglev); the
//           gradient Eq. (inexclu) is obtained by forward-mode differentiation (dual.hpp)
//           of those same formulas with the complex held fixed.
//
// parity pins (tests/test_oracle_*.py): isolated and two-sphere closed forms, the paper's
// two-sphere derivative jump (Sec. "dSASA", singularity at external tangency), an
// independent per-sphere Gauss-Bonnet exact area (gauss_bonnet below: exposed arcs of
// the cap arrangement, no triangulation), Monte-Carlo / dense-point areas, brute-force
// regularity of the triangulation, Euler characteristics of C, rigid-motion / permutation
// invariance, translation / rotation identities of the gradient and finite differences.
#include "exact.hpp"
#include "dual.hpp"

#include <array>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <numeric>
#include <set>
#include <string>
#include <unordered_map>
#include <vector>

namespace oracle {

static const double PI = 3.14159265358979323846;

struct Pt { double x, y, z, R; };   // R = fl(r + probe); far points have R = 0

struct Counters { long orient = 0, power = 0, sos = 0, alpha = 0; };

// ------------------------------------------------------------------ exact predicates
struct Geo {
    std::vector<Pt> pts;     // atoms 0..n-1, then 4 far points
    std::vector<BV> P;       // exact coordinates
    std::vector<Big> W;      // exact weights R^2
    int n = 0;
    Counters cnt;

    BV q(int k, int a) const { return P[k] - P[a]; }
    // lifted value of k relative to a: |p_k - p_a|^2 - w_k + w_a
    Big lift(const BV& qk, int k, int a) const { return dot(qk, qk) - W[k] + W[a]; }

    int orient(int a, int b, int c, int d) {
        ++cnt.orient;
        BV qb = q(b, a), qc = q(c, a), qd = q(d, a);
        return sgn(dot(qb, cross(qc, qd)));
    }

    // Does e have negative power with respect to the orthosphere of the positively oriented
    // tetrahedron (a,b,c,d)?  Ties are broken by Simulation of Simplicity on the weights:
    // w_k -> w_k + delta_k with delta_k infinitesimal, delta of a lower index dominating.
    bool conflict(int a, int b, int c, int d, int e) {
        ++cnt.power;
        BV qb = q(b, a), qc = q(c, a), qd = q(d, a), qe = q(e, a);
        Big lb = lift(qb, b, a), lc = lift(qc, c, a), ld = lift(qd, d, a), le = lift(qe, e, a);
        BV xcd = cross(qc, qd), xdb = cross(qd, qb), xbc = cross(qb, qc);
        Big D = dot(qb, xcd);
        BV Zv = xcd * lb + xdb * lc + xbc * ld;
        // sign(pi_e - psi) = sign(F) for D > 0
        Big F = le * D - dot(qe, Zv);
        int s = sgn(F);
        if (s != 0) return s < 0;
        ++cnt.sos;
        // dF/dl_k; l_k = |q_k|^2 - w_k + w_a
        Big dfe = D, dfb = -dot(qe, xcd), dfc = -dot(qe, xdb), dfd = -dot(qe, xbc);
        std::array<std::pair<int, Big>, 5> coef = {{
            {a, dfb + dfc + dfd + dfe}, {b, -dfb}, {c, -dfc}, {d, -dfd}, {e, -dfe}}};
        std::sort(coef.begin(), coef.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
        for (auto& kv : coef)
            if (sgn(kv.second) != 0) return sgn(kv.second) < 0;
        return false;
    }

    // sign of the orthosphere power psi of a tetrahedron (any orientation)
    int tet_psi(int a, int b, int c, int d) {
        ++cnt.alpha;
        BV qb = q(b, a), qc = q(c, a), qd = q(d, a);
        Big lb = lift(qb, b, a), lc = lift(qc, c, a), ld = lift(qd, d, a);
        BV xcd = cross(qc, qd), xdb = cross(qd, qb), xbc = cross(qb, qc);
        Big D = dot(qb, xcd);
        BV Zv = xcd * lb + xdb * lc + xbc * ld;   // z = Zv / (2D)
        return sgn(dot(Zv, Zv) - big(4.0) * W[a] * D * D);
    }
    // triangle orthocentre data (relative to a): z = Z / (2 |n|^2)
    void tri_z(int a, int b, int c, BV& Z, Big& n2) {
        BV qb = q(b, a), qc = q(c, a);
        Big lb = lift(qb, b, a), lc = lift(qc, c, a);
        BV nn = cross(qb, qc);
        n2 = dot(nn, nn);
        Z = cross(qc, nn) * lb + cross(nn, qb) * lc;
    }
    int tri_psi(int a, int b, int c) {
        ++cnt.alpha;
        BV Z; Big n2;
        tri_z(a, b, c, Z, n2);
        return sgn(dot(Z, Z) - big(4.0) * W[a] * n2 * n2);
    }
    // e attaches triangle (a,b,c): power of e at the orthocentre below psi
    bool tri_attached(int a, int b, int c, int e) {
        ++cnt.alpha;
        BV Z; Big n2;
        tri_z(a, b, c, Z, n2);
        BV qe = q(e, a);
        return sgn(lift(qe, e, a) * n2 - dot(qe, Z)) < 0;
    }
    int edge_psi(int a, int b) {
        ++cnt.alpha;
        BV qb = q(b, a);
        Big lb = lift(qb, b, a);
        return sgn(lb * lb - big(4.0) * W[a] * dot(qb, qb));
    }
    bool edge_attached(int a, int b, int e) {
        ++cnt.alpha;
        BV qb = q(b, a), qe = q(e, a);
        Big lb = lift(qb, b, a), le = lift(qe, e, a);
        return sgn(le * dot(qb, qb) - lb * dot(qe, qb)) < 0;
    }
    bool vertex_attached(int a, int e) {
        ++cnt.alpha;
        BV qe = q(e, a);
        return sgn(lift(qe, e, a)) < 0;
    }
};

// ------------------------------------------------------------------ regular triangulation
struct Tet { int v[4]; int nb[4]; };

struct RT {
    Geo& g;
    std::vector<Tet> T;
    std::vector<char> alive;
    std::vector<int> freel;
    std::vector<int> mark;
    int stamp = 0;
    int last = 0;
    uint64_t rs = 0x2545F4914F6CDD1DULL;
    std::vector<char> redundant;
    long degenerate_hits = 0;

    explicit RT(Geo& geo) : g(geo) {}

    int rnd4() { rs ^= rs << 13; rs ^= rs >> 7; rs ^= rs << 17; return (int)(rs & 3); }

    int new_tet(const Tet& t) {
        int id;
        if (!freel.empty()) { id = freel.back(); freel.pop_back(); T[id] = t; alive[id] = 1; mark[id] = 0; }
        else { id = (int)T.size(); T.push_back(t); alive.push_back(1); mark.push_back(0); }
        return id;
    }

    int orient_replace(int t, int k, int p) {
        int v[4] = {T[t].v[0], T[t].v[1], T[t].v[2], T[t].v[3]};
        v[k] = p;
        return g.orient(v[0], v[1], v[2], v[3]);
    }
    bool in_conflict(int t, int p) {
        const int* v = T[t].v;
        return g.conflict(v[0], v[1], v[2], v[3], p);
    }

    int locate(int p) {
        int t = last;
        if (!alive[t]) { for (t = 0; !alive[t]; ++t) {} }
        for (long it = 0; it < 100000000L; ++it) {
            int rot = rnd4(), moved = 0;
            for (int kk = 0; kk < 4; ++kk) {
                int k = (kk + rot) & 3;
                if (T[t].nb[k] < 0) continue;
                if (orient_replace(t, k, p) < 0) { t = T[t].nb[k]; moved = 1; break; }
            }
            if (!moved) return t;
        }
        throw std::runtime_error("point location did not terminate");
    }

    void init(const int far[4]) {
        Tet t;
        for (int k = 0; k < 4; ++k) { t.v[k] = far[k]; t.nb[k] = -1; }
        if (g.orient(t.v[0], t.v[1], t.v[2], t.v[3]) < 0) std::swap(t.v[0], t.v[1]);
        last = new_tet(t);
    }

    // Bowyer-Watson insertion of point p
    void insert(int p) {
        int t0 = locate(p);
        if (!in_conflict(t0, p)) {
            // p lies in t0 (possibly on its boundary); if a tetrahedron sharing a face on
            // which p lies is in conflict, start there, else p is redundant.
            int alt = -1;
            for (int k = 0; k < 4 && alt < 0; ++k) {
                int nb = T[t0].nb[k];
                if (nb >= 0 && orient_replace(t0, k, p) == 0 && in_conflict(nb, p)) alt = nb;
            }
            if (alt < 0) { redundant[p] = 1; return; }
            ++degenerate_hits;
            t0 = alt;
        }
        ++stamp;
        const int IN = 2 * stamp, OUT = 2 * stamp + 1;
        std::vector<int> cav = {t0};
        mark[t0] = IN;
        std::vector<std::pair<int, int>> bnd;
        for (size_t i = 0; i < cav.size(); ++i) {
            int t = cav[i];
            for (int k = 0; k < 4; ++k) {
                int nb = T[t].nb[k];
                if (nb < 0) { bnd.push_back({t, k}); continue; }
                if (mark[nb] == IN) continue;
                if (mark[nb] != OUT) {
                    if (in_conflict(nb, p)) { mark[nb] = IN; cav.push_back(nb); continue; }
                    mark[nb] = OUT;
                }
                bnd.push_back({t, k});
            }
        }
        std::map<std::pair<int, int>, std::pair<int, int>> open;
        std::vector<int> created;
        for (auto& bf : bnd) {
            int t = bf.first, k = bf.second;
            Tet nt = T[t];
            nt.v[k] = p;
            for (int m = 0; m < 4; ++m) nt.nb[m] = -1;
            nt.nb[k] = T[t].nb[k];
            created.push_back(-1);
            int id = new_tet(nt);  // may reuse a slot of a dead tet, never a cavity tet (killed below)
            created.back() = id;
            int out = nt.nb[k];
            if (out >= 0)
                for (int m = 0; m < 4; ++m)
                    if (T[out].nb[m] == t) T[out].nb[m] = id;
            for (int m = 0; m < 4; ++m) {
                if (m == k) continue;
                int e0 = -1, e1 = -1;
                for (int j = 0; j < 4; ++j) {
                    if (j == m || j == k) continue;
                    if (e0 < 0) e0 = nt.v[j]; else e1 = nt.v[j];
                }
                std::pair<int, int> key = {std::min(e0, e1), std::max(e0, e1)};
                auto it = open.find(key);
                if (it == open.end()) open[key] = {id, m};
                else {
                    T[id].nb[m] = it->second.first;
                    T[it->second.first].nb[it->second.second] = id;
                    open.erase(it);
                }
            }
        }
        if (!open.empty()) throw std::runtime_error("cavity boundary is not closed");
        for (int t : cav) { alive[t] = 0; freel.push_back(t); }
        last = created.back();
    }
};

// Morton key for a locality-preserving insertion order
static uint64_t spread(uint64_t x) {
    x &= 0x1fffff;
    x = (x | x << 32) & 0x1f00000000ffffULL;
    x = (x | x << 16) & 0x1f0000ff0000ffULL;
    x = (x | x << 8) & 0x100f00f00f00f00fULL;
    x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
    x = (x | x << 2) & 0x1249249249249249ULL;
    return x;
}

// ------------------------------------------------------------------ the oracle result
struct Result {
    int n = 0;
    Geo g;
    std::vector<std::array<int, 4>> rt_tets;      // tetrahedra with 4 atoms (sorted)
    std::vector<std::array<int, 4>> all_tets;     // every tetrahedron (far points n..n+3 too)
    long rt_tets_total = 0;                        // including the ones with far points
    std::vector<char> redundant;
    // the dual complex C (sorted index tuples)
    std::vector<int> kv;
    std::vector<std::array<int, 2>> ke;
    std::vector<std::array<int, 3>> kt;
    std::vector<std::array<int, 4>> kT;
    long rt_tris = 0, rt_edges = 0;
    // number of triangulation tetrahedra (far ones included) around each atom / edge: a
    // vertex or edge all of whose tetrahedra are in C is interior (coefficient exactly 0)
    std::vector<int> star_all;
    std::map<std::array<int, 2>, int> edge_star_all;
    double t_rt = 0, t_alpha = 0;
    long degenerate_hits = 0;
};

using Clock = std::chrono::steady_clock;
static double secs(Clock::time_point a) { return std::chrono::duration<double>(Clock::now() - a).count(); }

static void build(Result& res, int n, const double* xyz, const double* radii, double probe) {
    auto t0 = Clock::now();
    Geo& g = res.g;
    g.n = n;
    res.n = n;
    g.pts.resize(n + 4);
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i = 0; i < n; ++i) {
        g.pts[i] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], radii[i] + probe};
        for (int k = 0; k < 3; ++k) { lo[k] = std::min(lo[k], xyz[3 * i + k]); hi[k] = std::max(hi[k], xyz[3 * i + k]); }
    }
    if (n == 0) { lo[0] = lo[1] = lo[2] = hi[0] = hi[1] = hi[2] = 0; }
    double c[3], diam = 0;
    for (int k = 0; k < 3; ++k) { c[k] = 0.5 * (lo[k] + hi[k]); diam = std::max(diam, hi[k] - lo[k]); }
    double L = 64.0 * (diam + 16.0);
    const double s[4][3] = {{1, 1, 1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
    for (int k = 0; k < 4; ++k)
        g.pts[n + k] = {c[0] + L * s[k][0], c[1] + L * s[k][1], c[2] + L * s[k][2], 0.0};
    g.P.resize(n + 4);
    g.W.resize(n + 4);
    for (int i = 0; i < n + 4; ++i) {
        g.P[i] = {big(g.pts[i].x), big(g.pts[i].y), big(g.pts[i].z)};
        Big R = big(g.pts[i].R);
        g.W[i] = R * R;
    }
    res.redundant.assign(n, 0);

    // exact duplicates of a centre: keep the larger ball (lower index on a tie); the
    // others are redundant (their balls lie inside the kept one)
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        const Pt &A = g.pts[a], &B = g.pts[b];
        if (A.x != B.x) return A.x < B.x;
        if (A.y != B.y) return A.y < B.y;
        if (A.z != B.z) return A.z < B.z;
        if (A.R != B.R) return A.R > B.R;
        return a < b;
    });
    for (int k = 1; k < n; ++k) {
        const Pt &A = g.pts[order[k - 1]], &B = g.pts[order[k]];
        if (A.x == B.x && A.y == B.y && A.z == B.z) res.redundant[order[k]] = 1;
    }

    RT rt(g);
    rt.redundant.assign(n + 4, 0);
    int far[4] = {n, n + 1, n + 2, n + 3};
    rt.init(far);
    // insertion order: Morton order of a 2^21 grid over the bounding box
    std::vector<std::pair<uint64_t, int>> ord;
    double sc = diam > 0 ? (double)((1 << 21) - 1) / diam : 0.0;
    for (int i = 0; i < n; ++i) {
        if (res.redundant[i]) continue;
        uint64_t ix = (uint64_t)((g.pts[i].x - lo[0]) * sc), iy = (uint64_t)((g.pts[i].y - lo[1]) * sc),
                 iz = (uint64_t)((g.pts[i].z - lo[2]) * sc);
        ord.push_back({spread(ix) | spread(iy) << 1 | spread(iz) << 2, i});
    }
    std::sort(ord.begin(), ord.end());
    for (auto& o : ord) rt.insert(o.second);
    res.degenerate_hits = rt.degenerate_hits;

    // collect
    std::vector<char> isvert(n, 0);
    for (size_t t = 0; t < rt.T.size(); ++t) {
        if (!rt.alive[t]) continue;
        ++res.rt_tets_total;
        bool real = true;
        for (int k = 0; k < 4; ++k) {
            int v = rt.T[t].v[k];
            if (v >= n) real = false; else isvert[v] = 1;
        }
        if (real) {
            std::array<int, 4> a = {rt.T[t].v[0], rt.T[t].v[1], rt.T[t].v[2], rt.T[t].v[3]};
            std::sort(a.begin(), a.end());
            res.rt_tets.push_back(a);
        }
    }
    for (int i = 0; i < n; ++i)
        if (!isvert[i]) res.redundant[i] = 1;
    res.t_rt = secs(t0);

    // ---------------- Step 2: alpha = 0 complex
    auto t1 = Clock::now();
    // triangles with their cofaces' opposite vertices; edges with their link vertices
    std::map<std::array<int, 3>, std::vector<int>> tri_opp;      // opposite vertices
    std::map<std::array<int, 3>, std::vector<int>> tri_cof;      // coface tet ids (real only)
    std::map<std::array<int, 2>, std::set<int>> edge_link;
    std::map<int, std::set<int>> vert_link;
    std::vector<std::array<int, 4>> alive_tets;
    for (size_t t = 0; t < rt.T.size(); ++t)
        if (rt.alive[t]) alive_tets.push_back({rt.T[t].v[0], rt.T[t].v[1], rt.T[t].v[2], rt.T[t].v[3]});
    res.all_tets = alive_tets;
    std::map<std::array<int, 4>, int> tet_id;
    std::vector<char> tetK;
    for (auto& a : res.rt_tets) {
        tet_id[a] = (int)tetK.size();
        tetK.push_back(g.tet_psi(a[0], a[1], a[2], a[3]) <= 0);
    }
    res.star_all.assign(n, 0);
    for (auto& v : alive_tets) {
        for (int a = 0; a < 4; ++a) {
            if (v[a] < n) res.star_all[v[a]] += 1;
            for (int b = a + 1; b < 4; ++b)
                if (v[a] < n && v[b] < n) res.edge_star_all[{std::min(v[a], v[b]), std::max(v[a], v[b])}] += 1;
        }
        std::array<int, 4> s4 = v;
        std::sort(s4.begin(), s4.end());
        int tid = (s4[3] < n) ? tet_id[s4] : -1;
        for (int k = 0; k < 4; ++k) {
            std::array<int, 3> f;
            int m = 0;
            for (int j = 0; j < 4; ++j) if (j != k) f[m++] = v[j];
            std::sort(f.begin(), f.end());
            if (f[2] < n) {
                tri_opp[f].push_back(v[k]);
                if (tid >= 0) tri_cof[f].push_back(tid);
            }
        }
        for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b) {
                int x = std::min(v[a], v[b]), y = std::max(v[a], v[b]);
                if (y >= n) continue;
                auto& L = edge_link[{x, y}];
                for (int j = 0; j < 4; ++j) if (j != a && j != b) L.insert(v[j]);
                vert_link[x].insert(y);
                vert_link[y].insert(x);
            }
        for (int a = 0; a < 4; ++a)
            if (v[a] < n)
                for (int j = 0; j < 4; ++j) if (j != a) vert_link[v[a]].insert(v[j]);
    }
    res.rt_tris = (long)tri_opp.size();
    res.rt_edges = (long)edge_link.size();
    std::map<std::array<int, 3>, char> triK;
    for (auto& kv : tri_opp) {
        const auto& f = kv.first;
        bool inK = false;
        for (int tid : tri_cof[f]) inK = inK || tetK[tid];
        if (!inK && g.tri_psi(f[0], f[1], f[2]) <= 0) {
            bool att = false;
            for (int e : kv.second) att = att || g.tri_attached(f[0], f[1], f[2], e);
            inK = !att;
        }
        triK[f] = inK;
    }
    std::map<std::array<int, 2>, char> edgeK;
    for (auto& kv : edge_link) {
        const auto& e = kv.first;
        bool inK = false;
        for (int c3 : kv.second) {
            if (c3 >= n) continue;
            std::array<int, 3> f = {e[0], e[1], c3};
            std::sort(f.begin(), f.end());
            auto it = triK.find(f);
            if (it != triK.end() && it->second) { inK = true; break; }
        }
        if (!inK && g.edge_psi(e[0], e[1]) <= 0) {
            bool att = false;
            for (int c3 : kv.second) att = att || g.edge_attached(e[0], e[1], c3);
            inK = !att;
        }
        edgeK[e] = inK;
    }
    std::vector<char> vK(n, 0);
    for (auto& kv : edgeK)
        if (kv.second) { vK[kv.first[0]] = 1; vK[kv.first[1]] = 1; }
    for (int i = 0; i < n; ++i) {
        if (res.redundant[i] || vK[i]) continue;
        bool att = false;
        for (int e : vert_link[i]) att = att || g.vertex_attached(i, e);
        vK[i] = !att;
    }
    for (int i = 0; i < n; ++i) if (vK[i]) res.kv.push_back(i);
    for (auto& kv : edgeK) if (kv.second) res.ke.push_back(kv.first);
    for (auto& kv : triK) if (kv.second) res.kt.push_back(kv.first);
    for (size_t k = 0; k < res.rt_tets.size(); ++k) if (tetK[k]) res.kT.push_back(res.rt_tets[k]);
    std::sort(res.kT.begin(), res.kT.end());
    std::sort(res.rt_tets.begin(), res.rt_tets.end());
    res.t_alpha = secs(t1);
}

// ------------------------------------------------------------------ area terms (Step 3)
// normalised inner solid angle at p0 of the tetrahedron (p0,p1,p2,p3): Van Oosterom-Strackee
static Dual omega(const DV& p0, const DV& p1, const DV& p2, const DV& p3) {
    DV a = p1 - p0, b = p2 - p0, c = p3 - p0;
    Dual la = norm(a), lb = norm(b), lc = norm(c);
    Dual num = fabs(dot(a, cross(b, c)));
    Dual den = la * lb * lc + dot(a, b) * lc + dot(a, c) * lb + dot(b, c) * la;
    return atan2(num, den) * (1.0 / (2.0 * PI));
}
// normalised inner dihedral angle along edge (pu,pv) between the faces towards pc and pd
static Dual phi(const DV& pu, const DV& pv, const DV& pc, const DV& pd) {
    DV e = pv - pu;
    DV u = cross(e, pc - pu), v = cross(e, pd - pu);
    return atan2(norm(cross(u, v)), dot(u, v)) * (1.0 / (2.0 * PI));
}
// S_ij^(i) = 2 pi R_i h_i: the cap of sphere i inside ball j
static Dual cap(const DV& pi, const DV& pj, double Ri, double Rj) {
    Dual d = norm(pj - pi);
    Dual t = (d * d + Dual(Ri * Ri - Rj * Rj)) / (d * 2.0);
    return (Dual(Ri) - t) * (2.0 * PI * Ri);
}
// one of the two points common to the three sphere surfaces
static DV triple_point(const DV& p1, const DV& p2, const DV& p3, double R1, double R2, double R3, bool* ok) {
    DV q2 = p2 - p1, q3 = p3 - p1;
    Dual l2 = dot(q2, q2) + Dual(R1 * R1 - R2 * R2), l3 = dot(q3, q3) + Dual(R1 * R1 - R3 * R3);
    DV nn = cross(q2, q3);
    Dual n2 = dot(nn, nn);
    DV Z = cross(q3, nn) * l2 + cross(nn, q2) * l3;
    DV z = Z * (Dual(0.5) / n2);
    Dual psi = dot(z, z) - Dual(R1 * R1);
    *ok = psi.v < 0;
    Dual s = sqrt(-psi);
    return p1 + z + nn * (s / sqrt(n2));
}
// S_ijk^(i): area of sphere i inside balls j and k, Eq. (trianglev):
// 1/2 S = Phi^x_ij S_ij^(i) + Phi^x_ik S_ik^(i) - Omega^x_i S_i with the tetrahedron (i,j,k,x)
static Dual tri_term(const DV& pi, const DV& pj, const DV& pk, double Ri, double Rj, double Rk, bool* ok) {
    DV x = triple_point(pi, pj, pk, Ri, Rj, Rk, ok);
    Dual a = phi(pi, pj, pk, x) * cap(pi, pj, Ri, Rj);
    Dual b = phi(pi, pk, pj, x) * cap(pi, pk, Ri, Rk);
    Dual c = omega(pi, pj, pk, x) * (4.0 * PI * Ri * Ri);
    return (a + b - c) * 2.0;
}

struct Areas {
    std::vector<long double> A;
    std::vector<double> G;
    long n_tri_bad = 0;
};

// Exterior classification shared by the term loops (the sums of Eq. sainexclu run over the
// boundary of C): a vertex / edge whose every triangulation tetrahedron is in C has
// coefficient 0; ntet counts the tetrahedra of C on each triangle.
struct TermPrep {
    std::vector<int> kstar;
    std::map<std::array<int, 2>, int> kedge;
    std::map<std::array<int, 3>, int> ntet;
};

static void prepare_terms(const Result& res, TermPrep& p) {
    p.kstar.assign(res.n, 0);
    for (auto& T : res.kT)
        for (int s = 0; s < 4; ++s) {
            p.kstar[T[s]] += 1;
            for (int t = s + 1; t < 4; ++t) p.kedge[{T[s], T[t]}] += 1;
            std::array<int, 3> f;
            int m = 0;
            for (int j = 0; j < 4; ++j) if (j != s) f[m++] = T[j];
            p.ntet[f] += 1;
        }
}

// The terms of Eq. (sainexclu) and, if want_grad, their gradient (Eq. inexclu): the share
// `part` of `nparts` of the vertices, tetrahedra, edges and triangles of C (every nparts-th
// one; part 0 of 1 is all of them in order), added to out (sized by the caller).
static void accumulate_terms(const Result& res, const TermPrep& p, const double* w, bool want_grad, Areas& out,
                             int part, int nparts) {
    const Geo& g = res.g;
    auto W = [&](int i) { return w ? w[i] : 1.0; };
    auto pt = [&](int i) { return &g.pts[i].x; };
    auto R = [&](int i) { return g.pts[i].R; };
    // accumulate a term owned by atom `own` that involves atoms ids[0..m)
    auto add = [&](int own, const Dual& val, const int* ids, int m) {
        out.A[own] += (long double)val.v;
        if (!want_grad) return;
        double wo = W(own);
        for (int s = 0; s < m; ++s)
            for (int k = 0; k < 3; ++k) out.G[3 * ids[s] + k] += wo * val.d[3 * s + k];
    };
    auto vert_interior = [&](int i) { return p.kstar[i] == res.star_all[i]; };
    auto edge_interior = [&](int a, int b) {
        std::array<int, 2> e = {std::min(a, b), std::max(a, b)};
        auto it = p.kedge.find(e);
        return it != p.kedge.end() && it->second == res.edge_star_all.at(e);
    };
    // vertex constant part 4 pi R^2
    for (size_t q = part; q < res.kv.size(); q += nparts) {
        int i = res.kv[q];
        if (!vert_interior(i)) out.A[i] += (long double)(4.0 * PI * R(i) * R(i));
    }
    // tetrahedra: -4 pi R_v^2 omega_v(T) for each vertex, +cap_u(v) phi_uv(T) for each edge/direction
    for (size_t q = part; q < res.kT.size(); q += nparts) {
        auto& T = res.kT[q];
        DV P[4];
        for (int s = 0; s < 4; ++s) P[s] = seed_point(pt(T[s]), s);
        for (int s = 0; s < 4; ++s) {
            int o[3], m = 0;
            for (int j = 0; j < 4; ++j) if (j != s) o[m++] = j;
            if (!vert_interior(T[s])) {
                Dual om = omega(P[s], P[o[0]], P[o[1]], P[o[2]]) * (-4.0 * PI * R(T[s]) * R(T[s]));
                add(T[s], om, T.data(), 4);
            }
            for (int e = 0; e < 3; ++e) {
                int v = o[e], c1 = o[(e + 1) % 3], c2 = o[(e + 2) % 3];
                if (edge_interior(T[s], T[v])) continue;
                Dual ph = phi(P[s], P[v], P[c1], P[c2]) * cap(P[s], P[v], R(T[s]), R(T[v]));
                add(T[s], ph, T.data(), 4);
            }
        }
    }
    // edges: -cap_i(j) for both directions
    for (size_t q = part; q < res.ke.size(); q += nparts) {
        auto& E = res.ke[q];
        if (edge_interior(E[0], E[1])) continue;
        for (int s = 0; s < 2; ++s) {
            int i = E[s], j = E[1 - s];
            DV Pi = seed_point(pt(i), 0), Pj = seed_point(pt(j), 1);
            int ids[2] = {i, j};
            add(i, cap(Pi, Pj, R(i), R(j)) * -1.0, ids, 2);
        }
    }
    // triangles: c_ijk S_ijk^(i) with c = 1 - #coface tetrahedra in C / 2
    for (size_t q = part; q < res.kt.size(); q += nparts) {
        auto& F = res.kt[q];
        auto it = p.ntet.find(F);
        double cc = 1.0 - 0.5 * (it != p.ntet.end() ? it->second : 0);
        if (cc == 0.0) continue;
        for (int s = 0; s < 3; ++s) {
            int i = F[s], j = F[(s + 1) % 3], k = F[(s + 2) % 3];
            DV Pi = seed_point(pt(i), 0), Pj = seed_point(pt(j), 1), Pk = seed_point(pt(k), 2);
            bool ok = true;
            Dual S = tri_term(Pi, Pj, Pk, R(i), R(j), R(k), &ok) * cc;
            if (!ok) { ++out.n_tri_bad; continue; }
            int ids[3] = {i, j, k};
            add(i, S, ids, 3);
        }
    }
}

static void compute_areas(const Result& res, const double* w, bool want_grad, Areas& out) {
    out.A.assign(res.n, 0.0L);
    out.G.assign(want_grad ? 3 * res.n : 0, 0.0);
    TermPrep p;
    prepare_terms(res, p);
    accumulate_terms(res, p, w, want_grad, out, 0, 1);
}

// The same terms split over `nthreads` OpenMP threads (timing of the area and gradient stage
// on all host cores; the triangulation stays serial).  Each thread sums its share, the
// shares are added in thread order: the values equal compute_areas' up to the order of
// summation.
static void compute_areas_parallel(const Result& res, const double* w, bool want_grad, Areas& out, int nthreads) {
    out.A.assign(res.n, 0.0L);
    out.G.assign(want_grad ? 3 * res.n : 0, 0.0);
    TermPrep p;
    prepare_terms(res, p);
    std::vector<Areas> parts(nthreads);
#pragma omp parallel for num_threads(nthreads) schedule(static, 1)
    for (int t = 0; t < nthreads; ++t) {
        parts[t].A.assign(res.n, 0.0L);
        parts[t].G.assign(want_grad ? 3 * res.n : 0, 0.0);
        accumulate_terms(res, p, w, want_grad, parts[t], t, nthreads);
    }
    for (int t = 0; t < nthreads; ++t) {
        for (int i = 0; i < res.n; ++i) out.A[i] += parts[t].A[i];
        for (size_t k = 0; k < out.G.size(); ++k) out.G[k] += parts[t].G[k];
        out.n_tri_bad += parts[t].n_tri_bad;
    }
}

// Numbers of the terms compute_areas evaluates (the same loops, counting instead of
// evaluating): out[0] vertex constants 4 pi R^2, out[1] solid-angle terms omega, out[2]
// dihedral terms phi (each with its cap factor), out[3] edge caps, out[4] triangle terms
// S_ijk^(i); used for the benchmark's work model.
static void count_terms(const Result& res, long* out) {
    int n = res.n;
    for (int k = 0; k < 5; ++k) out[k] = 0;
    std::vector<int> kstar(n, 0);
    std::map<std::array<int, 2>, int> kedge;
    for (auto& T : res.kT)
        for (int s = 0; s < 4; ++s) {
            kstar[T[s]] += 1;
            for (int t = s + 1; t < 4; ++t) kedge[{T[s], T[t]}] += 1;
        }
    auto vert_interior = [&](int i) { return kstar[i] == res.star_all[i]; };
    auto edge_interior = [&](int a, int b) {
        std::array<int, 2> e = {std::min(a, b), std::max(a, b)};
        auto it = kedge.find(e);
        return it != kedge.end() && it->second == res.edge_star_all.at(e);
    };
    for (int i : res.kv)
        if (!vert_interior(i)) out[0] += 1;
    for (auto& T : res.kT)
        for (int s = 0; s < 4; ++s) {
            if (!vert_interior(T[s])) out[1] += 1;
            for (int v = 0; v < 4; ++v)
                if (v != s && !edge_interior(T[s], T[v])) out[2] += 1;
        }
    for (auto& E : res.ke)
        if (!edge_interior(E[0], E[1])) out[3] += 2;
    std::map<std::array<int, 3>, int> ntet;
    for (auto& T : res.kT)
        for (int s = 0; s < 4; ++s) {
            std::array<int, 3> f;
            int m = 0;
            for (int j = 0; j < 4; ++j) if (j != s) f[m++] = T[j];
            ntet[f] += 1;
        }
    for (auto& F : res.kt) {
        double cc = 1.0 - 0.5 * (ntet.count(F) ? ntet[F] : 0);
        if (cc != 0.0) out[4] += 3;
    }
}

// ------------------------------------------------------------------ Gauss-Bonnet check
// Exact exposed area of each sphere from the arrangement of its caps (independent of the
// triangulation): area(E) = sum over boundary cycles gamma of [A(D_gamma) - 4 pi 1(s in D_gamma)]
// + 4 pi 1(s in E), with A(D_gamma) from Gauss-Bonnet on the unit sphere and the 0/1
// indicators from a coarse numerical winding integral about a reference direction s.
struct V3 { double x, y, z; };
static V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
static V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
static V3 operator*(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
static double dotv(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static V3 crossv(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
static V3 unit(V3 a) { return a * (1.0 / std::sqrt(dotv(a, a))); }

static void basis(V3 n, V3& e1, V3& e2) {
    V3 t = std::fabs(n.x) < 0.6 ? V3{1, 0, 0} : (std::fabs(n.y) < 0.6 ? V3{0, 1, 0} : V3{0, 0, 1});
    e1 = unit(crossv(n, t));
    e2 = crossv(n, e1);
}

static int gb_sphere(int i, int n, const double* xyz, const double* radii, double probe,
                     const std::vector<int>& nbrs, double* area) {
    V3 pi = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
    double Ri = radii[i] + probe;
    struct Circ { V3 nrm, e1, e2; double c, s; };
    std::vector<Circ> C;
    for (int j : nbrs) {
        V3 pj = {xyz[3 * j], xyz[3 * j + 1], xyz[3 * j + 2]};
        double Rj = radii[j] + probe;
        V3 d3 = pj - pi;
        double d = std::sqrt(dotv(d3, d3));
        if (!(d < Ri + Rj)) continue;
        if (d == 0.0) {
            if (Rj > Ri || (Rj == Ri && j < i)) { *area = 0.0; return 0; }
            continue;
        }
        double c = (d * d + Ri * Ri - Rj * Rj) / (2.0 * d * Ri);
        if (c <= -1.0) { *area = 0.0; return 0; }
        if (c >= 1.0) continue;
        Circ ci;
        ci.nrm = d3 * (1.0 / d);
        ci.c = c;
        ci.s = std::sqrt(1.0 - c * c);
        basis(ci.nrm, ci.e1, ci.e2);
        C.push_back(ci);
    }
    int m = (int)C.size();
    auto covered = [&](V3 u, int skip1, int skip2) {
        for (int k = 0; k < m; ++k)
            if (k != skip1 && k != skip2 && dotv(u, C[k].nrm) > C[k].c) return true;
        return false;
    };
    // reference direction far from every circle
    V3 sref = {0, 0, 1};
    double best = -1;
    for (int t = 0; t < 200; ++t) {
        double z = 1.0 - (2.0 * t + 1.0) / 200.0, r = std::sqrt(std::max(0.0, 1 - z * z));
        double a = t * 2.399963229728653;
        V3 s = {r * std::cos(a), r * std::sin(a), z};
        double md = 10;
        for (auto& ci : C) md = std::min(md, std::fabs(std::acos(std::max(-1.0, std::min(1.0, dotv(s, ci.nrm)))) - std::acos(ci.c)));
        if (md > best) { best = md; sref = s; }
    }
    // intersection points
    struct IP { V3 u; int j, k; };
    std::vector<IP> pts;
    std::vector<std::vector<std::pair<double, int>>> on(m);   // (angle on circle, point id)
    for (int j = 0; j < m; ++j)
        for (int k = j + 1; k < m; ++k) {
            double gg = dotv(C[j].nrm, C[k].nrm), den = 1.0 - gg * gg;
            if (den < 1e-14) continue;
            double al = (C[j].c - gg * C[k].c) / den, be = (C[k].c - gg * C[j].c) / den;
            double h2 = 1.0 - (al * al + be * be + 2.0 * al * be * gg);
            if (h2 <= 0) continue;
            double ga = std::sqrt(h2 / den);
            V3 mm = crossv(C[j].nrm, C[k].nrm);
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                V3 u = C[j].nrm * al + C[k].nrm * be + mm * (sgn * ga);
                int id = (int)pts.size();
                pts.push_back({u, j, k});
                on[j].push_back({std::atan2(dotv(u, C[j].e2), dotv(u, C[j].e1)), id});
                on[k].push_back({std::atan2(dotv(u, C[k].e2), dotv(u, C[k].e1)), id});
            }
        }
    struct Arc { int circ, p0, p1; double a0, da; };   // clockwise from angle a0 by da
    std::vector<Arc> arcs;
    double total = 0.0;   // sum over cycles of A(D) - 4 pi 1(s in D), unit sphere
    auto circ_pt = [&](int j, double a) { return C[j].nrm * C[j].c + (C[j].e1 * std::cos(a) + C[j].e2 * std::sin(a)) * C[j].s; };
    for (int j = 0; j < m; ++j) {
        auto& L = on[j];
        if (L.empty()) {
            if (!covered(circ_pt(j, 0.0), j, -1)) {
                // full circle, clockwise: D = complement of cap j
                double AD = 2.0 * PI * (1.0 + C[j].c);
                int sin_d = dotv(sref, C[j].nrm) < C[j].c;
                total += AD - 4.0 * PI * sin_d;
            }
            continue;
        }
        std::sort(L.begin(), L.end());
        int q = (int)L.size();
        for (int t = 0; t < q; ++t) {
            // clockwise arc from L[t+1] down to L[t] (wrap for the last)
            double a_hi = (t + 1 < q) ? L[t + 1].first : L[0].first + 2.0 * PI;
            int p_hi = (t + 1 < q) ? L[t + 1].second : L[0].second;
            double a_lo = L[t].first;
            double da = a_hi - a_lo;
            if (da <= 0) continue;
            V3 mid = circ_pt(j, 0.5 * (a_hi + a_lo));
            if (covered(mid, j, -1)) continue;
            arcs.push_back({j, p_hi, L[t].second, a_hi, da});
        }
    }
    // link arcs into cycles
    std::multimap<int, int> starts;
    for (size_t a = 0; a < arcs.size(); ++a) starts.insert({arcs[a].p0, (int)a});
    std::vector<char> used(arcs.size(), 0);
    int bad = 0;
    for (size_t a0 = 0; a0 < arcs.size(); ++a0) {
        if (used[a0]) continue;
        double AD = 2.0 * PI, wind = 0.0;
        int a = (int)a0;
        V3 nref = sref * -1.0, f1, f2;
        basis(nref, f1, f2);
        for (int guard = 0; guard < 100000; ++guard) {
            used[a] = 1;
            const Arc& A = arcs[a];
            AD += C[A.circ].c * A.da;
            // winding integral of (1 - cos theta) dphi about nref along the arc
            const int M = 2048;
            V3 prev = circ_pt(A.circ, A.a0);
            double pphi = std::atan2(dotv(prev, f2), dotv(prev, f1));
            for (int s = 1; s <= M; ++s) {
                V3 cur = circ_pt(A.circ, A.a0 - A.da * s / M);
                double cphi = std::atan2(dotv(cur, f2), dotv(cur, f1));
                double dphi = cphi - pphi;
                while (dphi > PI) dphi -= 2 * PI;
                while (dphi < -PI) dphi += 2 * PI;
                V3 mid = unit(prev + cur);
                wind += (1.0 - dotv(mid, nref)) * dphi;
                prev = cur;
                pphi = cphi;
            }
            // next arc: the exposed arc leaving the end point on the other circle
            auto rng = starts.equal_range(A.p1);
            int nxt = -1;
            for (auto it = rng.first; it != rng.second; ++it)
                if (arcs[it->second].circ != A.circ) nxt = it->second;
            if (nxt < 0) { bad = 1; break; }
            V3 u = pts[A.p1].u;
            V3 tin = unit(crossv(u, C[A.circ].nrm)), tout = unit(crossv(u, C[arcs[nxt].circ].nrm));
            AD -= std::atan2(dotv(u, crossv(tin, tout)), dotv(tin, tout));
            a = nxt;
            if (a == (int)a0) break;
            if (used[a]) { bad = 1; break; }
        }
        double ind = (AD - wind) / (4.0 * PI);
        double r = std::round(ind);
        if (std::fabs(ind - r) > 0.05 || (r != 0.0 && r != 1.0)) bad = 1;
        total += AD - 4.0 * PI * r;
    }
    bool sE = !covered(sref, -1, -1);
    total += sE ? 4.0 * PI : 0.0;
    *area = Ri * Ri * total;
    return bad;
}

}  // namespace oracle

// ------------------------------------------------------------------ C ABI for ctypes
using namespace oracle;

// ---------------------------------------------------------------- molecular volume
// Per-atom volume V_i = vol(B_i cap L_i) (the power-cell partition of the union of balls,
// Sum_i V_i = vol(union B)).  By the divergence theorem over the closed surface
// boundary(B_i cap L_i), with the origin at p_i:
//   V_i = (1/3) [ R_i A_i + Sum_j h_ij a_ij ],
// where A_i is the exposed sphere area (the SASA of atom i), a_ij the area of the power-
// diagram face L_i cap L_j inside B_i, and h_ij = b_j / |q_j| the signed distance of that
// face's plane from p_i.  The vector area of a closed surface is zero, so the exposed
// sphere piece has vector area -Sum_j a_ij u_ij (u_ij the unit normal towards j), which is
// d vol(union B) / d p_i (moving sphere i by dp sweeps its exposed piece).
//
// Here the face polygon of the edge ij is the ring of power centres of the triangulation's
// tetrahedra around ij (far points included), and a_ij the area of its intersection with
// the disk B_i cap plane, summed over the fan of triangles from the disk centre.

// signed area of the triangle (0, a, b) intersected with the disk |x| <= r (2-D)
static double tri_disk_area(double ax, double ay, double bx, double by, double r) {
    auto cross = [](double ux, double uy, double vx, double vy) { return ux * vy - uy * vx; };
    auto sector = [&](double ux, double uy, double vx, double vy) {
        return 0.5 * r * r * std::atan2(cross(ux, uy, vx, vy), ux * vx + uy * vy);
    };
    const double r2 = r * r;
    const double aa = ax * ax + ay * ay, bb = bx * bx + by * by;
    const bool ain = aa <= r2, bin = bb <= r2;
    if (ain && bin) return 0.5 * cross(ax, ay, bx, by);
    // points a + t (b - a) on the circle: |a|^2 + 2 t a.d + t^2 |d|^2 = r^2
    const double dx = bx - ax, dy = by - ay;
    const double A = dx * dx + dy * dy, B = ax * dx + ay * dy, C = aa - r2;
    const double disc = B * B - A * C;
    if (ain) {   // leaves the disk at t1 in [0, 1]
        double t1 = (-B + std::sqrt(std::max(disc, 0.0))) / A;
        double px = ax + t1 * dx, py = ay + t1 * dy;
        return 0.5 * cross(ax, ay, px, py) + sector(px, py, bx, by);
    }
    if (bin) {   // enters at t0 in [0, 1]
        double t0 = (-B - std::sqrt(std::max(disc, 0.0))) / A;
        double px = ax + t0 * dx, py = ay + t0 * dy;
        return sector(ax, ay, px, py) + 0.5 * cross(px, py, bx, by);
    }
    if (A > 0 && disc > 0) {
        double sq = std::sqrt(disc), t0 = (-B - sq) / A, t1 = (-B + sq) / A;
        if (t0 > 0 && t1 < 1) {
            double px = ax + t0 * dx, py = ay + t0 * dy, qx = ax + t1 * dx, qy = ay + t1 * dy;
            return sector(ax, ay, px, py) + 0.5 * cross(px, py, qx, qy) + sector(qx, qy, bx, by);
        }
    }
    return sector(ax, ay, bx, by);
}

// First moment (integral of the position, 2-D) of the same signed region as tri_disk_area:
// the part of the triangle (0, a, b) inside the disk |x| <= r.  A straight piece (0, u, v)
// contributes its signed area times its centroid (u + v) / 3; a circular sector from u to v
// (|u| = |v| = r) contributes r^2 / 3 times (v - u) turned by -90 degrees, the integral of
// r^3 (cos t, sin t) / 3 over its angle.
static void tri_disk_moment(double ax, double ay, double bx, double by, double r, double& mx, double& my) {
    auto cross = [](double ux, double uy, double vx, double vy) { return ux * vy - uy * vx; };
    mx = my = 0.0;
    auto tri = [&](double ux, double uy, double vx, double vy) {
        const double w = 0.5 * cross(ux, uy, vx, vy) / 3.0;
        mx += w * (ux + vx);
        my += w * (uy + vy);
    };
    auto sector = [&](double ux, double uy, double vx, double vy) {
        mx += r * r / 3.0 * (vy - uy);
        my += r * r / 3.0 * (ux - vx);
    };
    const double r2 = r * r;
    const double aa = ax * ax + ay * ay, bb = bx * bx + by * by;
    const bool ain = aa <= r2, bin = bb <= r2;
    if (ain && bin) { tri(ax, ay, bx, by); return; }
    const double dx = bx - ax, dy = by - ay;
    const double A = dx * dx + dy * dy, B = ax * dx + ay * dy, C = aa - r2;
    const double disc = B * B - A * C;
    if (ain) {
        double t1 = (-B + std::sqrt(std::max(disc, 0.0))) / A;
        double px = ax + t1 * dx, py = ay + t1 * dy;
        tri(ax, ay, px, py);
        sector(px, py, bx, by);
        return;
    }
    if (bin) {
        double t0 = (-B - std::sqrt(std::max(disc, 0.0))) / A;
        double px = ax + t0 * dx, py = ay + t0 * dy;
        sector(ax, ay, px, py);
        tri(px, py, bx, by);
        return;
    }
    if (A > 0 && disc > 0) {
        double sq = std::sqrt(disc), t0 = (-B - sq) / A, t1 = (-B + sq) / A;
        if (t0 > 0 && t1 < 1) {
            double px = ax + t0 * dx, py = ay + t0 * dy, qx = ax + t1 * dx, qy = ay + t1 * dy;
            sector(ax, ay, px, py);
            tri(px, py, qx, qy);
            sector(qx, qy, bx, by);
            return;
        }
    }
    sector(ax, ay, bx, by);
}

// Volumes V_i = vol(B_i cap L_i) and, with weights w (NULL = ones), the gradient
// d(sum_i w_i V_i)/dp.  Moving p_j moves only the face of L_i towards j, so
// dV_i/dp_j = s (p_j - C) / |p_j - p_i| with s the area and C the centroid of that face's part
// inside B_i (the same polygon for cell j: on the bisector the two balls have equal power);
// dV_i/dp_i = -sum_j dV_i/dp_j (translation).  In the frame of atom k the gradient entry is
//   g_k = sum_faces [(w_k - w_j) m - w_k s q] / |q|,  q = p_j - p_k, m = s (C - p_k).
static void compute_volumes(const Result& res, const std::vector<long double>& A, std::vector<double>& vol,
                            std::vector<double>& grad, const double* w = nullptr) {
    const Geo& g = res.g;
    const int n = res.n;
    vol.assign(n, 0.0);
    grad.assign(3 * n, 0.0);
    // link of every edge of C: for each tetrahedron around ij the two other vertices
    std::map<std::array<int, 2>, std::vector<std::array<int, 2>>> ring;
    std::set<std::array<int, 2>> inC(res.ke.begin(), res.ke.end());
    for (auto& v : res.all_tets)
        for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b) {
                std::array<int, 2> e = {std::min(v[a], v[b]), std::max(v[a], v[b])};
                if (!inC.count(e)) continue;
                std::array<int, 2> o;
                int m = 0;
                for (int c = 0; c < 4; ++c) if (c != a && c != b) o[m++] = v[c];
                ring[e].push_back(o);
            }
    // power centre of the tetrahedron (own, j, k, l) relative to p_own: q_m . z = b_m
    auto plane = [&](int own, int m, double q[3], double& b) {
        const Pt &P = g.pts[own], &M = g.pts[m];
        q[0] = M.x - P.x; q[1] = M.y - P.y; q[2] = M.z - P.z;
        b = 0.5 * ((q[0] * q[0] + q[1] * q[1] + q[2] * q[2]) - M.R * M.R + P.R * P.R);
    };
    auto centre = [&](int own, int j, int k, int l, double z[3]) {
        double qa[3], qb[3], qc[3], ba, bb, bc;
        plane(own, j, qa, ba); plane(own, k, qb, bb); plane(own, l, qc, bc);
        V3 A3 = {qa[0], qa[1], qa[2]}, B3 = {qb[0], qb[1], qb[2]}, C3 = {qc[0], qc[1], qc[2]};
        V3 bcx = crossv(B3, C3), cax = crossv(C3, A3), abx = crossv(A3, B3);
        double D = dotv(A3, bcx);
        V3 Z = (bcx * ba + cax * bb + abx * bc) * (1.0 / D);
        z[0] = Z.x; z[1] = Z.y; z[2] = Z.z;
    };
    for (auto& kv : ring) {
        const int ei = kv.first[0], ej = kv.first[1];
        // order the ring: consecutive tetrahedra share one link vertex
        std::vector<std::array<int, 2>> L = kv.second;
        std::vector<int> cyc;
        {
            std::vector<char> used(L.size(), 0);
            int cur = 0;
            used[0] = 1;
            cyc.push_back(0);
            int next_v = L[0][1];
            for (size_t s = 1; s < L.size(); ++s) {
                int found = -1;
                for (size_t t = 0; t < L.size(); ++t)
                    if (!used[t] && (L[t][0] == next_v || L[t][1] == next_v)) { found = (int)t; break; }
                if (found < 0) break;
                used[found] = 1;
                cyc.push_back(found);
                next_v = L[found][0] == next_v ? L[found][1] : L[found][0];
                cur = found;
            }
            (void)cur;
        }
        for (int side = 0; side < 2; ++side) {
            const int own = side == 0 ? ei : ej, oth = side == 0 ? ej : ei;
            const double Ri = g.pts[own].R;
            double q[3], b;
            plane(own, oth, q, b);
            const double qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2], qn = std::sqrt(qq);
            const double u[3] = {q[0] / qn, q[1] / qn, q[2] / qn};
            const double h = b / qn;            // signed distance of the face plane from p_own
            const double rho2 = Ri * Ri - h * h;
            if (rho2 <= 0) continue;
            const double c[3] = {u[0] * h, u[1] * h, u[2] * h};
            // in-plane basis
            V3 nn = {u[0], u[1], u[2]}, e1, e2;
            basis(nn, e1, e2);
            std::vector<std::array<double, 2>> poly;
            for (int t : cyc) {
                double z[3];
                centre(own, oth, L[t][0], L[t][1], z);
                V3 d = {z[0] - c[0], z[1] - c[1], z[2] - c[2]};
                poly.push_back({dotv(d, e1), dotv(d, e2)});
            }
            double area = 0.0, m1 = 0.0, m2 = 0.0;
            const double r = std::sqrt(rho2);
            for (size_t k = 0; k < poly.size(); ++k) {
                const auto& P0 = poly[k];
                const auto& P1 = poly[(k + 1) % poly.size()];
                area += tri_disk_area(P0[0], P0[1], P1[0], P1[1], r);
                double mx, my;
                tri_disk_moment(P0[0], P0[1], P1[0], P1[1], r, mx, my);
                m1 += mx;
                m2 += my;
            }
            if (area < 0) { area = -area; m1 = -m1; m2 = -m2; }   // the ring's orientation
            vol[own] += h * area / 3.0;
            const double wo = w ? w[own] : 1.0, wt = w ? w[oth] : 1.0;
            // first moment of the in-ball face part relative to p_own: area c + in-plane part
            const double mom[3] = {area * c[0] + m1 * e1.x + m2 * e2.x, area * c[1] + m1 * e1.y + m2 * e2.y,
                                   area * c[2] + m1 * e1.z + m2 * e2.z};
            for (int k = 0; k < 3; ++k) grad[3 * own + k] += ((wo - wt) * mom[k] - wo * area * q[k]) / qn;
        }
    }
    for (int i = 0; i < n; ++i) vol[i] += g.pts[i].R * (double)A[i] / 3.0;
}

struct OracleHandle {
    Result res;
    std::string err;
};

extern "C" {

OracleHandle* oracle_build(int n, const double* xyz, const double* radii, double probe, char* err, int errlen) {
    auto h = std::make_unique<OracleHandle>();
    try {
        build(h->res, n, xyz, radii, probe);
    } catch (const std::exception& e) {
        if (err && errlen > 0) { std::snprintf(err, (size_t)errlen, "%s", e.what()); }
        return nullptr;
    }
    return h.release();
}

void oracle_free(OracleHandle* h) { delete h; }

// counts: [0] rt tets (4 atoms), [1] rt tets incl. far, [2] |C0|, [3] |C1|, [4] |C2|, [5] |C3|,
// [6] redundant atoms, [7] rt triangles (atoms only), [8] rt edges, [9] exact power tests,
// [10] SoS fallbacks, [11] alpha predicates, [12] orient tests, [13] degenerate insertions
void oracle_counts(const OracleHandle* h, long* out) {
    const Result& r = h->res;
    long red = 0;
    for (char c : r.redundant) red += c;
    long v[14] = {(long)r.rt_tets.size(), r.rt_tets_total, (long)r.kv.size(), (long)r.ke.size(),
                  (long)r.kt.size(), (long)r.kT.size(), red, r.rt_tris, r.rt_edges, r.g.cnt.power,
                  r.g.cnt.sos, r.g.cnt.alpha, r.g.cnt.orient, r.degenerate_hits};
    for (int k = 0; k < 14; ++k) out[k] = v[k];
}

void oracle_times(const OracleHandle* h, double* out) { out[0] = h->res.t_rt; out[1] = h->res.t_alpha; }

void oracle_term_counts(const OracleHandle* h, long* out) { count_terms(h->res, out); }

// dim 0..3: the dual complex's simplices (sorted tuples, lexicographic); dim 4: all
// triangulation tetrahedra with four atoms
void oracle_simplices(const OracleHandle* h, int dim, int* out) {
    const Result& r = h->res;
    size_t k = 0;
    if (dim == 0) for (int v : r.kv) out[k++] = v;
    if (dim == 1) for (auto& e : r.ke) { out[k++] = e[0]; out[k++] = e[1]; }
    if (dim == 2) for (auto& t : r.kt) { out[k++] = t[0]; out[k++] = t[1]; out[k++] = t[2]; }
    if (dim == 3) for (auto& t : r.kT) for (int j = 0; j < 4; ++j) out[k++] = t[j];
    if (dim == 4) for (auto& t : r.rt_tets) for (int j = 0; j < 4; ++j) out[k++] = t[j];
}

void oracle_redundant(const OracleHandle* h, unsigned char* out) {
    for (int i = 0; i < h->res.n; ++i) out[i] = (unsigned char)h->res.redundant[i];
}

// areas[n]; grad[3n] (may be NULL) = d(sum_i w_i A_i)/dx; weights NULL = ones.
// returns the number of triangles without a triple point (must be 0)
long oracle_areas(const OracleHandle* h, const double* weights, double* areas, double* grad, double* total) {
    Areas a;
    compute_areas(h->res, weights, grad != nullptr, a);
    long double tot = 0;
    for (int i = 0; i < h->res.n; ++i) { areas[i] = (double)a.A[i]; tot += a.A[i]; }
    if (total) *total = (double)tot;
    if (grad) for (int k = 0; k < 3 * h->res.n; ++k) grad[k] = a.G[k];
    return a.n_tri_bad;
}

// as oracle_areas with the term loops on nthreads OpenMP threads (timing only); returns the
// number of threads the build supports in *used (1 without OpenMP)
long oracle_areas_parallel(const OracleHandle* h, const double* weights, double* areas, double* grad, double* total,
                           int nthreads, int* used) {
#ifdef _OPENMP
    const int t = nthreads > 0 ? nthreads : 1;
#else
    const int t = 1;
#endif
    if (used) *used = t;
    Areas a;
    compute_areas_parallel(h->res, weights, grad != nullptr, a, t);
    long double tot = 0;
    for (int i = 0; i < h->res.n; ++i) { areas[i] = (double)a.A[i]; tot += a.A[i]; }
    if (total) *total = (double)tot;
    if (grad) for (int k = 0; k < 3 * h->res.n; ++k) grad[k] = a.G[k];
    return a.n_tri_bad;
}

// per-atom volumes vol(B_i cap L_i) [n], d(sum_i w_i V_i)/dx [3n] (may be NULL; weights NULL
// = ones: the gradient of the union volume), total volume
long oracle_volumes(const OracleHandle* h, const double* weights, double* volumes, double* grad, double* total) {
    Areas a;
    compute_areas(h->res, nullptr, false, a);
    std::vector<double> v, g;
    compute_volumes(h->res, a.A, v, g, weights);
    long double tot = 0;
    for (int i = 0; i < h->res.n; ++i) { volumes[i] = v[i]; tot += v[i]; }
    if (total) *total = (double)tot;
    if (grad) for (int k = 0; k < 3 * h->res.n; ++k) grad[k] = g[k];
    return a.n_tri_bad;
}

// Gauss-Bonnet exposed areas; returns the number of spheres whose arc structure was not
// generic (their value is unreliable)
int oracle_gauss_bonnet(int n, const double* xyz, const double* radii, double probe, double* areas) {
    double rmax = 0;
    for (int i = 0; i < n; ++i) rmax = std::max(rmax, radii[i] + probe);
    double cell = 2.0 * rmax + 1e-9;
    std::unordered_map<long long, std::vector<int>> grid;
    auto key = [&](long long x, long long y, long long z) { return (x * 73856093LL) ^ (y * 19349663LL) ^ (z * 83492791LL); };
    std::vector<std::array<long long, 3>> cid(n);
    for (int i = 0; i < n; ++i) {
        for (int k = 0; k < 3; ++k) cid[i][k] = (long long)std::floor(xyz[3 * i + k] / cell);
        grid[key(cid[i][0], cid[i][1], cid[i][2])].push_back(i);
    }
    int bad = 0;
    for (int i = 0; i < n; ++i) {
        std::vector<int> nb;
        for (int dx = -1; dx <= 1; ++dx)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dz = -1; dz <= 1; ++dz) {
                    auto it = grid.find(key(cid[i][0] + dx, cid[i][1] + dy, cid[i][2] + dz));
                    if (it == grid.end()) continue;
                    for (int j : it->second) {
                        if (j == i) continue;
                        if (std::llabs(cid[j][0] - cid[i][0]) > 1 || std::llabs(cid[j][1] - cid[i][1]) > 1 ||
                            std::llabs(cid[j][2] - cid[i][2]) > 1) continue;
                        nb.push_back(j);
                    }
                }
        std::sort(nb.begin(), nb.end());
        nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
        bad += gb_sphere(i, n, xyz, radii, probe, nb, &areas[i]);
    }
    return bad;
}

// The triangle term S_123^(1) of Eq. (trianglev) for three spheres (radii already include
// the probe), with its gradient (9 values, d/dp1, d/dp2, d/dp3). Returns 0 if no triple point.
int oracle_tri_term(const double* p1, const double* p2, const double* p3, double R1, double R2, double R3,
                    double* value, double* grad9) {
    DV P1 = seed_point(p1, 0), P2 = seed_point(p2, 1), P3 = seed_point(p3, 2);
    bool ok = true;
    Dual S = tri_term(P1, P2, P3, R1, R2, R3, &ok);
    *value = S.v;
    if (grad9) for (int k = 0; k < 9; ++k) grad9[k] = S.d[k];
    return ok ? 1 : 0;
}

// exact sign predicates exposed for tests: kind 0 orient(a,b,c,d), 1 conflict(a,b,c,d;e),
// 2 tet psi(a,b,c,d), 3 triangle psi(a,b,c), 4 edge psi(a,b), 5 e attaches triangle (a,b,c),
// 6 e attaches edge (a,b), 7 e attaches vertex a (5-7 return 1 when attached, else 0)
int oracle_predicate(int kind, int npts, const double* xyzR, const int* ids) {
    Geo g;
    g.n = npts;
    for (int i = 0; i < npts; ++i) {
        g.pts.push_back({xyzR[4 * i], xyzR[4 * i + 1], xyzR[4 * i + 2], xyzR[4 * i + 3]});
        g.P.push_back({big(xyzR[4 * i]), big(xyzR[4 * i + 1]), big(xyzR[4 * i + 2])});
        Big R = big(xyzR[4 * i + 3]);
        g.W.push_back(R * R);
    }
    switch (kind) {
        case 0: return g.orient(ids[0], ids[1], ids[2], ids[3]);
        case 1: return g.conflict(ids[0], ids[1], ids[2], ids[3], ids[4]) ? -1 : 1;
        case 2: return g.tet_psi(ids[0], ids[1], ids[2], ids[3]);
        case 3: return g.tri_psi(ids[0], ids[1], ids[2]);
        case 4: return g.edge_psi(ids[0], ids[1]);
        case 5: return g.tri_attached(ids[0], ids[1], ids[2], ids[3]) ? 1 : 0;
        case 6: return g.edge_attached(ids[0], ids[1], ids[2]) ? 1 : 0;
        case 7: return g.vertex_attached(ids[0], ids[1]) ? 1 : 0;
    }
    return 0;
}

}  // extern "C"
