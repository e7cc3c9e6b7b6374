// The per-atom kernels: a warp builds atom i's restricted Laguerre cell, classifies the
// simplices of the dual complex C that contain i, and evaluates A_i and the gradient entry
// of atom i (and, on request, the atom's molecular-volume share).
//
//   Step 1 (paper): the weighted Delaunay tetrahedra around i are the vertices of the power
//     cell L_i.  The warp starts from a cube (6 ghost planes at distance h > R_i) and clips
//     it by the power bisector of every neighbour whose ball overlaps B_i (all other
//     neighbours cannot cut L_i inside B_i, so L_i cap B_i is exact).  The cell is stored as
//     its dual triangulation: a vertex = a triangle (a, b, c) of plane ids, counter-clockwise
//     seen from outside, with the three adjacent triangles.  Clipping by plane m removes the
//     vertices strictly beyond m (an exact predicate), and re-triangulates the hole with a
//     fan around m along the boundary cycle of the removed region.
//   Step 2: a cell vertex (a,b,c) is a tetrahedron of C iff it lies in B_i (psi <= 0); a cell
//     edge (a,b) is a triangle of C iff it meets B_i (its orthocentre lies on it with psi <= 0,
//     or an end vertex is in C); a face a is an edge of C iff it meets B_i; i is a vertex of C
//     iff its cell meets B_i.  A vertex / edge / triangle whose tetrahedra close around it is
//     interior (coefficient exactly 0, skipped).
//   Step 3: A_i by Eq. (sainexclu); the gradient entry of atom i gathers, over the simplices
//     of C containing i, the derivative of every atom's terms (Eq. inexclu) - no atomics.
//
// One warp per atom (two per block); the cell lives in shared memory (plane table, triangle
// table) and in registers (each lane caches the homogeneous coordinates of up to NT / 32
// cell vertices).  The fast path runs the steps as separate kernels that hand the cell over
// through a per-atom record in HBM (PH_CELL: Step 1; PH_CLASS: Step 2; PH_TERMS: Step 3;
// PH_VOL: the volume), so that each kernel's code fits the instruction cache.  When all atoms
// fit in one wave, Steps 1 and 2 run as one kernel (PH_CC), so that classifications overlap
// the slowest cells.  With carried cells, Step 1 is PH_CARRY (on calls reusing the neighbour
// lists, each atom's cell from the previous call, kept when exact predicates certify it) and
// then PH_CELL over the atoms it could not keep.  The fused form (PH_ALL) serves the
// large-capacity pass and the no-allocation entry point.
#pragma once
#include "dsasa_kernels.cuh"
#include "dsasa_math.cuh"

#include <stddef.h>
#include <stdint.h>

namespace dsasa {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int NG = 6;            // ghost planes (the initial cube)
constexpr uint8_t NONE = 0xff;
// warps per block (a warp that finishes frees its slot at once): fused, cell, classification
// and terms kernels
constexpr int WARPS = 1, WARPS_CELL = 2, WARPS_CLASS = 2, WARPS_TERMS = 2;
// resident blocks per SM that each kernel's register budget is sized for (one warp each)
constexpr int MINB = 32, MINB_CELL = 18, MINB_CLASS = 18, MINB_TERMS = 18;

// kernel phases: the whole computation in one kernel, or three kernels that pass the cell
// through a global record per atom: the cell construction (gather, sort, clipping), the
// classification (Steps 2a-2c: which simplices of the cell are in C), and the area terms and
// gradient.  Each kernel's code then fits the instruction cache.
enum { PH_ALL = 0, PH_CELL = 1, PH_CLASS = 2, PH_TERMS = 3, PH_VOL = 4, PH_CC = 5, PH_CARRY = 6 };
enum { CELL_OK = 0, CELL_DONE = 1 };   // record flag: CELL_DONE = outputs already written

// Per-warp cell storage.  NE plane entries (0..5 ghosts, then the candidates in sorted
// order), NT cell-vertex slots (NT / 32 per lane).  Two capacities are compiled: 64 / 64
// holds every atom of the molecular workloads measured (at most 58 overlapping neighbours,
// 54 vertex slots); atoms that do not fit are deferred to a 128 / 128 pass.
template <class R, int NE, int NT> struct Smem {
    using Real = R;
    static constexpr int kNE = NE, kNT = NT;
    alignas(16) R pq[NE][4];   // plane q.x, q.y, q.z, b (relative to p_i)
    R pB[NE];             // magnitude proxy of b for the filters
    int pg[NE];           // global atom index (>= 0) or -1 - ghost id
    uint8_t start[NE];    // a vertex slot on the face of this plane
    // boundary edges of the current cut, by number: (a, b, kept neighbour slot, new slot, edge
    // index in the kept neighbour) packed 7/7/7/7/2 bits; the new slot by first and last plane
    unsigned bedge[NE];
    uint8_t bslot[NE], eslot[NE];
    uint8_t ord[NE];      // clipping order (entry ids)
    uint8_t eflag[NE];    // face summary: bit0 edge in C, bit1 interior (closed)
    R ephi[NE];           // Phi_ia of the face
    uchar4 tv[NT];        // cell vertex = triangle of plane ids (x = NONE: dead slot)
    uchar4 ta[NT];        // neighbour slots across edges (v0 v1), (v1 v2), (v2 v0)
    uint8_t kf[NT];       // 0 not in C, 1 tetrahedron of C, 2 involves a ghost plane
    unsigned tf[NT];      // bit k: the triangle of edge k is in C; bit 4+k: it is processed here
    unsigned skey[NE];    // orderable sort key of each candidate
    uint16_t tl[NT * 3 / 2 + 2];   // compacted exterior triangles (slot << 2 | edge)
    uint8_t rem[NT];
    uint8_t rsl[NT];      // removed slots in order
    uint8_t fs[NT];       // free slot stack
    int hw, nfree, bad;
};

// The cell of one atom between the two kernels (first NG + nc plane entries, first hw
// vertex slots used).
template <class R, int NE, int NT> struct CellRec {
    alignas(16) R pq[NE][4];
    R pB[NE];
    int pg[NE];
    uchar4 tv[NT];
    uchar4 ta[NT];
    uint8_t start[NE];
    uint8_t kf[NT];       // classification (the Smem fields of the same names)
    uint8_t tf[NT];
    uint8_t eflag[NE];
    int iK, icl;
    int nc, hw, flag;
    int atom;             // the atom whose cell this is (-1: no cell), for carrying it to the next call
};
using CellRecF = CellRec<float, 64, 64>;
using CellRecD = CellRec<double, 64, 64>;
static_assert(offsetof(CellRecF, iK) % 16 == 0 && offsetof(CellRecD, iK) % 16 == 0,
              "the record header (iK, icl, nc, hw) is read as one 16-byte load");
// The plane rows move in 16-byte pieces (copy_row, load_row, store_row): every row of the
// shared table and of a record must start on a 16-byte boundary.  Records are indexed as an
// array of CellRec (and the per-warp tables as an array of Smem), so their sizes must keep
// the next element's rows aligned too.
template <class R, int NE, int NT> constexpr bool rows_aligned() {
    using SM = Smem<R, NE, NT>;
    using RC = CellRec<R, NE, NT>;
    return offsetof(SM, pq) % 16 == 0 && sizeof(R[4]) % 16 == 0 && sizeof(SM) % 16 == 0 &&
           offsetof(RC, pq) % 16 == 0 && sizeof(RC) % 16 == 0 && alignof(SM) >= 16 && alignof(RC) >= 16;
}
static_assert(rows_aligned<float, 64, 64>() && rows_aligned<double, 64, 64>() && rows_aligned<float, 128, 128>() &&
                  rows_aligned<double, 128, 128>(),
              "16-byte plane-row moves need 16-byte aligned rows in every table and record");

// one plane row (4 values of R) between the shared table and a cell record, 16-byte moves
template <class R> __device__ __forceinline__ void copy_row(R* dst, const R* src) {
    if constexpr (sizeof(R) == 4) {
        *(float4*)dst = *(const float4*)src;
    } else {
        ((double2*)dst)[0] = ((const double2*)src)[0];
        ((double2*)dst)[1] = ((const double2*)src)[1];
    }
}

// a plane row held in registers (16-byte loads and stores)
template <class R> struct Row4 {
    R v[4];
};
template <class R> __device__ __forceinline__ Row4<R> load_row(const R* src) {
    Row4<R> r;
    if constexpr (sizeof(R) == 4) {
        const float4 f = *(const float4*)src;
        r.v[0] = f.x; r.v[1] = f.y; r.v[2] = f.z; r.v[3] = f.w;
    } else {
        const double2 d0 = ((const double2*)src)[0], d1 = ((const double2*)src)[1];
        r.v[0] = d0.x; r.v[1] = d0.y; r.v[2] = d1.x; r.v[3] = d1.y;
    }
    return r;
}
template <class R> __device__ __forceinline__ void store_row(R* dst, const Row4<R>& r) {
    if constexpr (sizeof(R) == 4) {
        *(float4*)dst = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
    } else {
        ((double2*)dst)[0] = make_double2(r.v[0], r.v[1]);
        ((double2*)dst)[1] = make_double2(r.v[2], r.v[3]);
    }
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ int warp_sum_i(int v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}
// A lane's sum of gradient contributions.  In the FP32 form every contribution is added
// exactly as a fixed-point integer (the float value times 2^40, rounded to an int64): the sum
// is exact and independent of the summation order (the contributions gathered for one atom
// largely cancel, and a plain float sum would carry an error of about 2^-24 times the largest
// partial sum); 2^-40 is far below the contributions' own rounding and 2^63 / 2^40 leaves room
// for sums up to 8e6.  The FP64 form sums in double.
constexpr float GFIX = 1099511627776.0f;   // 2^40
template <class R> struct GAcc;
template <> struct GAcc<float> {
    long long x = 0, y = 0, z = 0;
    __device__ __forceinline__ void add(float a, float b, float c) {
        x += __float2ll_rn(a * GFIX);
        y += __float2ll_rn(b * GFIX);
        z += __float2ll_rn(c * GFIX);
    }
    // warp sum (exact: every lane ends with the same value)
    __device__ __forceinline__ void reduce(double& gx, double& gy, double& gz) {
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_xor_sync(FULL, x, o);
            y += __shfl_xor_sync(FULL, y, o);
            z += __shfl_xor_sync(FULL, z, o);
        }
        gx = (double)x * (1.0 / (double)GFIX);
        gy = (double)y * (1.0 / (double)GFIX);
        gz = (double)z * (1.0 / (double)GFIX);
    }
};
template <> struct GAcc<double> {
    double x = 0.0, y = 0.0, z = 0.0;
    __device__ __forceinline__ void add(double a, double b, double c) { x += a; y += b; z += c; }
    __device__ __forceinline__ void reduce(double& gx, double& gy, double& gz) {
        gx = warp_sum_d(x);
        gy = warp_sum_d(y);
        gz = warp_sum_d(z);
    }
};
__device__ __forceinline__ uint8_t tv_get(const uchar4& v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }
template <class SM> __device__ __forceinline__ void ta_set(SM* S, int t, int k, uint8_t s) {
    ((uint8_t*)&S->ta[t & (SM::kNT - 1)])[k] = s;
}

// ------------------------------------------------------------------ global plane access
struct Ctx {
    const double* xyz;
    const double* R;
    double pi[3];
    double Ri;
    double h;
    int i;
    int n;          // atoms (the range of plane owners)
    int* status;
};

__device__ void plane64_of(const Ctx& c, int g, double q[3], double& b, double& babs, bool& exact) {
    if (g < 0) {
        ghost_plane64(-1 - g, c.h, q, b);
        babs = fabs(b);
        exact = true;
        return;
    }
    g = DS_IDX(g, c.n, c.status);
    double pk[3] = {c.xyz[3 * g], c.xyz[3 * g + 1], c.xyz[3 * g + 2]};
    plane64(c.pi, c.Ri, pk, c.R[g], q, b, babs);
    exact = false;
}
__device__ PlaneN<FA<double>> fa64_of(const Ctx& c, int g) {
    double q[3], b, babs;
    bool ex;
    plane64_of(c, g, q, b, babs, ex);
    return fa_plane64(q, b, babs, ex);
}
__device__ PlaneN<XP> xp_of(const Ctx& c, int g) {
    if (g < 0) return xp_ghost(-1 - g, c.h);
    g = DS_IDX(g, c.n, c.status);
    double pk[3] = {c.xyz[3 * g], c.xyz[3 * g + 1], c.xyz[3 * g + 2]};
    return xp_plane(c.pi, c.Ri, pk, c.R[g]);
}

// one more atom of atom i's molecule has final outputs (lane 0 wrote them): count it after a
// system-scope fence; the molecule's last atom raises its ready flag (out of line: cold code)
__device__ __noinline__ void molecule_count(const AtomArgs& A, int i) {
    __threadfence_system();
    const int m = A.molid[i];
    const int size = (int)(A.mol_off[m + 1] - A.mol_off[m]);
    if (atomicAdd(A.mol_done + m, 1) + 1 == size) {
        // every other atom of the molecule fenced its outputs before counting itself, so the
        // outputs are complete; tell the host
        __threadfence_system();
        *(volatile int*)(A.mol_ready + m) = 1;
    }
}

// predicate kinds
enum { PK_CLIP = 0, PK_TET = 1, PK_TRI = 2, PK_TRIB = 3, PK_EDGE = 4, PK_EDGEB = 5, PK_VERT = 6 };

template <class N> __device__ N eval_kind(int kind, const PlaneN<N>* P, const N& wi) {
    switch (kind) {
        case PK_CLIP: return pred_clip(P[0], P[1], P[2], P[3]);
        case PK_TET: return pred_tet_psi(P[0], P[1], P[2], wi);
        case PK_TRI: return pred_tri_psi(P[0], P[1], wi);
        case PK_TRIB: return pred_tri_beyond(P[0], P[1], P[2]);
        case PK_EDGE: return pred_edge_psi(P[0], wi);
        case PK_EDGEB: return pred_edge_beyond(P[0], P[1]);
        default: return P[0].b;
    }
}
__device__ __forceinline__ int kind_planes(int kind) {
    return kind == PK_CLIP ? 4 : (kind == PK_TET || kind == PK_TRIB) ? 3 : (kind == PK_TRI || kind == PK_EDGEB) ? 2 : 1;
}

// Slow path: FP64 filter (unless skip64), then exact expansions.  An exact zero of the clip
// test (a vertex exactly on a bisector: co-spherical atoms) is broken by Simulation of
// Simplicity on the weights, as the regular triangulation breaks its ties (sos_clip_sign);
// an exact zero of a test of the dual complex (psi = 0, an orthocentre exactly on a plane) is
// a decision of its own (psi <= 0 is in C; "beyond" is strict) and is returned as 0.
__device__ __noinline__ int resolve_exact(const Ctx& c, int kind, int g0, int g1, int g2, int g3, bool try64) {
    int gs[4] = {g0, g1, g2, g3};
    int np = kind_planes(kind);
    if (try64) {
        PlaneN<FA<double>> P[4];
        for (int k = 0; k < np; ++k) P[k] = fa64_of(c, gs[k]);
        FA<double> wi = {c.Ri * c.Ri, c.Ri * c.Ri};
        int s = fa_sign(eval_kind(kind, P, wi), G64, TINY64);
        if (s != 0) return s;
    }
    PlaneN<XP> P[4];
    for (int k = 0; k < np; ++k) P[k] = xp_of(c, gs[k]);
    XP wi = xp_sq(c.Ri);
    XP v = eval_kind(kind, P, wi);
    if (v.ovf) {
        atomicOr(c.status, ST_UNRESOLVED);
        return v.n ? (v.c[v.n - 1] > 0 ? 1 : -1) : 0;
    }
    int s = xp_sign(v);
    if (s == 0 && kind == PK_CLIP) {
        s = sos_clip_sign(P, gs, c.i);
        if (s == 0) atomicOr(c.status, ST_DEGENERATE);   // coincident atoms: no perturbation separates them
    }
    return s;
}

// filter planes from the shared table
template <class SM, class R = typename SM::Real> __device__ __forceinline__ PlaneN<FA<R>> fplane(const SM* S, int e) {
    e &= SM::kNE - 1;
    PlaneN<FA<R>> P;
    P.q = {{S->pq[e][0], fabs(S->pq[e][0])}, {S->pq[e][1], fabs(S->pq[e][1])}, {S->pq[e][2], fabs(S->pq[e][2])}};
    P.b = {S->pq[e][3], S->pB[e]};
    return P;
}
// homogeneous cell vertex (Dv, D) of the planes of triangle v, with magnitudes for the filter
template <class R> struct VtxFA { R v[4], a[4]; };
template <class SM, class R = typename SM::Real> __device__ __forceinline__ VtxFA<R> vertex_fa_inl(const SM* S, uchar4 v) {
    PlaneN<FA<R>> Pa = fplane(S, v.x), Pb = fplane(S, v.y), Pc = fplane(S, v.z);
    V3<FA<R>> Dv;
    FA<R> D;
    vertex_hom(Pa, Pb, Pc, Dv, D);
    return {{Dv.x.v, Dv.y.v, Dv.z.v, D.v}, {Dv.x.a, Dv.y.a, Dv.z.a, D.a}};
}
// out of line (the kernels that also classify or evaluate terms keep their code small)
template <class SM, class R = typename SM::Real> __device__ __noinline__ VtxFA<R> vertex_fa(const SM* S, uchar4 v) {
    return vertex_fa_inl(S, v);
}
// Volume pieces of the restricted cell (molecular volume, the paper's named extension).  For
// every face f of the cell (plane q_f . z = b_f, unit normal u_f, signed distance h_f from
// p_i), the polygon is split by the fan from the centre of the disk B_i cap plane_f into
// the area s_f inside the ball and o_f outside it.  By the divergence theorem over the
// closed surface of B_i cap L_i:  V_i = (R_i A_i + sum_f h_f s_f) / 3.  The exposed sphere
// piece has vector area -sum_f s_f u_f = d vol(union) / d p_i; since the whole cell's faces
// have zero vector area, that is +sum_f o_f u_f, which vanishes exactly (no cancellation)
// when the cell lies inside the ball.  With volume weights (vw != NULL) the gradient of
// sum_i w_i V_i also needs, for every face towards an atom k, the first moment m_f of its part
// inside the ball (relative to p_i): moving p_k moves only that face, by
// dV_i/dp_k = (s_f q_k - m_f) / |q_k|, and the face is the same polygon in k's cell; the
// weighted entry is w_i (the unweighted one) + sum_f (w_i - w_k) m_f / |q_f| (wx, wy, wz).
// Per lane: partial sums over faces.
template <class SM, class R = typename SM::Real>
__device__ void cell_volume_terms(const SM* S, int nc, R Ri, int lane, const double* vw, R wi, int n, int* status,
                                  R& hs, R& nx, R& ny, R& nz, R& wx, R& wy, R& wz) {
    constexpr int NT = SM::kNT, NE = SM::kNE;
    hs = nx = ny = nz = wx = wy = wz = (R)0;
    for (int a = lane; a < NG + nc; a += 32) {
        const int st0 = S->start[a];
        if (st0 == NONE) continue;
        const int st = st0 & (NT - 1);
        {
            const uchar4 v = S->tv[st];
            if (!(v.x == a || v.y == a || v.z == a)) continue;   // face clipped away
        }
        const R qx = S->pq[a][0], qy = S->pq[a][1], qz = S->pq[a][2], b = S->pq[a][3];
        const R inv = (R)1 / ds_sqrt(qx * qx + qy * qy + qz * qz);
        const R h = b * inv;
        const R rho2 = Ri * Ri - h * h;
        const R r = rho2 > (R)0 ? ds_sqrt(rho2) : (R)0;
        const P3<R> u = {qx * inv, qy * inv, qz * inv};
        const P3<R> tt = fabs(u.x) < (R)0.6 ? P3<R>{(R)1, (R)0, (R)0} : (fabs(u.y) < (R)0.6 ? P3<R>{(R)0, (R)1, (R)0} : P3<R>{(R)0, (R)0, (R)1});
        P3<R> e1 = cross3(u, tt);
        e1 = e1 * ((R)1 / norm3(e1));
        const P3<R> e2 = cross3(u, e1);
        int t = st;
        R fx = 0, fy = 0, px = 0, py = 0, sin_ = 0, sout = 0, m1 = 0, m2 = 0;
        const int gk = S->pg[a];   // < 0: a ghost plane
        const bool moments = vw != nullptr && gk >= 0 && r > (R)0;
        auto fan = [&](R ax, R ay, R bx, R by) {
            const R full = (R)0.5 * (ax * by - ay * bx);
            if (r > (R)0 && ax * ax + ay * ay <= rho2 && bx * bx + by * by <= rho2) {
                sin_ += full;   // wholly inside: nothing outside
            } else {
                const R in = r > (R)0 ? tri_disk_area_ol(ax, ay, bx, by, r) : (R)0;
                sin_ += in;
                sout += full - in;
            }
            if (moments) {
                const T2<R> mm = tri_disk_moment_ol(ax, ay, bx, by, r);
                m1 += mm.x;
                m2 += mm.y;
            }
        };
        for (int step = 0; step < NT; ++step) {
            const uchar4 v = S->tv[t];
            // cell vertex (planes v.x, v.y, v.z): z = Dv / D
            const P3<R> A3 = ppos(S, v.x), B3 = ppos(S, v.y), C3 = ppos(S, v.z);
            const R ba = S->pq[v.x & (NE - 1)][3], bb = S->pq[v.y & (NE - 1)][3], bc = S->pq[v.z & (NE - 1)][3];
            const P3<R> xbc = cross3(B3, C3), xca = cross3(C3, A3), xab = cross3(A3, B3);
            const R D = dot3(A3, xbc);
            const P3<R> z = (xbc * ba + xca * bb + xab * bc) * ((R)1 / D);
            const P3<R> d = {z.x - u.x * h, z.y - u.y * h, z.z - u.z * h};
            const R cx = dot3(d, e1), cy = dot3(d, e2);
            if (step == 0) { fx = cx; fy = cy; }
            else fan(px, py, cx, cy);
            px = cx;
            py = cy;
            const int k = v.x == a ? 0 : (v.y == a ? 1 : 2);
            t = tv_get(S->ta[t], k) & (NT - 1);
            if (t == st) break;
        }
        fan(px, py, fx, fy);
        // the fan runs around the face the same way for every face of the cell: a common sign
        const R sg = sin_ + sout < (R)0 ? (R)-1 : (R)1;
        hs += h * sin_ * sg;
        nx += sout * sg * u.x;
        ny += sout * sg * u.y;
        nz += sout * sg * u.z;
        if (moments) {
            // m_f = s_f (h u) + m1 e1 + m2 e2, scaled by (w_i - w_k) / |q_f|
            const R f = (wi - (R)vw[DS_IDX(gk, n, status)]) * inv * sg;
            wx += f * (sin_ * h * u.x + m1 * e1.x + m2 * e2.x);
            wy += f * (sin_ * h * u.y + m1 * e1.y + m2 * e2.y);
            wz += f * (sin_ * h * u.z + m1 * e1.z + m2 * e2.z);
        }
    }
}

template <class R> struct Gam;
template <> struct Gam<float> {
    static constexpr float g = G32, gclip = G32_CLIP, tiny = TINY32;
    static constexpr bool try64 = true;
};
template <> struct Gam<double> {
    static constexpr double g = G64, gclip = G64, tiny = TINY64;
    static constexpr bool try64 = false;
};

template <int KIND, class N> __device__ __forceinline__ N eval_k(const PlaneN<N>* P, const N& wi) {
    if constexpr (KIND == PK_CLIP) return pred_clip(P[0], P[1], P[2], P[3]);
    else if constexpr (KIND == PK_TET) return pred_tet_psi(P[0], P[1], P[2], wi);
    else if constexpr (KIND == PK_TRI) return pred_tri_psi(P[0], P[1], wi);
    else if constexpr (KIND == PK_TRIB) return pred_tri_beyond(P[0], P[1], P[2]);
    else if constexpr (KIND == PK_EDGE) return pred_edge_psi(P[0], wi);
    else if constexpr (KIND == PK_EDGEB) return pred_edge_beyond(P[0], P[1]);
    else return P[0].b;
}

// sign of predicate KIND on shared-table planes e0..e3 (FP32/FP64 filter, then slow path)
template <int KIND, class SM, class R = typename SM::Real>
__device__ __noinline__ int psign(const SM* S, const Ctx& c, const FA<R>& wi, int e0, int e1, int e2 = 0, int e3 = 0) {
    PlaneN<FA<R>> P[4] = {fplane(S, e0), fplane(S, e1), fplane(S, e2), fplane(S, e3)};
    int s = fa_sign(eval_k<KIND>(P, wi), Gam<R>::g, Gam<R>::tiny);
    if (s != 0) return s;
    const int kind = KIND;
    constexpr int M = SM::kNE - 1;
    return resolve_exact(c, kind, S->pg[e0 & M], S->pg[e1 & M], S->pg[e2 & M], S->pg[e3 & M], Gam<R>::try64);
}

// the filter alone (inline): the certified sign, or 0 when the filter leaves it open
template <int KIND, class SM, class R = typename SM::Real>
__device__ __forceinline__ int fsign(const SM* S, const FA<R>& wi, int e0, int e1, int e2 = 0) {
    PlaneN<FA<R>> P[4] = {fplane(S, e0), fplane(S, e1), fplane(S, e2), fplane(S, e2)};
    return fa_sign(eval_k<KIND>(P, wi), Gam<R>::g, Gam<R>::tiny);
}

template <class SM, class R = typename SM::Real> __device__ __forceinline__ P3<R> ppos(const SM* S, int e) {
    e &= SM::kNE - 1;
    return {S->pq[e][0], S->pq[e][1], S->pq[e][2]};
}

// ------------------------------------------------------------------ the initial cube
// Corner t of the cube of the 6 ghost planes (bit 0 / 1 / 2 of t: the -x / -y / -z side): the
// triangle of its three planes, oriented like every cell vertex (positive orientation).
__host__ __device__ constexpr int cube_corner_plane(int t, int k) {
    const int sx = (t & 1) ? -1 : 1, sy = (t & 2) ? -1 : 1, sz = (t & 4) ? -1 : 1;
    const int px = sx > 0 ? 0 : 1, py = sy > 0 ? 2 : 3, pz = sz > 0 ? 4 : 5;
    const bool even = sx * sy * sz > 0;
    return k == 0 ? (even ? px : py) : (k == 1 ? (even ? py : px) : pz);
}
// The corner across edge k (from plane k to plane k + 1 of the triangle) of every corner,
// one byte per corner: the cube's adjacency, computed at compile time.
__host__ __device__ constexpr unsigned long long cube_adjacency(int k) {
    unsigned long long packed = 0;
    for (int t = 0; t < 8; ++t) {
        const int a = cube_corner_plane(t, k), b = cube_corner_plane(t, (k + 1) % 3);
        for (int t2 = 0; t2 < 8; ++t2)
            for (int k2 = 0; k2 < 3; ++k2)
                if (cube_corner_plane(t2, k2) == b && cube_corner_plane(t2, (k2 + 1) % 3) == a)
                    packed |= (unsigned long long)t2 << (8 * t);
    }
    return packed;
}
constexpr unsigned long long CUBE_ADJ0 = cube_adjacency(0), CUBE_ADJ1 = cube_adjacency(1),
                             CUBE_ADJ2 = cube_adjacency(2);
static_assert(CUBE_ADJ0 == 0x0302010007060504ull && CUBE_ADJ1 == 0x0507040602000301ull &&
                  CUBE_ADJ2 == 0x0604070501030002ull,
              "every edge of the cube's triangulation has exactly one neighbour across it");

// ------------------------------------------------------------------ carried cells
// The incremental update of C across MD steps.  On a call that reuses the neighbour lists
// (every atom within half the skin of its last rebuild), the cell that the previous call
// built for atom i is carried to the current positions when exact predicates certify it,
// instead of being clipped again from the cube.
//
// Any set F of planes of other atoms may bound the cell: each half-space contains the true
// Laguerre cell, and the half-space of an atom whose ball does not meet B_i contains B_i, so
// the cell cut by F and by the current candidates meets B_i exactly where the cell of the
// candidates does (its vertices inside B_i, and so every simplex of C, are the same).  The
// record gives F (the previous cell's faces, ghosts included) and the dual triangulation of
// their polytope.  With every vertex recomputed from its three current planes, the structure
// is that polytope when (i) every vertex has a certified positive orientation and (ii) every
// vertex lies strictly inside every other face plane of F.  Then each vertex is a simple
// vertex of the polytope, and its edge along the line of two of its planes ends at the
// structure's neighbour across that edge: both lie on the line, each strictly inside the
// other's third plane and strictly inside every remaining plane.  The structure, closed under
// that adjacency, holds every vertex of the polytope (whose vertex-edge graph is connected),
// and the polytope is bounded.  When, in addition, no current candidate outside F removes a
// vertex, the structure is the cell.  The carry kernel (PH_CARRY) keeps exactly those cells;
// every other atom (no usable record, a failed certification, a new candidate that cuts, or
// lists not reused) goes to a redo list that the plain cell kernel then builds from the cube,
// so the carry kernel holds no clipping code.
//
// carry_cell reads the record, checks its structure (plane ids in range, every edge's two
// triangles pointing at each other with the edge reversed, every face's start slot on that
// face, V = 2F - 4 for the closed triangulation of a sphere), renumbers the faces NG.. in
// record order with the other candidates after them, and sets up the shared tables:
// triangles, adjacency, free slots (the dead slots below the high-water mark), the test order
// (ghost faces, faces, other candidates) and each face's start slot, staged in rem[] for the
// caller.  It returns nc | ncert << 8 | nclip << 16 | nalive << 24, or 0 when the record
// gives no usable structure.
template <class SM, class RC>
__device__ __noinline__ int carry_cell(SM* S, const RC* rec, int i, int n, int nc, int lane) {
    constexpr int NE = SM::kNE, NT = SM::kNT, KMAX = NE - NG;
    static_assert(NE == 64 && NT == 64, "the record is read as two entries per lane; start slots are staged in rem");
    // every load of the record at once, one memory round trip (the arrays are read whole;
    // entries past the record's counts are ignored)
    const int4 hd = *reinterpret_cast<const int4*>(&rec->iK);   // iK, icl, nc, hw
    const int tag = rec->atom;
    int rpg[2];
    uint8_t rst[2];
    uchar4 rtv[2], rta[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int e = lane + 32 * h;
        rpg[h] = rec->pg[e];
        rst[h] = rec->start[e];
        rtv[h] = rec->tv[e];
        rta[h] = rec->ta[e];
    }
    const int nco = hd.z, hwo = hd.w;
    if (tag != i || nco < 0 || nco > KMAX || hwo < 4 || hwo > NT) return 0;
    const int npo = NG + nco;
    const uchar4 none = make_uchar4(NONE, NONE, NONE, 0);
    for (int k = lane; k < nc; k += 32) S->bedge[k] = (unsigned)S->pg[NG + k];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int e = lane + 32 * h;
        if (e < npo) {
            S->skey[e] = (unsigned)rpg[h];
            S->bslot[e] = rst[h];
            S->eslot[e] = NONE;
        }
        S->tv[e] = e < hwo ? rtv[h] : none;
        S->ta[e] = e < hwo ? rta[h] : none;
        S->rem[e] = NONE;
        S->kf[e] = 0;
        S->tf[e] = 0;
    }
    __syncwarp();
    bool ok = true;
    int live = 0;
    for (int t = lane; t < hwo; t += 32) {
        const uchar4 v = S->tv[t];
        if (v.x == NONE) continue;
        ++live;
        if (v.x >= npo || v.y >= npo || v.z >= npo || v.x == v.y || v.y == v.z || v.z == v.x) {
            ok = false;
            continue;
        }
        S->eslot[v.x] = 1;
        S->eslot[v.y] = 1;
        S->eslot[v.z] = 1;
        const uchar4 adj = S->ta[t];
        for (int k = 0; k < 3; ++k) {
            const int t2 = tv_get(adj, k);
            if (t2 >= hwo) { ok = false; break; }
            const uchar4 w = S->tv[t2];
            const uint8_t a = tv_get(v, k), b = tv_get(v, (k + 1) % 3);
            int k2 = -1;
            for (int h = 0; h < 3; ++h)
                if (tv_get(w, h) == b && tv_get(w, (h + 1) % 3) == a) k2 = h;
            if (k2 < 0 || tv_get(S->ta[t2], k2) != t) { ok = false; break; }
        }
    }
    ok = __all_sync(FULL, ok);
    live = warp_sum_i(live);
    __syncwarp();
    if (!ok) return 0;
    // the faces: ghosts keep their ids, the others become NG, NG + 1, ... (record order);
    // each face's start slot must be a live triangle of that face
    int nF = 0, ngf = 0;
    for (int e0 = 0; e0 < npo; e0 += 32) {
        const int e = e0 + lane;
        const bool f = e < npo && S->eslot[e] == 1;
        if (f) {
            const int st = S->bslot[e];
            const uchar4 v = st < hwo ? S->tv[st] : none;
            if (!(v.x == e || v.y == e || v.z == e)) ok = false;
        }
        const unsigned bg = __ballot_sync(FULL, f && e < NG), ba = __ballot_sync(FULL, f && e >= NG);
        if (f && e >= NG) {
            const int r = nF + __popc(ba & lanemask_lt());
            const int g = (int)S->skey[e];
            if (g < 0 || g >= n || g == i) ok = false;
            S->pg[NG + r] = g;
            S->rem[NG + r] = S->bslot[e];
            S->eslot[e] = (uint8_t)(NG + r);
        } else if (f) {
            S->rem[e] = S->bslot[e];
            S->eslot[e] = (uint8_t)e;
        } else if (e < npo) {
            S->eslot[e] = NONE;
        }
        nF += __popc(ba);
        ngf += __popc(bg);
    }
    ok = __all_sync(FULL, ok) && live == 2 * (nF + ngf) - 4;
    if (!ok) return 0;
    __syncwarp();
    // the current candidates that are not faces, after the faces
    int nnew = 0;
    for (int k0 = 0; k0 < nc; k0 += 32) {
        const int k = k0 + lane;
        int g = -1;
        bool add = false;
        if (k < nc) {
            g = (int)S->bedge[k];
            add = true;
            for (int f = 0; f < nF; ++f)
                if (S->pg[NG + f] == g) add = false;
        }
        const unsigned bn = __ballot_sync(FULL, add);
        const int r = nF + nnew + __popc(bn & lanemask_lt());
        if (add && r < KMAX) S->pg[NG + r] = g;
        nnew += __popc(bn);
    }
    const int ncn = nF + nnew;
    if (ncn > KMAX) return 0;
    // clipping order: ghost faces, faces, new candidates
    {
        const bool gf = lane < NG && S->eslot[lane] != NONE;
        const unsigned bg = __ballot_sync(FULL, gf);
        if (gf) S->ord[__popc(bg & lanemask_lt())] = (uint8_t)lane;
    }
    for (int k = lane; k < ncn; k += 32) S->ord[ngf + k] = (uint8_t)(NG + k);
    // triangles in the new numbering; the dead slots below the high-water mark are free
    int nfree = 0;
    for (int t0 = 0; t0 < hwo; t0 += 32) {
        const int t = t0 + lane;
        bool dead = false;
        if (t < hwo) {
            const uchar4 v = S->tv[t];
            if (v.x == NONE) dead = true;
            else S->tv[t] = make_uchar4(S->eslot[v.x], S->eslot[v.y], S->eslot[v.z], 0);
        }
        const unsigned bd = __ballot_sync(FULL, dead);
        if (dead) S->fs[nfree + __popc(bd & lanemask_lt())] = (uint8_t)t;
        nfree += __popc(bd);
    }
    if (lane == 0) {
        S->hw = hwo;
        S->nfree = nfree;
        S->bad = 0;
    }
    __syncwarp();
    return ncn | (ngf + nF) << 8 | (ngf + ncn) << 16 | live << 24;
}

// ------------------------------------------------------------------ the kernel
__host__ __device__ constexpr int minb(int ph) {
    return (ph == PH_CELL || ph == PH_CC || ph == PH_CARRY) ? MINB_CELL : (ph == PH_CLASS ? MINB_CLASS : ((ph == PH_TERMS || ph == PH_VOL) ? MINB_TERMS : MINB));
}
__host__ __device__ constexpr int warps_of(int ph) {
    return (ph == PH_CELL || ph == PH_CC || ph == PH_CARRY) ? WARPS_CELL : (ph == PH_CLASS ? WARPS_CLASS : ((ph == PH_TERMS || ph == PH_VOL) ? WARPS_TERMS : WARPS));
}
template <class R, bool GRAD, int NE, int NT, int PHX>
__global__ void __launch_bounds__(warps_of(PHX) * 32, minb(PHX)) k_atoms(AtomArgs A) {
    // PH_CARRY: the carried cells of list-reusing calls (the other atoms go to the redo list)
    constexpr bool CARRY = PHX == PH_CARRY;
    constexpr int PH = CARRY ? PH_CELL : PHX;
    constexpr int WARPS = warps_of(PH);
    constexpr int SPL = NT / 32;      // vertex slots per lane
    constexpr int KMAX = NE - NG;     // overlapping neighbours per atom
    const bool EXPORT = A.rec != nullptr;
    // the large-capacity pass works on the atoms the fast pass deferred
    const bool deferred = A.work_list != nullptr;
    const bool can_defer = A.defer_list != nullptr;
    __shared__ Smem<R, NE, NT> smem_all[WARPS];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    Smem<R, NE, NT>* S = &smem_all[wib];
    const int nwarps = gridDim.x * WARPS;
    grid_dep_trigger();
    grid_dep_wait();   // the previous kernel of the call (cell list, cell records) is complete
    const int total = deferred ? *A.work_count : A.n;

    for (int s0 = blockIdx.x * WARPS + wib; s0 < total; s0 += nwarps) {
        const int s = DS_IDX(deferred ? A.work_list[s0] : s0, A.n, A.status);
        const int i = DS_IDX(A.sidx[s], A.n, A.status);
        const float4 fi = A.sf4[s];
        const MolGrid G = A.grids[A.molid[i]];
        Ctx c;
        c.xyz = A.xyz;
        c.R = A.R;
        c.pi[0] = A.xyz[3 * i];
        c.pi[1] = A.xyz[3 * i + 1];
        c.pi[2] = A.xyz[3 * i + 2];
        c.Ri = A.R[i];
        c.h = ghost_h(c.Ri);
        c.i = i;
        c.n = A.n;
        c.status = A.status;
        const R Rr = (R)c.Ri;
        const FA<R> wi = {Rr * Rr, Rr * Rr};
        CellRec<R, NE, NT>* rec = (CellRec<R, NE, NT>*)A.cells + s;
        auto done = [&]() {   // the outputs of this atom are written: tell the terms kernel
            if ((PH == PH_CELL || PH == PH_CLASS || PH == PH_CC) && lane == 0) rec->flag = CELL_DONE;
        };
        auto no_cell = [&]() {   // the record holds no cell of this atom (nothing to carry)
            if ((PH == PH_CELL || PH == PH_CC) && lane == 0) rec->atom = -1;
        };
        // PH_CARRY: this atom's cell is built by the cell kernel that follows, from the redo list
        auto redo = [&]() {
            if (lane == 0) A.redo_list[DS_IDX(atomicAdd(A.redo_count, 1), A.n, A.status)] = s;
            __syncwarp();
        };
        // the outputs of this atom are final (lane 0 wrote them): count it for its molecule
        // after a system-scope fence; the molecule's last atom raises its ready flag, which a
        // host may poll in mapped memory while the kernels run
        auto finished = [&]() {
            if (A.mol_done && lane == 0) molecule_count(A, i);
        };

        int nc = 0;
        int nrounds = 1;     // vertex-slot rounds in use: slots < 32 * nrounds (warp-uniform)
        // per-lane vertex caches (homogeneous z = Dv / D with magnitudes for the filter)
        // (V).  FP32 form: for a first loose filter, the sum of the four filter magnitudes (Vs,
        // rounded up); a test that the loose bound leaves open recomputes the magnitudes.  FP64
        // form: the four magnitudes (Va; measured faster there).
        constexpr bool LOOSE = sizeof(R) == 4;
        R V[SPL][4], Vs[SPL], Va[SPL][LOOSE ? 1 : 4];
        unsigned alive = 0;
        auto compute_vertex = [&](int r, int t) {
            // inline in the split cell and classification kernels (measured faster there), a
            // call in the kernels that hold more code
            VtxFA<R> q;
            if constexpr (PH == PH_CELL || PH == PH_CLASS) q = vertex_fa_inl(S, S->tv[t]);
            else q = vertex_fa(S, S->tv[t]);
            for (int k = 0; k < 4; ++k) V[r][k] = q.v[k];
            if constexpr (LOOSE) Vs[r] = ((q.a[0] + q.a[1]) + (q.a[2] + q.a[3])) * (R)1.000001;
            else
                for (int k = 0; k < 4; ++k) Va[r][k] = q.a[k];
        };

        // molecular volume of the atom from its classified cell (lane 0 writes); the gradient
        // entry of sum_k w_k V_k (w = ones without volume weights)
        auto write_volume = [&](double Ai) {
            R hs, nx, ny, nz, wx, wy, wz;
            const double wv = A.vw ? A.vw[i] : 1.0;
            cell_volume_terms(S, nc, Rr, lane, A.vgrad ? A.vw : nullptr, (R)wv, A.n, A.status, hs, nx, ny, nz, wx, wy, wz);
            const double hsum = warp_sum_d((double)hs);
            const double gx = warp_sum_d((double)nx), gy = warp_sum_d((double)ny), gz = warp_sum_d((double)nz);
            double ex = 0.0, ey = 0.0, ez = 0.0;
            if (A.vgrad && A.vw) { ex = warp_sum_d((double)wx); ey = warp_sum_d((double)wy); ez = warp_sum_d((double)wz); }
            if (lane == 0) {
                A.vol[i] = (c.Ri * Ai + hsum) / 3.0;
                if (A.vgrad) { A.vgrad[3 * i] = wv * gx + ex; A.vgrad[3 * i + 1] = wv * gy + ey; A.vgrad[3 * i + 2] = wv * gz + ez; }
            }
        };

        if constexpr (PH == PH_ALL || PH == PH_CELL || PH == PH_CC) {
        // ---------------- neighbour candidates: balls that may overlap B_i (from this atom's
        // Verlet list when every atom stayed within half the skin of its reference position)
        // Verlet lists of one molecule (indexed by atom, scalar reuse flag) or of a batch of
        // resident molecules (molecule m's lists at its arena slot mol_base[m], entries local
        // to the molecule, per-molecule reuse flag)
        const int mi = A.molid[i];
        const bool slot = A.nbl != nullptr && (A.mol_base == nullptr || A.mol_base[mi] >= 0);
        const int lofs = A.mol_base ? (int)A.mol_off[mi] : 0;                 // list entry = atom - lofs
        const size_t li = A.mol_base ? (size_t)(A.mol_base[mi] + (i - lofs)) : (size_t)i;   // list slot of i
        const bool reuse = slot && (A.mol_base ? A.mol_reuse[mi] != 0 : (A.reuse != nullptr && *A.reuse != 0));
        if constexpr (CARRY) {
            if (!reuse) { redo(); continue; }
        }
        if (reuse) {
            // the list holds every atom within R_i + R_j + skin at the last rebuild; keep the
            // ones whose balls overlap B_i now (float64, with a relative slack of 1e-9)
            const int nl = A.nbn[li];
            for (int b0 = 0; b0 < nl; b0 += 32) {
                const int k = b0 + lane;
                bool ok = false;
                int j = -1;
                if (k < nl) {
                    j = DS_IDX(A.nbl[li * NBL_CAP + k] + lofs, A.n, A.status);
                    const double dx = A.xyz[3 * j] - c.pi[0], dy = A.xyz[3 * j + 1] - c.pi[1], dz = A.xyz[3 * j + 2] - c.pi[2];
                    const double rr = c.Ri + A.R[j];
                    ok = dx * dx + dy * dy + dz * dz < rr * rr * (1.0 + 1e-9);
                }
                unsigned bal = __ballot_sync(FULL, ok);
                int pos = nc + __popc(bal & lanemask_lt());
                if (ok && pos < KMAX) S->pg[NG + pos] = j;
                nc += __popc(bal);
            }
        } else {
            // with Verlet lists (skin > 0) the gather also finds the atoms of the skin band:
            // they go to the atom's list in global memory (nl entries), while the plane table
            // keeps only the balls that overlap B_i now (the float64 test of the reuse path)
            const bool store_lists = slot;
            int nl = 0;
            {
                int cx = min(max((int)floorf((fi.x - G.lo[0]) * G.inv_cell), 0), G.dims[0] - 1);
                int cy = min(max((int)floorf((fi.y - G.lo[1]) * G.inv_cell), 0), G.dims[1] - 1);
                int cz = min(max((int)floorf((fi.z - G.lo[2]) * G.inv_cell), 0), G.dims[2] - 1);
                // one candidate per lane: the FP32 overlap test with the grid's certified slack,
                // the Verlet-list entry and the float64 test, the append to the plane table
                auto gather_one = [&](bool valid, float4 fj, int j) {
                    bool ok = false;
                    if (valid) {
                        float dx = fj.x - fi.x, dy2 = fj.y - fi.y, dz2 = fj.z - fi.z;
                        float rr = fi.w + fj.w + G.margin;
                        ok = (j != i) && (dx * dx + dy2 * dy2 + dz2 * dz2 < rr * rr);
                    }
                    if (store_lists) {
                        const unsigned bl = __ballot_sync(FULL, ok);
                        const int lp = nl + __popc(bl & lanemask_lt());
                        if (ok && lp < NBL_CAP) A.nbl[li * NBL_CAP + lp] = j - lofs;
                        nl += __popc(bl);
                    }
                    if (store_lists || A.skin_band) {
                        if (ok) {
                            const double ddx = A.xyz[3 * j] - c.pi[0], ddy = A.xyz[3 * j + 1] - c.pi[1],
                                         ddz = A.xyz[3 * j + 2] - c.pi[2];
                            const double rr64 = c.Ri + A.R[j];
                            ok = ddx * ddx + ddy * ddy + ddz * ddz < rr64 * rr64 * (1.0 + 1e-9);
                        }
                    }
                    unsigned bal = __ballot_sync(FULL, ok);
                    int pos = nc + __popc(bal & lanemask_lt());
                    if (ok && pos < KMAX) S->pg[NG + pos] = j;
                    nc += __popc(bal);
                };
                // sorted positions [beg, end): the atoms that may overlap B_i
                auto gather_range = [&](int beg, int end) {
                    for (int b0 = beg; b0 < end; b0 += 32) {
                        const int k = b0 + lane;
                        float4 fj = make_float4(0.f, 0.f, 0.f, 0.f);
                        int j = -1;
                        if (k < end) { fj = A.sf4[k]; j = DS_IDX(A.sidx[k], A.n, A.status); }
                        gather_one(k < end, fj, j);
                    }
                };
                if constexpr (PH == PH_CELL) {
                    // the 9 rows (dz, dy) of 3 cells along x: lane r < 9 looks up row r's range (the
                    // 18 lookups in one memory round trip); the first 32 atoms of the 3 rows of one
                    // dz are loaded together (one round trip for the three), longer rows finish by
                    // rounds.  Measured faster in the split cell kernel (50k globule: 569 -> 548 us)
                    // and slower in the one-wave kernel, which keeps the row loop
                    int rbeg = 0, rend = 0;
                    if (lane < 9) {
                        const int z = cz + lane / 3 - 1, y = cy + lane % 3 - 1;
                        if (z >= 0 && z < G.dims[2] && y >= 0 && y < G.dims[1]) {
                            const int row = G.base + (z * G.dims[1] + y) * G.dims[0];
                            const int x0 = max(cx - 1, 0), x1 = min(cx + 1, G.dims[0] - 1);
                            rbeg = A.cstart[row + x0];
                            rend = A.cstart[row + x1 + 1];
                        }
                    }
#pragma unroll 1
                    for (int r0 = 0; r0 < 9; r0 += 3) {
                        float4 rf[3];
                        int rj[3];
#pragma unroll
                        for (int u = 0; u < 3; ++u) {
                            const int k = __shfl_sync(FULL, rbeg, r0 + u) + lane;
                            rf[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                            rj[u] = -1;
                            if (k < __shfl_sync(FULL, rend, r0 + u)) {
                                rf[u] = A.sf4[k];
                                rj[u] = DS_IDX(A.sidx[k], A.n, A.status);
                            }
                        }
#pragma unroll 1
                        for (int u = 0; u < 3; ++u) {
                            const int e = __shfl_sync(FULL, rend, r0 + u);
                            int b0 = __shfl_sync(FULL, rbeg, r0 + u);
                            float4 fj = u == 0 ? rf[0] : (u == 1 ? rf[1] : rf[2]);
                            int j = u == 0 ? rj[0] : (u == 1 ? rj[1] : rj[2]);
                            for (;;) {
                                gather_one(b0 + lane < e, fj, j);
                                b0 += 32;
                                if (b0 >= e) break;
                                const int k = b0 + lane;
                                fj = make_float4(0.f, 0.f, 0.f, 0.f);
                                j = -1;
                                if (k < e) { fj = A.sf4[k]; j = DS_IDX(A.sidx[k], A.n, A.status); }
                            }
                        }
                    }
                } else {
                    for (int dz = -1; dz <= 1; ++dz) {
                        int z = cz + dz;
                        if (z < 0 || z >= G.dims[2]) continue;
                        for (int dy = -1; dy <= 1; ++dy) {
                            int y = cy + dy;
                            if (y < 0 || y >= G.dims[1]) continue;
                            int row = G.base + (z * G.dims[1] + y) * G.dims[0];
                            int x0 = max(cx - 1, 0), x1 = min(cx + 1, G.dims[0] - 1);
                            gather_range(A.cstart[row + x0], A.cstart[row + x1 + 1]);
                        }
                    }
                }
            }
            if (store_lists && lane == 0) {
                // the list's length and the reference position for the next calls; a list
                // longer than its capacity makes the next call rebuild (a deferred atom writes
                // the same list again in the large-capacity pass): one molecule's lists are
                // all marked by lists_bad, a resident slot's by a negative length
                if (nl <= NBL_CAP) A.nbn[li] = nl;
                else if (A.mol_base) A.nbn[li] = -1;
                else atomicOr(A.lists_bad, 1);
                for (int k = 0; k < 3; ++k) A.ref_xyz[3 * li + k] = A.xyz[3 * i + k];
                A.ref_rad[li] = A.radii_in[i];
            }
        }
        if constexpr (CARRY) {
            if (nc > KMAX) { redo(); continue; }
        }
        if (nc > KMAX && can_defer) {
            if (lane == 0) A.defer_list[DS_IDX(atomicAdd(A.defer_count, 1), A.n, A.status)] = s;
            no_cell();
            done();
            __syncwarp();
            continue;
        }
        if (nc > KMAX) {
            if (lane == 0) {
                atomicOr(A.status, ST_CAND_OVF);
                A.areas[i] = __longlong_as_double(0x7ff8000000000000ll);
                if (A.grad) { A.grad[3 * i] = A.grad[3 * i + 1] = A.grad[3 * i + 2] = __longlong_as_double(0x7ff8000000000000ll); }
                if (A.vol) A.vol[i] = __longlong_as_double(0x7ff8000000000000ll);
            }
            no_cell();
            finished();
            done();
            __syncwarp();
            continue;
        }

        // ---------------- PH_CARRY: the previous call's cell carried over (list-reusing calls);
        // an atom whose record gives no usable structure, or whose carried cell is not certified
        // or is cut by a new candidate, goes to the redo list
        constexpr bool carried = CARRY;
        int ncert = 0, nclip = nc;   // planes that certify the carried cell; the other candidates
        if constexpr (CARRY) {
            const int cc = carry_cell(S, rec, i, A.n, nc, lane);
            if (cc == 0) { redo(); continue; }
            nc = cc & 255;
            ncert = (cc >> 8) & 255;
            nclip = (cc >> 16) & 255;
        }

        // ---------------- plane table: ghosts 0..5, candidates NG..NG+nc-1; sort keys
        unsigned long long key[SPL];
        unsigned pay[SPL];
        for (int r = 0; r < SPL; ++r) { key[r] = ~0ull; pay[r] = 0; }
        for (int e = lane; e < NG + nc; e += 32) {
            double q[3], b, babs;
            bool ex;
            int g = e < NG ? -1 - e : S->pg[e];
            plane64_of(c, g, q, b, babs, ex);
            if (e < NG) S->pg[e] = g;
            for (int k = 0; k < 3; ++k) S->pq[e][k] = (R)q[k];
            S->pq[e][3] = (R)b;
            // magnitude proxy of b in float: |b_f| (1 + 2^-22) + 2^-26 babs, rounded up (the float
            // evaluation loses at most 2 ulp, covered by the larger factors)
            if (sizeof(R) == 4) S->pB[e] = (R)(fabsf((float)b) * 1.0000003f + (float)babs * 1.5e-8f);
            else S->pB[e] = (R)(ex ? fabs(b) : 8.0 * babs);
            S->start[e] = NONE;
            if (e >= NG) {
                // sort key: signed distance of the bisector from p_i (ties: atom index)
                float qx = (float)q[0], qy = (float)q[1], qz = (float)q[2];
                float kf = (float)b * rsqrtf(qx * qx + qy * qy + qz * qz + 1e-30f);
                unsigned u = __float_as_uint(kf);
                S->skey[e] = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
            }
            S->eflag[e] = 0;
        }
        __syncwarp();
        if constexpr (!carried) {
        for (int r = 0; r < SPL; ++r) {
            int el = r * 32 + lane;
            if (el < nc) {
                key[r] = ((unsigned long long)S->skey[NG + el] << 32) | (unsigned)S->pg[NG + el];
                pay[r] = NG + el;
            }
        }
        __syncwarp();
        // bitonic sort of the first ns (key, payload) pairs, element e = r*32 + lane; the
        // padding keys are the largest, so sorting a power-of-two prefix that holds all nc
        // candidates sorts them all
        const int ns = nc <= 32 ? 32 : (nc <= 64 ? 64 : NT);
        const int nsr = ns >> 5;
        for (int k = 2; k <= ns; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                if (j >= 32) {
                    // rounds r and r ^ (j / 32) in this lane's registers (the partner round is
                    // a compile-time index in every unrolled branch, so key and pay stay in
                    // registers)
                    const int jr = j >> 5;
#pragma unroll
                    for (int JR = 1; JR < SPL; JR <<= 1) {
                        if (jr != JR) continue;
#pragma unroll
                        for (int r = 0; r < SPL; ++r) {
                            const int r2 = r ^ JR;
                            if (r2 > r && r2 < nsr) {
                                int e = r * 32 + lane;
                                bool up = (e & k) == 0;
                                bool sw = up ? (key[r] > key[r2]) : (key[r] < key[r2]);
                                if (sw) {
                                    unsigned long long tk = key[r]; key[r] = key[r2]; key[r2] = tk;
                                    unsigned tp = pay[r]; pay[r] = pay[r2]; pay[r2] = tp;
                                }
                            }
                        }
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < SPL; ++r) {
                        if (r >= nsr) break;
                        int e = r * 32 + lane;
                        unsigned long long ok = __shfl_xor_sync(FULL, key[r], j);
                        unsigned op = __shfl_xor_sync(FULL, pay[r], j);
                        bool up = (e & k) == 0;
                        bool lower = (lane & j) == 0;
                        bool take = (lower == up) ? (ok < key[r]) : (ok > key[r]);
                        if (take) { key[r] = ok; pay[r] = op; }
                    }
                }
            }
        }
        // renumber the candidate planes in sorted order, so that every later summation
        // order depends only on the geometry (not on the order atoms sit in their cells)
        {
            R tq[SPL][4], tb[SPL];
            int tg[SPL];
#pragma unroll
            for (int r = 0; r < SPL; ++r) {
                int e = r * 32 + lane;
                if (e < nc) {
                    int src = pay[r] & (NE - 1);
                    for (int k = 0; k < 4; ++k) tq[r][k] = S->pq[src][k];
                    tb[r] = S->pB[src];
                    tg[r] = S->pg[src];
                }
            }
            __syncwarp();
#pragma unroll
            for (int r = 0; r < SPL; ++r) {
                int e = r * 32 + lane;
                if (e < nc) {
                    for (int k = 0; k < 4; ++k) S->pq[NG + e][k] = tq[r][k];
                    S->pB[NG + e] = tb[r];
                    S->pg[NG + e] = tg[r];
                    S->ord[e] = (uint8_t)(NG + e);
                }
            }
            __syncwarp();
        }

        // ---------------- initial cell: the cube of the 6 ghost planes (8 vertices)
        for (int t = lane; t < NT; t += 32) {
            uchar4 v = make_uchar4(NONE, NONE, NONE, 0);
            if (t < 8)
                v = make_uchar4((uint8_t)cube_corner_plane(t, 0), (uint8_t)cube_corner_plane(t, 1),
                                (uint8_t)cube_corner_plane(t, 2), 0);
            S->tv[t] = v;
            S->rem[t] = 0;
            S->kf[t] = 0;
            S->tf[t] = 0;
        }
        if (lane == 0) { S->hw = 8; S->nfree = 0; S->bad = 0; }
        if (lane < 8) {
            const int sh = 8 * lane;
            S->ta[lane] = make_uchar4((uint8_t)(CUBE_ADJ0 >> sh), (uint8_t)(CUBE_ADJ1 >> sh), (uint8_t)(CUBE_ADJ2 >> sh), 0);
        }
        if (lane < NG) S->start[lane] = (lane & 1) ? 7 : 0;   // +x,+y,+z at corner 0; -x,-y,-z at 7
        __syncwarp();
        } else {
            // the carried faces' start slots (staged by carry_cell), the clipping marks cleared
            for (int e = lane; e < NG + nc; e += 32) S->start[e] = S->rem[e];
            __syncwarp();
            for (int t = lane; t < NT; t += 32) S->rem[t] = 0;
            __syncwarp();
        }

        const int hw0 = carried ? S->hw : 8;
        nrounds = (hw0 + 31) >> 5;
#pragma unroll
        for (int r = 0; r < SPL; ++r) {
            int t = r * 32 + lane;
            if (t < hw0 && (!CARRY || S->tv[t].x != NONE)) { compute_vertex(r, t); alive |= 1u << r; }
        }
        bool empty = false;
        int nalive = 8;      // live cell vertices (warp-uniform)
        if constexpr (CARRY) {
            // the certification: (i) every carried vertex has a certified positive orientation;
            // (ii) every face plane keeps every vertex not on it strictly inside.  The new
            // candidates are tested in the same sweep (planes outer, the lane's vertices inner,
            // one warp vote at the end): one that removes a vertex sends the atom to the redo list,
            // and so does any test that the FP32 (FP64) filter leaves open
            bool fail = false, cut = false;
#pragma unroll
            for (int r = 0; r < SPL; ++r) {
                if (!(alive >> r & 1)) continue;
                FA<R> D;
                D.v = V[r][3];
                if constexpr (LOOSE) D.a = Vs[r];
                else D.a = Va[r][3];
                if (fa_sign(D, Gam<R>::g, Gam<R>::tiny) <= 0) fail = true;
            }
            for (int kk = 0; kk < nclip; ++kk) {
                const int m = S->ord[kk] & (NE - 1);
                const bool cert = kk < ncert;
                const PlaneN<FA<R>> M = fplane(S, m);
                const R qmax = fmax(fmax(M.q.x.a, M.q.y.a), fmax(M.q.z.a, M.b.a));
#pragma unroll
                for (int r = 0; r < SPL; ++r) {
                    if (r >= nrounds) break;
                    if (!(alive >> r & 1)) continue;
                    const uchar4 v = S->tv[r * 32 + lane];
                    if (cert && (v.x == m || v.y == m || v.z == m)) continue;   // a vertex on the face
                    FA<R> sv;
                    sv.v = M.q.x.v * V[r][0] + M.q.y.v * V[r][1] + M.q.z.v * V[r][2] - M.b.v * V[r][3];
                    if constexpr (LOOSE) sv.a = qmax * Vs[r];
                    else sv.a = M.q.x.a * Va[r][0] + M.q.y.a * Va[r][1] + M.q.z.a * Va[r][2] + M.b.a * Va[r][3];
                    // the filters only: a test they leave open sends the atom to the redo
                    // list (no call in the loop; such tests are rare)
                    const int sg = fa_sign(sv, Gam<R>::gclip, Gam<R>::tiny);
                    if (sg > 0 && !cert) cut = true;
                    else if (sg >= 0) fail = true;
                }
            }
            if (__any_sync(FULL, fail || cut)) { redo(); continue; }
        }

        // ---------------- clipping by the sorted neighbour planes.  The loop makes no call on
        // the clip tests: a test that the filter leaves open ends the inner loop, that plane's
        // tests are resolved outside it (tight magnitudes, then exact predicates), and the loop
        // resumes at the same plane with the resolved signs.  (A call inside the loop made the
        // compiler keep the loop's state in local memory.)
        if constexpr (!CARRY) {
        int kk = 0;
        unsigned rsv = 0;          // removal bits of plane kk resolved outside the loop
        bool resolved = false, open_tests = false;
        for (;;) {
        for (; kk < nclip && !empty; ++kk) {
            const int m = S->ord[kk] & (NE - 1);
            unsigned remv = 0;
            if (resolved) {
                remv = rsv;
                resolved = false;
            } else {
                const PlaneN<FA<R>> M = fplane(S, m);
                // sum_k |q_k| a_k <= max_k |q_k| * sum_k a_k: the loose magnitude of the clip test
                const R qmax = fmax(fmax(M.q.x.a, M.q.y.a), fmax(M.q.z.a, M.b.a));
                bool open = false;
#pragma unroll
                for (int r = 0; r < SPL; ++r) {
                    if (r >= nrounds) break;
                    if (!(alive >> r & 1)) continue;
                    FA<R> sv;
                    sv.v = M.q.x.v * V[r][0] + M.q.y.v * V[r][1] + M.q.z.v * V[r][2] - M.b.v * V[r][3];
                    if constexpr (LOOSE) sv.a = qmax * Vs[r];
                    else sv.a = M.q.x.a * Va[r][0] + M.q.y.a * Va[r][1] + M.q.z.a * Va[r][2] + M.b.a * Va[r][3];
                    const int sg = fa_sign(sv, Gam<R>::gclip, Gam<R>::tiny);
                    if (sg > 0) remv |= 1u << r;
                    else if (sg == 0) open = true;
                }
                open_tests = __any_sync(FULL, open);
                if (open_tests) break;
            }
            unsigned bal[SPL];
            int nrem = 0;
#pragma unroll
            for (int r = 0; r < SPL; ++r) {
                bal[r] = r < nrounds ? __ballot_sync(FULL, remv >> r & 1) : 0u;
                nrem += __popc(bal[r]);
            }
            if (nrem == 0) continue;
            if (nrem == nalive) { empty = true; break; }
            // the ordered list of removed slots (round-major)
            int before = 0;
#pragma unroll
            for (int r = 0; r < SPL; ++r) {
                if (r >= nrounds) break;
                int t = r * 32 + lane;
                if (remv >> r & 1) S->rsl[before + __popc(bal[r] & lanemask_lt())] = (uint8_t)t;
                before += __popc(bal[r]);
            }
            auto removed = [&](int t2) -> bool {   // slot t2 removed by this cut (ballot bits)
                unsigned w = bal[0];
#pragma unroll
                for (int r = 1; r < SPL; ++r)
                    if ((t2 >> 5) == r) w = bal[r];
                return (w >> (t2 & 31)) & 1u;
            };
            __syncwarp();
            // boundary edges of the removed region, one lane per edge of a removed triangle:
            // edge (a -> b) whose neighbour is kept; the new face m gets the triangle (a, b, m)
            // in the slot of boundary edge number e (the e-th removed slot, then free slots)
            const int hw = S->hw, nfree = S->nfree;
            int nb = 0;
            for (int c0 = 0; c0 < 3 * nrem; c0 += 32) {
                const int e3 = c0 + lane;
                bool isb = false;
                uint8_t a = 0, b = 0, t2 = 0, k2 = 0;
                if (e3 < 3 * nrem) {
                    const int t = S->rsl[e3 / 3], k = e3 - 3 * (e3 / 3);
                    const uchar4 v = S->tv[t], adj = S->ta[t];
                    t2 = tv_get(adj, k) & (NT - 1);
                    if (!removed(t2)) {
                        isb = true;
                        a = tv_get(v, k) & (NE - 1);
                        b = tv_get(v, (k + 1) % 3) & (NE - 1);
                        const uchar4 adj2 = S->ta[t2];
                        k2 = adj2.x == t ? 0 : (adj2.y == t ? 1 : 2);
                    }
                }
                const unsigned bb = __ballot_sync(FULL, isb);
                if (isb) {
                    const int e = nb + __popc(bb & lanemask_lt());
                    int slot;
                    if (e < nrem) slot = S->rsl[e];
                    else {
                        int x = e - nrem;
                        slot = x < nfree ? S->fs[nfree - 1 - x] : hw + (x - nfree);
                    }
                    S->bedge[e & (NE - 1)] = (unsigned)a | ((unsigned)b << 7) | ((unsigned)t2 << 14) |
                                             ((unsigned)(slot & 127) << 21) | ((unsigned)k2 << 28);
                    S->bslot[a] = (uint8_t)slot;   // the new triangle on the edge that starts at a
                    S->eslot[b] = (uint8_t)slot;   // ... and ends at b
                }
                nb += __popc(bb);
            }
            const int extra = nb - nrem;
            if (hw + max(0, extra - nfree) > NT || nb > NE) {
                __syncwarp();
                if (lane == 0) S->bad = 2;
                __syncwarp();
                break;
            }
            __syncwarp();
            for (int e = lane; e < nb; e += 32) {
                const unsigned w = S->bedge[e];
                const uint8_t a = w & 127, b = (w >> 7) & 127, t2 = (w >> 14) & 127;
                const int sl = (w >> 21) & (NT - 1);
                S->tv[sl] = make_uchar4(a, b, (uint8_t)m, 0);
                S->ta[sl] = make_uchar4(t2, S->bslot[b & (NE - 1)], S->eslot[a & (NE - 1)], 0);
                ta_set(S, t2, (w >> 28) & 3, (uint8_t)sl);
                S->start[a] = (uint8_t)sl;
                S->rem[sl] = 2;
            }
            if (lane == 0) S->start[m] = (uint8_t)((S->bedge[0] >> 21) & (NT - 1));
            __syncwarp();
            // leftover removed slots become free; update the slot allocator
            if (extra < 0) {
                for (int y = lane; y < -extra; y += 32) {
                    int sl = S->rsl[nb + y];
                    S->tv[sl] = make_uchar4(NONE, NONE, NONE, 0);
                    S->fs[nfree + y] = (uint8_t)sl;
                }
            }
            const int hw2 = extra <= nfree ? hw : hw + (extra - nfree);
            if (lane == 0) {
                if (extra <= nfree) S->nfree = nfree - extra;
                else { S->nfree = 0; S->hw = hw2; }
            }
            nalive += extra;
            nrounds = (hw2 + 31) >> 5;
            __syncwarp();
#pragma unroll
            for (int r = 0; r < SPL; ++r) {
                if (r >= nrounds) break;
                int t = r * 32 + lane;
                if (S->rem[t] == 2) {
                    compute_vertex(r, t);
                    alive |= 1u << r;
                    S->rem[t] = 0;
                } else if (remv >> r & 1) {
                    alive &= ~(1u << r);
                }
            }
            __syncwarp();
        }
        if (!open_tests) break;
        // the tests of plane kk that the filter left open: tight magnitudes, then exact
        {
            open_tests = false;
            const int m = S->ord[kk] & (NE - 1);
            const PlaneN<FA<R>> M = fplane(S, m);
            rsv = 0;
            for (int r = 0; r < nrounds; ++r) {
                if (!(alive >> r & 1)) continue;
                const uchar4 v = S->tv[r * 32 + lane];
                const VtxFA<R> q = vertex_fa(S, v);
                FA<R> sv;
                sv.v = M.q.x.v * q.v[0] + M.q.y.v * q.v[1] + M.q.z.v * q.v[2] - M.b.v * q.v[3];
                sv.a = M.q.x.a * q.a[0] + M.q.y.a * q.a[1] + M.q.z.a * q.a[2] + M.b.a * q.a[3];
                int sg = fa_sign(sv, Gam<R>::gclip, Gam<R>::tiny);
                if (sg == 0)
                    sg = resolve_exact(c, PK_CLIP, S->pg[v.x & (NE - 1)], S->pg[v.y & (NE - 1)],
                                       S->pg[v.z & (NE - 1)], S->pg[m], Gam<R>::try64);
                if (sg > 0) rsv |= 1u << r;
            }
            resolved = true;
        }
        }
        }
        __syncwarp();
        const bool bad = S->bad != 0;
        if (bad && S->bad == 2 && can_defer) {
            if (lane == 0) A.defer_list[DS_IDX(atomicAdd(A.defer_count, 1), A.n, A.status)] = s;
            no_cell();
            done();
            __syncwarp();
            continue;
        }
        if (bad) {
            if (lane == 0) {
                atomicOr(A.status, S->bad == 2 ? ST_TRI_OVF : ST_BADCELL);
                A.areas[i] = __longlong_as_double(0x7ff8000000000000ll);
                if (A.grad) { A.grad[3 * i] = A.grad[3 * i + 1] = A.grad[3 * i + 2] = __longlong_as_double(0x7ff8000000000000ll); }
                if (A.vol) A.vol[i] = __longlong_as_double(0x7ff8000000000000ll);
            }
            no_cell();
            finished();
            done();
            __syncwarp();
            continue;
        }
        if (empty) {
            // the Laguerre cell is empty (redundant ball): A_i = 0 and no simplex of C holds i
            if (lane == 0) {
                A.areas[i] = 0.0;
                if (A.grad) { A.grad[3 * i] = A.grad[3 * i + 1] = A.grad[3 * i + 2] = 0.0; }
                if (A.vol) A.vol[i] = 0.0;
                if (A.vgrad) { A.vgrad[3 * i] = A.vgrad[3 * i + 1] = A.vgrad[3 * i + 2] = 0.0; }
            }
            no_cell();
            finished();
            done();
            __syncwarp();
            continue;
        }
        if constexpr (PH == PH_CELL || PH == PH_CC) {
            // hand the cell to the terms kernel
            const int np = NG + nc, hw = S->hw;
            for (int e = lane; e < np; e += 32) {
                copy_row(rec->pq[e], S->pq[e]);
                rec->pB[e] = S->pB[e];
                rec->pg[e] = S->pg[e];
                rec->start[e] = S->start[e];
            }
            for (int t = lane; t < hw; t += 32) {
                rec->tv[t] = S->tv[t];
                rec->ta[t] = S->ta[t];
            }
            if (lane == 0) {
                rec->nc = nc;
                rec->hw = hw;
                rec->flag = CELL_OK;
                rec->atom = i;
            }
            __syncwarp();
            if constexpr (PH == PH_CELL) continue;
        }
        } else {
            // ---------------- the cell built by the cell kernel: the header, then every load of
            // the record before any shared-memory store (one memory round trip, not one per
            // table); two plane rows and two vertex slots per lane
            static_assert(NE <= 64 && NT <= 64, "a record holds at most 64 planes and 64 vertex slots");
            const int flag = rec->flag;
            const int4 hd = *reinterpret_cast<const int4*>(&rec->iK);   // iK, icl, nc, hw
            if (flag != CELL_OK) continue;
            nc = hd.z;
            const int np = NG + nc, hw = hd.w;
            nrounds = (hw + 31) >> 5;
            constexpr bool BATCH_LOADS = PH == PH_CLASS || PH == PH_VOL;
            if constexpr (BATCH_LOADS) {
                Row4<R> rq[2];
                R rb[2];
                int rg[2];
                uint8_t rs[2], ref[2] = {0, 0}, rkf[2] = {0, 0}, rtf[2] = {0, 0};
                uchar4 rtv[2], rta[2];
    #pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int e = lane + 32 * h;
                    if (e < np) {
                        rq[h] = load_row(rec->pq[e]);
                        rb[h] = rec->pB[e];
                        rg[h] = rec->pg[e];
                        rs[h] = rec->start[e];
                        if constexpr (PH == PH_TERMS || PH == PH_VOL) ref[h] = rec->eflag[e];
                    }
                    rtv[h] = rta[h] = make_uchar4(NONE, NONE, NONE, 0);
                    if (e < hw) {
                        rtv[h] = rec->tv[e];
                        rta[h] = rec->ta[e];
                        if constexpr (PH == PH_TERMS) {
                            rkf[h] = rec->kf[e];
                            rtf[h] = rec->tf[e];
                        }
                    }
                }
    #pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int e = lane + 32 * h;
                    if (e < np) {
                        store_row(S->pq[e], rq[h]);
                        S->pB[e] = rb[h];
                        S->pg[e] = rg[h];
                        S->start[e] = rs[h];
                        if constexpr (PH == PH_TERMS || PH == PH_VOL) S->eflag[e] = ref[h];
                    }
                    if (e < 32 * nrounds) {
                        S->tv[e] = rtv[h];
                        S->ta[e] = rta[h];
                        if constexpr (PH == PH_TERMS) {
                            S->kf[e] = rkf[h];
                            S->tf[e] = rtf[h];
                        }
                    }
                }
            } else {
                for (int e = lane; e < np; e += 32) {
                    copy_row(S->pq[e], rec->pq[e]);
                    S->pB[e] = rec->pB[e];
                    S->pg[e] = rec->pg[e];
                    S->start[e] = rec->start[e];
                }
                for (int t = lane; t < 32 * nrounds; t += 32) {
                    S->tv[t] = t < hw ? rec->tv[t] : make_uchar4(NONE, NONE, NONE, 0);
                    S->ta[t] = t < hw ? rec->ta[t] : make_uchar4(NONE, NONE, NONE, 0);
                }
                if constexpr (PH == PH_TERMS || PH == PH_VOL)
                    for (int e = lane; e < np; e += 32) S->eflag[e] = rec->eflag[e];
                if constexpr (PH == PH_TERMS) {
                    for (int t = lane; t < 32 * nrounds; t += 32) {
                        S->kf[t] = t < hw ? rec->kf[t] : 0;
                        S->tf[t] = t < hw ? rec->tf[t] : 0;
                    }
                }
            }
            if (lane == 0) { S->hw = hw; S->bad = 0; }
            __syncwarp();
#pragma unroll
            for (int r = 0; r < SPL; ++r) {
                if (r >= nrounds) break;
                int t = r * 32 + lane;
                if (S->tv[t].x != NONE) {
                    if constexpr (PH == PH_CLASS) compute_vertex(r, t);
                    alive |= 1u << r;
                }
            }
            __syncwarp();
            if constexpr (PH == PH_VOL) {
                if (!(rec->iK)) {
                    if (lane == 0) {
                        A.vol[i] = 0.0;
                        if (A.vgrad) { A.vgrad[3 * i] = A.vgrad[3 * i + 1] = A.vgrad[3 * i + 2] = 0.0; }
                    }
                    continue;
                }
                write_volume(A.areas[i]);
                __syncwarp();
                continue;
            }
        }

        // ---------------- Step 2a: tetrahedra of C (cell vertices inside B_i)
        unsigned kmask = 0;
        if constexpr (PH == PH_TERMS) {
#pragma unroll
            for (int r = 0; r < SPL; ++r)
                if ((alive >> r & 1) && S->kf[r * 32 + lane] == 1) kmask |= 1u << r;
        } else {
        // The classification loops make no call on their predicates: a test that the filter
        // leaves open is marked and resolved after the loop (tight magnitudes, exact).
        unsigned open2a = 0;   // rounds whose tetrahedron test the loose filter left open
#pragma unroll
        for (int r = 0; r < SPL; ++r) {
            if (r >= nrounds) break;
            int t = r * 32 + lane;
            uint8_t f = 0;
            if (alive >> r & 1) {
                uchar4 v = S->tv[t];
                if (v.x < NG || v.y < NG || v.z < NG) f = 2;
                else {
                    FA<R> P;
                    P.v = V[r][0] * V[r][0] + V[r][1] * V[r][1] + V[r][2] * V[r][2] - wi.v * V[r][3] * V[r][3];
                    // sum_k a_k^2 + w a_3^2 <= max(1, w) (sum_k a_k)^2 (loose), then the magnitudes
                    if constexpr (LOOSE) P.a = fmax((R)1, wi.a) * Vs[r] * Vs[r] * (R)1.000001;
                    else P.a = Va[r][0] * Va[r][0] + Va[r][1] * Va[r][1] + Va[r][2] * Va[r][2] + wi.a * Va[r][3] * Va[r][3];
                    const int sg = fa_sign(P, Gam<R>::g, Gam<R>::tiny);
                    if (sg == 0) open2a |= 1u << r;
                    f = sg < 0 ? 1 : 0;
                    if (f) kmask |= 1u << r;
                }
            }
            S->kf[t] = f;
            S->tf[t] = 0;
        }
        if (__any_sync(FULL, open2a != 0)) {
            for (int r = 0; r < nrounds; ++r) {
                if (!(open2a >> r & 1)) continue;
                const int t = r * 32 + lane;
                const uchar4 v = S->tv[t];
                const VtxFA<R> q = vertex_fa(S, v);
                FA<R> P;
                P.v = q.v[0] * q.v[0] + q.v[1] * q.v[1] + q.v[2] * q.v[2] - wi.v * q.v[3] * q.v[3];
                P.a = q.a[0] * q.a[0] + q.a[1] * q.a[1] + q.a[2] * q.a[2] + wi.a * q.a[3] * q.a[3];
                int sg = fa_sign(P, Gam<R>::g, Gam<R>::tiny);
                if (sg == 0) sg = resolve_exact(c, PK_TET, S->pg[v.x], S->pg[v.y], S->pg[v.z], 0, Gam<R>::try64);
                if (sg <= 0) {
                    S->kf[t] = 1;
                    kmask |= 1u << r;
                }
            }
        }
        __syncwarp();

        // ---------------- Step 2b: triangles of C (cell edges meeting B_i)
        unsigned open2b = 0;   // (round, edge) pairs whose filters left a sign open: bit 3 r + k
#pragma unroll
        for (int r = 0; r < SPL; ++r) {
            if (r >= nrounds) break;
            if (!(alive >> r & 1)) continue;
            int t = r * 32 + lane;
            uchar4 v = S->tv[t], adj = S->ta[t];
            for (int k = 0; k < 3; ++k) {
                int t2 = tv_get(adj, k) & (NT - 1);
                if (t2 < t) continue;   // each cell edge once (t2 == t impossible)
                uint8_t a = tv_get(v, k), b = tv_get(v, (k + 1) % 3), cc = tv_get(v, (k + 2) % 3);
                if (a < NG || b < NG) continue;
                uchar4 w = S->tv[t2];
                uint8_t d = (w.x != a && w.x != b) ? w.x : ((w.y != a && w.y != b) ? w.y : w.z);
                bool inK = S->kf[t] == 1 || S->kf[t2] == 1;
                if (!inK) {
                    // psi of (i, a, b) <= 0 and no attaching plane (cc, d): filters only
                    const int s1 = fsign<PK_TRI>(S, wi, a, b);
                    if (s1 == 0) { open2b |= 1u << (3 * r + k); continue; }
                    if (s1 < 0) {
                        const int s2 = cc < NG ? -1 : fsign<PK_TRIB>(S, wi, a, b, cc);
                        if (s2 == 0) { open2b |= 1u << (3 * r + k); continue; }
                        if (s2 < 0) {
                            const int s3 = d < NG ? -1 : fsign<PK_TRIB>(S, wi, a, b, d);
                            if (s3 == 0) { open2b |= 1u << (3 * r + k); continue; }
                            inK = s3 < 0;
                        }
                    }
                }
                if (inK) {
                    uchar4 adj2 = S->ta[t2];
                    int k2 = adj2.x == t ? 0 : (adj2.y == t ? 1 : 2);
                    atomicOr(&S->tf[t], (1u << k) | (16u << k));
                    atomicOr(&S->tf[t2], 1u << k2);
                }
            }
        }
        if (__any_sync(FULL, open2b != 0)) {
            // the edges whose filters left a sign open, with exact predicates
            for (int r = 0; r < nrounds; ++r) {
                for (int k = 0; k < 3; ++k) {
                    if (!(open2b >> (3 * r + k) & 1)) continue;
                    const int t = r * 32 + lane;
                    const uchar4 v = S->tv[t];
                    const int t2 = tv_get(S->ta[t], k) & (NT - 1);
                    const uint8_t a = tv_get(v, k), b = tv_get(v, (k + 1) % 3), cc = tv_get(v, (k + 2) % 3);
                    const uchar4 w = S->tv[t2];
                    const uint8_t d = (w.x != a && w.x != b) ? w.x : ((w.y != a && w.y != b) ? w.y : w.z);
                    if (psign<PK_TRI>(S, c, wi, a, b) <= 0 && (cc < NG || psign<PK_TRIB>(S, c, wi, a, b, cc) <= 0) &&
                        (d < NG || psign<PK_TRIB>(S, c, wi, a, b, d) <= 0)) {
                        const uchar4 adj2 = S->ta[t2];
                        const int k2 = adj2.x == t ? 0 : (adj2.y == t ? 1 : 2);
                        atomicOr(&S->tf[t], (1u << k) | (16u << k));
                        atomicOr(&S->tf[t2], 1u << k2);
                    }
                }
            }
        }
        __syncwarp();
        }

        // ---------------- Step 2c / 3: faces (edges of C), area terms, gradient gathers
        // Vectors, angles and the gradient are evaluated in R (float in the mixed mode).  The
        // area terms are combined in FP64 in a form where pi multiplies only quantities of the
        // radii and distances (pi, R_i and R_i^2 rounded to float would bias every term the
        // same way, and the terms cancel about 30-fold in A_i); no FP64 division is used.
        const R zero = (R)0;
        const double TWO_PI = 6.283185307179586476925;
        double area_acc = 0.0;
        GAcc<R> gacc;
        const double wi_w = A.w ? A.w[i] : 1.0;
        const R wif = (R)wi_w;
        // Mixed mode: the radius quantities (R, R^2, R_i -+ R_j, 2 pi) enter as float pairs and
        // the lane's terms are summed in float-float (no FP64 instruction per term); the
        // per-atom constants 4 pi R_i^2 and c 2 pi R_i^2 are added once in FP64 at the end.
        constexpr bool FFM = sizeof(R) == 4;
        const float2 ri2 = A.Rhl[i];
        const FF Ri_ff = {ri2.x, ri2.y}, Ri2_ff = ff_mul(Ri_ff, Ri_ff);
        FF acc_ff = {0.f, 0.f};
        float cf_sum = 0.f;
        float vtx_const = 0.f;   // 2 when the vertex term is present: its 4 pi R_i^2 = 2 (2 pi R_i^2)
        const float TWO_PI_H = 6.28318548202514648f, TWO_PI_L = -1.74845553e-07f;   // 2 pi = H + L
        int myEK = 0;
        // edge term of A_i and its gradient gathers, for an edge (i, a) of C that is not closed;
        // phi_sum and gsum sum the dihedral angles (and their d/dp_i) of its tetrahedra
        auto edge_term = [&](int a, const P3<R>& pa, R phi_sum, const P3<R>& gsum) {
            // edge term of A_i (Eqs. phiedge, edge): - Phi_ia S_ia^(i) with
            // S_ia^(i) = 2 pi R_i h_i and Phi_ia = 1 - sum(theta) / 2 pi, i.e.
            // R_i h_i (sum(theta) - 2 pi); h_i = (R_i + R_a - d)(R_a - R_i + d) / 2d
            int ga = DS_IDX(S->pg[a], A.n, A.status);
            const R dr = norm3(pa), inv2d = (R)0.5 / dr;
            R Raf, dR2;
            if constexpr (FFM) {
                const float2 ra2 = A.Rhl[ga];
                const FF Ra = {ra2.x, ra2.y}, Sp = ff_add(Ri_ff, Ra), Dm = ff_sub(Ra, Ri_ff);
                const float hi = ((Sp.h - dr) + Sp.l) * ((Dm.h + dr) + Dm.l) * inv2d;
                acc_ff = ff_add(acc_ff, ff_mul_f(Ri_ff, hi * ((phi_sum - TWO_PI_H) - TWO_PI_L)));
                Raf = Ra.h;
                dR2 = ff_mul(ff_sub(Ri_ff, Ra), Sp).h;
            } else {
                const double Ra = A.R[ga];
                const double d = (double)dr;
                const double hi = ((c.Ri + Ra) - d) * ((Ra - c.Ri) + d) * (double)inv2d;
                area_acc += c.Ri * hi * ((double)phi_sum - TWO_PI);
                Raf = (R)Ra;
                dR2 = (R)((c.Ri - Ra) * (c.Ri + Ra));
            }
            if (GRAD) {
                const R waf = A.w ? (R)A.w[ga] : (R)1;
                const R ti = (dr * dr + dR2) * inv2d, ta = (dr * dr - dR2) * inv2d;
                const R phi = (R)1 - phi_sum * (R)(1.0 / TWO_PI);
                // vertex + edge parts of the dihedral derivatives around ia (Eq. inexclu)
                const R kap = -(wif * Rr * ti + waf * Raf * ta);
                // cap derivatives (Eq. edge): -Phi (2 pi / d)(w_i R_i t_a + w_a R_a t_i) u
                const R cf = -phi * (R)TWO_PI / (dr * dr) * (wif * Rr * ta + waf * Raf * ti);
                gacc.add(kap * gsum.x + cf * pa.x, kap * gsum.y + cf * pa.y, kap * gsum.z + cf * pa.z);
            }
        };
        if constexpr (PH != PH_TERMS) {
        // faces whose edge test the filters left open (bit = the lane's face iteration), and
        // which of them are closed; resolved after the loop (the fused kernel decides in place)
        unsigned open2c = 0, closed2c = 0;
        int it2c = 0;
        for (int a = NG + lane; a < NG + nc; a += 32, ++it2c) {
            uint8_t flag = 0;
            R phi_sum = zero;
            int st = S->start[a];
            bool active = false;
            if (st != NONE) {
                uchar4 v = S->tv[st & (NT - 1)];
                active = v.x == a || v.y == a || v.z == a;
            }
            if (active) {
                int t = st & (NT - 1);
                int nv = 0, nk = 0;
                bool ghost = false, triK = false, inside = true;
                P3<R> gsum = {zero, zero, zero};
                const P3<R> O = {zero, zero, zero};
                const P3<R> pa = ppos(S, a);
                for (int step = 0; step < NT; ++step) {
                    uchar4 v = S->tv[t];
                    int k = v.x == a ? 0 : (v.y == a ? 1 : 2);
                    uint8_t b = tv_get(v, (k + 1) % 3), cc = tv_get(v, (k + 2) % 3);
                    ++nv;
                    if (S->kf[t] == 2) ghost = true;
                    if (S->kf[t] == 1) {
                        ++nk;
                        if constexpr (PH == PH_ALL) {
                            P3<R> pb = ppos(S, b), pc = ppos(S, cc);
                            phi_sum += dihedral_ol(O, pa, pb, pc);
                            // (i, a, b, c) is positively oriented: (a, b, c) is counter-clockwise
                            if (GRAD) gsum = gsum + dihedral_grad_u_ol(O, pa, pb, pc, (R)1);
                        }
                    }
                    if ((S->tf[t] >> k) & 1) triK = true;
                    int nx = tv_get(S->ta[t], k) & (NT - 1);
                    t = nx;
                    if (t == (st & (NT - 1))) break;
                    if (step == NT - 1) S->bad = 3;
                }
                bool closed = (nk == nv) && !ghost;
                bool eK = triK;
                if constexpr (PH == PH_ALL) {
                    if (!eK && psign<PK_EDGE>(S, c, wi, a, 0) <= 0) {
                        // is the edge orthocentre inside the face polygon?  walk again over its sides
                        t = st & (NT - 1);
                        for (int step = 0; step < NT && inside; ++step) {
                            uchar4 v = S->tv[t];
                            int k = v.x == a ? 0 : (v.y == a ? 1 : 2);
                            uint8_t b = tv_get(v, (k + 1) % 3);
                            if (b >= NG && psign<PK_EDGEB>(S, c, wi, a, b) > 0) inside = false;
                            t = tv_get(S->ta[t], k) & (NT - 1);
                            if (t == (st & (NT - 1))) break;
                        }
                        eK = inside;
                    }
                } else if (!eK) {
                    // the same tests with the filters only; an open one defers the face
                    const int se = fsign<PK_EDGE>(S, wi, a, a);
                    bool open = se == 0;
                    if (se < 0) {
                        bool out = false;
                        t = st & (NT - 1);
                        for (int step = 0; step < NT; ++step) {
                            uchar4 v = S->tv[t];
                            int k = v.x == a ? 0 : (v.y == a ? 1 : 2);
                            uint8_t b = tv_get(v, (k + 1) % 3);
                            if (b >= NG) {
                                const int sb = fsign<PK_EDGEB>(S, wi, a, b);
                                if (sb > 0) { out = true; break; }
                                if (sb == 0) open = true;
                            }
                            t = tv_get(S->ta[t], k) & (NT - 1);
                            if (t == (st & (NT - 1))) break;
                        }
                        if (out) open = false;
                        else if (!open) eK = true;
                    }
                    if (open) {
                        open2c |= 1u << it2c;
                        if (closed) closed2c |= 1u << it2c;
                    }
                }
                if (eK) {
                    flag = 1 | (closed ? 2 : 0);
                    myEK = 1;
                    if constexpr (PH == PH_ALL)
                        if (!closed) edge_term(a, pa, phi_sum, gsum);
                }
            }
            S->eflag[a] = flag;
        }
        if (PH != PH_ALL && __any_sync(FULL, open2c != 0)) {
            // the deferred faces, with exact predicates
            it2c = 0;
            for (int a = NG + lane; a < NG + nc; a += 32, ++it2c) {
                if (!(open2c >> it2c & 1)) continue;
                const int st = S->start[a] & (NT - 1);
                bool eK = false;
                if (psign<PK_EDGE>(S, c, wi, a, 0) <= 0) {
                    eK = true;
                    int t = st;
                    for (int step = 0; step < NT; ++step) {
                        const uchar4 v = S->tv[t];
                        const int k = v.x == a ? 0 : (v.y == a ? 1 : 2);
                        const uint8_t b = tv_get(v, (k + 1) % 3);
                        if (b >= NG && psign<PK_EDGEB>(S, c, wi, a, b) > 0) { eK = false; break; }
                        t = tv_get(S->ta[t], k) & (NT - 1);
                        if (t == st) break;
                    }
                }
                if (eK) {
                    S->eflag[a] = 1 | ((closed2c >> it2c & 1) ? 2 : 0);
                    myEK = 1;
                }
            }
        }
        __syncwarp();
        } else {
        // the faces that are edges of C and not closed (classified by the previous kernel)
        for (int a = NG + lane; a < NG + nc; a += 32) {
            if ((S->eflag[a] & 3) != 1) continue;
            const int st = S->start[a] & (NT - 1);
            const P3<R> O = {zero, zero, zero};
            const P3<R> pa = ppos(S, a);
            R phi_sum = zero;
            P3<R> gsum = {zero, zero, zero};
            int t = st;
            for (int step = 0; step < NT; ++step) {
                uchar4 v = S->tv[t];
                int k = v.x == a ? 0 : (v.y == a ? 1 : 2);
                if (S->kf[t] == 1) {
                    P3<R> pb = ppos(S, tv_get(v, (k + 1) % 3)), pc = ppos(S, tv_get(v, (k + 2) % 3));
                    phi_sum += dihedral(O, pa, pb, pc);
                    if (GRAD) gsum = gsum + dihedral_grad_u_in(O, pa, pb, pc, (R)1);
                }
                t = tv_get(S->ta[t], k) & (NT - 1);
                if (t == st) break;
            }
            edge_term(a, pa, phi_sum, gsum);
        }
        __syncwarp();
        }

        // vertex i in C?  (an edge of C holds it, or p_i lies in its own cell)
        bool iK, icl;
        if constexpr (PH == PH_TERMS) {
            iK = rec->iK != 0;
            icl = rec->icl != 0;
        } else {
        iK = __any_sync(FULL, myEK);
        icl = true;   // cell entirely inside B_i: interior vertex
#pragma unroll
        for (int r = 0; r < SPL; ++r)
            if ((alive >> r & 1) && !(kmask >> r & 1)) icl = false;
        icl = __all_sync(FULL, icl);
        if (!iK) {
            bool ok = true;
            for (int a = NG + lane; a < NG + nc; a += 32) {
                int st = S->start[a];
                if (st == NONE) continue;
                uchar4 v = S->tv[st & (NT - 1)];
                if (!(v.x == a || v.y == a || v.z == a)) continue;
                FA<R> b = {S->pq[a][3], S->pB[a]};
                int sg = fa_sign(b, Gam<R>::g, Gam<R>::tiny);
                if (sg == 0) sg = resolve_exact(c, PK_VERT, S->pg[a], 0, 0, 0, Gam<R>::try64);
                if (sg < 0) ok = false;
            }
            iK = __all_sync(FULL, ok);
        }

        }
        if constexpr (PH == PH_CLASS || PH == PH_CC) {
            __syncwarp();
            if (S->bad) {
                if (lane == 0) {
                    atomicOr(A.status, ST_BADCELL);
                    A.areas[i] = __longlong_as_double(0x7ff8000000000000ll);
                    if (A.grad) { A.grad[3 * i] = A.grad[3 * i + 1] = A.grad[3 * i + 2] = __longlong_as_double(0x7ff8000000000000ll); }
                    if (A.vol) A.vol[i] = __longlong_as_double(0x7ff8000000000000ll);
                }
                finished();
                done();
                __syncwarp();
                continue;
            }
            if (!iK && !EXPORT) {
                // no simplex of C holds i: A_i = 0 (and V_i = 0) and no gradient gathers
                if (lane == 0) {
                    A.areas[i] = 0.0;
                    if (A.grad) { A.grad[3 * i] = A.grad[3 * i + 1] = A.grad[3 * i + 2] = 0.0; }
                    if (A.vol) A.vol[i] = 0.0;
                    if (A.vgrad) { A.vgrad[3 * i] = A.vgrad[3 * i + 1] = A.vgrad[3 * i + 2] = 0.0; }
                }
                finished();
                done();
                __syncwarp();
                continue;
            }
            for (int e = lane; e < NG + nc; e += 32) rec->eflag[e] = S->eflag[e];
            for (int t = lane; t < S->hw; t += 32) {
                rec->kf[t] = S->kf[t];
                rec->tf[t] = (uint8_t)S->tf[t];
            }
            if (lane == 0) {
                rec->iK = iK;
                rec->icl = icl;
            }
            __syncwarp();
            continue;
        }

        // vertex term Omega_i 4 pi R_i^2 (Eq. vertex), Omega_i = 1 - sum of solid angles / 4 pi
        // (with the half solid angles h_T of its tetrahedra: Omega_i 4 pi R_i^2 = 4 pi R_i^2 - 2 R_i^2 sum h_T)
        if (iK && !icl) {
            R om = zero;
#pragma unroll
            for (int r = 0; r < SPL; ++r) {
                if (!(kmask >> r & 1)) continue;
                uchar4 v = S->tv[r * 32 + lane];
                om += solid_angle_half(ppos(S, v.x), ppos(S, v.y), ppos(S, v.z));
            }
            if constexpr (FFM) {
                // - 2 R_i^2 (half solid angles) in float-float; the 4 pi R_i^2 is added once below
                acc_ff = ff_add(acc_ff, ff_mul_f(Ri2_ff, -2.f * om));
                vtx_const = 2.f;
            } else {
                double omd = warp_sum_d((double)om);
                if (lane == 0) area_acc += c.Ri * c.Ri * (2.0 * TWO_PI - 2.0 * omd);
            }
        }

        // triangle terms: c_iab S_iab^(i) (Eq. trianglev) and the gradient of the triangle
        // terms of i, a and b (Eq. triangle) and of the dihedral (wing) terms that do not
        // cancel.  The exterior triangles are first compacted into a list so that the lanes
        // share the work evenly.
        int ntl = 0;
#pragma unroll
        for (int r = 0; r < SPL; ++r) {
            if (r >= nrounds) break;
            int t = r * 32 + lane;
            unsigned f = (alive >> r & 1) ? S->tf[t] : 0u;
            for (int k = 0; k < 3; ++k) {
                bool want = (f >> (4 + k)) & 1;   // processed by its canonical owner only
                if (want) {
                    int t2 = tv_get(S->ta[t], k) & (NT - 1);
                    want = !(S->kf[t] == 1 && S->kf[t2] == 1);   // interior: coefficient 0
                }
                unsigned bl = __ballot_sync(FULL, want);
                if (want) S->tl[ntl + __popc(bl & lanemask_lt())] = (uint16_t)((t << 2) | k);
                ntl += __popc(bl);
            }
        }
        __syncwarp();
        // With the gradient, four lanes per exterior triangle: parts 0-2 evaluate the lens
        // gradient of owner i, a or b (one call on all those lanes), part 3 the area term; part
        // 0 adds the wing dihedral term when one tetrahedron of C holds the triangle.
        constexpr int GT = GRAD ? 4 : 1;
        for (int j = lane; j < GT * ntl; j += 32) {
            {
                const int e = j / GT, part = GRAD ? (j & 3) : 3;
                const int t = S->tl[e] >> 2, k = S->tl[e] & 3;
                uchar4 v = S->tv[t];
                uint8_t a = tv_get(v, k), b = tv_get(v, (k + 1) % 3), cc = tv_get(v, (k + 2) % 3);
                int t2 = tv_get(S->ta[t], k) & (NT - 1);
                int nk = (S->kf[t] == 1) + (S->kf[t2] == 1);
                const R cff = (R)1 - (R)0.5 * (R)nk;
                P3<R> pa = ppos(S, a), pb = ppos(S, b);
                int ga = DS_IDX(S->pg[a], A.n, A.status), gb = DS_IDX(S->pg[b], A.n, A.status);
                R Raf, Rbf, dRab;
                if constexpr (FFM) {
                    const float2 ra2 = A.Rhl[ga], rb2 = A.Rhl[gb];
                    const FF Ra = {ra2.x, ra2.y}, Rb = {rb2.x, rb2.y};
                    if (part == 3) {
                        FF v = tri_term_ff(pa, pb, Ri_ff, Ra, Rb, Ri2_ff, -1.f);
                        acc_ff = ff_add(acc_ff, FF{cff * v.h, cff * v.l});
                        cf_sum += cff;
                    }
                    Raf = Ra.h;
                    Rbf = Rb.h;
                    dRab = ff_mul(ff_sub(Ra, Rb), ff_add(Ra, Rb)).h;
                } else {
                    const double Ra = A.R[ga], Rb = A.R[gb];
                    if (part == 3) area_acc += (double)cff * tri_term_mixed_ol(pa, pb, c.Ri, Ra, Rb);
                    Raf = (R)Ra;
                    Rbf = (R)Rb;
                    dRab = (R)((Ra - Rb) * (Ra + Rb));
                }
                if (GRAD && part < 3) {
                    const P3<R> O = {zero, zero, zero};
                    const R waf = A.w ? (R)A.w[ga] : (R)1, wbf = A.w ? (R)A.w[gb] : (R)1;

                    // owner i: d/dp_i = -(g2 + g3); owner a: p_i is the second centre; owner b
                    const P3<R> u = part == 0 ? pa : (part == 1 ? O - pa : O - pb);
                    const P3<R> w = part == 0 ? pb : (part == 1 ? pb - pa : pa - pb);
                    const R r0 = part == 0 ? Rr : (part == 1 ? Raf : Rbf);
                    const R r1 = part == 0 ? Raf : Rr;
                    const R r2 = part == 2 ? Raf : Rbf;
                    P3x2f<R> lg = lens_grad_in(u, w, r0, r1, r2, (R)-1);
                    if (FFM && lg.refine) {
                        // The lens gradient is linear in the height s_t of the triple points over
                        // the plane of the centres, whose float value (R^2 - |z|^2) errs by about
                        // 2^-24 R^2 / s_t: for the few lens gradients (about 0.4 %) whose s_t^2 is
                        // below 0.01 R^2 it is taken from the float64 coordinates (the same for the
                        // three owners: it depends on the three spheres only) and the gradient
                        // redone.  Each FP64 instruction occupies a GB300 sub-partition for 64
                        // cycles, so the FP64 work is kept that rare and short (Gram form).
                        const P3<double> qa = {A.xyz[3 * ga] - c.pi[0], A.xyz[3 * ga + 1] - c.pi[1], A.xyz[3 * ga + 2] - c.pi[2]};
                        const P3<double> qb = {A.xyz[3 * gb] - c.pi[0], A.xyz[3 * gb + 1] - c.pi[1], A.xyz[3 * gb + 2] - c.pi[2]};
                        const float s2 = triple_height2_gram(qa, qb, c.Ri, A.R[ga], A.R[gb]);
                        lg = lens_grad_in(u, w, r0, r1, r2, (R)(s2 > 0.f ? sqrtf(s2) : 0.f));
                    }
                    const R f = cff * (part == 0 ? -wif : (part == 1 ? waf : wbf));
                    R sx = f * (part == 0 ? lg.a.x + lg.b.x : lg.a.x);
                    R sy = f * (part == 0 ? lg.a.y + lg.b.y : lg.a.y);
                    R sz = f * (part == 0 ? lg.a.z + lg.b.z : lg.a.z);
                    if (part == 0 && nk == 1) {
                        // the single tetrahedron of C on this triangle: (i, a, b, x); its
                        // orientation is + when it is the cell vertex t, - when it is t2
                        uchar4 w2 = S->tv[t2];
                        uint8_t xo = (w2.x != a && w2.x != b) ? w2.x : ((w2.y != a && w2.y != b) ? w2.y : w2.z);
                        bool on_t = S->kf[t] == 1;
                        uint8_t x = on_t ? cc : xo;
                        const R dab = norm3(pb - pa), inv2 = (R)0.5 / dab;
                        const R tab = (dab * dab + dRab) * inv2, tba = (dab * dab - dRab) * inv2;
                        const R kap = -(waf * Raf * tab + wbf * Rbf * tba);
                        P3<R> gc = dihedral_grad_c_in(pa, pb, O, ppos(S, x), on_t ? (R)1 : (R)-1);
                        sx += kap * gc.x; sy += kap * gc.y; sz += kap * gc.z;
                    }
                    gacc.add(sx, sy, sz);
                }
            }
        }

        double gxd = 0.0, gyd = 0.0, gzd = 0.0;
        if constexpr (FFM) {
            // one float-float warp sum of every lane's terms (the same order on every run; lane 0's
            // value is used), then the per-atom constants (2 + c) 2 pi R_i^2 in FP64
            FF tot = acc_ff;
            for (int o = 16; o > 0; o >>= 1)
                tot = ff_add(tot, FF{__shfl_xor_sync(FULL, tot.h, o), __shfl_xor_sync(FULL, tot.l, o)});
            for (int o = 16; o > 0; o >>= 1) cf_sum += __shfl_xor_sync(FULL, cf_sum, o);
            area_acc = ff_to_double(tot) + ((double)cf_sum + (double)vtx_const) * TWO_PI * c.Ri * c.Ri;
        } else {
            area_acc = warp_sum_d(area_acc);
        }
        if (GRAD) gacc.reduce(gxd, gyd, gzd);
        __syncwarp();
        if (lane == 0) {
            if (S->bad) {
                atomicOr(A.status, ST_BADCELL);
                area_acc = __longlong_as_double(0x7ff8000000000000ll);
            }
            A.areas[i] = iK ? area_acc : 0.0;
            if (GRAD && A.grad) {
                A.grad[3 * i] = iK ? gxd : 0.0;
                A.grad[3 * i + 1] = iK ? gyd : 0.0;
                A.grad[3 * i + 2] = iK ? gzd : 0.0;
            }
        }
        if (!(PH == PH_ALL && A.vol)) finished();
        if constexpr (PH == PH_ALL) {
            if (A.vol) {
                if (iK) write_volume(area_acc);
                else if (lane == 0) {
                    A.vol[i] = 0.0;
                    if (A.vgrad) { A.vgrad[3 * i] = A.vgrad[3 * i + 1] = A.vgrad[3 * i + 2] = 0.0; }
                }
            }
        }

        // ---------------- optional export of the simplices of C containing i
        if (EXPORT) {
            auto emit = [&](int v0, int v1, int v2, int v3) {
                unsigned long long pos = atomicAdd(A.nrec, 1ull);
                if ((long long)pos < A.max_rec) {
                    int* rr = A.rec + 5 * pos;
                    int tmp[4] = {v0, v1, v2, v3};
                    // sort the atom indices (-1 last)
                    for (int p = 0; p < 4; ++p)
                        for (int q2 = p + 1; q2 < 4; ++q2) {
                            bool sw = (tmp[q2] >= 0) && (tmp[p] < 0 || tmp[q2] < tmp[p]);
                            if (sw) { int x = tmp[p]; tmp[p] = tmp[q2]; tmp[q2] = x; }
                        }
                    rr[0] = i; rr[1] = tmp[0]; rr[2] = tmp[1]; rr[3] = tmp[2]; rr[4] = tmp[3];
                }
            };
            if (lane == 0 && iK) emit(i, -1, -1, -1);
            for (int a = NG + lane; a < NG + nc; a += 32)
                if (S->eflag[a] & 1) emit(i, S->pg[a], -1, -1);
#pragma unroll
            for (int r = 0; r < SPL; ++r) {
                if (!(alive >> r & 1)) continue;
                int t = r * 32 + lane;
                uchar4 v = S->tv[t];
                if (kmask >> r & 1) emit(i, S->pg[v.x], S->pg[v.y], S->pg[v.z]);
                unsigned f = S->tf[t];
                for (int k = 0; k < 3; ++k)
                    if ((f >> (4 + k)) & 1) emit(i, S->pg[tv_get(v, k)], S->pg[tv_get(v, (k + 1) % 3)], -1);
            }
        }
        __syncwarp();
    }
}

}  // namespace

#ifndef DSASA_ATOMS_NO_LAUNCH
// Whether every atom's warp of the cell kernel is resident at once (one wave).  Then the fused
// cell + classification kernel runs an atom's classification while other atoms are still
// clipping (the slowest cells set the end of the wave); with more atoms the split kernels keep
// each kernel's instruction stream in the cache, which is worth more.
template <class R> bool cells_in_one_wave(int n) {
    static int cap = -1;
    if (cap < 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_atoms<R, false, 64, 64, PH_CC>, WARPS_CELL * 32, 0);
        cap = sms * per * WARPS_CELL;
    }
    return n <= cap;
}

// Fast pass (64 planes, 64 vertex slots) over all atoms: with a cell store, the cell,
// classification and terms kernels, else the fused kernel.  The atoms it defers get the fused 128 / 128
// pass, whose grid reads the deferred count from device memory (no host sync).  The deferred
// count must be zero when the first kernel starts (the cell-list build clears it).
template <class R>
cudaError_t launch_atoms_t(const AtomArgs& a, bool grad, cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    int blocks = (a.n + WARPS - 1) / WARPS;
    AtomArgs fast = a;
    fast.work_list = nullptr;
    fast.work_count = nullptr;
    AtomArgs big = a;
    big.defer_list = nullptr;
    big.defer_count = nullptr;
    big.work_list = a.defer_list;
    big.work_count = a.defer_count;
    big.cells = nullptr;
    fast.ev = big.ev = nullptr;
    // the deferred atoms are few: a small grid that loops over them (most calls have none)
    int big_blocks = blocks < 64 ? blocks : 64;
    const bool g = grad && a.rec == nullptr;
    auto mark = [&](int k) {
        if (a.ev) cudaEventRecord(a.ev[k], s);
    };
    // every kernel after the cell-list build is a programmatic dependent launch in the mixed
    // form (measured: 3 % faster on a 5k-atom molecule); the all-FP64 form's kernels ran 3 %
    // slower that way and are launched in plain stream order
    cudaError_t err = cudaSuccess;
    auto go = [&](auto kernel, int grid, int block, const AtomArgs& args) {
        cudaError_t e = launch_dependent(kernel, grid, block, s, sizeof(R) == 4, args);
        if (err == cudaSuccess) err = e;
        note_launches(1);
    };
    if (a.cells) {
        auto nb = [&](int w) { return (a.n + w - 1) / w; };
        if (!a.carry && cells_in_one_wave<R>(a.n)) {
            go(k_atoms<R, false, 64, 64, PH_CC>, nb(WARPS_CELL), WARPS_CELL * 32, fast);
            mark(0);
            mark(1);
        } else {
            if (a.carry) {
                // the carried cells, then the cell kernel over the redo list (its grid covers
                // every atom; the warps past the list's length return at once)
                go(k_atoms<R, false, 64, 64, PH_CARRY>, nb(WARPS_CELL), WARPS_CELL * 32, fast);
                AtomArgs redo = fast;
                redo.work_list = a.redo_list;
                redo.work_count = a.redo_count;
                go(k_atoms<R, false, 64, 64, PH_CELL>, nb(WARPS_CELL), WARPS_CELL * 32, redo);
            } else {
                go(k_atoms<R, false, 64, 64, PH_CELL>, nb(WARPS_CELL), WARPS_CELL * 32, fast);
            }
            mark(0);
            go(k_atoms<R, false, 64, 64, PH_CLASS>, nb(WARPS_CLASS), WARPS_CLASS * 32, fast);
            mark(1);
        }
        if (g) go(k_atoms<R, true, 64, 64, PH_TERMS>, nb(WARPS_TERMS), WARPS_TERMS * 32, fast);
        else go(k_atoms<R, false, 64, 64, PH_TERMS>, nb(WARPS_TERMS), WARPS_TERMS * 32, fast);
        if (a.vol) go(k_atoms<R, false, 64, 64, PH_VOL>, nb(WARPS_TERMS), WARPS_TERMS * 32, fast);
        mark(2);
    } else {
        if (g) go(k_atoms<R, true, 64, 64, PH_ALL>, blocks, WARPS * 32, fast);
        else go(k_atoms<R, false, 64, 64, PH_ALL>, blocks, WARPS * 32, fast);
        mark(0);
        mark(1);
        mark(2);
    }
    if (a.defer_list) {
        if (g) go(k_atoms<R, true, 128, 128, PH_ALL>, big_blocks, WARPS * 32, big);
        else go(k_atoms<R, false, 128, 128, PH_ALL>, big_blocks, WARPS * 32, big);
    }
    mark(3);
    return err != cudaSuccess ? err : cudaGetLastError();
}
#endif

}  // namespace dsasa
