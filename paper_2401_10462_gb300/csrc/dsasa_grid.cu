// Cell-list build for the neighbour search (input preparation and binning).
//
// Atoms are binned per molecule into cubic cells of edge >= 2 R_max + skin + slack, so every
// pair of overlapping balls |p_i - p_j| < R_i + R_j lies in the same or adjacent cells.  The
// binning is a counting sort (atomic counts -> exclusive scan -> scatter); the order inside a
// cell is not deterministic, which is harmless because each atom later sorts its candidate
// list by (plane distance, atom index).  The sorted float4 copy (x, y, z, R) gives coalesced
// neighbour-tile loads in the atom kernel.
#include "dsasa_kernels.cuh"

#include <math.h>

namespace dsasa {

namespace {

__device__ __forceinline__ unsigned fenc(float f) {
    unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fdec(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__global__ void k_bbox_init(unsigned* bbox, int n_mol, int* zero_word) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m == 0 && zero_word) { zero_word[0] = 0; zero_word[1] = 0; }
    if (m >= n_mol) return;
    unsigned lo = fenc(INFINITY), hi = fenc(-INFINITY);
    for (int k = 0; k < 3; ++k) { bbox[8 * m + k] = lo; bbox[8 * m + 3 + k] = hi; }
    bbox[8 * m + 6] = fenc(0.0f);
    bbox[8 * m + 7] = 0;
}

__global__ void k_prep(BuildArgs a) {
    if (a.skip && *a.skip) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = i < a.n;
    const unsigned mask = __ballot_sync(0xffffffffu, act);
    if (!act) return;
    int m = 0;
    if (a.offsets) {
        int lo = 0, hi = a.n_mol - 1;   // last m with offsets[m] <= i
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (a.offsets[mid] <= i) lo = mid; else hi = mid - 1;
        }
        m = lo;
    }
    double x = a.xyz[3 * i], y = a.xyz[3 * i + 1], z = a.xyz[3 * i + 2];
    double R = a.radii[i] + a.probe;
    if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(R)) || !(R > 0.0)) {
        atomicOr(a.status, ST_INPUT);
        x = y = z = 0.0;
        R = 1.0;
    }
    a.R[i] = R;
    { float h = (float)R; a.Rhl[i] = make_float2(h, (float)(R - (double)h)); }
    a.molid[i] = m;
    float4 f = make_float4((float)x, (float)y, (float)z, (float)R);
    a.f4[i] = f;
    // bounding box of the molecule: reduced over the warp first when its atoms share one
    // molecule (one atomic per warp instead of one per atom on the same 7 words)
    unsigned lo3[3] = {fenc(f.x), fenc(f.y), fenc(f.z)};
    unsigned hi4[4] = {lo3[0], lo3[1], lo3[2], fenc(f.w)};
    const int first = __ffs(mask) - 1;
    const int m0 = __shfl_sync(mask, m, first);
    unsigned* bb = a.bbox + 8 * m;
    if (__all_sync(mask, m == m0)) {
        for (int k = 0; k < 3; ++k) lo3[k] = __reduce_min_sync(mask, lo3[k]);
        for (int k = 0; k < 4; ++k) hi4[k] = __reduce_max_sync(mask, hi4[k]);
        if ((int)(threadIdx.x & 31) != first) return;
    }
    atomicMin(bb + 0, lo3[0]);
    atomicMin(bb + 1, lo3[1]);
    atomicMin(bb + 2, lo3[2]);
    atomicMax(bb + 3, hi4[0]);
    atomicMax(bb + 4, hi4[1]);
    atomicMax(bb + 5, hi4[2]);
    atomicMax(bb + 6, hi4[3]);
}

// Grid of one molecule from its encoded bounding box (bb: min x y z, max x y z, max R) and
// atom count: cell size and dimensions; the cell count is returned in base.
__device__ MolGrid make_grid(const unsigned* bb, long long nm, double skin) {
    MolGrid g;
    if (nm <= 0) {
        for (int k = 0; k < 3; ++k) { g.lo[k] = 0.f; g.dims[k] = 1; }
        g.inv_cell = 1.f;
        g.margin = 0.f;
        g.rmax = 0.f;
        g.base = 1;
        return g;
    }
    float lo[3], hi[3], amax = 0.f;
    for (int k = 0; k < 3; ++k) {
        lo[k] = fdec(bb[k]);
        hi[k] = fdec(bb[3 + k]);
        amax = fmaxf(amax, fmaxf(fabsf(lo[k]), fabsf(hi[k])));
    }
    float rmax = fdec(bb[6]);
    // float rounding of coordinates (|x| 2^-24 each), of the difference and of R: slack
    float margin = 1e-5f + 4.0e-7f * (amax + 16.0f);
    float cell = 2.0f * rmax + (float)skin + 2.0f * margin + 1e-3f;
    double cap = 8.0 * (double)nm + 64.0;
    int dims[3];
    for (int it = 0; it < 64; ++it) {
        double prod = 1.0;
        for (int k = 0; k < 3; ++k) {
            dims[k] = (int)fminf((hi[k] - lo[k]) / cell, 1e6f) + 1;
            prod *= dims[k];
        }
        if (prod <= cap) break;
        cell *= (float)fmax(1.01, cbrt(prod / cap) * 1.01);
    }
    for (int k = 0; k < 3; ++k) { g.lo[k] = lo[k]; g.dims[k] = dims[k]; }
    g.inv_cell = 1.0f / cell;
    g.margin = margin + (float)skin;   // candidates within R_i + R_j + skin (Verlet lists)
    g.rmax = rmax;
    g.base = dims[0] * dims[1] * dims[2];
    return g;
}

// per molecule: cell size and dimensions (cell count stored in base for the scan below)
__global__ void k_grid_local(BuildArgs a) {
    if (a.skip && *a.skip) return;
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= a.n_mol) return;
    long long nm = a.offsets ? (a.offsets[m + 1] - a.offsets[m]) : a.n;
    a.grids[m] = make_grid(a.bbox + 8 * m, nm, a.skin);
}

// exclusive scan of the per-molecule cell counts (one block)
__global__ void k_grid_scan(BuildArgs a) {
    if (a.skip && *a.skip) return;
    __shared__ int carry;
    __shared__ int ws[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < a.n_mol; b0 += blockDim.x) {
        int m = b0 + threadIdx.x;
        int v = m < a.n_mol ? a.grids[m].base : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if ((threadIdx.x & 31) >= o) x += y;
        }
        if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            int s = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, s, o);
                if (threadIdx.x >= o) s += y;
            }
            ws[threadIdx.x] = s;
        }
        __syncthreads();
        int wpre = (threadIdx.x >= 32) ? ws[(threadIdx.x >> 5) - 1] : 0;
        int excl = carry + wpre + x - v;
        if (m < a.n_mol) a.grids[m].base = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *a.ncells_out = carry;
        if (carry > a.max_cells) atomicOr(a.status, ST_GRID_OVF);
    }
}

__device__ __forceinline__ int cell_of(const MolGrid& g, float4 f) {
    int cx = min(max((int)floorf((f.x - g.lo[0]) * g.inv_cell), 0), g.dims[0] - 1);
    int cy = min(max((int)floorf((f.y - g.lo[1]) * g.inv_cell), 0), g.dims[1] - 1);
    int cz = min(max((int)floorf((f.z - g.lo[2]) * g.inv_cell), 0), g.dims[2] - 1);
    return g.base + (cz * g.dims[1] + cy) * g.dims[0] + cx;
}

__global__ void k_count(BuildArgs a) {
    if (a.skip && *a.skip) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const MolGrid g = a.grids[a.molid[i]];
    int c = cell_of(g, a.f4[i]);
    if (c >= a.max_cells) c = a.max_cells - 1;   // only after a reported overflow
    a.cell[i] = c;
    a.rank[i] = atomicAdd(&a.counts[c], 1);
}

// ---- exclusive scan of counts[0..len) into cstart (3 phases, tile = 256 threads x 16)
constexpr int SCAN_T = 256, SCAN_V = 16, SCAN_TILE = SCAN_T * SCAN_V;

__device__ int block_excl_scan(int v, int* total) {
    __shared__ int ws[SCAN_T / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = lane < SCAN_T / 32 ? ws[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < SCAN_T / 32) ws[lane] = s;
    }
    __syncthreads();
    int pre = (w > 0 ? ws[w - 1] : 0) + x - v;
    *total = ws[SCAN_T / 32 - 1];
    __syncthreads();
    return pre;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_reduce(const int* in, int len, int* bsum) {
    int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_V;
    int s = 0;
    for (int k = 0; k < SCAN_V; ++k) s += (base + k < len) ? in[base + k] : 0;
    int tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}
__global__ void __launch_bounds__(SCAN_T) k_scan_top(int* bsum, int nb) {
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nb; b0 += SCAN_T) {
        int v = (b0 + threadIdx.x < nb) ? bsum[b0 + threadIdx.x] : 0;
        int tot;
        int pre = block_excl_scan(v, &tot);
        if (b0 + threadIdx.x < nb) bsum[b0 + threadIdx.x] = carry + pre;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
}
__global__ void __launch_bounds__(SCAN_T) k_scan_down(const int* in, int len, const int* bsum, int* out) {
    int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_V;
    int v[SCAN_V];
    int s = 0;
    for (int k = 0; k < SCAN_V; ++k) { v[k] = (base + k < len) ? in[base + k] : 0; s += v[k]; }
    int tot;
    int pre = block_excl_scan(s, &tot) + bsum[blockIdx.x];
    for (int k = 0; k < SCAN_V; ++k) {
        if (base + k <= len) out[base + k] = pre;   // out has len + 1 entries
        pre += v[k];
    }
}

__global__ void k_scatter(BuildArgs a) {
    grid_dep_trigger();
    if (a.skip && *a.skip) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    int pos = a.cstart[a.cell[i]] + a.rank[i];
    a.sidx[pos] = i;
    a.sf4[pos] = a.f4[i];
}

// The whole build for one molecule of at most kSmallAtoms atoms in one kernel (the
// multi-kernel path's launch overheads dominate at that size).  Same grid, same cells.  One
// thread per atom for the input pass (its FP64 work and conversions spread over several SMs);
// each block leaves its partial bounding box in a.sync and takes a ticket, and the block that
// takes the last ticket (nothing waits) finishes the build: box, grid, counting sort in shared
// memory, scan, scatter.  It then resets the ticket for the next call.
constexpr int kSmallAtoms = 16384, kSmallT = 1024, kSmallCells = 8192, kSmallBlocks = kSmallAtoms / kSmallT;
static_assert(kSmallBlocks * 8 + 1 <= BUILD_SYNC_WORDS, "block-exchange area too small");
__device__ __forceinline__ unsigned box_init(int k) {
    return k < 3 ? fenc(INFINITY) : (k < 6 ? fenc(-INFINITY) : (k == 6 ? fenc(0.0f) : 0u));
}
__global__ void __launch_bounds__(kSmallT) k_build_small(BuildArgs a) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.zero_word) { a.zero_word[0] = 0; a.zero_word[1] = 0; }
    grid_dep_trigger();
    if (a.skip && *a.skip) return;
    __shared__ unsigned bb[8];
    __shared__ MolGrid g;
    __shared__ int ws[kSmallT / 32];
    __shared__ int scount[kSmallCells];
    __shared__ bool last;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid < 8) bb[tid] = box_init(tid);
    __syncthreads();
    unsigned lo[3] = {fenc(INFINITY), fenc(INFINITY), fenc(INFINITY)};
    unsigned hi[4] = {fenc(-INFINITY), fenc(-INFINITY), fenc(-INFINITY), fenc(0.0f)};
    {
        const int i = blockIdx.x * kSmallT + tid;
        if (i < a.n) {
            double x = a.xyz[3 * i], y = a.xyz[3 * i + 1], z = a.xyz[3 * i + 2];
            double R = a.radii[i] + a.probe;
            if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(R)) || !(R > 0.0)) {
                atomicOr(a.status, ST_INPUT);
                x = y = z = 0.0;
                R = 1.0;
            }
            a.R[i] = R;
            { float h = (float)R; a.Rhl[i] = make_float2(h, (float)(R - (double)h)); }
            a.molid[i] = 0;
            float4 f = make_float4((float)x, (float)y, (float)z, (float)R);
            a.f4[i] = f;
            unsigned e[4] = {fenc(f.x), fenc(f.y), fenc(f.z), fenc(f.w)};
            for (int k = 0; k < 3; ++k) { lo[k] = min(lo[k], e[k]); hi[k] = max(hi[k], e[k]); }
            hi[3] = max(hi[3], e[3]);
        }
    }
    for (int k = 0; k < 3; ++k) {
        lo[k] = __reduce_min_sync(0xffffffffu, lo[k]);
        hi[k] = __reduce_max_sync(0xffffffffu, hi[k]);
    }
    hi[3] = __reduce_max_sync(0xffffffffu, hi[3]);
    if (lane == 0) {
        for (int k = 0; k < 3; ++k) { atomicMin(&bb[k], lo[k]); atomicMax(&bb[3 + k], hi[k]); }
        atomicMax(&bb[6], hi[3]);
    }
    __syncthreads();
    // partial box out, every thread's writes made visible, then the ticket
    if (tid < 8) a.sync[8 * blockIdx.x + tid] = bb[tid];
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(a.sync + 8 * kSmallBlocks, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (tid < 8) {
        unsigned v = box_init(tid);
        for (int b = 0; b < (int)gridDim.x; ++b) {
            const unsigned p = __ldcg(a.sync + 8 * b + tid);
            v = tid < 3 ? min(v, p) : (tid < 7 ? max(v, p) : 0u);
        }
        bb[tid] = v;
    }
    if (tid == 0) a.sync[8 * kSmallBlocks] = 0u;   // ticket back to zero for the next call
    __syncthreads();
    if (tid == 0) {
        MolGrid gg = make_grid(bb, a.n, a.skin);
        const int ncells = gg.base;
        gg.base = 0;
        g = gg;
        a.grids[0] = gg;
        *a.ncells_out = ncells;
        if (ncells > a.max_cells) atomicOr(a.status, ST_GRID_OVF);
        for (int k = 0; k < 8; ++k) a.bbox[k] = bb[k];
    }
    __syncthreads();
    const int ncells = min(g.dims[0] * g.dims[1] * g.dims[2], a.max_cells);
    // counts in shared memory when the grid is small enough (the usual case), else in HBM
    const bool sm = ncells + 1 <= kSmallCells;
    int* cnt = sm ? scount : a.counts;
    for (int c = tid; c <= ncells; c += kSmallT) cnt[c] = 0;
    __syncthreads();
#pragma unroll 4
    for (int i = tid; i < a.n; i += kSmallT) {
        int c = cell_of(g, __ldcg(a.f4 + i));   // written by other blocks of this grid
        if (c >= a.max_cells) c = a.max_cells - 1;   // only after a reported overflow
        a.cell[i] = c;
        a.rank[i] = atomicAdd(&cnt[c], 1);
    }
    __syncthreads();
    // exclusive scan of counts[0 .. ncells] into cstart: each thread scans a contiguous run
    // of cells, one block scan over the run totals (the shared copy keeps the starts)
    const int per = (ncells + 1 + kSmallT - 1) / kSmallT;
    const int c0 = min(tid * per, ncells + 1), c1 = min(c0 + per, ncells + 1);
    int run = 0;
    for (int c = c0; c < c1; ++c) run += c < ncells ? cnt[c] : 0;
    int x = run;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = ws[lane];
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        ws[lane] = t;
    }
    __syncthreads();
    int pre = (w > 0 ? ws[w - 1] : 0) + x - run;
    for (int c = c0; c < c1; ++c) {
        const int v = c < ncells ? cnt[c] : 0;
        a.cstart[c] = pre;
        if (sm) cnt[c] = pre;
        pre += v;
    }
    __syncthreads();
#pragma unroll 4
    for (int i = tid; i < a.n; i += kSmallT) {
        int pos = (sm ? cnt[a.cell[i]] : a.cstart[a.cell[i]]) + a.rank[i];
        a.sidx[pos] = i;
        a.sf4[pos] = __ldcg(a.f4 + i);
    }
}

cudaError_t launch_build_multi(const BuildArgs& a, cudaStream_t s) {
    const int T = 256;
    int nb = (a.n + T - 1) / T;
    k_bbox_init<<<(a.n_mol + T - 1) / T, T, 0, s>>>(a.bbox, a.n_mol, a.zero_word);
    k_prep<<<nb, T, 0, s>>>(a);
    k_grid_local<<<(a.n_mol + T - 1) / T, T, 0, s>>>(a);
    k_grid_scan<<<1, 1024, 0, s>>>(a);
    cudaMemsetAsync(a.counts, 0, sizeof(int) * (size_t)(a.max_cells + 1), s);
    k_count<<<nb, T, 0, s>>>(a);
    int len = a.max_cells;   // scan the whole capacity: cells past the used range are zero
    int nt = (len + 1 + SCAN_TILE - 1) / SCAN_TILE;
    k_scan_reduce<<<nt, SCAN_T, 0, s>>>(a.counts, len, a.blocksums);
    k_scan_top<<<1, SCAN_T, 0, s>>>(a.blocksums, nt);
    k_scan_down<<<nt, SCAN_T, 0, s>>>(a.counts, len, a.blocksums, a.cstart);
    k_scatter<<<nb, T, 0, s>>>(a);
    note_launches(9);
    return cudaGetLastError();
}

}  // namespace

size_t scan_scratch_ints(int max_cells) { return (size_t)(max_cells + 1 + SCAN_TILE - 1) / SCAN_TILE + 1; }

namespace {

// Verlet skin test (see dsasa_kernels.cuh)
__global__ void k_verlet_check(const double* xyz, const double* radii, const double* ref_xyz, const double* ref_rad,
                               int n, int* vstate) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float d2 = 0.f;
    int changed = 0;
    if (i < n) {
        double dx = xyz[3 * i] - ref_xyz[3 * i], dy = xyz[3 * i + 1] - ref_xyz[3 * i + 1], dz = xyz[3 * i + 2] - ref_xyz[3 * i + 2];
        double dd = dx * dx + dy * dy + dz * dz;
        d2 = (float)dd * (1.f + 1e-6f);   // rounded up: the test stays conservative
        if (!(dd == dd)) d2 = INFINITY;
        changed = radii[i] != ref_rad[i];
    }
    const unsigned d2max = __reduce_max_sync(0xffffffffu, __float_as_uint(d2));   // d2 >= 0: bits order as values
    changed = __reduce_or_sync(0xffffffffu, changed);
    if ((threadIdx.x & 31) == 0) {
        atomicMax((unsigned*)&vstate[0], d2max);
        if (changed) atomicOr(&vstate[1], 1);
    }
}
__global__ void k_verlet_decide(int* vstate, int valid, float lim2) {
    const float d2 = __uint_as_float((unsigned)vstate[0]);
    const int reuse = valid && vstate[1] == 0 && vstate[3] == 0 && d2 <= lim2;
    vstate[2] = reuse;
    if (!reuse) vstate[3] = 0;   // the lists are rebuilt by this call
}

// The same test for a batch of resident molecules, per molecule m (atoms [off[m], off[m+1]),
// lists at arena slot base[m] + local index; base[m] < 0: no lists): vmol[3m] the largest
// squared displacement since the lists were built (float bits, rounded up), vmol[3m + 1] a
// radius changed, vmol[3m + 2] some atom has no valid list (negative length).
__global__ void k_verlet_check_batch(const double* xyz, const double* radii, const double* ref_xyz,
                                     const double* ref_rad, const int* nbn, const long long* off,
                                     const long long* base, int n, int n_mol, int* vmol) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = n_mol - 1;   // last m with off[m] <= i
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    const int m = lo;
    if (base[m] < 0) return;
    const size_t li = (size_t)(base[m] + (i - off[m]));
    const double dx = xyz[3 * i] - ref_xyz[3 * li], dy = xyz[3 * i + 1] - ref_xyz[3 * li + 1],
                 dz = xyz[3 * i + 2] - ref_xyz[3 * li + 2];
    const double dd = dx * dx + dy * dy + dz * dz;
    const float d2 = dd == dd ? (float)dd * (1.f + 1e-6f) : INFINITY;
    atomicMax((unsigned*)&vmol[3 * m], __float_as_uint(d2));
    if (radii[i] != ref_rad[li]) atomicOr(&vmol[3 * m + 1], 1);
    if (nbn[li] < 0) atomicOr(&vmol[3 * m + 2], 1);
}
__global__ void k_verlet_decide_batch(const int* vmol, const long long* base, int n_mol, float lim2, int* reuse) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_mol) return;
    reuse[m] = base[m] >= 0 && vmol[3 * m + 1] == 0 && vmol[3 * m + 2] == 0 &&
               __uint_as_float((unsigned)vmol[3 * m]) <= lim2;
}

}  // namespace

cudaError_t launch_verlet_check_batch(const double* xyz, const double* radii, const double* ref_xyz,
                                      const double* ref_rad, const int* nbn, const long long* off,
                                      const long long* base, int n, int n_mol, double skin, int* vmol, int* reuse,
                                      cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(vmol, 0, sizeof(int) * 3 * (size_t)n_mol, s);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        k_verlet_check_batch<<<(n + 255) / 256, 256, 0, s>>>(xyz, radii, ref_xyz, ref_rad, nbn, off, base, n, n_mol, vmol);
        note_launches(1);
    }
    const float lim2 = (float)(0.25 * skin * skin) * (1.f - 1e-6f);
    k_verlet_decide_batch<<<(n_mol + 127) / 128, 128, 0, s>>>(vmol, base, n_mol, lim2, reuse);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_verlet_check(const double* xyz, const double* radii, const double* ref_xyz, const double* ref_rad,
                                int n, int valid, double skin, int* vstate, cudaStream_t s) {
    cudaMemsetAsync(vstate, 0, 2 * sizeof(int), s);
    if (valid && n > 0) {
        k_verlet_check<<<(n + 255) / 256, 256, 0, s>>>(xyz, radii, ref_xyz, ref_rad, n, vstate);
        note_launches(1);
    }
    // (skin / 2)^2, rounded down in float
    float lim2 = (float)(0.25 * skin * skin) * (1.f - 1e-6f);
    k_verlet_decide<<<1, 1, 0, s>>>(vstate, valid, lim2);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_build(const BuildArgs& a, cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    if (a.n_mol == 1 && a.n <= kSmallAtoms) {
        k_build_small<<<(a.n + kSmallT - 1) / kSmallT, kSmallT, 0, s>>>(a);
        note_launches(1);
        return cudaGetLastError();
    }
    return launch_build_multi(a, s);
}

}  // namespace dsasa
