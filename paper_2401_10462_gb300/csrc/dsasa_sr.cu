// Shrake-Rupley numerical SASA on the GPU: an on-device cross-check of the exact areas.
//
// m unit vectors s_k (supplied by the caller) are placed on every probe-inflated sphere; a
// point is exposed when it lies strictly outside every other ball that overlaps the
// sphere, and A_i = 4 pi R_i^2 (exposed points) / m (Shrake & Rupley 1973, the numerical
// method the paper's accuracy comparison uses).  Every point is tested against every
// overlapping neighbour (no early exit): the work is a fixed m x k_i distance tests per atom,
// which makes the kernel a plain FP32 stream.  The per-point decision uses float32 operations
// without contraction (x = R_i s_k, q = float(p_j - p_i), d2 = (dx dx + dy dy) + dz dz,
// covered iff d2 <= R_j^2) so that the exposed counts can be compared exactly with a host
// evaluation of the same arithmetic; the neighbour set uses the exact float64 test
// |p_i - p_j|^2 < (R_i + R_j)^2.
//
// One warp per atom: the neighbours are gathered from the 27 cells of the cell list into
// shared memory (coordinates relative to p_i, R_j^2), then each lane tests 4 points at a
// time against every neighbour (one shared-memory broadcast per neighbour for 4 points).
#include "dsasa_kernels.cuh"

namespace dsasa {

namespace {

constexpr int SR_WARPS = 4;      // atoms per block
constexpr int SR_KN = 128;       // overlapping neighbours per atom (more: capacity error)
constexpr int SR_PPL = 4;        // points per lane per pass

struct SRSmem {
    float4 nb[SR_KN];            // q_j (float(p_j - p_i)), R_j^2
};

__global__ void __launch_bounds__(SR_WARPS * 32) k_shrake_rupley(SRArgs A) {
    __shared__ SRSmem smem_all[SR_WARPS];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    SRSmem* S = &smem_all[wib];
    const int s = blockIdx.x * SR_WARPS + wib;
    if (s >= A.n) return;
    const int i = A.sidx[s];
    const float4 fi = A.sf4[s];
    const MolGrid G = A.grids[A.molid[i]];
    const double pix = A.xyz[3 * i], piy = A.xyz[3 * i + 1], piz = A.xyz[3 * i + 2], Ri = A.R[i];

    // overlapping neighbours from the 27 cells (float prefilter with the grid's slack, then
    // the exact float64 test)
    int nn = 0;
    bool ovf = false;
    {
        int cx = min(max((int)floorf((fi.x - G.lo[0]) * G.inv_cell), 0), G.dims[0] - 1);
        int cy = min(max((int)floorf((fi.y - G.lo[1]) * G.inv_cell), 0), G.dims[1] - 1);
        int cz = min(max((int)floorf((fi.z - G.lo[2]) * G.inv_cell), 0), G.dims[2] - 1);
        for (int dz = -1; dz <= 1; ++dz) {
            int z = cz + dz;
            if (z < 0 || z >= G.dims[2]) continue;
            for (int dy = -1; dy <= 1; ++dy) {
                int y = cy + dy;
                if (y < 0 || y >= G.dims[1]) continue;
                int row = G.base + (z * G.dims[1] + y) * G.dims[0];
                int x0 = max(cx - 1, 0), x1 = min(cx + 1, G.dims[0] - 1);
                int beg = A.cstart[row + x0], end = A.cstart[row + x1 + 1];
                for (int b0 = beg; b0 < end; b0 += 32) {
                    int k = b0 + lane;
                    bool ok = false;
                    float4 nbv = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (k < end) {
                        float4 fj = A.sf4[k];
                        float ddx = fj.x - fi.x, ddy = fj.y - fi.y, ddz = fj.z - fi.z;
                        float rr = fi.w + fj.w + G.margin;
                        int j = A.sidx[k];
                        if (j != i && ddx * ddx + ddy * ddy + ddz * ddz < rr * rr) {
                            const double qx = __dsub_rn(A.xyz[3 * j], pix), qy = __dsub_rn(A.xyz[3 * j + 1], piy),
                                         qz = __dsub_rn(A.xyz[3 * j + 2], piz);
                            const double dd = __dadd_rn(__dadd_rn(__dmul_rn(qx, qx), __dmul_rn(qy, qy)), __dmul_rn(qz, qz));
                            const double Rj = A.R[j];
                            const double rs = __dadd_rn(Rj, Ri);
                            if (dd < __dmul_rn(rs, rs)) {
                                ok = true;
                                const float Rjf = (float)Rj;
                                nbv = make_float4((float)qx, (float)qy, (float)qz, __fmul_rn(Rjf, Rjf));
                            }
                        }
                    }
                    unsigned bal = __ballot_sync(0xffffffffu, ok);
                    unsigned lt;
                    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
                    int pos = nn + __popc(bal & lt);
                    if (ok) {
                        if (pos < SR_KN) S->nb[pos] = nbv;
                        else ovf = true;
                    }
                    nn += __popc(bal);
                }
            }
        }
    }
    __syncwarp();
    if (__any_sync(0xffffffffu, ovf) || nn > SR_KN) {
        if (lane == 0) {
            atomicOr(A.status, ST_CAND_OVF);
            A.areas[i] = __longlong_as_double(0x7ff8000000000000ll);
            if (A.exposed) A.exposed[i] = -1;
        }
        return;
    }
    const float Rf = (float)Ri;
    int cnt = 0;
    for (int k0 = 0; k0 < A.m; k0 += 32 * SR_PPL) {
        float px[SR_PPL], py[SR_PPL], pz[SR_PPL];
        bool cov[SR_PPL];
#pragma unroll
        for (int p = 0; p < SR_PPL; ++p) {
            const int k = k0 + p * 32 + lane;
            const bool have = k < A.m;
            px[p] = have ? __fmul_rn(Rf, A.pts[3 * k]) : 0.f;
            py[p] = have ? __fmul_rn(Rf, A.pts[3 * k + 1]) : 0.f;
            pz[p] = have ? __fmul_rn(Rf, A.pts[3 * k + 2]) : 0.f;
            cov[p] = !have;
        }
        for (int j = 0; j < nn; ++j) {
            const float4 q = S->nb[j];
#pragma unroll
            for (int p = 0; p < SR_PPL; ++p) {
                const float dx = __fsub_rn(px[p], q.x), dy = __fsub_rn(py[p], q.y), dz = __fsub_rn(pz[p], q.z);
                const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
                cov[p] = cov[p] || d2 <= q.w;
            }
        }
#pragma unroll
        for (int p = 0; p < SR_PPL; ++p) cnt += cov[p] ? 0 : 1;
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) {
        A.areas[i] = 4.0 * 3.14159265358979323846 * Ri * Ri * (double)cnt / (double)A.m;
        if (A.exposed) A.exposed[i] = cnt;
        if (A.tests) atomicAdd(A.tests, (unsigned long long)A.m * (unsigned long long)nn);
    }
}

}  // namespace

cudaError_t launch_sr(const SRArgs& a, cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    k_shrake_rupley<<<(a.n + SR_WARPS - 1) / SR_WARPS, SR_WARPS * 32, 0, s>>>(a);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace dsasa
