// Shared declarations of the dSASA CUDA kernels (host side and device side).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace dsasa {

// Programmatic dependent launch (the kernels of one call run back to back on one stream): a
// kernel launched by launch_dependent may be scheduled while the previous kernel of the
// stream is still running; it calls grid_dep_wait() before it touches anything, which returns
// once that kernel has completed and its writes are visible.  grid_dep_trigger() lets the
// next kernel be scheduled once every block of this one has started.  Both are no-ops for a
// kernel launched without the attribute.
#ifdef __CUDACC__
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
#endif
template <class... K, class... A>
cudaError_t launch_dependent(void (*kernel)(K...), int grid, int block, cudaStream_t s, bool early, A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = early ? 1 : 0;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

// host: adds k to the library-wide count of kernel launches (dsasa_kernel_launches)
void note_launches(int k);

// words of the single-molecule cell-list build's block-exchange area: 16 partial bounding
// boxes of 8 words, then the completion ticket
constexpr int BUILD_SYNC_WORDS = 16 * 8 + 1;

// device status bits (ORed by kernels, read by dsasa_status_sync)
enum : int {
    ST_CAND_OVF = 1,      // more overlapping neighbours than one warp's candidate table holds
    ST_TRI_OVF = 2,       // cell needed more vertex slots than available
    ST_UNRESOLVED = 4,    // exact expansion capacity exceeded
    ST_DEGENERATE = 8,    // a clip tie that Simulation of Simplicity cannot break (coincident atoms)
    ST_BADCELL = 16,      // inconsistent cell structure detected (atom output set to NaN)
    ST_INPUT = 32,        // non-finite input
    ST_EXPORT_OVF = 64,   // complex export buffer too small
    ST_GRID_OVF = 128,    // cell grid larger than its capacity
    ST_CHECK = 256        // a bounds check of the checked build failed (the access was redirected)
};

// The checked build (-DDSASA_CHECKED): every data-dependent index into a global array of
// atoms (sorted positions, neighbour entries, plane owners, work lists) is verified on the
// device.  A bad index sets ST_CHECK and is replaced by 0, so the access stays inside the
// array; the results of that call are then not to be used.  The normal build checks nothing.
#ifdef DSASA_CHECKED
__device__ __forceinline__ int ds_checked(int idx, int lim, int* status) {
    if ((unsigned)idx < (unsigned)lim) return idx;
    atomicOr(status, ST_CHECK);
    return 0;
}
#define DS_IDX(idx, lim, status) ds_checked((idx), (lim), (status))
#else
#define DS_IDX(idx, lim, status) (idx)
#endif

// cell grid of one molecule: cells of edge `cell` starting at `lo`, cell id = base + local
struct MolGrid {
    float lo[3];
    float inv_cell;
    int dims[3];
    int base;         // first global cell of this molecule
    float margin;     // conservative slack of the FP32 neighbour test (A)
    float rmax;       // largest probe-inflated radius of the molecule
    int pad[2];
};

struct BuildArgs {
    const double* xyz;
    const double* radii;
    double probe;
    int n;
    int n_mol;
    const long long* offsets;   // device, n_mol + 1 (NULL: one molecule)
    double skin;
    const int* skip;   // non-NULL and *skip != 0: the previous cell list is reused (nothing to do)
    int* zero_word;    // non-NULL: zero_word[0..1] set to 0 by the build's first kernel (the next atom
                       // kernels' deferred count, and a spare word)
    int max_cells;
    // outputs / scratch
    double* R;         // n
    float2* Rhl;       // n: R as a float pair (hi, lo), for the float-float area terms
    float4* f4;        // n  (x, y, z, R) float
    int* molid;        // n
    int* rank;         // n
    int* cell;         // n
    unsigned* bbox;    // n_mol * 8 (ordered-int encoded: min xyz, max xyz, rmax, pad)
    MolGrid* grids;    // n_mol
    int* counts;       // max_cells + 1
    int* cstart;       // max_cells + 1
    int* sidx;         // n
    float4* sf4;       // n
    int* blocksums;    // scan scratch
    unsigned* sync;    // BUILD_SYNC_WORDS, zero between calls: single-molecule build's partial boxes + ticket
    int* status;
    int* ncells_out;   // device int: total cells used
};

struct AtomArgs {
    const double* xyz;
    const double* R;
    const float2* Rhl;      // R as (hi, lo) floats
    const float4* sf4;
    const int* sidx;
    const int* molid;
    const int* cstart;
    const MolGrid* grids;
    const double* w;        // NULL = ones
    double* areas;
    double* grad;           // NULL = no gradient
    double* vol;            // per-atom volumes vol(B_i cap L_i); NULL = not computed
    double* vgrad;          // d(sum_i vw_i V_i) / dx (n x 3); NULL = not computed
    const double* vw;       // volume weights vw (n); NULL = ones (the union volume's gradient)
    // per-molecule completion (NULL = off; not with volumes): every atom adds 1 to
    // mol_done[molid] (device memory, zero at the start) once its area and gradient are final,
    // after a system-scope fence; the molecule's last atom then sets mol_ready[molid] = 1
    // (caller memory, which may be mapped host memory)
    int* mol_done;
    int* mol_ready;
    const long long* mol_off;   // batch offsets (n_mol + 1, device): molecule m is [off[m], off[m+1])
    // resident Verlet lists of a batch (NULL = none): molecule m's lists live at arena index
    // mol_base[m] + (i - mol_off[m]) with molecule-local entries (mol_base[m] < 0: no lists);
    // mol_reuse[m] != 0: reuse them; an atom whose list overflows marks its slot invalid
    const long long* mol_base;
    const int* mol_reuse;
    // the cell list holds the skin band too (skin > 0): keep only the balls that overlap B_i
    // now in the plane table
    int skin_band;
    // single-molecule calls with neighbour lists: the carry kernel keeps each atom's cell from
    // the previous call where it can (list-reusing calls) and appends the other atoms (sorted
    // positions) to redo_list, counted in *redo_count (zero when the kernels start); the cell
    // kernel then builds those
    int carry;
    int* redo_list;
    int* redo_count;
    int n;
    int* status;
    // complex export (NULL = off): records {i, v0, v1, v2, v3}
    int* rec;
    long long max_rec;
    unsigned long long* nrec;
    // deferral: the fast pass appends sorted positions it cannot hold to defer_list; the
    // large pass reads work_list[0 .. *work_count)
    int* defer_list;
    int* defer_count;       // zero when the first atom kernel starts (cleared by the cell-list build)
    const int* work_list;
    const int* work_count;
    // per-atom cell records (by sorted position) between the cell kernel and the terms
    // kernel; NULL = one fused kernel
    void* cells;
    // optional timing: events recorded on the stream after the cell, classification, terms
    // and large-capacity kernels (NULL = none)
    cudaEvent_t* ev;
    // Verlet neighbour lists (single molecule, skin > 0; NULL = none): candidates of atom i
    // at nbl[i * NBL_CAP .. + nbn[i]).  *reuse != 0: take the candidates from the lists (the
    // cell list was not rebuilt); else gather them from the cell list and store them with
    // the reference coordinates and radii.  Either way only the balls that overlap B_i at
    // the current positions enter the plane table.  *lists_bad is set when a list cannot
    // hold its atom's candidates (the next call rebuilds).
    int* nbl;
    int* nbn;
    const int* reuse;
    int* lists_bad;
    double* ref_xyz;
    double* ref_rad;
    const double* radii_in;
};
constexpr int NBL_CAP = 122;   // list capacity per atom (atoms within R_i + R_j + skin)

// Shrake-Rupley numerical SASA (cross-check): m unit vectors pts[3m] (device)
struct SRArgs {
    const double* xyz;
    const double* R;
    const float4* sf4;
    const int* sidx;
    const int* molid;
    const int* cstart;
    const MolGrid* grids;
    const float* pts;
    int m;
    int n;
    double* areas;
    int* exposed;                 // NULL = not written
    unsigned long long* tests;    // NULL = not counted: point-neighbour tests performed
    int* status;
};

cudaError_t launch_build(const BuildArgs& a, cudaStream_t s);
// Verlet skin test: vstate[2] = reuse the lists (valid, every atom within skin/2 of its
// reference position, radii unchanged, no list overflow); vstate[0..1] scratch, [3] overflow
cudaError_t launch_verlet_check(const double* xyz, const double* radii, const double* ref_xyz, const double* ref_rad,
                                int n, int valid, double skin, int* vstate, cudaStream_t s);
// the Verlet skin test of a batch of resident molecules: reuse[m] for each molecule (see
// k_verlet_check_batch); vmol: 3 ints per molecule of scratch
cudaError_t launch_verlet_check_batch(const double* xyz, const double* radii, const double* ref_xyz,
                                      const double* ref_rad, const int* nbn, const long long* off,
                                      const long long* base, int n, int n_mol, double skin, int* vmol, int* reuse,
                                      cudaStream_t s);
cudaError_t launch_sr(const SRArgs& a, cudaStream_t s);
cudaError_t launch_atoms_f32(const AtomArgs& a, bool grad, cudaStream_t s);
cudaError_t launch_atoms_f64(const AtomArgs& a, bool grad, cudaStream_t s);
// whether n atoms fit one wave of the fused cell + classification kernel (mixed / FP64 form)
bool atoms_one_wave_f32(int n);
bool atoms_one_wave_f64(int n);
size_t scan_scratch_ints(int max_cells);
size_t cell_record_bytes();

}  // namespace dsasa
