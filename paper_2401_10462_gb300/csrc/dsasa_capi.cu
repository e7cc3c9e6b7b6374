// C ABI of the dSASA library (declared in include/dsasa.h): context, capacity management,
// argument validation, launches and the device status word.
#include "../../include/dsasa.h"
#include "dsasa_kernels.cuh"

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

using namespace dsasa;

constexpr int kTimingRing = 256;

namespace {
std::atomic<long long> g_launches{0};   // kernels launched by this library (all contexts)
std::atomic<int> g_fail_allocs{0};      // dsasa_debug_fail_allocations: allocations left to fail

// every device allocation of the library goes through here (so that the error path of an
// exhausted device can be tested without exhausting a device)
cudaError_t dev_alloc(void** p, size_t bytes) {
    int left = g_fail_allocs.load();
    while (left > 0) {
        if (g_fail_allocs.compare_exchange_weak(left, left - 1)) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
    }
    return cudaMalloc(p, bytes);
}
}
void dsasa::note_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// Resident Verlet lists of molecules kept on the device across calls (serving): per arena
// atom, the candidate list (molecule-local indices), its length (negative: no valid list)
// and the coordinates and radius at the list's build.
struct dsasa_arena {
    int device = 0;
    int64_t cap = 0;
    int* nbl = nullptr;
    int* nbn = nullptr;
    double* ref_xyz = nullptr;
    double* ref_rad = nullptr;
};

struct dsasa_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    dsasa_config cfg{};
    // capacities
    int64_t cap_atoms = 0;
    int64_t cap_mol = 0;
    int64_t cap_cells = 0;
    // scratch
    double* R = nullptr;
    float2* Rhl = nullptr;
    float4* f4 = nullptr;
    int* molid = nullptr;
    int* rank = nullptr;
    int* cell = nullptr;
    int* sidx = nullptr;
    float4* sf4 = nullptr;
    unsigned* bbox = nullptr;
    MolGrid* grids = nullptr;
    int* counts = nullptr;
    int* cstart = nullptr;
    int* blocksums = nullptr;
    unsigned* bsync = nullptr;   // single-molecule build: partial boxes + ticket (zero between calls)
    long long* offsets = nullptr;
    int* defer = nullptr;       // atoms the fast kernel pass defers to the large pass
    int* redo = nullptr;        // atoms whose cell the carry kernel could not keep
    int64_t carry_n = 0;        // atoms of the last call when it carried cells, else 0
    // per-molecule arrays of a batch: arena slot, reuse decision, skin-test scratch, completion
    long long* mol_base = nullptr;
    int* mol_reuse = nullptr;
    int* vmol = nullptr;
    int* mol_done = nullptr;
    unsigned char* cells = nullptr;   // per-atom cell records between the cell and terms kernels
    // Verlet lists (skin > 0): candidates per atom, reference coordinates / radii, state
    int* nbl = nullptr;
    int* nbn = nullptr;
    double* ref_xyz = nullptr;
    double* ref_rad = nullptr;
    int* vstate = nullptr;        // [0] max displacement^2 (float bits), [1] radii changed, [2] reuse, [3] overflow
    int64_t lists_n = 0;          // the lists hold this many atoms of the last single-molecule call
    double lists_probe = -1.0;
    int* status = nullptr;      // [0] status bits, [1] total cells, [2] deferred count, [3] redo count
    // optional per-kernel timing: events of up to kTimingRing calls since the last read
    bool timing = false;
    int n_timed = 0;
    cudaEvent_t ev[kTimingRing][DSASA_NPHASE + 1] = {};
    unsigned long long* nrec = nullptr;
    unsigned long long* sr_tests = nullptr;   // Shrake-Rupley point-neighbour tests of the last call
    // staging for the host-buffer entry point
    int64_t cap_host = 0;
    double* h_xyz = nullptr;
    double* h_rad = nullptr;
    double* h_w = nullptr;
    double* h_area = nullptr;
    double* h_grad = nullptr;
    char err[512] = {0};
};

namespace {

const char* const kVersion = "dsasa-gb300 0.1 (sm_103a)";

dsasa_status fail(dsasa_ctx* c, dsasa_status st, const char* fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        std::vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

dsasa_status cuda_fail(dsasa_ctx* c, cudaError_t e, const char* what) {
    return fail(c, e == cudaErrorMemoryAllocation ? DSASA_ERR_OOM : DSASA_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

template <class T> void dfree(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

void free_scratch(dsasa_ctx* c) {
    dfree(c->R); dfree(c->Rhl); dfree(c->f4); dfree(c->molid); dfree(c->rank); dfree(c->cell); dfree(c->sidx); dfree(c->sf4);
    dfree(c->bbox); dfree(c->grids); dfree(c->counts); dfree(c->cstart); dfree(c->blocksums); dfree(c->bsync); dfree(c->offsets);
    dfree(c->defer); dfree(c->redo); dfree(c->cells); dfree(c->mol_base); dfree(c->mol_reuse); dfree(c->vmol); dfree(c->mol_done);
    dfree(c->nbl); dfree(c->nbn); dfree(c->ref_xyz); dfree(c->ref_rad); dfree(c->vstate);
    c->lists_n = 0;
    c->cap_atoms = c->cap_mol = c->cap_cells = 0;
}
void free_host_staging(dsasa_ctx* c) {
    dfree(c->h_xyz); dfree(c->h_rad); dfree(c->h_w); dfree(c->h_area); dfree(c->h_grad);
    c->cap_host = 0;
}

int64_t cells_for(int64_t n, int64_t n_mol) { return 8 * n + 64 * n_mol + 64; }

dsasa_status ensure(dsasa_ctx* c, int64_t n, int64_t n_mol) {
    int64_t need_cells = cells_for(n, n_mol);
    if (n <= c->cap_atoms && n_mol <= c->cap_mol && need_cells <= c->cap_cells) return DSASA_OK;
    if (c->cfg.max_atoms > 0 && c->cap_atoms > 0)
        return fail(c, DSASA_ERR_CAPACITY, "n=%lld molecules=%lld exceed the fixed capacity (max_atoms=%lld)",
                    (long long)n, (long long)n_mol, (long long)c->cfg.max_atoms);
    if (n > 0x3fffffff || need_cells > 0x7ffffff0)
        return fail(c, DSASA_ERR_CAPACITY, "n=%lld is beyond the 32-bit index range of the kernels", (long long)n);
    // the stream may still use the old buffers
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
    free_scratch(c);
    int64_t na = n + n / 4 + 256, nm = n_mol + n_mol / 4 + 4;
    if (c->cfg.max_atoms > 0) { na = std::max<int64_t>(n, c->cfg.max_atoms); nm = std::max<int64_t>(nm, 4096); }
    int64_t nc = cells_for(na, nm);
    if (c->cfg.max_cells > 0 && c->cfg.max_cells < nc) nc = std::max<int64_t>(c->cfg.max_cells, 64);
    int64_t nbs = (int64_t)scan_scratch_ints((int)nc) + 16;
#define ALLOC(ptr, count)                                                               \
    e = dev_alloc((void**)&c->ptr, sizeof(*c->ptr) * (size_t)(count));                 \
    if (e != cudaSuccess) { free_scratch(c); return cuda_fail(c, e, "cudaMalloc " #ptr); }
    ALLOC(R, na) ALLOC(Rhl, na) ALLOC(f4, na) ALLOC(molid, na) ALLOC(rank, na) ALLOC(cell, na) ALLOC(sidx, na) ALLOC(sf4, na)
    ALLOC(bbox, 8 * nm) ALLOC(grids, nm) ALLOC(counts, nc + 1) ALLOC(cstart, nc + 1) ALLOC(blocksums, nbs)
    ALLOC(offsets, nm + 1) ALLOC(defer, na) ALLOC(redo, na) ALLOC(cells, na * (int64_t)cell_record_bytes()) ALLOC(bsync, BUILD_SYNC_WORDS)
    ALLOC(mol_base, nm) ALLOC(mol_reuse, nm) ALLOC(vmol, 3 * nm) ALLOC(mol_done, nm)
    e = cudaMemsetAsync(c->bsync, 0, sizeof(unsigned) * BUILD_SYNC_WORDS, c->stream);
    if (e != cudaSuccess) { free_scratch(c); return cuda_fail(c, e, "memset"); }
    if (c->cfg.skin > 0.0) {
        ALLOC(nbl, na * NBL_CAP) ALLOC(nbn, na) ALLOC(ref_xyz, 3 * na) ALLOC(ref_rad, na) ALLOC(vstate, 4)
        e = cudaMemsetAsync(c->vstate, 0, 4 * sizeof(int), c->stream);
        if (e != cudaSuccess) { free_scratch(c); return cuda_fail(c, e, "memset"); }
    }
#undef ALLOC
    c->cap_atoms = na;
    c->cap_mol = nm;
    c->cap_cells = nc;
    return DSASA_OK;
}

// the cell list of the inputs in the context's scratch (enqueued on its stream)
cudaError_t build_cells(dsasa_ctx* c, const double* coords, const double* radii, double probe, int64_t n, int n_mol,
                        const long long* offsets_dev, const int* skip = nullptr,
                        int* zero_word = nullptr) {
    BuildArgs b{};
    b.skip = skip;
    b.xyz = coords;
    b.radii = radii;
    b.probe = probe;
    b.n = (int)n;
    b.n_mol = n_mol;
    b.offsets = offsets_dev;
    b.skin = c->cfg.skin;
    b.max_cells = (int)c->cap_cells;
    b.R = c->R; b.Rhl = c->Rhl; b.f4 = c->f4; b.molid = c->molid; b.rank = c->rank; b.cell = c->cell;
    b.bbox = c->bbox; b.grids = c->grids; b.counts = c->counts; b.cstart = c->cstart; b.sidx = c->sidx;
    b.sf4 = c->sf4; b.blocksums = c->blocksums; b.sync = c->bsync; b.zero_word = zero_word; b.status = c->status; b.ncells_out = c->status + 1;
    return launch_build(b, c->stream);
}

// the serving extras of a batch: completion flags and resident lists
struct BatchExtras {
    int* mol_ready = nullptr;       // caller memory, n_mol ints, zero on entry
    dsasa_arena* arena = nullptr;   // resident lists (mol_base / mol_reuse already on the device)
};

dsasa_status run(dsasa_ctx* c, const double* coords, const double* radii, double probe, int64_t n, int n_mol,
                 const long long* offsets_dev, const double* w, double* areas, double* grad, int* rec,
                 int64_t max_rec, double* vol = nullptr, double* vgrad = nullptr, const double* vw = nullptr,
                 const BatchExtras& bx = BatchExtras()) {
    dsasa_status st = ensure(c, n, n_mol);
    if (st != DSASA_OK) return st;
    cudaEvent_t* ev = (c->timing && c->n_timed < kTimingRing) ? c->ev[c->n_timed++] : nullptr;
    if (ev) cudaEventRecord(ev[0], c->stream);
    // Verlet lists of one molecule: reused on the device when every atom stayed within half
    // the skin (a batch with resident lists decides per molecule before this call)
    const bool lists = c->nbl != nullptr && n_mol == 1 && bx.arena == nullptr;
    if (lists) {
        const int valid = c->lists_n == n && c->lists_probe == probe;
        cudaError_t ev_e = launch_verlet_check(coords, radii, c->ref_xyz, c->ref_rad, (int)n, valid, c->cfg.skin,
                                               c->vstate, c->stream);
        if (ev_e != cudaSuccess) return cuda_fail(c, ev_e, "Verlet check launch");
    }
    // the build also clears the deferred-atom count of the atom kernels that follow it
    cudaError_t e = build_cells(c, coords, radii, probe, n, n_mol, offsets_dev, lists ? c->vstate + 2 : nullptr,
                                c->status + 2);
    if (e != cudaSuccess) return cuda_fail(c, e, "cell-list launch");
    if (ev) cudaEventRecord(ev[1], c->stream);
    AtomArgs a{};

    a.xyz = coords;
    a.R = c->R;
    a.Rhl = c->Rhl;
    a.sf4 = c->sf4;
    a.sidx = c->sidx;
    a.molid = c->molid;
    a.cstart = c->cstart;
    a.grids = c->grids;
    a.w = w;
    a.areas = areas;
    a.grad = grad;
    a.vol = vol;
    a.vgrad = vol ? vgrad : nullptr;
    a.vw = vol ? vw : nullptr;
    a.n = (int)n;
    a.status = c->status;
    a.rec = rec;
    a.max_rec = max_rec;
    a.nrec = c->nrec;
    a.defer_list = c->defer;
    a.defer_count = c->status + 2;
    a.cells = c->cells;
    a.ev = ev ? ev + 2 : nullptr;
    if (lists) {
        a.nbl = c->nbl;
        a.nbn = c->nbn;
        a.reuse = c->vstate + 2;
        a.lists_bad = c->vstate + 3;
        a.ref_xyz = c->ref_xyz;
        a.ref_rad = c->ref_rad;
        a.radii_in = radii;
    }
    a.skin_band = c->cfg.skin > 0.0;
    // carried cells: always (carry 2), or (carry 1) for molecules of more than one wave of the
    // fused cell kernel, where they pay (within one wave the fused kernel is faster)
    if (lists && c->cfg.carry != 0) {
        const bool one_wave = c->cfg.precision == DSASA_FP64 ? atoms_one_wave_f64((int)n) : atoms_one_wave_f32((int)n);
        a.carry = c->cfg.carry == 2 || !one_wave;
    }
    a.redo_list = c->redo;
    a.redo_count = c->status + 3;   // cleared by the cell-list build
    a.mol_off = offsets_dev;
    if (bx.arena) {
        a.nbl = bx.arena->nbl;
        a.nbn = bx.arena->nbn;
        a.ref_xyz = bx.arena->ref_xyz;
        a.ref_rad = bx.arena->ref_rad;
        a.radii_in = radii;
        a.mol_base = c->mol_base;
        a.mol_reuse = c->mol_reuse;
    }
    if (bx.mol_ready) {
        e = cudaMemsetAsync(c->mol_done, 0, sizeof(int) * (size_t)n_mol, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "memset");
        a.mol_done = c->mol_done;
        a.mol_ready = bx.mol_ready;
    }
    e = c->cfg.precision == DSASA_FP64 ? launch_atoms_f64(a, grad != nullptr, c->stream)
                                       : launch_atoms_f32(a, grad != nullptr, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "atom kernel launch");
    // the lists now describe this call's molecule (or none: another layout overwrote the cells)
    c->lists_n = lists ? n : 0;
    c->carry_n = a.carry ? n : 0;
    c->lists_probe = probe;
    return DSASA_OK;
}

dsasa_status check_common(dsasa_ctx* c, const double* coords, const double* radii, double probe, int64_t n,
                          const double* areas) {
    if (!c) return DSASA_ERR_ARG;
    if (n < 0) return fail(c, DSASA_ERR_ARG, "n must be >= 0 (got %lld)", (long long)n);
    if (!std::isfinite(probe) || probe < 0) return fail(c, DSASA_ERR_ARG, "probe must be finite and >= 0");
    if (n > 0 && (!coords || !radii || !areas)) return fail(c, DSASA_ERR_ARG, "coords, radii and areas_out must be non-NULL");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    return DSASA_OK;
}

}  // namespace

// NVTX range over one entry point (host side: argument checks, allocation, enqueue), visible
// in a profiler's timeline next to the kernels it launched; free when no tool is attached
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

extern "C" {

void dsasa_default_config(dsasa_config* cfg) {
    if (!cfg) return;
    cfg->precision = DSASA_MIXED;
    cfg->skin = 0.0;
    cfg->max_atoms = 0;
    cfg->max_cells = 0;
    cfg->carry = 1;
}

const char* dsasa_version(void) { return kVersion; }

dsasa_status dsasa_create(dsasa_ctx** out, int device, void* cuda_stream, const dsasa_config* cfg) {
    if (!out) return DSASA_ERR_ARG;
    *out = nullptr;
    dsasa_ctx* c = new (std::nothrow) dsasa_ctx();
    if (!c) return DSASA_ERR_OOM;
    if (cfg) c->cfg = *cfg; else dsasa_default_config(&c->cfg);
    if ((c->cfg.precision != DSASA_MIXED && c->cfg.precision != DSASA_FP64) || !(c->cfg.skin >= 0.0) ||
        c->cfg.carry < 0 || c->cfg.carry > 2 ||
        c->cfg.max_atoms < 0 || c->cfg.max_cells < 0) {
        delete c;
        return DSASA_ERR_ARG;
    }
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = dev_alloc((void**)&c->status, 4 * sizeof(int));
    if (e == cudaSuccess) e = dev_alloc((void**)&c->nrec, sizeof(unsigned long long));
    if (e == cudaSuccess) e = dev_alloc((void**)&c->sr_tests, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, 4 * sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        if (c->status) cudaFree(c->status);
        if (c->nrec) cudaFree(c->nrec);
        if (c->sr_tests) cudaFree(c->sr_tests);
        delete c;
        return e == cudaErrorMemoryAllocation ? DSASA_ERR_OOM : DSASA_ERR_CUDA;
    }
    if (c->cfg.max_atoms > 0) {
        dsasa_status st = ensure(c, c->cfg.max_atoms, 1);
        if (st != DSASA_OK) { dsasa_destroy(c); return st; }
    }
    *out = c;
    return DSASA_OK;
}

dsasa_status dsasa_set_stream(dsasa_ctx* c, void* cuda_stream) {
    if (!c) return DSASA_ERR_ARG;
    c->stream = (cudaStream_t)cuda_stream;
    return DSASA_OK;
}

dsasa_status dsasa_set_precision(dsasa_ctx* c, int precision) {
    if (!c) return DSASA_ERR_ARG;
    if (precision != DSASA_MIXED && precision != DSASA_FP64) return fail(c, DSASA_ERR_ARG, "unknown precision %d", precision);
    c->cfg.precision = precision;
    return DSASA_OK;
}

dsasa_status dsasa_compute_vjp(dsasa_ctx* c, const double* coords, const double* radii, double probe, int64_t n,
                               const double* area_weights, double* areas_out, double* grad_out) {
    NvtxRange nvtx_range("dsasa_compute_vjp");
    dsasa_status st = check_common(c, coords, radii, probe, n, areas_out);
    if (st != DSASA_OK || n == 0) return st;
    return run(c, coords, radii, probe, n, 1, nullptr, area_weights, areas_out, grad_out, nullptr, 0);
}

dsasa_status dsasa_compute(dsasa_ctx* c, const double* coords, const double* radii, double probe, int64_t n,
                           double* areas_out, double* grad_out) {
    NvtxRange nvtx_range("dsasa_compute");
    return dsasa_compute_vjp(c, coords, radii, probe, n, nullptr, areas_out, grad_out);
}

dsasa_status dsasa_compute_volume(dsasa_ctx* c, const double* coords, const double* radii, double probe, int64_t n,
                                  double* areas_out, double* grad_out, double* volumes_out, double* vol_grad_out) {
    NvtxRange nvtx_range("dsasa_compute_volume");
    dsasa_status st = check_common(c, coords, radii, probe, n, areas_out);
    if (st != DSASA_OK || n == 0) return st;
    if (!volumes_out) return fail(c, DSASA_ERR_ARG, "volumes_out is NULL");
    return run(c, coords, radii, probe, n, 1, nullptr, nullptr, areas_out, grad_out, nullptr, 0, volumes_out,
               vol_grad_out);
}

dsasa_status dsasa_compute_volume_vjp(dsasa_ctx* c, const double* coords, const double* radii, double probe,
                                      int64_t n, const double* volume_weights, double* areas_out, double* volumes_out,
                                      double* vol_grad_out) {
    NvtxRange nvtx_range("dsasa_compute_volume_vjp");
    dsasa_status st = check_common(c, coords, radii, probe, n, areas_out);
    if (st != DSASA_OK || n == 0) return st;
    if (!volumes_out || !vol_grad_out) return fail(c, DSASA_ERR_ARG, "volumes_out and vol_grad_out are required");
    return run(c, coords, radii, probe, n, 1, nullptr, nullptr, areas_out, nullptr, nullptr, 0, volumes_out,
               vol_grad_out, volume_weights);
}

dsasa_status dsasa_compute_sr(dsasa_ctx* c, const double* coords, const double* radii, double probe, int64_t n,
                              const float* unit_points, int m, double* areas_out, int32_t* exposed_out) {
    NvtxRange nvtx_range("dsasa_compute_sr");
    dsasa_status st = check_common(c, coords, radii, probe, n, areas_out);
    if (st != DSASA_OK || n == 0) return st;
    if (!unit_points || m <= 0) return fail(c, DSASA_ERR_ARG, "need m > 0 unit points");
    st = ensure(c, n, 1);
    if (st != DSASA_OK) return st;
    cudaError_t e = build_cells(c, coords, radii, probe, n, 1, nullptr);
    if (e != cudaSuccess) return cuda_fail(c, e, "cell-list launch");
    c->lists_n = 0;   // the cell list now belongs to this call
    SRArgs a{};
    a.xyz = coords;
    a.R = c->R;
    a.sf4 = c->sf4;
    a.sidx = c->sidx;
    a.molid = c->molid;
    a.cstart = c->cstart;
    a.grids = c->grids;
    a.pts = unit_points;
    a.m = m;
    a.n = (int)n;
    a.areas = areas_out;
    a.exposed = exposed_out;
    a.tests = c->sr_tests;
    a.status = c->status;
    if (c->sr_tests) cudaMemsetAsync(c->sr_tests, 0, sizeof(unsigned long long), c->stream);
    e = launch_sr(a, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "Shrake-Rupley launch");
    return DSASA_OK;
}

dsasa_status dsasa_lists_reused(dsasa_ctx* c, int* reused) {
    if (!c || !reused) return DSASA_ERR_ARG;
    *reused = 0;
    if (!c->vstate) return DSASA_OK;
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    int h[4] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(h, c->vstate, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "list state read");
    *reused = h[2];
    return DSASA_OK;
}

dsasa_status dsasa_cells_carried(dsasa_ctx* c, int64_t* carried) {
    if (!c || !carried) return DSASA_ERR_ARG;
    *carried = 0;
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    int h = 0;
    if (e == cudaSuccess && c->carry_n > 0) e = cudaMemcpy(&h, c->status + 3, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "redo count read");
    *carried = c->carry_n > 0 ? c->carry_n - h : 0;   // every atom is carried or redone
    return DSASA_OK;
}

dsasa_status dsasa_sr_tests(dsasa_ctx* c, int64_t* tests) {
    if (!c || !tests) return DSASA_ERR_ARG;
    unsigned long long h = 0;
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaMemcpy(&h, c->sr_tests, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "test count read");
    *tests = (int64_t)h;
    return DSASA_OK;
}

dsasa_status dsasa_compute_batch(dsasa_ctx* c, int n_mol, const int64_t* atom_offsets, const double* coords,
                                 const double* radii, double probe, const double* area_weights, double* areas_out,
                                 double* grad_out) {
    NvtxRange nvtx_range("dsasa_compute_batch");
    if (!c) return DSASA_ERR_ARG;
    if (n_mol < 0 || (n_mol > 0 && !atom_offsets)) return fail(c, DSASA_ERR_ARG, "invalid molecule offsets");
    if (n_mol == 0) return DSASA_OK;
    if (atom_offsets[0] != 0) return fail(c, DSASA_ERR_ARG, "atom_offsets[0] must be 0");
    for (int m = 0; m < n_mol; ++m)
        if (atom_offsets[m + 1] < atom_offsets[m]) return fail(c, DSASA_ERR_ARG, "atom_offsets must be non-decreasing");
    int64_t n = atom_offsets[n_mol];
    dsasa_status st = check_common(c, coords, radii, probe, n, areas_out);
    if (st != DSASA_OK || n == 0) return st;
    st = ensure(c, n, n_mol);
    if (st != DSASA_OK) return st;
    cudaError_t e = cudaMemcpyAsync(c->offsets, atom_offsets, sizeof(long long) * (size_t)(n_mol + 1),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "offsets upload");
    return run(c, coords, radii, probe, n, n_mol, c->offsets, area_weights, areas_out, grad_out, nullptr, 0);
}

dsasa_status dsasa_arena_create(dsasa_arena** out, int device, int64_t capacity_atoms) {
    if (!out || capacity_atoms <= 0 || capacity_atoms > 0x3fffffff) return DSASA_ERR_ARG;
    *out = nullptr;
    dsasa_arena* r = new (std::nothrow) dsasa_arena();
    if (!r) return DSASA_ERR_OOM;
    r->device = device;
    r->cap = capacity_atoms;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = dev_alloc((void**)&r->nbl, sizeof(int) * (size_t)capacity_atoms * NBL_CAP);
    if (e == cudaSuccess) e = dev_alloc((void**)&r->nbn, sizeof(int) * (size_t)capacity_atoms);
    if (e == cudaSuccess) e = dev_alloc((void**)&r->ref_xyz, sizeof(double) * 3 * (size_t)capacity_atoms);
    if (e == cudaSuccess) e = dev_alloc((void**)&r->ref_rad, sizeof(double) * (size_t)capacity_atoms);
    if (e == cudaSuccess) e = cudaMemset(r->nbn, 0xff, sizeof(int) * (size_t)capacity_atoms);   // no valid list
    if (e != cudaSuccess) {
        dsasa_arena_destroy(r);
        return e == cudaErrorMemoryAllocation ? DSASA_ERR_OOM : DSASA_ERR_CUDA;
    }
    *out = r;
    return DSASA_OK;
}

dsasa_status dsasa_arena_invalidate(dsasa_arena* r, int64_t base, int64_t n, void* cuda_stream) {
    if (!r || base < 0 || n < 0 || base + n > r->cap) return DSASA_ERR_ARG;
    if (n == 0) return DSASA_OK;
    cudaError_t e = cudaSetDevice(r->device);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(r->nbn + base, 0xff, sizeof(int) * (size_t)n, (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? DSASA_OK : DSASA_ERR_CUDA;
}

void dsasa_arena_destroy(dsasa_arena* r) {
    if (!r) return;
    cudaSetDevice(r->device);
    cudaDeviceSynchronize();
    if (r->nbl) cudaFree(r->nbl);
    if (r->nbn) cudaFree(r->nbn);
    if (r->ref_xyz) cudaFree(r->ref_xyz);
    if (r->ref_rad) cudaFree(r->ref_rad);
    delete r;
}

dsasa_status dsasa_compute_batch_resident(dsasa_ctx* c, dsasa_arena* arena, int n_mol, const int64_t* atom_offsets,
                                          const int64_t* arena_base, const double* coords, const double* radii,
                                          double probe, const double* area_weights, double* areas_out,
                                          double* grad_out, int32_t* mol_ready) {
    NvtxRange nvtx_range("dsasa_compute_batch_resident");
    if (!c) return DSASA_ERR_ARG;
    if (n_mol < 0 || (n_mol > 0 && !atom_offsets)) return fail(c, DSASA_ERR_ARG, "invalid molecule offsets");
    if (n_mol == 0) return DSASA_OK;
    if (atom_offsets[0] != 0) return fail(c, DSASA_ERR_ARG, "atom_offsets[0] must be 0");
    for (int m = 0; m < n_mol; ++m)
        if (atom_offsets[m + 1] <= atom_offsets[m]) return fail(c, DSASA_ERR_ARG, "every molecule needs atoms");
    if ((arena == nullptr) != (arena_base == nullptr)) return fail(c, DSASA_ERR_ARG, "arena and arena_base go together");
    if (arena) {
        if (!(c->cfg.skin > 0.0)) return fail(c, DSASA_ERR_ARG, "resident lists need a context with skin > 0");
        if (arena->device != c->device) return fail(c, DSASA_ERR_ARG, "the arena lives on another device");
        for (int m = 0; m < n_mol; ++m)
            if (arena_base[m] >= 0 && arena_base[m] + (atom_offsets[m + 1] - atom_offsets[m]) > arena->cap)
                return fail(c, DSASA_ERR_CAPACITY, "molecule %d does not fit the arena at %lld", m, (long long)arena_base[m]);
    }
    int64_t n = atom_offsets[n_mol];
    dsasa_status st = check_common(c, coords, radii, probe, n, areas_out);
    if (st != DSASA_OK) return st;
    st = ensure(c, n, n_mol);
    if (st != DSASA_OK) return st;
    cudaError_t e = cudaMemcpyAsync(c->offsets, atom_offsets, sizeof(long long) * (size_t)(n_mol + 1),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "offsets upload");
    BatchExtras bx;
    bx.mol_ready = mol_ready;
    if (arena) {
        e = cudaMemcpyAsync(c->mol_base, arena_base, sizeof(long long) * (size_t)n_mol, cudaMemcpyHostToDevice,
                            c->stream);
        if (e == cudaSuccess)
            e = launch_verlet_check_batch(coords, radii, arena->ref_xyz, arena->ref_rad, arena->nbn, c->offsets,
                                          c->mol_base, (int)n, n_mol, c->cfg.skin, c->vmol, c->mol_reuse, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "resident list check");
        bx.arena = arena;
    }
    return run(c, coords, radii, probe, n, n_mol, c->offsets, area_weights, areas_out, grad_out, nullptr, 0, nullptr,
               nullptr, nullptr, bx);
}

dsasa_status dsasa_batch_reused(dsasa_ctx* c, int n_mol, int32_t* reused_host) {
    if (!c || n_mol < 0 || (n_mol > 0 && !reused_host) || n_mol > c->cap_mol) return DSASA_ERR_ARG;
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess && n_mol > 0)
        e = cudaMemcpy(reused_host, c->mol_reuse, sizeof(int) * (size_t)n_mol, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "reuse flags read");
    return DSASA_OK;
}

dsasa_status dsasa_compute_host(dsasa_ctx* c, const double* coords_host, const double* radii_host, double probe,
                                int64_t n, const double* weights_host, double* areas_host, double* grad_host) {
    NvtxRange nvtx_range("dsasa_compute_host");
    dsasa_status st = check_common(c, coords_host, radii_host, probe, n, areas_host);
    if (st != DSASA_OK || n == 0) return st;
    cudaError_t e;
    // Pinned (page-locked) host buffers are mapped into the device's address space: the
    // kernels then read the inputs and write the outputs in host memory themselves, over the
    // coherent CPU-GPU link, with no staging copy either way.  Pageable buffers are copied.
    auto mapped = [](const void* h) -> void* {
        if (!h) return nullptr;
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, h) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
    };
    {
        const double* dx = (const double*)mapped(coords_host);
        const double* dr = (const double*)mapped(radii_host);
        const double* dw = (const double*)mapped(weights_host);
        double* da = (double*)mapped(areas_host);
        double* dg = (double*)mapped(grad_host);
        if (dx && dr && da && (!weights_host || dw) && (!grad_host || dg)) {
            st = run(c, dx, dr, probe, n, 1, nullptr, dw, da, dg, nullptr, 0);
            if (st != DSASA_OK) return st;
            e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
            return DSASA_OK;
        }
    }
    if (n > c->cap_host) {
        if (c->cfg.max_atoms > 0 && n > c->cfg.max_atoms)
            return fail(c, DSASA_ERR_CAPACITY, "n=%lld exceeds max_atoms", (long long)n);
        e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
        free_host_staging(c);
        int64_t cap = n + n / 4 + 256;
#define ALLOC(ptr, count)                                                           \
    e = dev_alloc((void**)&c->ptr, sizeof(double) * (size_t)(count));             \
    if (e != cudaSuccess) { free_host_staging(c); return cuda_fail(c, e, "cudaMalloc " #ptr); }
        ALLOC(h_xyz, 3 * cap) ALLOC(h_rad, cap) ALLOC(h_w, cap) ALLOC(h_area, cap) ALLOC(h_grad, 3 * cap)
#undef ALLOC
        c->cap_host = cap;
    }
    e = cudaMemcpyAsync(c->h_xyz, coords_host, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_rad, radii_host, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && weights_host)
        e = cudaMemcpyAsync(c->h_w, weights_host, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "host-to-device copy");
    st = run(c, c->h_xyz, c->h_rad, probe, n, 1, nullptr, weights_host ? c->h_w : nullptr, c->h_area,
             grad_host ? c->h_grad : nullptr, nullptr, 0);
    if (st != DSASA_OK) return st;
    e = cudaMemcpyAsync(areas_host, c->h_area, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && grad_host)
        e = cudaMemcpyAsync(grad_host, c->h_grad, sizeof(double) * 3 * (size_t)n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "device-to-host copy");
    return DSASA_OK;
}

dsasa_status dsasa_status_sync(dsasa_ctx* c) {
    NvtxRange nvtx_range("dsasa_status_sync");
    if (!c) return DSASA_ERR_ARG;
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    int h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(h, c->status, sizeof(h), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "status read");
    int s = h[0];
    if (s == 0) return DSASA_OK;
    if (s & ST_INPUT) return fail(c, DSASA_ERR_INPUT, "non-finite coordinate or radius (status 0x%x)", s);
    if (s & (ST_CAND_OVF | ST_TRI_OVF | ST_GRID_OVF | ST_EXPORT_OVF))
        return fail(c, DSASA_ERR_CAPACITY, "a fixed per-atom or grid capacity was exceeded (status 0x%x)", s);
    if (s & ST_CHECK) return fail(c, DSASA_ERR_CHECK, "a device bounds check failed (checked build; status 0x%x)", s);
    if (s & (ST_UNRESOLVED | ST_BADCELL))
        return fail(c, DSASA_ERR_UNRESOLVED, "an exact predicate or a cell could not be resolved (status 0x%x)", s);
    return fail(c, DSASA_ERR_DEGENERATE, "an exactly degenerate configuration was met (status 0x%x)", s);
}

dsasa_status dsasa_deferred_count(dsasa_ctx* c, int64_t* deferred) {
    if (!c || !deferred) return DSASA_ERR_ARG;
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    int h[3] = {0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(h, c->status, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "deferred count read");
    *deferred = h[2];
    return DSASA_OK;
}

dsasa_status dsasa_export_complex(dsasa_ctx* c, const double* coords, const double* radii, double probe, int64_t n,
                                  int32_t* records, int64_t max_records, int64_t* n_records) {
    NvtxRange nvtx_range("dsasa_export_complex");
    if (!c || !n_records) return DSASA_ERR_ARG;
    *n_records = 0;
    if (!records && max_records > 0) return fail(c, DSASA_ERR_ARG, "records is NULL");
    // areas are produced as a by-product into the host staging buffer
    dsasa_status st = check_common(c, coords, radii, probe, n, coords);
    if (st != DSASA_OK || n == 0) return st;
    double* areas = nullptr;
    cudaError_t e = dev_alloc((void**)&areas, sizeof(double) * (size_t)n);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc export areas");
    e = cudaMemsetAsync(c->nrec, 0, sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) { cudaFree(areas); return cuda_fail(c, e, "memset"); }
    st = run(c, coords, radii, probe, n, 1, nullptr, nullptr, areas, nullptr, records ? records : (int32_t*)areas,
             records ? max_records : 0);
    unsigned long long cnt = 0;
    if (st == DSASA_OK) {
        e = cudaMemcpyAsync(&cnt, c->nrec, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) st = cuda_fail(c, e, "export count");
    }
    cudaFree(areas);
    if (st != DSASA_OK) return st;
    *n_records = (int64_t)cnt;
    if ((int64_t)cnt > max_records) return fail(c, DSASA_ERR_CAPACITY, "%llu records > capacity %lld", cnt, (long long)max_records);
    return DSASA_OK;
}

const char* dsasa_last_error(const dsasa_ctx* c) { return c ? c->err : "null context"; }

int64_t dsasa_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

void dsasa_debug_fail_allocations(int count) { g_fail_allocs.store(count > 0 ? count : 0); }

dsasa_status dsasa_set_timing(dsasa_ctx* c, int enable) {
    if (!c) return DSASA_ERR_ARG;
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess && enable && !c->ev[0][0]) {
        for (int k = 0; k < kTimingRing && e == cudaSuccess; ++k)
            for (int j = 0; j <= DSASA_NPHASE && e == cudaSuccess; ++j) e = cudaEventCreate(&c->ev[k][j]);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "timing events");
    c->timing = enable != 0;
    c->n_timed = 0;
    return DSASA_OK;
}

dsasa_status dsasa_kernel_times(dsasa_ctx* c, double* ms_out, int64_t* calls_out) {
    if (!c || !ms_out) return DSASA_ERR_ARG;
    for (int j = 0; j < DSASA_NPHASE; ++j) ms_out[j] = 0.0;
    if (calls_out) *calls_out = 0;
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    for (int k = 0; k < c->n_timed && e == cudaSuccess; ++k)
        for (int j = 0; j < DSASA_NPHASE && e == cudaSuccess; ++j) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, c->ev[k][j], c->ev[k][j + 1]);
            ms_out[j] += ms;
        }
    if (e != cudaSuccess) return cuda_fail(c, e, "timing read");
    if (calls_out) *calls_out = c->n_timed;
    c->n_timed = 0;
    return DSASA_OK;
}

void dsasa_destroy(dsasa_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
    for (int k = 0; k < kTimingRing; ++k)
        for (int j = 0; j <= DSASA_NPHASE; ++j)
            if (c->ev[k][j]) cudaEventDestroy(c->ev[k][j]);
    free_scratch(c);
    free_host_staging(c);
    if (c->status) cudaFree(c->status);
    if (c->nrec) cudaFree(c->nrec);
    if (c->sr_tests) cudaFree(c->sr_tests);
    delete c;
}

}  // extern "C"
