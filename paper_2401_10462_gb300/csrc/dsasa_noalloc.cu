// dsasa_compute_noalloc: the SASA + gradient computation without any device allocation.
//
// Some callers cannot let a library call cudaMalloc: a host application (an MD engine, a
// plugin host) that provisions a fixed device-memory budget up front and accounts for every
// byte, a process whose memory is owned by another framework's pool allocator, or a
// latency-critical loop that must never reach the CUDA allocator.  This entry point serves
// them: its scratch (cell list, sorted atom copies, status word) lives in one file-scope
// __device__ array of fixed size, so the call allocates nothing; the caller still passes its
// own input and output buffers.
//
// The array is reserved on every GPU that loads the library, for the life of the process.
#include "../../include/dsasa.h"
#include "dsasa_kernels.cuh"

#include <cuda_runtime.h>

using namespace dsasa;

namespace {

constexpr long long kMaxAtoms = DSASA_NOALLOC_MAX_ATOMS;
constexpr long long kMaxCells = 8 * kMaxAtoms + 64 + 64;   // the cell budget of one molecule
constexpr size_t al(size_t x) { return (x + 255) & ~size_t(255); }

// byte offsets of the regions inside the static scratch array (each 256-byte aligned)
constexpr size_t OFF_R = 0;
constexpr size_t OFF_RHL = al(OFF_R + sizeof(double) * kMaxAtoms);
constexpr size_t OFF_F4 = al(OFF_RHL + sizeof(float2) * kMaxAtoms);
constexpr size_t OFF_MOLID = al(OFF_F4 + sizeof(float4) * kMaxAtoms);
constexpr size_t OFF_RANK = al(OFF_MOLID + sizeof(int) * kMaxAtoms);
constexpr size_t OFF_CELL = al(OFF_RANK + sizeof(int) * kMaxAtoms);
constexpr size_t OFF_SIDX = al(OFF_CELL + sizeof(int) * kMaxAtoms);
constexpr size_t OFF_SF4 = al(OFF_SIDX + sizeof(int) * kMaxAtoms);
constexpr size_t OFF_BBOX = al(OFF_SF4 + sizeof(float4) * kMaxAtoms);
constexpr size_t OFF_GRID = al(OFF_BBOX + sizeof(unsigned) * 8);
constexpr size_t OFF_COUNTS = al(OFF_GRID + sizeof(MolGrid));
constexpr size_t OFF_CSTART = al(OFF_COUNTS + sizeof(int) * (kMaxCells + 1));
constexpr size_t OFF_BSUM = al(OFF_CSTART + sizeof(int) * (kMaxCells + 1));
constexpr size_t OFF_DEFER = al(OFF_BSUM + sizeof(int) * 4096);
constexpr size_t OFF_STATUS = al(OFF_DEFER + sizeof(int) * kMaxAtoms);
constexpr size_t OFF_SYNC = al(OFF_STATUS + sizeof(int) * 4);   // zero at load; the build leaves it zero
constexpr size_t kScratchBytes = al(OFF_SYNC + sizeof(unsigned) * BUILD_SYNC_WORDS);

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

}  // namespace

extern "C" dsasa_status dsasa_compute_noalloc(const double* coords, const double* radii, double probe, int64_t n,
                                              double* areas_out, double* grad_out, void* cuda_stream) {
    if (n < 0 || !(probe >= 0.0) || probe != probe || probe > 1e300) return DSASA_ERR_ARG;
    if (n == 0) return DSASA_OK;
    if (!coords || !radii || !areas_out) return DSASA_ERR_ARG;
    if (n > kMaxAtoms) return DSASA_ERR_CAPACITY;   // more atoms than the static scratch holds
    if ((long long)scan_scratch_ints((int)kMaxCells) > 4096) return DSASA_ERR_CAPACITY;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // The host-side name of the array is only a stand-in; its device address belongs to the
    // CUDA context that is current now (it changes after a device reset or under another
    // driver context), so it is looked up on every call, with that context current.  The
    // lookup is host work only; on the first call in a context it also loads the module,
    // which is why the first call must come before any stream capture.
    unsigned char* base = nullptr;
    {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return DSASA_ERR_CUDA;
        base = (unsigned char*)p;
    }
    int* status = (int*)(base + OFF_STATUS);
    // the array keeps the previous call's contents: clear what must start at zero (the
    // status word here; the cell counts are cleared inside the cell-list build)
    if (cudaMemsetAsync(status, 0, sizeof(int) * 4, s) != cudaSuccess) return DSASA_ERR_CUDA;
    BuildArgs b{};
    b.xyz = coords;
    b.radii = radii;
    b.probe = probe;
    b.n = (int)n;
    b.n_mol = 1;
    b.offsets = nullptr;
    b.skin = 0.0;
    b.max_cells = (int)kMaxCells;
    b.R = (double*)(base + OFF_R);
    b.Rhl = (float2*)(base + OFF_RHL);
    b.f4 = (float4*)(base + OFF_F4);
    b.molid = (int*)(base + OFF_MOLID);
    b.rank = (int*)(base + OFF_RANK);
    b.cell = (int*)(base + OFF_CELL);
    b.sidx = (int*)(base + OFF_SIDX);
    b.sf4 = (float4*)(base + OFF_SF4);
    b.bbox = (unsigned*)(base + OFF_BBOX);
    b.grids = (MolGrid*)(base + OFF_GRID);
    b.counts = (int*)(base + OFF_COUNTS);
    b.cstart = (int*)(base + OFF_CSTART);
    b.blocksums = (int*)(base + OFF_BSUM);
    b.sync = (unsigned*)(base + OFF_SYNC);
    b.zero_word = status + 2;   // the deferred count of the atom kernels (and a spare word)
    b.status = status;
    b.ncells_out = status + 1;
    if (launch_build(b, s) != cudaSuccess) return DSASA_ERR_CUDA;
    AtomArgs a{};
    a.xyz = coords;
    a.R = b.R;
    a.Rhl = b.Rhl;
    a.sf4 = b.sf4;
    a.sidx = b.sidx;
    a.molid = b.molid;
    a.cstart = b.cstart;
    a.grids = b.grids;
    a.w = nullptr;
    a.areas = areas_out;
    a.grad = grad_out;
    a.n = (int)n;
    a.status = status;
    a.defer_list = (int*)(base + OFF_DEFER);
    a.defer_count = status + 2;
    if (launch_atoms_f32(a, grad_out != nullptr, s) != cudaSuccess) return DSASA_ERR_CUDA;
    int h = 0;
    if (cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return DSASA_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return DSASA_ERR_CUDA;
    if (h == 0) return DSASA_OK;
    if (h & ST_INPUT) return DSASA_ERR_INPUT;
    if (h & (ST_CAND_OVF | ST_TRI_OVF | ST_GRID_OVF)) return DSASA_ERR_CAPACITY;
    if (h & (ST_UNRESOLVED | ST_BADCELL)) return DSASA_ERR_UNRESOLVED;
    return DSASA_ERR_DEGENERATE;
}
