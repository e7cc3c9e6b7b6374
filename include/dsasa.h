/*
 * dsasa.h - C ABI of the GB300 dSASA library (libdsasa.so).
 *
 * Computes, for N atoms with centres p_i and radii r_i, the solvent accessible surface
 * area A_i of every atom and the gradient of sum_i w_i A_i with respect to the centres,
 * by the exact inclusion-exclusion method of the paper (Sec. "dSASA: an analytical method
 * for SASA"):
 *   - weighted points p'_i = (p_i, d_i) with d_i = R_i^2, R_i = fl64(r_i + probe);
 *   - the weighted Delaunay tetrahedrization (Step 1) is built locally per atom as the
 *     power (Laguerre) cell L_i clipped by the atom's overlapping neighbours;
 *   - the dual complex C (Step 2) is its alpha = 0 subcomplex: a simplex is in C iff the
 *     Laguerre-intersection cells LI_i = L_i cap B_i of its vertices intersect;
 *   - A_i follows Eq. (sainexclu) with the vertex, edge and triangle terms of
 *     Eqs. (vertex), (phiedge)/(edge) and (trianglev); the gradient follows Eq. (inexclu)
 *     with Eq. (triangle), evaluated as a per-atom gather (no atomics, deterministic).
 *
 * Conventions shared by every entry point
 *   - All array arguments of dsasa_compute* are DEVICE pointers (cudaMalloc'd or torch CUDA
 *     tensors) on the context's device, unless the name ends in _host.  The caller owns
 *     them; the library never frees or retains them past the call.
 *   - coords: double[n][3], row-major (x, y, z of atom i at coords[3i..3i+2]), Angstrom.
 *   - radii: double[n], van der Waals radii WITHOUT the probe, Angstrom.
 *   - areas_out: double[n], A_i in Angstrom^2.  grad_out: double[n][3] or NULL.
 *   - Work is enqueued on the context's stream and returns immediately.  Argument errors
 *     are returned synchronously and nothing is enqueued.  Errors found on the device
 *     (capacity overflow, unresolved exact predicate) are recorded in a device status word
 *     that dsasa_status_sync() reads; the atoms concerned get NaN outputs.  Nothing aborts,
 *     nothing calls __trap, every device loop is bounded.
 *   - The context owns its scratch (cell list, sorted atom copies, status word).  It grows
 *     scratch on demand unless cfg.max_atoms fixes the capacity (then a larger n returns
 *     DSASA_ERR_CAPACITY).  With a fixed capacity no call allocates, so calls can be
 *     captured in a CUDA graph after one warm-up call.
 *   - A context is not thread-safe; use one context per host thread / stream.
 */
#ifndef DSASA_H
#define DSASA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dsasa_ctx dsasa_ctx;

typedef enum {
    DSASA_OK = 0,
    DSASA_ERR_ARG = 1,           /* invalid argument (NULL pointer, n < 0, non-finite probe, ...) */
    DSASA_ERR_OOM = 2,           /* device allocation failed */
    DSASA_ERR_CAPACITY = 3,      /* a fixed capacity was exceeded (atoms, neighbours, cell faces) */
    DSASA_ERR_UNRESOLVED = 4,    /* an exact predicate exceeded its expansion capacity */
    DSASA_ERR_CUDA = 5,          /* a CUDA runtime call failed (see dsasa_last_error) */
    DSASA_ERR_UNIMPLEMENTED = 6,
    DSASA_ERR_DEGENERATE = 7,    /* a tie that Simulation of Simplicity cannot break was met
                                    (coincident atoms); exact ties of co-spherical or
                                    co-planar atoms are broken as the regular triangulation
                                    breaks them and are not errors */
    DSASA_ERR_INPUT = 8,         /* non-finite coordinate or radius found on the device */
    DSASA_ERR_CHECK = 9          /* the checked build (compiled with DSASA_CHECKED) found an
                                    index out of its array on the device; the access was
                                    redirected inside the array and the call's results are void */
} dsasa_status;

/* Precision of the arithmetic (the predicates that decide which simplices exist are exact
 * in both modes):
 *   DSASA_MIXED - the geometry of every area and gradient term (vectors, triple points,
 *                 sqrt, atan2) in FP32; the radius quantities (R_i, R_i^2, R_i^2 - R_j^2)
 *                 enter the area terms as float-float pairs and all area terms of an atom are
 *                 one float-float warp sum; the per-atom constants (multiples of 2 pi R_i^2)
 *                 are added once in FP64.  The gradient contributions of an atom are summed
 *                 in int64 fixed point (2^-40; each FP32 term rounded once, the sum exact and
 *                 independent of its order).  Predicates are filtered in FP32, then FP64, then
 *                 decided by exact expansions.  The one FP32 quantity that cancels without
 *                 bound, the height of a triangle's triple points over the plane of its
 *                 centres (R_i^2 - |z|^2), is taken from the float64 coordinates when its
 *                 square is below 0.01 R_i^2: the lens gradient is linear in it.
 *                 Limit: the neighbour vectors enter the terms rounded to float, which leaves
 *                 an absolute gradient error of up to about 3e-5 (A^2 / A) per atom; an atom
 *                 whose gradient is below about 0.03 (nearly buried, or a sliver) can
 *                 therefore miss a 1e-3 relative bound with a 1e-2 floor.  DSASA_FP64 has no
 *                 such limit.
 *   DSASA_FP64  - every term in FP64; predicates filtered in FP64, then exact. */
enum { DSASA_MIXED = 0, DSASA_FP64 = 1 };

typedef struct {
    int precision;      /* DSASA_MIXED or DSASA_FP64 */
    double skin;        /* Verlet skin in Angstrom (>= 0).  0: the cell list is rebuilt every call.
                         * > 0: single-molecule calls keep per-atom candidate lists (atoms
                         * within R_i + R_j + skin) on the device and reuse them, without
                         * rebuilding the cell list, while every atom stays within skin / 2 of
                         * its position at the last rebuild and n, the radii and the probe are
                         * unchanged (tested on the device: graph-capturable).  The simplices
                         * are recomputed every call; results do not depend on reuse beyond
                         * rounding. */
    int64_t max_atoms;  /* fixed capacity in atoms, or 0 to grow on demand */
    int64_t max_cells;  /* cap on cell-list cells (0 = default 2^22); larger boxes use coarser cells */
    int carry;          /* with skin > 0, on calls that reuse the lists: keep each atom's cell
                         * from the previous call (its faces' planes at the current positions)
                         * when exact predicates certify that it is still the cell and no new
                         * neighbour cuts it; the other cells are built afresh.  The incremental
                         * update of the complex across MD steps (the paper's Conclusions).  The
                         * simplices of the complex are the same as a fresh build's, the areas
                         * and gradient equal up to the rounding of the terms.  0: off; 1
                         * (default): for molecules of more than one wave of the fused cell
                         * kernel (about 5,400 atoms on a GB300), where it pays; 2: always. */
} dsasa_config;

/* Fills cfg with defaults: MIXED, skin 0, grow on demand, default cell cap, carry 1 (auto). */
void dsasa_default_config(dsasa_config* cfg);

/* Creates a context on `device` (CUDA ordinal) bound to `cuda_stream` (a cudaStream_t, or
 * NULL for the legacy default stream).  cfg may be NULL (defaults).  On success *out holds
 * the context (free it with dsasa_destroy). */
dsasa_status dsasa_create(dsasa_ctx** out, int device, void* cuda_stream, const dsasa_config* cfg);

/* Rebinds the context to another stream of the same device. */
dsasa_status dsasa_set_stream(dsasa_ctx* ctx, void* cuda_stream);

/* Changes the precision mode (DSASA_MIXED / DSASA_FP64) of later calls. */
dsasa_status dsasa_set_precision(dsasa_ctx* ctx, int precision);

/* SASA per atom and, if grad_out != NULL, grad_out[j] = d(sum_i A_i)/d(p_j).
 * Paper: Eqs. (sainexclu) and (inexclu).  n = 0 is valid (nothing is enqueued). */
dsasa_status dsasa_compute(dsasa_ctx* ctx, const double* coords, const double* radii, double probe,
                           int64_t n, double* areas_out, double* grad_out);

/* Molecular volume (an extension the paper names; no equation of the paper defines it):
 * as dsasa_compute, and also volumes_out[i] = vol(B_i cap L_i), the part of the probe-
 * inflated ball of atom i in its power (Laguerre) cell, so that sum_i volumes_out[i] is the
 * volume of the union of the balls (the solvent-accessible volume); and, if vol_grad_out !=
 * NULL, vol_grad_out[j] = d(sum_i V_i)/d(p_j) (double[n][3]).  Computed from the same cell
 * by the divergence theorem: V_i = (R_i A_i + sum_j h_ij s_ij) / 3 with s_ij the area of the
 * cell face ij inside B_i and h_ij its plane's distance from p_i; the gradient is minus the
 * faces' vector area.  areas_out and volumes_out are required (double[n], device). */
dsasa_status dsasa_compute_volume(dsasa_ctx* ctx, const double* coords, const double* radii, double probe,
                                  int64_t n, double* areas_out, double* grad_out, double* volumes_out,
                                  double* vol_grad_out);

/* Weighted molecular-volume gradient (the vector-Jacobian product of the per-atom volumes,
 * which reverse-mode differentiation of an energy sum_i c_i V_i needs): as
 * dsasa_compute_volume, with vol_grad_out[j] = d(sum_i w_i V_i)/d(p_j) for volume_weights w
 * (double[n], device; NULL means all ones, the union volume's gradient).  Moving p_j moves
 * only the face of each neighbour's cell towards j, so dV_i/dp_j = (s q - m) / |q| with s
 * the area and m the first moment (relative to p_i) of that face's part inside B_i,
 * q = p_j - p_i; the face is the same polygon in j's cell.  volumes_out and vol_grad_out
 * are required (device). */
dsasa_status dsasa_compute_volume_vjp(dsasa_ctx* ctx, const double* coords, const double* radii, double probe,
                                      int64_t n, const double* volume_weights, double* areas_out,
                                      double* volumes_out, double* vol_grad_out);

/* Shrake-Rupley numerical SASA, an on-device cross-check of the exact areas (no equation of
 * the paper; the numerical method of its accuracy comparison): unit_points is float[m][3]
 * (device, caller-owned) of unit vectors placed on every probe-inflated sphere; a point is
 * exposed when strictly outside every other ball overlapping the sphere;
 * areas_out[i] = 4 pi R_i^2 exposed_i / m and, if exposed_out != NULL, exposed_out[i] =
 * exposed_i (int32[n], device; -1 with a NaN area past 128 overlapping neighbours, reported
 * as DSASA_ERR_CAPACITY by dsasa_status_sync).  The per-point decision is taken in float32
 * without contraction: x = R_i s_k, q = float(p_j - p_i), d2 = (dx dx + dy dy) + dz dz,
 * covered iff d2 <= R_j^2; overlapping means |p_i - p_j|^2 < (R_i + R_j)^2 in float64. */
dsasa_status dsasa_compute_sr(dsasa_ctx* ctx, const double* coords, const double* radii, double probe,
                              int64_t n, const float* unit_points, int m, double* areas_out, int32_t* exposed_out);

/* Diagnostics: synchronises and writes 1 to *reused if the last call reused the Verlet
 * lists (skin > 0), else 0. */
dsasa_status dsasa_lists_reused(dsasa_ctx* ctx, int* reused);

/* Diagnostics: synchronises and writes the number of atoms whose cell the last call carried
 * from the previous call (dsasa_config.carry), else 0. */
dsasa_status dsasa_cells_carried(dsasa_ctx* ctx, int64_t* carried);

/* Diagnostics: synchronises and writes the number of point-neighbour tests the last
 * dsasa_compute_sr call performed (sum over atoms of m x overlapping neighbours). */
dsasa_status dsasa_sr_tests(dsasa_ctx* ctx, int64_t* tests);

/* As dsasa_compute, with grad_out[j] = d(sum_i w_i A_i)/d(p_j) for area_weights w
 * (double[n], device; NULL means all ones).  This vector-Jacobian product is what
 * reverse-mode differentiation of an energy sum_i gamma_i A_i needs. */
dsasa_status dsasa_compute_vjp(dsasa_ctx* ctx, const double* coords, const double* radii, double probe,
                               int64_t n, const double* area_weights, double* areas_out, double* grad_out);

/* Several independent molecules in one launch.  Molecule m owns atoms
 * [atom_offsets[m], atom_offsets[m+1]) of the concatenated device arrays; atom_offsets is a
 * HOST array of n_mol + 1 increasing values starting at 0.  Atoms of different molecules
 * never interact.  area_weights may be NULL; grad_out may be NULL. */
dsasa_status dsasa_compute_batch(dsasa_ctx* ctx, int n_mol, const int64_t* atom_offsets,
                                 const double* coords, const double* radii, double probe,
                                 const double* area_weights, double* areas_out, double* grad_out);

/* Resident Verlet lists for serving (no paper counterpart: neighbour lists kept on the
 * device across requests): an arena of capacity_atoms atom slots on
 * `device` holding, per atom, its candidate list (atoms within R_i + R_j + skin at the
 * list's build, molecule-local indices), the list length and the coordinates and radius
 * at the build.  The caller assigns each resident molecule a slot range [base, base + n)
 * and passes base to dsasa_compute_batch_resident; contexts that share an arena must use
 * the same skin and probe, and two calls in flight at once must not use the same slots.
 * A new arena holds no valid list.  dsasa_arena_invalidate marks the lists of a slot range
 * invalid (asynchronously on `cuda_stream`), as needed when a slot is given to another
 * molecule.  dsasa_arena_destroy synchronises the device and frees the arena. */
typedef struct dsasa_arena dsasa_arena;
dsasa_status dsasa_arena_create(dsasa_arena** out, int device, int64_t capacity_atoms);
dsasa_status dsasa_arena_invalidate(dsasa_arena* arena, int64_t base, int64_t n, void* cuda_stream);
void dsasa_arena_destroy(dsasa_arena* arena);

/* The serving form of dsasa_compute_batch (continuous batching; no paper counterpart): one
 * pass of the kernels over all molecules of the batch, as dsasa_compute_batch, with
 *   - arena / arena_base: NULL, or the resident lists: arena_base is a HOST array of n_mol
 *     values, molecule m's first slot in the arena or -1 for a molecule without resident
 *     lists.  Per molecule the device decides, as for one molecule (see dsasa_config.skin),
 *     whether its lists can be reused (every atom within skin / 2 of its position at the
 *     lists' build, radii unchanged, every list valid); reused or rebuilt, the results are the
 *     same up to rounding.  Needs a context with skin > 0 on the arena's device.
 *   - mol_ready: NULL, or n_mol int32 (caller memory the device can write: device memory or
 *     mapped / pinned host memory, zero on entry).  mol_ready[m] becomes 1 once molecule m's
 *     areas and gradient are final in areas_out / grad_out, while the kernels of the batch are
 *     still running, so a host polling pinned host memory can return finished molecules early.
 *     areas_out / grad_out may themselves be mapped host memory (zero-copy outputs).
 * Every molecule needs at least one atom; the other arguments as dsasa_compute_batch. */
dsasa_status dsasa_compute_batch_resident(dsasa_ctx* ctx, dsasa_arena* arena, int n_mol,
                                          const int64_t* atom_offsets, const int64_t* arena_base,
                                          const double* coords, const double* radii, double probe,
                                          const double* area_weights, double* areas_out, double* grad_out,
                                          int32_t* mol_ready);

/* Diagnostics: synchronises and writes, for the n_mol molecules of the last resident batch,
 * 1 if its lists were reused (0: rebuilt or none). */
dsasa_status dsasa_batch_reused(dsasa_ctx* ctx, int n_mol, int32_t* reused_host);

/* End-to-end convenience on HOST buffers: runs dsasa_compute_vjp on coords/radii/weights in
 * host memory, leaves areas (and grad if grad_host != NULL) in host memory and synchronises
 * the stream.  When every buffer is pinned (page-locked, hence mapped into the device's
 * address space) the kernels read and write them in place over the CPU-GPU link, with no
 * copy; otherwise (pageable memory) the inputs are copied to device staging buffers and the
 * outputs back.  weights_host may be NULL. */
dsasa_status dsasa_compute_host(dsasa_ctx* ctx, const double* coords_host, const double* radii_host,
                                double probe, int64_t n, const double* weights_host,
                                double* areas_host, double* grad_host);

/* Synchronises the context's stream and returns the device status of the calls since the
 * previous dsasa_status_sync (then clears it).  DSASA_OK if every atom was resolved. */
dsasa_status dsasa_status_sync(dsasa_ctx* ctx);

/* Diagnostics (no paper counterpart): synchronises the stream and writes to *deferred how
 * many atoms of the most recent compute call had a cell larger than the fast pass holds
 * (64 neighbour planes or 64 cell vertices) and were finished by the large-capacity pass. */
dsasa_status dsasa_deferred_count(dsasa_ctx* ctx, int64_t* deferred);

/* Per-kernel timing (diagnostics, no paper counterpart).  With timing enabled, each compute
 * call records CUDA events on the context's stream around its kernels; dsasa_kernel_times
 * synchronises the stream, writes to ms_out[DSASA_NPHASE] the summed device milliseconds per
 * phase over the calls since the last read (at most 256 calls are recorded) and their number
 * to *calls_out (may be NULL), and resets the sums.  Phases: */
#define DSASA_NPHASE 5
#define DSASA_PHASE_CELL_LIST 0   /* cell-list build (input pass, grid, scan, scatter) */
#define DSASA_PHASE_CELL 1        /* restricted power cell per atom (gather, sort, clipping); when
                                     all atoms fit one wave of the GPU this kernel also classifies,
                                     and DSASA_PHASE_CLASSIFY is (near) zero */
#define DSASA_PHASE_CLASSIFY 2    /* simplices of the cell in C (Steps 2a-2c) */
#define DSASA_PHASE_TERMS 3       /* area terms and gradient gathers */
#define DSASA_PHASE_LARGE 4       /* the large-capacity pass over deferred atoms */
dsasa_status dsasa_set_timing(dsasa_ctx* ctx, int enable);
dsasa_status dsasa_kernel_times(dsasa_ctx* ctx, double* ms_out, int64_t* calls_out);

/* Number of CUDA kernels this library has launched since it was loaded, over all contexts and
 * the no-allocation entry point (host-side count of launch statements; cudaMemsetAsync is not
 * counted).  Diagnostics, no paper counterpart; thread-safe. */
int64_t dsasa_kernel_launches(void);

/* Test hook for the error path of an exhausted device (no paper counterpart): the next
 * `count` device allocations that the library attempts fail as if cudaMalloc had returned
 * cudaErrorMemoryAllocation (nothing is allocated; the call that needed the memory returns
 * DSASA_ERR_OOM and leaves its context usable).  count <= 0 clears it.  Thread-safe. */
void dsasa_debug_fail_allocations(int count);

/* Diagnostic export of the dual complex C as seen by each atom's local cell.  For every atom
 * i and every simplex of C that contains i, one record of 5 int32 is written to `records`
 * (device, capacity `max_records`): {i, v0, v1, v2, v3} with the simplex's atom indices in
 * increasing order and -1 in unused slots (a vertex, an edge, a triangle or a tetrahedron).
 * *n_records (host) receives the number of records (when it exceeds max_records, only the
 * first max_records were written and DSASA_ERR_CAPACITY is returned).  Synchronises. */
dsasa_status dsasa_export_complex(dsasa_ctx* ctx, const double* coords, const double* radii, double probe,
                                  int64_t n, int32_t* records, int64_t max_records, int64_t* n_records);

/* Largest n that dsasa_compute_noalloc accepts. */
#define DSASA_NOALLOC_MAX_ATOMS 32768

/* dsasa_compute without any device allocation, for callers that must not have a library call
 * cudaMalloc or cudaFree: for example an application that provisions a fixed device-memory
 * budget up front, or code whose device memory belongs to another framework's pool.  (The
 * paper has no counterpart to this entry point; it concerns memory ownership only.)
 *   - Same inputs and outputs as dsasa_compute (device pointers, caller-owned; grad_out may be
 *     NULL), computed in the DSASA_MIXED precision on `cuda_stream` (a cudaStream_t or NULL)
 *     of the current device; no context is involved.
 *   - Its scratch is one static device array of about 4.3 MB, sized for at most
 *     DSASA_NOALLOC_MAX_ATOMS atoms and reserved on every GPU that loads the library until
 *     the process exits.  n > DSASA_NOALLOC_MAX_ATOMS returns DSASA_ERR_CAPACITY and enqueues
 *     nothing; n = 0 returns DSASA_OK.
 *   - Every call looks up the device address of that array in the CUDA context current on
 *     the calling thread (the address belongs to the context, not to the device ordinal).
 *     The first call in a context also loads the library's device code there; make that
 *     first call before any stream capture begins.
 *   - Every call shares the one array, which keeps the previous call's contents: calls that
 *     overlap on the GPU (other streams, other host threads) race.  Serialise them.
 *   - Blocking: the call synchronises `cuda_stream` and returns the device status of this
 *     call (DSASA_OK, DSASA_ERR_INPUT, DSASA_ERR_CAPACITY, DSASA_ERR_UNRESOLVED or
 *     DSASA_ERR_DEGENERATE with the meanings above); argument errors return DSASA_ERR_ARG. */
dsasa_status dsasa_compute_noalloc(const double* coords, const double* radii, double probe, int64_t n,
                                   double* areas_out, double* grad_out, void* cuda_stream);

/* Message describing the last error of this context ("" if none). */
const char* dsasa_last_error(const dsasa_ctx* ctx);

/* Releases the context and its scratch.  NULL is a no-op. */
void dsasa_destroy(dsasa_ctx* ctx);

/* Library version string. */
const char* dsasa_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DSASA_H */
