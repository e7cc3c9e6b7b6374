// All-FP64 instantiation of the per-atom kernel: FP64 terms, FP64 -> exact predicates
// (see dsasa_atoms.cuh); also the mixed form's FP64 large-capacity pass.
#include "dsasa_atoms.cuh"

namespace dsasa {
cudaError_t launch_atoms_f64(const AtomArgs& a, bool grad, cudaStream_t s) { return launch_atoms_t<double>(a, grad, s); }
// The large-capacity pass in FP64 over a work list (the mixed form's deferred atoms and the
// atoms its cancellation detector flagged), launched in plain stream order after the mixed
// form's kernels.
cudaError_t launch_large_f64(const AtomArgs& big, bool grad, int blocks, cudaStream_t s) {
    if (grad) k_atoms<double, true, 128, 128, PH_ALL><<<blocks, WARPS * 32, 0, s>>>(big);
    else k_atoms<double, false, 128, 128, PH_ALL><<<blocks, WARPS * 32, 0, s>>>(big);
    return cudaGetLastError();
}
}  // namespace dsasa
