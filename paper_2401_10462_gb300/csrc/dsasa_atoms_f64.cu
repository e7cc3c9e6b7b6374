// All-FP64 instantiation of the per-atom kernel: FP64 terms, FP64 -> exact predicates
// (see dsasa_atoms.cuh).
#include "dsasa_atoms.cuh"

namespace dsasa {
cudaError_t launch_atoms_f64(const AtomArgs& a, bool grad, cudaStream_t s) { return launch_atoms_t<double>(a, grad, s); }
bool atoms_one_wave_f64(int n) { return cells_in_one_wave<double>(n); }
}  // namespace dsasa
