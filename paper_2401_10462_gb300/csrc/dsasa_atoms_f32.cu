// Mixed-precision instantiation of the per-atom kernel: FP32 terms, FP32 -> FP64 -> exact
// predicates (see dsasa_atoms.cuh).
#include "dsasa_atoms.cuh"

namespace dsasa {
cudaError_t launch_atoms_f32(const AtomArgs& a, bool grad, cudaStream_t s) { return launch_atoms_t<float>(a, grad, s); }
}  // namespace dsasa
