// Mixed-precision instantiation of the per-atom kernel: FP32 terms, FP32 -> FP64 -> exact
// predicates (see dsasa_atoms.cuh).
#include "dsasa_atoms.cuh"

namespace dsasa {
cudaError_t launch_atoms_f32(const AtomArgs& a, bool grad, cudaStream_t s) { return launch_atoms_t<float>(a, grad, s); }
bool atoms_one_wave_f32(int n) { return cells_in_one_wave<float>(n); }
// bytes of one atom's cell record between the two kernels (the larger of the two precisions)
size_t cell_record_bytes() {
    return sizeof(CellRec<double, 64, 64>) > sizeof(CellRec<float, 64, 64>) ? sizeof(CellRec<double, 64, 64>)
                                                                            : sizeof(CellRec<float, 64, 64>);
}
}  // namespace dsasa
