// Instantiation of the refinement kernels with half Krylov storage (u_g = half, u_p = single),
// for u = single and u = double: the one-reduction MGS only.
#include "ir_kernel.cuh"

namespace spai {
void ir_kernels_fhf(int rm, bool ls, IrKernels* k) { ir_kernels_ls<float, __half, float>(rm, ls, k); }
void ir_kernels_dhf(int rm, bool ls, IrKernels* k) { ir_kernels_ls<double, __half, float>(rm, ls, k); }
}  // namespace spai
