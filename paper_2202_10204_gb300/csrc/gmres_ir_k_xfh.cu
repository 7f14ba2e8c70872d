// Instantiation of the refinement kernels with half Krylov storage (u_g = single, u_p = half),
// for u = single and u = double: the one-reduction MGS only.
#include "ir_kernel.cuh"

namespace spai {
void ir_kernels_ffh(int rm, bool ls, IrKernels* k) { ir_kernels_ls<float, float, __half>(rm, ls, k); }
void ir_kernels_dfh(int rm, bool ls, IrKernels* k) { ir_kernels_ls<double, float, __half>(rm, ls, k); }
}  // namespace spai
