// Instantiation of the refinement kernels with half Krylov storage (u_g = u_p = half),
// for u = single and u = double: the one-reduction MGS only.
#include "ir_kernel.cuh"

namespace spai {
void ir_kernels_fhh(int rm, bool ls, IrKernels* k) { ir_kernels_ls<float, __half, __half>(rm, ls, k); }
void ir_kernels_dhh(int rm, bool ls, IrKernels* k) { ir_kernels_ls<double, __half, __half>(rm, ls, k); }
}  // namespace spai
