// Instantiation of the refinement kernels for (u, u_g, u_p) = (float, float, double):
// one translation unit per tuple, so that nvcc compiles them in parallel.
#include "ir_kernel.cuh"

namespace spai {
void ir_kernels_ffd(int rm, bool ls, IrKernels* k) { ir_kernels_t<float, float, double>(rm, ls, k); }
}  // namespace spai
