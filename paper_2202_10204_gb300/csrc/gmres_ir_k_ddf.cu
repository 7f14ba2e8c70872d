// Instantiation of the refinement kernels for (u, u_g, u_p) = (double, double, float):
// one translation unit per tuple, so that nvcc compiles them in parallel.
#include "ir_kernel.cuh"

namespace spai {
void ir_kernels_ddf(int rm, bool ls, IrKernels* k) { ir_kernels_t<double, double, float>(rm, ls, k); }
}  // namespace spai
