// Instantiation of the shared-memory tile SPAI kernel (spai_mid.cuh) for u_f = double.
#include "spai_mid.cuh"

namespace spai {

int launch_spai_mid_bin_double(const SpaiArgs& a, int bin, int num_sms, size_t smem_cap, cudaStream_t s)
{
    return launch_spai_mid_bin_t<double>(a, bin, num_sms, smem_cap, s);
}

}  // namespace spai
