// Instantiation of the SPAI column kernel for u_f = single.
#include "spai_column.cuh"
#include "spai_cta.cuh"

int launch_spai_single(const spai::SpaiArgs& a, bool adaptive, int num_sms, size_t smem_cap, cudaStream_t s)
{
    return spai::launch_spai_t<float>(a, adaptive, num_sms, smem_cap, s);
}
