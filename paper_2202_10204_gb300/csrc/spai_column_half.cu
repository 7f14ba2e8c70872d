// Instantiation of the SPAI column kernel for u_f = half.
#include "spai_column.cuh"
#include "spai_cta.cuh"
#include "spai_big.cuh"

int launch_spai_half(const spai::SpaiArgs& a, bool adaptive, int num_sms, size_t smem_cap, cudaStream_t s)
{
    return spai::launch_spai_t<__half>(a, adaptive, num_sms, smem_cap, s);
}

int launch_spai_big_half(const spai::SpaiArgs& a, bool adaptive, const int32_t* list, const int* count, int grid,
                          unsigned char* slab, size_t slab_bytes, int mcap, int ccap, cudaStream_t s)
{
    return spai::launch_spai_big_t<__half>(a, adaptive, list, count, grid, slab, slab_bytes, mcap, ccap, s);
}
