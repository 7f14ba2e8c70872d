// Device-side building blocks shared by the SPAI and GMRES-IR kernels:
// precision storage types, warp/block reductions, double-double arithmetic
// and a bounded grid-wide barrier for co-resident (cooperative) launches.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/spai_ir.h"

namespace spai {

// ---------------------------------------------------------------- precision

template <class S> struct Compute { typedef float T; };       // half, float -> float
template <> struct Compute<double> { typedef double T; };     // double -> double

__device__ __forceinline__ float to_c(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_c(float v) { return v; }
__device__ __forceinline__ double to_c(double v) { return v; }

template <class S> __device__ __forceinline__ S from_f(float v);
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <class S> __device__ __forceinline__ S from_d(double v);
template <> __device__ __forceinline__ __half from_d<__half>(double v) { return __double2half(v); }
template <> __device__ __forceinline__ float from_d<float>(double v) { return __double2float_rn(v); }
template <> __device__ __forceinline__ double from_d<double>(double v) { return v; }

// round a compute-type value to the storage precision S, returned in the
// compute type (the "store in u_f" step of the FP16-storage model)
template <class S> __device__ __forceinline__ typename Compute<S>::T rnd(typename Compute<S>::T v);
template <> __device__ __forceinline__ float rnd<__half>(float v) { return __half2float(__float2half_rn(v)); }
template <> __device__ __forceinline__ float rnd<float>(float v) { return v; }
template <> __device__ __forceinline__ double rnd<double>(double v) { return v; }

template <class T> __device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }
template <> __device__ __forceinline__ __half ldcg<__half>(const __half* p)
{
    unsigned short r;
    asm volatile("ld.global.cg.u16 %0, [%1];" : "=h"(r) : "l"(p));
    return __ushort_as_half(r);
}

// ---------------------------------------------------------------- reductions

template <class T> __device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <class T> __device__ __forceinline__ T warp_max(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// sum within aligned groups of L lanes (L a power of two <= 32)
template <int L, class T> __device__ __forceinline__ T group_sum(T v)
{
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block-wide sum; every thread gets the result.  red must
// hold 33 elements of T in shared memory.
template <class T> __device__ T block_sum(T v, T* red)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        T t = lane < nw ? red[lane] : T(0);
        t = warp_sum(t);
        if (lane == 0) red[32] = t;
    }
    __syncthreads();
    T r = red[32];
    __syncthreads();
    return r;
}
template <class T> __device__ T block_max(T v, T* red)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_max(v);
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        T t = lane < nw ? red[lane] : T(0);
        t = warp_max(t);
        if (lane == 0) red[32] = t;
    }
    __syncthreads();
    T r = red[32];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------- double-double
// Error-free transformations (Knuth TwoSum, FMA-based TwoProd; Dekker 1971,
// Ogita-Rump-Oishi 2005) used for the quad-precision residual.

__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e)
{
    s = a + b;
    double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void two_prod(double a, double b, double& p, double& e)
{
    p = a * b;
    e = fma(a, b, -p);
}
// (hi, lo) += a (double)
__device__ __forceinline__ void dd_add(double& hi, double& lo, double a)
{
    double s, e;
    two_sum(hi, a, s, e);
    e += lo;
    hi = s + e;
    lo = e - (hi - s);
}
// (hi, lo) -= a * b exactly-rounded product accumulation
__device__ __forceinline__ void dd_sub_prod(double& hi, double& lo, double a, double b)
{
    double p, pe;
    two_prod(a, b, p, pe);
    double s, e;
    two_sum(hi, -p, s, e);
    e += lo - pe;
    hi = s + e;
    lo = e - (hi - s);
}

// ---------------------------------------------------------------- grid barrier
// A barrier over all blocks of a co-resident (cooperative) launch.  The
// counter is monotonic: barrier number e completes when it reaches
// e * gridDim.x.  Every wait is bounded by a clock budget; on expiry the
// block records SPAI_ERR_TIMEOUT in *err and the barrier returns false, and
// any block that sees a non-zero *err also returns false, so all blocks
// leave the kernel.

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_i32(const int* p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct GridBarrier {
    unsigned* count;   // zeroed before the launch
    int* err;          // zeroed before the launch
    long long limit;   // clock64 cycles before a wait gives up
    unsigned nblocks;  // blocks taking part (the grid, or one system's blocks of a batch)
};

struct NoBarrierWork {
    __device__ void operator()() const {}
};

// `epoch` is a per-block counter kept in shared memory by the caller and
// advanced identically by every block.  `work` runs on thread 0 after the
// block has arrived and before it starts waiting for the others (short
// serial work hides in the wait); the wait's clock budget starts after it.
template <class Work = NoBarrierWork>
__device__ __forceinline__ bool grid_sync(const GridBarrier& gb, unsigned* epoch, int* s_flag,
                                          const Work& work = Work())
{
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned e = *epoch + 1u;
        *epoch = e;
        const unsigned target = e * gb.nblocks;
        // release: the bar.sync above orders the block's writes before it
        red_release_add_u32(gb.count, 1u);
        work();
        int ok = 1;
        const long long t0 = clock64();
        unsigned spins = 0;
        while (ld_acquire_u32(gb.count) < target) {
            if (((++spins) & 63u) == 0u) {
                if (ld_relaxed_i32(gb.err) != 0) { ok = 0; break; }
                if (clock64() - t0 > gb.limit) {
                    atomicCAS(gb.err, 0, SPAI_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

}  // namespace spai

// The structural check of a CSR on the device, one thread per row: rowptr[0]
// = 0, rowptr[n] = nnz, rows in order and inside [0, nnz], columns inside
// [0, n) and strictly ascending (flag 1); empty rows (flag 2) unless
// allow_empty.  Internal linkage: each translation unit that launches it
// has its own copy.
static __global__ void k_csr_check(int64_t n, int64_t nnz, const int64_t* __restrict__ rp,
                                   const int32_t* __restrict__ col, int* __restrict__ flags, int allow_empty)
{
    int f = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = rp[i], e = rp[i + 1];
        if ((i == 0 && b != 0) || (i == n - 1 && e != nnz)) f |= 1;
        if (b < 0 || e < b || e > nnz) { f |= 1; continue; }
        if (e == b) {
            if (!allow_empty) f |= 2;
            continue;
        }
        int prev = -1;
        for (int64_t q = b; q < e; q++) {
            const int c = col[q];
            if (c < 0 || c >= n || c <= prev) { f |= 1; break; }
            prev = c;
        }
    }
    if (f) atomicOr(flags, f);
}

#define SPAI_CUDA_TRY(expr)                                   \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) {                              \
            spai_set_last_cuda_error(_e);                     \
            return _e == cudaErrorMemoryAllocation ? SPAI_ERR_NO_MEMORY : SPAI_ERR_CUDA; \
        }                                                     \
    } while (0)

void spai_set_last_cuda_error(cudaError_t e);
