// SPAI construction on the GPU: Algorithm 1 (Grote-Huckle / Sedlacek variant)
// run on B = A^T D (Section 4 scaling), giving the left preconditioner
// P = M^T D (Section 3: run on A^T, transpose).
//
// Steps (each a kernel):
//   k_scale        d_j = 1 / max_i |a_ji|: every column of A^T (row of A) to max-abs 1
//   k_bvals        b = fl(a_ij d_j) in u_f, once per nonzero of A (the gather reads these)
//   k_col_count / k_col_fill / k_col_sort
//                  structure of A^T (column lists of A) for pattern(A), pattern(A^2)
//                  and the candidate sets N_l of the adaptive step
//   k_pattern      initial J_k (identity, pattern(A), pattern(A^2)) with the fill cap,
//                  and |I_k| for sizing the per-column tiles
//   k_spai         (spai_column.cuh) one warp per column: gather, Householder QR,
//                  back substitution, explicit residual, adaptive augmentation
//                  (k_spai_cta, spai_cta.cuh: one CTA per column for shadows of up
//                  to 512 rows; k_spai_big, spai_big.cuh: larger shadows, the
//                  tile in global memory)
//   k_assemble     P row k = m_k * d(J_k) in CSR (column k of M is row k of P)
#include <climits>
#include <cstdio>
#include <cstring>

#include "common.cuh"
#include "internal.h"
#include "spai_big.cuh"

using namespace spai;

namespace {

constexpr int MAX_FILL = SPAI_MAX_FILL;
constexpr int MMAX_LIMIT = SPAI_MMAX_LIMIT;

// ---------------------------------------------------------------- scaling

// a != 0.0 on the bits (every value but +0 and -0), off the slow FP64 pipe
__device__ __forceinline__ bool nonzero_bits(double a) { return (__double_as_longlong(a) << 1) != 0; }

// also sets *zeros when A stores an explicit zero (the pattern kernel then
// tests the values; otherwise the structure alone is the nonzero pattern)
__global__ void k_scale(int64_t n, const int64_t* __restrict__ rp, const double* __restrict__ val,
                        int scale, double* __restrict__ d, int* __restrict__ err, int* __restrict__ zeros)
{
    bool z = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double mx = 0.0;
        bool fin = true;
        for (int64_t q = rp[i]; q < rp[i + 1]; q++) {
            double a = val[q];
            if (!isfinite(a)) fin = false;
            if (!nonzero_bits(a)) z = true;
            mx = fmax(mx, fabs(a));
        }
        if (!fin) atomicCAS(err, 0, SPAI_ERR_NONFINITE);
        if (mx == 0.0) atomicCAS(err, 0, SPAI_ERR_ZERO_ROW);
        d[i] = scale ? (mx > 0.0 ? 1.0 / mx : 1.0) : 1.0;
    }
    if (z) atomicOr(zeros, 1);
}

// b = fl_S(a_ij d_j) for every nonzero of row j of A, once, in the storage
// precision the column kernels read; explicit zeros get the marker pattern
template <class S>
__global__ void k_bvals(int64_t n, const int64_t* __restrict__ rp, const double* __restrict__ val,
                        const double* __restrict__ d, S* __restrict__ bv)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const double dj = d[j];
        for (int64_t q = rp[j]; q < rp[j + 1]; q++) {
            const double a = val[q];
            bv[q] = a != 0.0 ? from_d<S>(a * dj) : bmark<S>();
        }
    }
}

// ---------------------------------------------------------------- A^T structure

__global__ void k_col_count(int64_t nnz, const int32_t* __restrict__ col, int32_t* __restrict__ cnt)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[col[q]], 1);
}

__global__ void k_col_fill(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const int64_t* __restrict__ cp, int32_t* __restrict__ cursor, int32_t* __restrict__ ri)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int64_t q = rp[i]; q < rp[i + 1]; q++) {
            int j = col[q];
            int slot = atomicAdd(&cursor[j], 1);
            ri[cp[j] + slot] = (int32_t)i;
        }
}

// insertion sort of each column's row list (lists are short)
__global__ void k_col_sort(int64_t n, const int64_t* __restrict__ cp, int32_t* __restrict__ ri)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        int64_t b = cp[j], e = cp[j + 1];
        for (int64_t x = b + 1; x < e; x++) {
            int32_t v = ri[x];
            int64_t y = x - 1;
            while (y >= b && ri[y] > v) { ri[y + 1] = ri[y]; y--; }
            ri[y + 1] = v;
        }
    }
}

// ---------------------------------------------------------------- scans

__global__ void k_block_sums(int64_t n, const int32_t* __restrict__ in, int64_t* __restrict__ sums, int64_t chunk)
{
    __shared__ int64_t red[33];
    int64_t b = blockIdx.x * chunk, e = min(n, b + chunk);
    int64_t acc = 0;
    for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) acc += in[i];
    acc = block_sum<int64_t>(acc, red);
    if (threadIdx.x == 0) sums[blockIdx.x] = acc;
}

__global__ void k_scan_sums(int nb, int64_t* sums)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int64_t acc = 0;
        for (int i = 0; i < nb; i++) { int64_t v = sums[i]; sums[i] = acc; acc += v; }
        sums[nb] = acc;
    }
}

// exclusive scan of each chunk, offset by the chunk's prefix; out has n+1 entries
__global__ void k_scan_chunks(int64_t n, const int32_t* __restrict__ in, const int64_t* __restrict__ sums,
                              int64_t* __restrict__ out, int64_t chunk)
{
    __shared__ int64_t wsum[32];
    __shared__ int64_t carry;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t b = blockIdx.x * chunk, e = min(n, b + chunk);
    if (threadIdx.x == 0) carry = sums[blockIdx.x];
    __syncthreads();
    for (int64_t base = b; base < e; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        int64_t v = i < e ? in[i] : 0;
        int64_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            int64_t t = lane < nw ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int64_t y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            if (lane < nw) wsum[lane] = t;
        }
        __syncthreads();
        int64_t pre = carry + (w > 0 ? wsum[w - 1] : 0) + x - v;
        if (i < e) out[i] = pre;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = pre + v;
        __syncthreads();
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = sums[gridDim.x];
}

}  // namespace

int scan_counts(int64_t n, const int32_t* in, int64_t* out, cudaStream_t s)
{
    // chunks of 4096 counts: one 1024-thread block scans a chunk in 4 passes
    const int64_t chunk = 4096;
    int nb = (int)((n + chunk - 1) / chunk);
    if (nb < 1) nb = 1;
    int64_t* sums = nullptr;
    int rc = dev_alloc((void**)&sums, sizeof(int64_t) * (nb + 1), s);
    if (rc) return rc;
    k_block_sums<<<nb, 256, 0, s>>>(n, in, sums, chunk);
    k_scan_sums<<<1, 32, 0, s>>>(nb, sums);
    k_scan_chunks<<<nb, 1024, 0, s>>>(n, in, sums, out, chunk);
    dev_free(sums, s);
    SPAI_CUDA_TRY(cudaGetLastError());
    return 0;
}

namespace {

// ---------------------------------------------------------------- sorted unions
// Sorted union of up to 32 sorted index lists held in shared memory, one per
// lane (lane l: lst[l*stride .. l*stride + len)).  The warp repeatedly takes
// the minimum head (one REDUX) and every lane holding it advances.  Writes
// the union to out[0..cap); returns its size.
__device__ int warp_union(const int32_t* lst, int stride, int len, int32_t* out, int cap)
{
    const int lane = threadIdx.x & 31;
    const int32_t* l = lst + lane * stride;
    int q = 0;
    int head = len > 0 ? l[0] : INT_MAX;
    int cnt = 0;
    while (true) {
        const int mn = __reduce_min_sync(0xffffffffu, head);
        if (mn == INT_MAX) break;
        if (lane == 0 && cnt < cap) out[cnt] = mn;
        cnt++;
        if (head == mn) {
            q++;
            head = q < len ? l[q] : INT_MAX;
        }
    }
    __syncwarp();
    return cnt;
}

// Load list `lane` = idx[b..e) into lst + lane*stride (at most stride
// entries); returns its length.
__device__ __forceinline__ int load_list(const int32_t* __restrict__ idx, int64_t b, int64_t e, int32_t* lst, int stride)
{
    const int lane = threadIdx.x & 31;
    int32_t* l = lst + lane * stride;
    int len = 0;
    for (int64_t q = b; q < e; q += 4) {
        int cc[4];
#pragma unroll
        for (int u = 0; u < 4; u++) cc[u] = q + u < e ? idx[q + u] : 0;
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (q + u < e && len < stride) l[len++] = cc[u];
    }
    return len;
}

// ---------------------------------------------------------------- pattern

// Initial pattern J_k (identity, pattern(A), pattern(A^2)), capped at F
// keeping k and then the nearest indices (ties to the smaller index), and
// the shadow size |I_k| = |union of the nonzero columns of rows j in J_k,
// plus k|.  One warp per column.  Per-warp shared memory: buf[cap] for the
// uncapped pattern, 32 lists of `stride` ints, and a hash set of tsz slots
// that counts the shadow (its size only is needed, so no sorted merge).
// Columns whose shadow exceeds big_thr are appended to big[] (count *nbig).
__global__ void k_pattern(int64_t n, int init, int F, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                          const double* __restrict__ val, const int64_t* __restrict__ cp,
                          const int32_t* __restrict__ ri, int32_t* __restrict__ Jidx, int32_t* __restrict__ Jcnt,
                          int32_t* __restrict__ Icnt, int cap, int stride, int tsz, int* __restrict__ err,
                          int* __restrict__ maxI, const int* __restrict__ zeros, int big_thr,
                          int32_t* __restrict__ big, int* __restrict__ nbig)
{
    const bool zv = *zeros != 0;  // A stores explicit zeros: test the values
    extern __shared__ int32_t pbuf[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    int32_t* buf = pbuf + (size_t)wib * (cap + 32 * stride + tsz);
    int32_t* lst = buf + cap;
    int32_t* tab = lst + 32 * stride;
    for (int t = lane; t < tsz; t += 32) tab[t] = -1;
    __syncwarp();
    int wmax = 0;  // the warp's largest shadow
    for (int64_t k = blockIdx.x * (int64_t)wpb + wib; k < n; k += (int64_t)gridDim.x * wpb) {
        int cnt = 0;
        if (init == SPAI_PAT_IDENTITY) {
            if (lane == 0) buf[0] = (int32_t)k;
            cnt = 1;
        } else if (init == SPAI_PAT_A) {
            const int64_t b = cp[k], e = cp[k + 1];
            cnt = (int)(e - b);
            if (cnt > cap) { if (lane == 0) atomicCAS(err, 0, SPAI_ERR_UNSUPPORTED); cnt = cap; }
            for (int t = lane; t < cnt; t += 32) buf[t] = ri[b + t];
        } else {
            // column k of A^2: union over i in column k of A of column i of A
            const int64_t b = cp[k];
            int64_t e = cp[k + 1];
            if (e - b > 32) { if (lane == 0) atomicCAS(err, 0, SPAI_ERR_UNSUPPORTED); e = b + 32; }
            int len = 0;
            if (lane < e - b) {
                const int i = ri[b + lane];
                len = load_list(ri, cp[i], cp[i + 1], lst, stride);
            }
            __syncwarp();
            cnt = warp_union(lst, stride, len, buf, cap);
            if (cnt > cap) { if (lane == 0) atomicCAS(err, 0, SPAI_ERR_UNSUPPORTED); cnt = cap; }
        }
        __syncwarp();
        // cap: the F entries nearest to k form a contiguous window of the sorted list
        int lo = 0, hi = cnt;
        if (cnt > F) {
            if (lane == 0) {
                int pk = 0;
                while (pk < cnt && buf[pk] < k) pk++;
                lo = pk; hi = pk;
                if (pk < cnt && buf[pk] == k) hi = pk + 1;
                while (hi - lo < F) {
                    const bool can_l = lo > 0, can_r = hi < cnt;
                    if (can_l && can_r) {
                        const long dl = (long)k - buf[lo - 1], dr = (long)buf[hi] - k;
                        if (dl <= dr) lo--; else hi++;
                    } else if (can_l) lo--;
                    else hi++;
                }
            }
            lo = __shfl_sync(0xffffffffu, lo, 0);
            hi = __shfl_sync(0xffffffffu, hi, 0);
        }
        const int nj = hi - lo;
        const int jl = lane < nj ? buf[lo + lane] : -1;
        if (lane < nj) Jidx[k * F + lane] = jl;  // entries past |J_k| are never read
        if (lane == 0) Jcnt[k] = nj;
        __syncwarp();
        // shadow size of the (initial) pattern: |{k} and the nonzero columns of rows J_k|,
        // counted in the first ts slots of the table, ts at least twice the entries
        // (a power of two, at most tsz): only those are cleared afterwards
        int64_t b = 0, e = 0;
        if (lane < nj) {
            b = rp[jl];
            e = rp[jl + 1];
        }
        int ts = 64;
        {
            int tot = (int)(e - b);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
            while (ts < 2 * (tot + 1) && ts < tsz) ts <<= 1;
        }
        const unsigned tmask = (unsigned)ts - 1u;
        const int tshift = __clz(ts) + 1;  // ts = 2^(31 - clz)
        int mine = lane == 0 ? hset_insert(tab, tmask, tshift, (int)k) : 0;
        // (four loads in flight per lane before the inserts)
        for (int64_t q = b; q < e; q += 4) {
            int c4[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                c4[u] = -1;
                if (q + u < e && (!zv || nonzero_bits(val[q + u]))) c4[u] = col[q + u];
            }
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (c4[u] >= 0) mine += hset_insert(tab, tmask, tshift, c4[u]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
        const int mI = mine;
        wmax = max(wmax, mI);
        if (lane == 0) {
            Icnt[k] = mI;
            if (mI > big_thr) big[atomicAdd(nbig, 1)] = (int32_t)k;  // for the large-shadow kernel
        }
        __syncwarp();
        for (int t = lane; t < ts; t += 32) tab[t] = -1;
        __syncwarp();
    }
    // one atomic per warp (one per column on a single address serialised the kernel)
    if (lane == 0 && wmax > 0) atomicMax(maxI, wmax);
}

// P in CSR from the padded per-column results: one thread per padded slot
// (k, c), so that the reads of the n x F arrays are coalesced
template <class S>
__global__ void k_assemble(int64_t n, int F, const int32_t* __restrict__ Jidx, const int32_t* __restrict__ Jcnt,
                           const double* __restrict__ Praw, const int64_t* __restrict__ prp,
                           int32_t* __restrict__ pcol, double* __restrict__ pval, S* __restrict__ pval_uf)
{
    const int64_t total = n * F;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / F;
        const int c = (int)(t - k * F);
        if (c < Jcnt[k]) {
            const int64_t o = prp[k] + c;
            const double v = Praw[t];
            pcol[o] = Jidx[t];
            pval[o] = v;
            pval_uf[o] = from_d<S>(v);
        }
    }
}

__global__ void k_flag_stats(int64_t n, const int32_t* __restrict__ flags, const int32_t* __restrict__ Jcnt,
                             unsigned long long* __restrict__ out /* conv, fillcap, nonfinite */, int* __restrict__ maxJ)
{
    unsigned long long c0 = 0, c1 = 0, c2 = 0;
    int mj = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        int f = flags[k];
        c0 += (f & CF_CONVERGED) ? 1 : 0;
        c1 += ((f & CF_FILLCAP) && !(f & CF_CONVERGED)) ? 1 : 0;
        c2 += (f & CF_NONFINITE) ? 1 : 0;
        mj = max(mj, (int)Jcnt[k]);
    }
    c0 = warp_sum(c0); c1 = warp_sum(c1); c2 = warp_sum(c2);
    int m2 = mj;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m2 = max(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], c0); atomicAdd(&out[1], c1); atomicAdd(&out[2], c2);
        atomicMax(maxJ, m2);
    }
}

// Fixed patterns: every column with a shadow of at most MMAX_LIMIT rows
// goes to the list of its kernel's bin (spai_bin).  k_bin_count counts the
// bins, the host places them one after another (boff), k_bin_place writes
// the lists; a column's place within its bin does not matter.  Both take
// one warp-aggregated atomic per bin present in a warp.
__device__ __forceinline__ int column_bin(int64_t k, int64_t n, const int32_t* Icnt, const int32_t* Jcnt)
{
    if (k >= n) return -1;
    const int m = Icnt[k];
    return m > MMAX_LIMIT ? -1 : spai_bin(m, Jcnt[k]);
}

__global__ void k_bin_count(int64_t n, const int32_t* __restrict__ Icnt, const int32_t* __restrict__ Jcnt,
                            int* __restrict__ cnt)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k0 = blockIdx.x * (int64_t)blockDim.x; k0 < n; k0 += stride) {
        const int b = column_bin(k0 + threadIdx.x, n, Icnt, Jcnt);
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        if (b >= 0 && lane == __ffs(peers) - 1) atomicAdd(&cnt[b], __popc(peers));
    }
}

__global__ void k_bin_place(int64_t n, const int32_t* __restrict__ Icnt, const int32_t* __restrict__ Jcnt,
                            const int64_t* __restrict__ boff, int* __restrict__ cursor, int32_t* __restrict__ list)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k0 = blockIdx.x * (int64_t)blockDim.x; k0 < n; k0 += stride) {
        const int64_t k = k0 + threadIdx.x;
        const int b = column_bin(k, n, Icnt, Jcnt);
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (b >= 0 && lane == leader) base = atomicAdd(&cursor[b], __popc(peers));
        base = __shfl_sync(peers, base, leader);
        if (b >= 0) list[boff[b] + base + __popc(peers & ((1u << lane) - 1u))] = (int32_t)k;
    }
}

// per matrix of a block-diagonal union: one block per matrix (grid-stride
// over matrices), the counts of k_flag_stats, max |I_k|, max |J_k|, nnz(P)
__global__ void k_seg_stats(int count, const int64_t* __restrict__ ro, const int32_t* __restrict__ flags,
                            const int32_t* __restrict__ Jcnt, const int32_t* __restrict__ Icnt,
                            const int64_t* __restrict__ prp, unsigned long long* __restrict__ out)
{
    __shared__ unsigned long long red[6];
    for (int i = blockIdx.x; i < count; i += gridDim.x) {
        if (threadIdx.x < 6) red[threadIdx.x] = 0;
        __syncthreads();
        unsigned long long c0 = 0, c1 = 0, c2 = 0;
        int mi = 0, mj = 0;
        for (int64_t k = ro[i] + threadIdx.x; k < ro[i + 1]; k += blockDim.x) {
            const int f = flags[k];
            c0 += (f & CF_CONVERGED) ? 1 : 0;
            c1 += ((f & CF_FILLCAP) && !(f & CF_CONVERGED)) ? 1 : 0;
            c2 += (f & CF_NONFINITE) ? 1 : 0;
            mi = max(mi, (int)Icnt[k]);
            mj = max(mj, (int)Jcnt[k]);
        }
        c0 = warp_sum(c0); c1 = warp_sum(c1); c2 = warp_sum(c2);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mi = max(mi, __shfl_xor_sync(0xffffffffu, mi, o));
            mj = max(mj, __shfl_xor_sync(0xffffffffu, mj, o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&red[0], c0); atomicAdd(&red[1], c1); atomicAdd(&red[2], c2);
            atomicMax(&red[3], (unsigned long long)mi); atomicMax(&red[4], (unsigned long long)mj);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int t = 0; t < 5; t++) out[6 * (size_t)i + t] = red[t];
            out[6 * (size_t)i + 5] = (unsigned long long)(prp[ro[i + 1]] - prp[ro[i]]);
        }
        __syncthreads();
    }
}

__global__ void k_max_row(int64_t n, const int64_t* __restrict__ rp, int* __restrict__ out)
{
    int mx = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        mx = max(mx, (int)(rp[i + 1] - rp[i]));
#pragma unroll
    for (int q = 16; q > 0; q >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, q));
    if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}

// ---------------------------------------------------------------- CSR transpose (right SPAI)

// entries of row i go to row col[q] of the transpose, at a slot taken from
// that row's cursor (order within a row fixed afterwards by k_tr_sort)
__global__ void k_tr_fill(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                          const double* __restrict__ val, const int64_t* __restrict__ rpT, int32_t* __restrict__ cursor,
                          int32_t* __restrict__ colT, double* __restrict__ valT)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int64_t q = rp[i]; q < rp[i + 1]; q++) {
            const int j = col[q];
            const int slot = atomicAdd(&cursor[j], 1);
            colT[rpT[j] + slot] = (int32_t)i;
            valT[rpT[j] + slot] = val[q];
        }
}

// insertion sort of each row by column index, carrying the values
__global__ void k_tr_sort(int64_t n, const int64_t* __restrict__ rp, int32_t* __restrict__ col, double* __restrict__ val)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = rp[i], e = rp[i + 1];
        for (int64_t x = b + 1; x < e; x++) {
            const int32_t c = col[x];
            const double v = val[x];
            int64_t y = x - 1;
            while (y >= b && col[y] > c) { col[y + 1] = col[y]; val[y + 1] = val[y]; y--; }
            col[y + 1] = c;
            val[y + 1] = v;
        }
    }
}

template <class S>
__global__ void k_round_to(int64_t m, const double* __restrict__ v, S* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = from_d<S>(v[i]);
}

// CSR (rowptr, col, val) of the transpose of an n x n CSR, in new device
// arrays (sorted column indices, deterministic whatever the atomic order)
int csr_transpose(int num_sms, cudaStream_t s, int64_t n, int64_t nnz, const int64_t* rp, const int32_t* col,
                  const double* val, int64_t** rpT, int32_t** colT, double** valT, int* nl)
{
    *rpT = nullptr; *colT = nullptr; *valT = nullptr;
    int32_t* cnt = nullptr;
    int rc = dev_alloc((void**)&cnt, sizeof(int32_t) * (n + 1), s);
    if (!rc) rc = dev_alloc((void**)rpT, sizeof(int64_t) * (n + 1), s);
    if (!rc) rc = dev_alloc((void**)colT, sizeof(int32_t) * (nnz > 0 ? nnz : 1), s);
    if (!rc) rc = dev_alloc((void**)valT, sizeof(double) * (nnz > 0 ? nnz : 1), s);
    const int tb = 256;
    const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((std::max(n, nnz) + tb - 1) / tb, (int64_t)num_sms * 32));
    if (!rc && cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (n + 1), s) != cudaSuccess) rc = SPAI_ERR_CUDA;
    if (!rc) {
        k_col_count<<<gb, tb, 0, s>>>(nnz, col, cnt);
        rc = scan_counts(n, cnt, *rpT, s);
        *nl += 4;
    }
    if (!rc && cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (n + 1), s) != cudaSuccess) rc = SPAI_ERR_CUDA;
    if (!rc) {
        k_tr_fill<<<gb, tb, 0, s>>>(n, rp, col, val, *rpT, cnt, *colT, *valT);
        k_tr_sort<<<gb, tb, 0, s>>>(n, *rpT, *colT, *valT);
        *nl += 2;
        if (cudaGetLastError() != cudaSuccess) rc = SPAI_ERR_CUDA;
    }
    dev_free(cnt, s);
    if (rc) {
        dev_free(*rpT, s); dev_free(*colT, s); dev_free(*valT, s);
        *rpT = nullptr; *colT = nullptr; *valT = nullptr;
    }
    return rc;
}

int spai_build_left(int device, int num_sms, cudaStream_t s, const DevCsr& A, const spai_opts* o,
                    spai_precond* P_out, spai_stats* st, const SpaiSegments* seg);

}  // namespace

// Algorithm 1 on A^T D (left, P = M^T D) or, with side = 1, on A D with P = D M
// (right).  The right construction is the left one run on A^T, transposed:
// the left run on A^T computes M ~ (A D)^{-1} column by column and assembles
// M^T D, whose transpose D M is the right preconditioner.
int spai_build_dev(int device, int num_sms, cudaStream_t s, const DevCsr& A, const spai_opts* o,
                   spai_precond* P_out, spai_stats* st, const SpaiSegments* seg)
{
    if (!o || !P_out) return SPAI_ERR_INVALID_ARG;
    if (o->side != 0 && o->side != 1) return SPAI_ERR_INVALID_ARG;
    if (o->side == 0) return spai_build_left(device, num_sms, s, A, o, P_out, st, seg);
    *P_out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SPAI_CUDA_TRY(cudaEventCreate(&e0));
    SPAI_CUDA_TRY(cudaEventCreate(&e1));
    int nl = 0, rc = 0;
    DevCsr At;
    At.n = A.n;
    At.nnz = A.nnz;
    At.owned = true;
    spai_opts ol = *o;
    ol.side = 0;
    spai_precond P = nullptr;
    int64_t* rpT = nullptr;
    int32_t* colT = nullptr;
    double* valT = nullptr;
    if (cudaEventRecord(e0, s) != cudaSuccess) rc = SPAI_ERR_CUDA;
    if (!rc) rc = csr_transpose(num_sms, s, A.n, A.nnz, A.rowptr, A.col, A.val, &At.rowptr, &At.col, &At.val, &nl);
    // (a block-diagonal union transposes block by block: the segments stay)
    if (!rc) rc = spai_build_left(device, num_sms, s, At, &ol, &P, st, seg);
    csr_release(&At, s);
    if (rc >= 0 && P) {
        const int wrc = rc;
        rc = csr_transpose(num_sms, s, P->n, P->nnz, P->rowptr, P->col, P->val, &rpT, &colT, &valT, &nl);
        if (!rc) {
            dev_free(P->rowptr, s);
            dev_free(P->col, s);
            dev_free(P->val, s);
            P->rowptr = rpT;
            P->col = colT;
            P->val = valT;
            // the u_f copy: the same values rounded to u_f
            const int tb = 256;
            const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((P->nnz + tb - 1) / tb, (int64_t)num_sms * 32));
            if (P->nnz > 0) {
                if (P->uf == SPAI_HALF) k_round_to<__half><<<gb, tb, 0, s>>>(P->nnz, P->val, (__half*)P->val_uf);
                else if (P->uf == SPAI_SINGLE) k_round_to<float><<<gb, tb, 0, s>>>(P->nnz, P->val, (float*)P->val_uf);
                else k_round_to<double><<<gb, tb, 0, s>>>(P->nnz, P->val, (double*)P->val_uf);
                nl++;
            }
            if (cudaGetLastError() != cudaSuccess) rc = SPAI_ERR_CUDA;
            if (!rc) rc = wrc;
        }
    }
    if (rc >= 0 && cudaEventRecord(e1, s) == cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess && st) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        st->ms = ms;  // the whole right construction, transposes included
        st->launches += nl;
    }
    if (rc < 0 && P) {
        spai_precond_free(P);
        P = nullptr;
    }
    *P_out = P;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

namespace {

int spai_build_left(int device, int num_sms, cudaStream_t s, const DevCsr& A, const spai_opts* o,
                    spai_precond* P_out, spai_stats* st, const SpaiSegments* seg)
{
    const int64_t n = A.n, nnz = A.nnz;
    if (!o || !P_out) return SPAI_ERR_INVALID_ARG;
    if (o->max_fill < 1 || o->max_fill > MAX_FILL) return SPAI_ERR_UNSUPPORTED;
    if (o->uf != SPAI_HALF && o->uf != SPAI_SINGLE && o->uf != SPAI_DOUBLE) return SPAI_ERR_UNSUPPORTED;
    if (o->init < SPAI_PAT_IDENTITY || o->init > SPAI_PAT_A2) return SPAI_ERR_INVALID_ARG;
    if (o->adaptive && o->beta < 1) return SPAI_ERR_INVALID_ARG;
    if (!(o->eps >= 0.0)) return SPAI_ERR_INVALID_ARG;
    const int F = o->max_fill;
    cudaEvent_t e0, e1, ek0, ek1;
    SPAI_CUDA_TRY(cudaEventCreate(&e0));
    SPAI_CUDA_TRY(cudaEventCreate(&e1));
    SPAI_CUDA_TRY(cudaEventCreate(&ek0));
    SPAI_CUDA_TRY(cudaEventCreate(&ek1));
    int nl = 0;  // kernels launched
    SPAI_CUDA_TRY(cudaEventRecord(e0, s));

    int rc = 0;
    // device scratch
    double* d = nullptr;
    int* err = nullptr;      // [0] error code, [1] max |I|, [2] max |J|, [3] [4] longest row and column,
                             // [5] explicit zeros, [6] columns for the large-shadow kernel,
                             // [8..21] columns per bin of the column kernels (fixed patterns),
                             // [24..37] the bins' cursors
    int32_t* big = nullptr;  // those columns
    int32_t* blist = nullptr;  // the bins' column lists
    int64_t* boff = nullptr;
    unsigned char* slab = nullptr;
    int32_t* ccount = nullptr;
    int64_t* cp = nullptr;
    int32_t* ri = nullptr;
    int32_t *Jidx = nullptr, *Jcnt = nullptr, *Icnt = nullptr, *flags = nullptr, *nsolve = nullptr;
    double *Praw = nullptr, *colres = nullptr;
    void* bval = nullptr;
    unsigned long long* fstat = nullptr;
    size_t ssz = o->uf == SPAI_HALF ? 2 : (o->uf == SPAI_SINGLE ? 4 : 8);
    spai_precond P = nullptr;
    int h_err[24] = {0};
    unsigned long long h_fstat[3] = {0, 0, 0};
    int maxrow = 0, maxcol = 0;
    const int optin = device_attr_cached(cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    const size_t smem_cap = optin > 0 ? (size_t)optin : (size_t)(100 * 1024);

#define TRY(x) do { rc = (x); if (rc) goto done; } while (0)
    TRY(dev_alloc((void**)&d, sizeof(double) * n, s));
    TRY(dev_alloc((void**)&err, sizeof(int) * 40, s));
    TRY(dev_alloc((void**)&boff, sizeof(int64_t) * SPAI_NBINS, s));
    TRY(dev_alloc((void**)&big, sizeof(int32_t) * n, s));
    TRY(dev_alloc((void**)&ccount, sizeof(int32_t) * (n + 1), s));
    TRY(dev_alloc((void**)&cp, sizeof(int64_t) * (n + 1), s));
    TRY(dev_alloc((void**)&ri, sizeof(int32_t) * (nnz > 0 ? nnz : 1), s));
    TRY(dev_alloc((void**)&Jidx, sizeof(int32_t) * n * F, s));
    TRY(dev_alloc((void**)&Jcnt, sizeof(int32_t) * n, s));
    TRY(dev_alloc((void**)&Icnt, sizeof(int32_t) * n, s));
    TRY(dev_alloc((void**)&flags, sizeof(int32_t) * n, s));
    TRY(dev_alloc((void**)&nsolve, sizeof(int32_t) * n, s));
    TRY(dev_alloc((void**)&Praw, sizeof(double) * n * F, s));
    TRY(dev_alloc((void**)&colres, sizeof(double) * n, s));
    TRY(dev_alloc(&bval, ssz * (nnz > 0 ? nnz : 1), s));
    TRY(dev_alloc((void**)&fstat, sizeof(unsigned long long) * 3, s));
    if (cudaMemsetAsync(err, 0, sizeof(int) * 40, s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
    if (cudaMemsetAsync(ccount, 0, sizeof(int32_t) * (n + 1), s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
    if (cudaMemsetAsync(fstat, 0, sizeof(unsigned long long) * 3, s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
    {
        int tb = 256;
        int gb = (int)std::min<int64_t>((n + tb - 1) / tb, (int64_t)num_sms * 32);
        if (gb < 1) gb = 1;
        k_scale<<<gb, tb, 0, s>>>(n, A.rowptr, A.val, o->scale, d, err, err + 5);
        if (o->uf == SPAI_HALF) k_bvals<__half><<<gb, tb, 0, s>>>(n, A.rowptr, A.val, d, (__half*)bval);
        else if (o->uf == SPAI_SINGLE) k_bvals<float><<<gb, tb, 0, s>>>(n, A.rowptr, A.val, d, (float*)bval);
        else k_bvals<double><<<gb, tb, 0, s>>>(n, A.rowptr, A.val, d, (double*)bval);
        nl += 2;
        int gq = (int)std::min<int64_t>((nnz + tb - 1) / tb, (int64_t)num_sms * 32);
        if (gq < 1) gq = 1;
        k_col_count<<<gq, tb, 0, s>>>(nnz, A.col, ccount);
        TRY(scan_counts(n, ccount, cp, s));
        nl += 1 + 3;
        if (cudaMemsetAsync(ccount, 0, sizeof(int32_t) * (n + 1), s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
        k_col_fill<<<gb, tb, 0, s>>>(n, A.rowptr, A.col, cp, ccount, ri);
        k_col_sort<<<gb, tb, 0, s>>>(n, cp, ri);
        nl += 2;
    }
    {
        // longest row and column of A: list capacities, and |I_k| <= max_fill * maxrow + 1
        int* mr = err + 3;
        k_max_row<<<(unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * 8) + 1, 256, 0, s>>>(n, A.rowptr, mr);
        k_max_row<<<(unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * 8) + 1, 256, 0, s>>>(n, cp, mr + 1);
        nl += 2;
        if (cudaMemcpyAsync(&maxrow, mr, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
        if (cudaMemcpyAsync(&maxcol, mr + 1, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
        if (cudaStreamSynchronize(s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
        if (maxrow < 1) maxrow = 1;
        if (maxcol < 1) maxcol = 1;
    }
    {
        // the pattern and its shadow sizes: per warp a buffer for the uncapped
        // pattern (pattern(A^2): at most maxcol^2 entries), 32 lists, and a hash
        // set of at least twice the shadow entries a column can bring
        const int cap = o->init == SPAI_PAT_A2 ? (int)std::min<int64_t>(1024, std::max<int64_t>(32, (int64_t)maxcol * maxcol))
                                               : std::max(32, maxcol);
        const int stride = std::max(maxrow, maxcol);
        int tsz = 64;
        while (tsz < 2 * ((int64_t)F * maxrow + 1)) tsz <<= 1;
        const int wpb = 4;
        const size_t sm = (size_t)(cap + 32 * stride + tsz) * 4 * wpb;
        if (sm > smem_cap) { rc = SPAI_ERR_UNSUPPORTED; goto done; }
        SPAI_CUDA_TRY(allow_max_dynamic_smem(k_pattern));
        int64_t blocks = std::min<int64_t>((n + wpb - 1) / wpb, (int64_t)num_sms * 64);
        if (blocks < 1) blocks = 1;
        // fixed patterns: the columns whose shadow exceeds the CTA tile go to the
        // large-shadow kernel (adaptive columns are handed over by the column
        // kernels when they outgrow them)
        const int big_thr = o->adaptive ? INT_MAX : MMAX_LIMIT;
        k_pattern<<<(unsigned)blocks, wpb * 32, sm, s>>>(n, o->init, F, A.rowptr, A.col, A.val, cp, ri, Jidx, Jcnt,
                                                        Icnt, cap, stride, tsz, err, err + 1, err + 5, big_thr, big,
                                                        err + 6);
        nl += 1;
        if (!o->adaptive) {
            k_bin_count<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * 8)), 256, 0, s>>>(
                n, Icnt, Jcnt, err + 8);
            nl++;
        }
        if (cudaGetLastError() != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
        if (cudaMemcpyAsync(h_err, err, sizeof(int) * 24, cudaMemcpyDeviceToHost, s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
        if (cudaStreamSynchronize(s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
        if (h_err[0]) { rc = h_err[0]; goto done; }
    }
    {
        SpaiArgs a;
        memset(&a, 0, sizeof(a));
        a.n = n; a.F = F; a.rp = A.rowptr; a.col = A.col; a.val = A.val; a.cp = cp; a.ri = ri; a.d = d; a.bval = bval;
        a.Jidx = Jidx; a.Jcnt = Jcnt; a.Praw = Praw; a.colres = colres; a.flags = flags;
        a.Icnt = Icnt; a.nsolve = nsolve; a.eps = o->eps;
        a.alpha = o->alpha < 0 ? (int)((n + o->beta - 1) / std::max(o->beta, 1)) : o->alpha;
        a.beta = o->beta; a.rho_restricted = o->rho_restricted; a.err = err;
        a.rl = maxrow;
        a.big = big;
        a.nbig = err + 6;
        if (!o->adaptive) {
            // the bins' lists, one after another
            int64_t off = 0;
            for (int b = 0; b < SPAI_NBINS; b++) {
                a.boff[b] = off;
                a.bcnt[b] = h_err[8 + b];
                off += h_err[8 + b];
            }
            TRY(dev_alloc((void**)&blist, sizeof(int32_t) * std::max<int64_t>(off, 1), s));
            if (cudaMemcpyAsync(boff, a.boff, sizeof(int64_t) * SPAI_NBINS, cudaMemcpyHostToDevice, s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
            k_bin_place<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * 8)), 256, 0, s>>>(
                n, Icnt, Jcnt, boff, err + 24, blist);
            nl++;
            if (cudaGetLastError() != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
            a.blist = blist;
        }
        // the warp and CTA kernels hold up to MMAX_LIMIT shadow rows; larger
        // shadows go to the large-shadow kernel below
        const int64_t mall = o->adaptive ? (int64_t)F * maxrow + 1 : (int64_t)h_err[1];
        int mneed = (int)std::min<int64_t>(mall, (int64_t)MMAX_LIMIT);
        if (mneed < 1) mneed = 1;
        a.mmax = (mneed + 31) & ~31;
        int cmax = 1;
        // raw candidate capacity: |I| * (largest column count of A); power of two
        while (cmax < (int64_t)a.mmax * maxcol) cmax <<= 1;
        a.cmax = cmax > 8192 ? 8192 : (cmax < 256 ? 256 : cmax);
        if (cudaEventRecord(ek0, s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
        if (o->uf == SPAI_HALF) TRY(launch_spai_half(a, o->adaptive != 0, num_sms, smem_cap, s));
        else if (o->uf == SPAI_SINGLE) TRY(launch_spai_single(a, o->adaptive != 0, num_sms, smem_cap, s));
        else TRY(launch_spai_double(a, o->adaptive != 0, num_sms, smem_cap, s));
        nl++;
        // the large-shadow kernel for the listed columns: fixed patterns know
        // their count from k_pattern; adaptive builds read what the column
        // kernels handed over
        int nbig = h_err[6];
        if (o->adaptive) {
            if (cudaMemcpyAsync(&nbig, err + 6, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
            if (cudaStreamSynchronize(s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
        }
        if (nbig > 0) {
            // every shadow has at most mall rows and every candidate list at most
            // mall * (longest column of A) entries
            int64_t cc = 1;
            if (o->adaptive)
                while (cc < mall * (int64_t)maxcol) cc <<= 1;
            if (mall > INT32_MAX / SPAI_LD || cc > INT32_MAX) { rc = SPAI_ERR_UNSUPPORTED; goto done; }
            const int mcap = (int)mall, ccap = (int)cc;
            const size_t per = o->uf == SPAI_DOUBLE ? big_slab_bytes<double>(mcap, maxrow, ccap)
                                                    : big_slab_bytes<float>(mcap, maxrow, ccap);
            // one slab per CTA; at most two CTAs per SM, and at most 4 GiB of slabs
            int grid = (int)std::min<int64_t>(nbig, 2 * (int64_t)num_sms);
            while (grid > 1 && (size_t)grid * per > ((size_t)4 << 30)) grid = (grid + 1) / 2;
            TRY(dev_alloc((void**)&slab, (size_t)grid * per, s));
            if (o->uf == SPAI_HALF) TRY(launch_spai_big_half(a, o->adaptive != 0, big, err + 6, grid, slab, per, mcap, ccap, s));
            else if (o->uf == SPAI_SINGLE) TRY(launch_spai_big_single(a, o->adaptive != 0, big, err + 6, grid, slab, per, mcap, ccap, s));
            else TRY(launch_spai_big_double(a, o->adaptive != 0, big, err + 6, grid, slab, per, mcap, ccap, s));
            nl++;
        }
        if (cudaEventRecord(ek1, s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
    }
    // assemble P
    P = new spai_precond_s();
    P->n = n; P->uf = o->uf; P->stream = s; P->device = device;
    TRY(dev_alloc((void**)&P->rowptr, sizeof(int64_t) * (n + 1), s));
    TRY(scan_counts(n, Jcnt, P->rowptr, s));
    nl += 3;
    if (cudaMemcpyAsync(&P->nnz, P->rowptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
    if (cudaStreamSynchronize(s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
    TRY(dev_alloc((void**)&P->col, sizeof(int32_t) * (P->nnz > 0 ? P->nnz : 1), s));
    TRY(dev_alloc((void**)&P->val, sizeof(double) * (P->nnz > 0 ? P->nnz : 1), s));
    TRY(dev_alloc(&P->val_uf, ssz * (P->nnz > 0 ? P->nnz : 1), s));
    {
        int tb = 256;
        int gb = (int)std::min<int64_t>((n + tb - 1) / tb, (int64_t)num_sms * 32);
        if (gb < 1) gb = 1;
        if (o->uf == SPAI_HALF)
            k_assemble<__half><<<gb, tb, 0, s>>>(n, F, Jidx, Jcnt, Praw, P->rowptr, P->col, P->val, (__half*)P->val_uf);
        else if (o->uf == SPAI_SINGLE)
            k_assemble<float><<<gb, tb, 0, s>>>(n, F, Jidx, Jcnt, Praw, P->rowptr, P->col, P->val, (float*)P->val_uf);
        else
            k_assemble<double><<<gb, tb, 0, s>>>(n, F, Jidx, Jcnt, Praw, P->rowptr, P->col, P->val, (double*)P->val_uf);
        k_flag_stats<<<gb, tb, 0, s>>>(n, flags, Jcnt, fstat, err + 2);
        nl += 2;
        if (seg && seg->count > 0) {
            k_seg_stats<<<(unsigned)std::min<int64_t>(seg->count, (int64_t)num_sms * 8), 256, 0, s>>>(
                seg->count, seg->ro, flags, Jcnt, Icnt, P->rowptr, seg->stats);
            nl++;
        }
        if (cudaGetLastError() != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
    }
    if (cudaEventRecord(e1, s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
    if (cudaMemcpyAsync(h_err, err, sizeof(int) * 3, cudaMemcpyDeviceToHost, s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
    if (cudaMemcpyAsync(h_fstat, fstat, sizeof(h_fstat), cudaMemcpyDeviceToHost, s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
    if (st) {
        if (st->colres && cudaMemcpyAsync(st->colres, colres, sizeof(double) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
        if (st->nJ && cudaMemcpyAsync(st->nJ, Jcnt, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
        if (st->nI && cudaMemcpyAsync(st->nI, Icnt, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
        if (st->flags && cudaMemcpyAsync(st->flags, flags, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
    if (h_err[0]) { rc = h_err[0]; goto done; }
    if (st) {
        st->n = n;
        st->nnz_P = P->nnz;
        st->cols_converged = (int64_t)h_fstat[0];
        st->cols_fillcap = (int64_t)h_fstat[1];
        st->cols_nonfinite = (int64_t)h_fstat[2];
        st->max_I = h_err[1];
        st->max_J = h_err[2];
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        st->ms = ms;
        cudaEventElapsedTime(&ms, ek0, ek1);
        st->ms_kernel = ms;
        st->launches = nl;
    }
    if (h_fstat[2] > 0) rc = SPAI_ERR_NONFINITE;
    else if (h_fstat[1] > 0) rc = SPAI_WARN_FILLCAP;
done:
#undef TRY
    dev_free(d, s); dev_free(err, s); dev_free(big, s); dev_free(blist, s); dev_free(boff, s); dev_free(slab, s); dev_free(ccount, s); dev_free(cp, s); dev_free(ri, s);
    dev_free(Jidx, s); dev_free(Jcnt, s); dev_free(Icnt, s); dev_free(flags, s); dev_free(nsolve, s);
    dev_free(Praw, s); dev_free(colres, s); dev_free(bval, s); dev_free(fstat, s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(ek0);
    cudaEventDestroy(ek1);
    if (rc < 0) {
        if (P) spai_precond_free(P);
        *P_out = nullptr;
        cudaStreamSynchronize(s);
        return rc;
    }
    *P_out = P;
    return rc;
}

}  // namespace
