// SPAI column kernel for fixed patterns with shadows of 65..512 rows: one
// warp per column, |I_k| <= 32 R rows and |J_k| <= NC columns.
//
// The warp kernel keeps one tile column per lane in registers, which caps
// the shadow at 64 rows; the CTA kernel spreads larger tiles over 8 or 16
// warps that synchronise at every Householder step, and a single warp does
// its gather.  Here one warp owns the column and the working tile X =
// [B(I_k,J_k) | e_k(I_k)] lives in shared memory, row-major and padded with
// zero rows to 32 R: lane l owns rows l, l + 32, ..., l + 32 (R-1), so every
// lane reads and updates only its own rows and no step needs a barrier.  The
// loops over steps and columns are not unrolled (the code stays in the
// instruction cache); each inner product is a lane-local sum over R rows and
// a warp sum, four columns at a time.  R is chosen per column as
// ceil(|I_k| / 32) (the bins of spai_bin), so few padding rows are computed.
//
// Per column:
//   1. gather: every lane takes entry e of each row J_k[t] of A (the u_f
//      values of B = A^T D; coalesced, all rows in flight at once) and
//      inserts its row index into a shared-memory hash set; the rows of I_k
//      are numbered in the order the traversal first meets them (k first,
//      then row J_k[0]'s entries, ...), which fixes the order of the tile's
//      rows for every run.  A second pass writes every value to its row of
//      the zeroed tile.  The order of the rows does not change the
//      least-squares problem; it only changes rounding, within the
//      tolerance of the oracle comparison;
//   2. Householder QR of X in place: per step c the norm of the pivot
//      column below row c, then for every later column (and e_k) its inner
//      product with the reflector and the update of every lane's rows,
//      rounded to u_f as stored (the arithmetic of the warp and CTA kernels:
//      v = x - alpha e_1 with alpha = -sign(x_0) ||x||, v^T v = 2 ||x||
//      (||x|| + |x_0|));
//   3. back substitution m_c = (y_c - sum_{t>c} R(c,t) m_t) / R(c,c), the
//      sum a warp sum over t (as in the CTA kernel);
//   4. explicit residual s = B(I,J) m - e_k: the rows of A are read again and
//      column t's entries added to s in order t = 0, 1, ... (per row of s
//      the same fused multiply-adds, in the same order, as the tile-based
//      kernels), then ||s||_2.
// Only fixed patterns (Algorithm 1 with a pattern that does not grow) come
// here; every column is computed independently of the others, so a column's
// result depends only on the column.
#pragma once

#include "spai_column.cuh"

namespace spai {

constexpr int mid_pow2(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

template <class S, int R, int NC>
struct MidCfg {
    typedef typename Compute<S>::T C;
    static constexpr int MM = 32 * R;              // tile rows
    static constexpr int HS = mid_pow2(2 * MM);    // hash slots (load at most one half)
    static constexpr int LDX = NC + 1;             // row stride of X: the NC columns and e_k (odd: no bank conflicts)
    static constexpr size_t bytes()
    {
        return (size_t)HS * 4 + (size_t)HS * 2 + 32 * 8 + 32 * 4 + 32 * sizeof(C) + (size_t)MM * sizeof(C) +
               (size_t)MM * LDX * sizeof(C) + 64;
    }
    static constexpr size_t stride() { return (bytes() + 15) & ~size_t(15); }
    // warps per block: two, or one where a warp's tile is large (finer occupancy steps)
    static constexpr int WPB = bytes() > 40 * 1024 ? 1 : 2;
};

__device__ __forceinline__ int mid_hash_shift(int hs)
{
    return 32 - (31 - __clz(hs));
}

// inserts key; returns its slot if it was not there yet, else -1
__device__ __forceinline__ int hset_insert_slot(int32_t* tab, unsigned mask, int shift, int key)
{
    unsigned h = hset_slot(key, shift);
    for (unsigned probe = 0; probe <= mask; probe++) {
        const int old = atomicCAS(&tab[h], -1, key);
        if (old == -1) return (int)h;
        if (old == key) return -1;
        h = (h + 1u) & mask;
    }
    return -1;
}

template <class S, int R, int NC>
__global__ void __launch_bounds__(32 * MidCfg<S, R, NC>::WPB) k_spai_mid(SpaiArgs a)
{
    typedef MidCfg<S, R, NC> Cfg;
    typedef typename Cfg::C C;
    constexpr int MM = Cfg::MM, HS = Cfg::HS, LDX = Cfg::LDX, WPB = Cfg::WPB;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned char* base = smem + (size_t)wib * Cfg::stride();
    int32_t* hk = (int32_t*)base;                                  // HS keys
    uint16_t* hr = (uint16_t*)(base + (size_t)HS * 4);             // HS: each key's row of the tile
    int64_t* rowq = (int64_t*)(base + (size_t)HS * 6);             // 32: first entry of row J[t] of A
    int32_t* rowl = (int32_t*)(base + (size_t)HS * 6 + 256);       // 32: its length
    C* mb = (C*)(base + (size_t)HS * 6 + 384);                     // 32: mbar
    C* sres = (C*)(base + (size_t)HS * 6 + 384 + 32 * sizeof(C));  // MM: s
    C* X = (C*)(((uintptr_t)(sres + MM) + 15) & ~(uintptr_t)15);   // MM x LDX, 16-byte aligned
    const unsigned FULL = 0xffffffffu;
    const unsigned hmask = HS - 1;
    const int hshift = mid_hash_shift(HS);
    const S* bv = (const S*)a.bval;
    const int F = a.F;
    C* Xl = X + lane * LDX;  // this lane's first row

    for (int64_t idx = blockIdx.x * (int64_t)WPB + wib; idx < a.nlist; idx += (int64_t)gridDim.x * WPB) {
        const int64_t k = a.list[idx];
        const int nj = a.Jcnt[k];
        if (nj > NC) {  // cannot happen: the column was binned by |J_k|
            if (lane == 0) atomicCAS(a.err, 0, SPAI_ERR_INTERNAL);
            continue;
        }
        const int jl = lane < nj ? a.Jidx[k * F + lane] : -1;
        // ---- 1. gather
        for (int t = lane; t < HS; t += 32) hk[t] = -1;
        {
            // zero the whole tile, padding rows included (16-byte stores)
            constexpr int n16 = (int)((MM * LDX * sizeof(C)) / 16);
            static_assert((MM * LDX * sizeof(C)) % 16 == 0, "tile size");
            for (int t = lane; t < n16; t += 32) reinterpret_cast<int4*>(X)[t] = make_int4(0, 0, 0, 0);
        }
        int len = 0;
        if (lane < nj) {
            const int64_t q0 = a.rp[jl];
            len = (int)(a.rp[jl + 1] - q0);
            rowq[lane] = q0;
            rowl[lane] = len;
        }
        const int maxlen = (int)__reduce_max_sync(FULL, (unsigned)len);
        __syncwarp();
        if (lane == 0) hr[hset_insert_slot(hk, hmask, hshift, (int)k)] = 0;  // e_k's row: row 0
        int m = 1;
        __syncwarp();
        for (int e0 = 0; e0 < maxlen; e0 += 32) {
            int ck[NC];
#pragma unroll
            for (int t = 0; t < NC; t++) {
                ck[t] = -1;
                if (t < nj && e0 + lane < rowl[t]) {
                    const int64_t q = rowq[t] + e0 + lane;
                    const S b = bv[q];
                    const int c = a.col[q];
                    ck[t] = bmarked<S>(b) ? -1 : c;
                }
            }
#pragma unroll
            for (int t = 0; t < NC; t++) {
                if (t < nj) {
                    const int slot = ck[t] >= 0 ? hset_insert_slot(hk, hmask, hshift, ck[t]) : -1;
                    const unsigned bal = __ballot_sync(FULL, slot >= 0);
                    if (slot >= 0) hr[slot] = (uint16_t)min(m + __popc(bal & ((1u << lane) - 1u)), 0xffff);
                    m += __popc(bal);
                }
            }
        }
        if (m > MM) {  // cannot happen: the column was binned by its shadow size
            if (lane == 0) atomicCAS(a.err, 0, SPAI_ERR_INTERNAL);
            __syncwarp();
            continue;
        }
        __syncwarp();
        for (int e0 = 0; e0 < maxlen; e0 += 32) {
#pragma unroll
            for (int t = 0; t < NC; t++) {
                if (t < nj && e0 + lane < rowl[t]) {
                    const int64_t q = rowq[t] + e0 + lane;
                    const S b = bv[q];
                    if (!bmarked<S>(b)) X[(int)hr[hset_find(hk, hmask, hshift, a.col[q])] * LDX + t] = to_c(b);
                }
            }
        }
        if (lane == 0) X[nj] = C(1);  // e_k: row 0, column nj
        __syncwarp();
        // ---- 2. Householder QR of X (each lane its own rows; padding rows stay zero)
        const int steps = nj < m ? nj : m;
        for (int c = 0; c < steps; c++) {
            C v[R];
#pragma unroll
            for (int i = 0; i < R; i++) v[i] = Xl[i * 32 * LDX + c];
            const C xl = v[0];
            if (lane < c) v[0] = C(0);  // rows >= c only
            C sp0 = 0, sp1 = 0;
#pragma unroll
            for (int i = 0; i < R; i += 2) {
                sp0 = fma(v[i], v[i], sp0);
                if (i + 1 < R) sp1 = fma(v[i + 1], v[i + 1], sp1);
            }
            const C sig2 = warp_sum(sp0 + sp1);
            const C x0 = __shfl_sync(FULL, xl, c);
            const C nrm = rnd<S>(sqrt(sig2));
            if (nrm != C(0)) {
                const C alpha = x0 >= C(0) ? -nrm : nrm;
                const C v0 = rnd<S>(x0 - alpha);
                const C vtv = C(2) * nrm * (nrm + fabs(x0));
                // the later columns and e_k (column nj), four at a time
                for (int t = c + 1; t <= nj; t += 4) {
                    const int nt = min(4, nj + 1 - t);
                    C xs[4][R];
                    C g[4];
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        g[u] = 0;
#pragma unroll
                        for (int i = 0; i < R; i++) xs[u][i] = u < nt ? Xl[i * 32 * LDX + t + u] : C(0);
                    }
#pragma unroll
                    for (int i = 0; i < R; i++)
#pragma unroll
                        for (int u = 0; u < 4; u++) g[u] = fma(v[i], xs[u][i], g[u]);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                        for (int u = 0; u < 4; u++) g[u] += __shfl_xor_sync(FULL, g[u], o);
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        if (u < nt) {
                            const C act = __shfl_sync(FULL, xs[u][0], c);
                            const C sv = g[u] + (v0 - x0) * act;
                            const C f = rnd<S>((sv + sv) / vtv);
                            if (lane > c) Xl[t + u] = rnd<S>(xs[u][0] - f * v[0]);
                            else if (lane == c) Xl[t + u] = rnd<S>(act - f * v0);
#pragma unroll
                            for (int i = 1; i < R; i++) Xl[i * 32 * LDX + t + u] = rnd<S>(xs[u][i] - f * v[i]);
                        }
                    }
                }
                if (lane == c) Xl[c] = alpha;
            }
        }
        __syncwarp();
        // ---- 3. back substitution: lane t holds m_t once computed
        int fl = 0;
        C mv = 0;
        for (int c = nj - 1; c >= 0; c--) {
            const C part = warp_sum((lane > c && lane < nj) ? X[c * LDX + lane] * mv : C(0));
            const C rcc = X[c * LDX + c];
            const C yc = X[c * LDX + nj];
            C mc = 0;
            if (c < m && rcc != C(0)) mc = rnd<S>(rnd<S>(yc - part) / rcc);
            else fl = CF_SINGULAR;
            if (lane == c) mv = mc;
        }
        if (lane < nj) mb[lane] = mv;
        for (int p = lane; p < m; p += 32) sres[p] = C(0);
        __syncwarp();
        // ---- 4. explicit residual s = B(I,J) m - e_k, column by column
        for (int e0 = 0; e0 < maxlen; e0 += 32) {
            for (int t = 0; t < nj; t++) {
                if (e0 + lane < rowl[t]) {
                    const int64_t q = rowq[t] + e0 + lane;
                    const S b = bv[q];
                    if (!bmarked<S>(b)) {
                        C& z = sres[hr[hset_find(hk, hmask, hshift, a.col[q])]];
                        z = fma(to_c(b), mb[t], z);
                    }
                }
                __syncwarp();
            }
        }
        C s2p = 0;
        for (int p = lane; p < m; p += 32) {
            const C sp = rnd<S>(rnd<S>(sres[p]) - (p == 0 ? C(1) : C(0)));
            s2p = fma(sp, sp, s2p);
        }
        const C snorm = rnd<S>(sqrt(warp_sum(s2p)));
        if (!isfinite((double)snorm)) fl |= CF_NONFINITE;
        if (snorm <= (C)a.eps) fl |= CF_CONVERGED;
        // ---- outputs: row k of P = mbar_k * d(J_k) (entries past |J_k| are never read)
        if (lane < nj) {
            a.Jidx[k * F + lane] = jl;
            a.Praw[k * F + lane] = (double)mv * a.d[jl];
            if (!isfinite((double)mv)) fl |= CF_NONFINITE;
        }
        fl = (int)__reduce_or_sync(FULL, (unsigned)fl);
        if (lane == 0) {
            a.Jcnt[k] = nj;
            a.colres[k] = (double)snorm;
            a.flags[k] = fl;
            a.Icnt[k] = m;
            a.nsolve[k] = 1;
        }
        __syncwarp();
    }
}

template <class S, int R, int NC>
int launch_spai_mid(const SpaiArgs& a, int num_sms, size_t smem_cap, cudaStream_t s)
{
    typedef MidCfg<S, R, NC> Cfg;
    const size_t smem = Cfg::stride() * Cfg::WPB;
    if (smem > smem_cap) return SPAI_ERR_UNSUPPORTED;
    void (*kern)(SpaiArgs) = k_spai_mid<S, R, NC>;
    SPAI_CUDA_TRY(allow_max_dynamic_smem(kern));
    int occ = 0;
    SPAI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * Cfg::WPB, smem));
    if (occ < 1) return SPAI_ERR_UNSUPPORTED;
    int64_t blocks = std::min<int64_t>((a.nlist + Cfg::WPB - 1) / Cfg::WPB, (int64_t)num_sms * occ);
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, 32 * Cfg::WPB, smem, s>>>(a);
    SPAI_CUDA_TRY(cudaGetLastError());
    return 0;
}

// ---- bins 2 .. SPAI_NBINS-1 of spai_bin, and the tuner of their tile shapes.
//
// A column's result does not depend on the tile it runs in as long as the
// tile holds it (R >= ceil(|I_k|/32), NC >= |J_k|): padding rows are zero and
// stay zero, so every inner product, update and norm sees the same values in
// the same order.  The tile shape is therefore only a cost choice.  For each
// bin the tuner times the candidate shapes (the bin's own tile, the next
// larger row counts, and a 32-column tile) on a sample of the bin's columns
// the first time a build has enough of them, and keeps the fastest per device,
// u_f and bin; later builds use it.  spai_tune_get / spai_tune_set read and
// force the choice.

constexpr int MID_TUNE_MIN = 8192;   // columns of a bin before it is tuned
constexpr int MID_TUNE_SAMPLE = 4096;
constexpr int MID_MAX_VARIANTS = 4;

// the bin's candidate tiles as (R, NC); returns their count
inline int mid_variants(int bin, int (*rv)[2])
{
    static const int R16[] = {3, 4, 5, 6, 7, 8, 10, 12, 16};
    static const int R32[] = {4, 8, 16};
    int Rb, nc;
    if (bin >= 2 && bin <= 10) { Rb = R16[bin - 2]; nc = 16; }
    else if (bin >= 11 && bin <= 13) { Rb = R32[bin - 11]; nc = 32; }
    else return 0;
    int cnt = 0;
    if (nc == 16) {
        for (int q = bin - 2; q < 9 && cnt < 3; q++) { rv[cnt][0] = R16[q]; rv[cnt][1] = 16; cnt++; }
    }
    for (int q = 0; q < 3 && cnt < MID_MAX_VARIANTS; q++)
        if (R32[q] >= Rb) { rv[cnt][0] = R32[q]; rv[cnt][1] = 32; cnt++; if (nc == 16) break; }
    return cnt;
}

template <class S>
int launch_spai_mid_shape(const SpaiArgs& a, int R, int NC, int num_sms, size_t smem_cap, cudaStream_t s)
{
    if (NC == 16) {
        switch (R) {
        case 3: return launch_spai_mid<S, 3, 16>(a, num_sms, smem_cap, s);
        case 4: return launch_spai_mid<S, 4, 16>(a, num_sms, smem_cap, s);
        case 5: return launch_spai_mid<S, 5, 16>(a, num_sms, smem_cap, s);
        case 6: return launch_spai_mid<S, 6, 16>(a, num_sms, smem_cap, s);
        case 7: return launch_spai_mid<S, 7, 16>(a, num_sms, smem_cap, s);
        case 8: return launch_spai_mid<S, 8, 16>(a, num_sms, smem_cap, s);
        case 10: return launch_spai_mid<S, 10, 16>(a, num_sms, smem_cap, s);
        case 12: return launch_spai_mid<S, 12, 16>(a, num_sms, smem_cap, s);
        case 16: return launch_spai_mid<S, 16, 16>(a, num_sms, smem_cap, s);
        }
    } else {
        switch (R) {
        case 4: return launch_spai_mid<S, 4, 32>(a, num_sms, smem_cap, s);
        case 8: return launch_spai_mid<S, 8, 32>(a, num_sms, smem_cap, s);
        case 16:
            if constexpr (!std::is_same<S, double>::value) return launch_spai_mid<S, 16, 32>(a, num_sms, smem_cap, s);
            break;
        }
    }
    return SPAI_ERR_INTERNAL;
}

// the tuner's choices: variant index per (device, u_f, bin), -1 until tuned
int mid_tune_get(int device, int uf, int bin);
void mid_tune_put(int device, int uf, int bin, int variant);

template <class S>
int launch_spai_mid_bin_t(const SpaiArgs& a, int bin, int num_sms, size_t smem_cap, cudaStream_t s)
{
    constexpr int uf = std::is_same<S, __half>::value ? SPAI_HALF : (std::is_same<S, float>::value ? SPAI_SINGLE : SPAI_DOUBLE);
    int rv[MID_MAX_VARIANTS][2];
    int nv = mid_variants(bin, rv);
    if (std::is_same<S, double>::value && bin == 13) return SPAI_ERR_INTERNAL;  // the CTA kernel's bin
    // shapes past what this type can hold (512 x 32 at double) are not candidates
    if (std::is_same<S, double>::value)
        while (nv > 1 && rv[nv - 1][0] == 16 && rv[nv - 1][1] == 32) nv--;
    if (nv == 0) return SPAI_ERR_INTERNAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SPAI_ERR_CUDA;
    int v = mid_tune_get(dev, uf, bin);
    if (v < 0 && nv > 1 && a.nlist >= MID_TUNE_MIN) {
        // time every candidate on the bin's first columns (twice each, the second counts);
        // every candidate writes the same results for them
        SpaiArgs t = a;
        t.nlist = std::min<int64_t>(a.nlist, MID_TUNE_SAMPLE);
        cudaEvent_t e0, e1;
        SPAI_CUDA_TRY(cudaEventCreate(&e0));
        SPAI_CUDA_TRY(cudaEventCreate(&e1));
        float best = 0.f;
        int rc = 0;
        for (int q = 0; q < nv && !rc; q++) {
            float ms = 0.f;
            for (int rep = 0; rep < 2 && !rc; rep++) {
                cudaEventRecord(e0, s);
                rc = launch_spai_mid_shape<S>(t, rv[q][0], rv[q][1], num_sms, smem_cap, s);
                cudaEventRecord(e1, s);
                if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = SPAI_ERR_CUDA;
                if (!rc) cudaEventElapsedTime(&ms, e0, e1);
            }
            // another shape replaces the bin's own tile only when clearly faster (timings
            // taken under a profiler or beside other work are noisy)
            if (!rc && (v < 0 || ms < (v == 0 ? 0.95f : 1.0f) * best)) { best = ms; v = q; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc) return rc;
        mid_tune_put(dev, uf, bin, v);
    }
    if (v < 0 || v >= nv) v = 0;
    return launch_spai_mid_shape<S>(a, rv[v][0], rv[v][1], num_sms, smem_cap, s);
}

}  // namespace spai
