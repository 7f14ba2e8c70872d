// SPAI column kernel for fixed patterns with shadows of 65..512 rows: one
// warp per column, |I_k| <= 32 R rows and |J_k| <= NC columns.
//
// The warp kernel keeps one tile column per lane in registers, which caps
// the shadow at 64 rows; the CTA kernel spreads larger tiles over 8 or 16
// warps that synchronise at every Householder step, and a single warp does
// its gather.  Here one warp owns the column and the working tile X =
// [B(I_k,J_k) | e_k(I_k)] lives in shared memory, row-major: lane l owns
// rows l, l + 32, ..., l + 32 (R-1), so every lane reads and updates only
// its own rows and no step needs a barrier.  The loops over steps and
// columns are not unrolled (the code stays in the instruction cache); each
// inner product is a lane-local sum over R rows and a warp sum, two columns
// at a time.
//
// Per column:
//   1. gather: every lane takes entry e of each row J_k[t] of A (the u_f
//      values of B = A^T D; coalesced, all rows in flight at once) and
//      inserts its row index into a shared-memory hash set (new keys
//      appended to I in arrival order, plus k); I_k is sorted (warp bitonic
//      sort), each hash slot records its key's rank, and a second pass
//      writes every value to its rank's row of the zeroed tile;
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

template <class S, int R, int NC>
struct MidCfg {
    typedef typename Compute<S>::T C;
    static constexpr int MM = 32 * R;      // tile rows
    static constexpr int HS = 64 * R;      // hash slots (load at most one half)
    static constexpr int LDX = NC + 1;     // row stride of X: the NC columns and e_k (odd: no bank conflicts)
    static constexpr size_t SV = (size_t)MM * (sizeof(C) > 4 ? sizeof(C) : 4);  // I, later s
    static constexpr size_t bytes()
    {
        return ((size_t)HS * 4 + (size_t)HS * 2 + 32 * 8 + 32 * 4 + 32 * sizeof(C) + SV + (size_t)MM * LDX * sizeof(C) +
                15) & ~size_t(15);
    }
    // warps per block: two, or one where a warp's tile is large (finer occupancy steps)
    static constexpr int WPB = bytes() > 40 * 1024 ? 1 : 2;
};

__device__ __forceinline__ int mid_hash_shift(int hs)
{
    return 32 - (31 - __clz(hs));
}

template <class S, int R, int NC>
__global__ void __launch_bounds__(32 * MidCfg<S, R, NC>::WPB) k_spai_mid(SpaiArgs a)
{
    typedef MidCfg<S, R, NC> Cfg;
    typedef typename Cfg::C C;
    constexpr int MM = Cfg::MM, HS = Cfg::HS, LDX = Cfg::LDX, WPB = Cfg::WPB;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned char* base = smem + (size_t)wib * Cfg::bytes();
    int32_t* hk = (int32_t*)base;                                  // HS keys
    uint16_t* hr = (uint16_t*)(base + (size_t)HS * 4);             // HS ranks
    int64_t* rowq = (int64_t*)(base + (size_t)HS * 6);             // 32: first entry of row J[t] of A
    int32_t* rowl = (int32_t*)(base + (size_t)HS * 6 + 256);       // 32: its length
    C* mb = (C*)(base + (size_t)HS * 6 + 384);                     // 32: mbar
    unsigned char* sv = base + (size_t)HS * 6 + 384 + 32 * sizeof(C);
    int32_t* I = (int32_t*)sv;                                     // MM: I_k (gather)
    C* sres = (C*)sv;                                              // MM: s (residual)
    C* X = (C*)(sv + Cfg::SV);                                     // MM x LDX
    const unsigned FULL = 0xffffffffu;
    const unsigned hmask = HS - 1;
    const int hshift = mid_hash_shift(HS);
    const S* bv = (const S*)a.bval;
    const int F = a.F;

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
        int len = 0;
        if (lane < nj) {
            const int64_t q0 = a.rp[jl];
            len = (int)(a.rp[jl + 1] - q0);
            rowq[lane] = q0;
            rowl[lane] = len;
        }
        const int maxlen = (int)__reduce_max_sync(FULL, (unsigned)len);
        __syncwarp();
        int m = 0;
        if (lane == 0) hset_insert(hk, hmask, hshift, (int)k);
        if (lane == 0) I[0] = (int)k;
        m = 1;
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
                    const bool isnew = ck[t] >= 0 && hset_insert(hk, hmask, hshift, ck[t]);
                    const unsigned bal = __ballot_sync(FULL, isnew);
                    if (isnew) {
                        const int pos = m + __popc(bal & ((1u << lane) - 1u));
                        if (pos < MM) I[pos] = ck[t];
                    }
                    m += __popc(bal);
                }
            }
        }
        __syncwarp();
        if (m > MM) {  // cannot happen: the column was binned by its shadow size
            if (lane == 0) atomicCAS(a.err, 0, SPAI_ERR_INTERNAL);
            continue;
        }
        for (int t = m + lane; t < MM; t += 32) I[t] = INT_MAX;
        __syncwarp();
        warp_bitonic_sort(I, MM);
        for (int p = lane; p < m; p += 32) hr[hset_find(hk, hmask, hshift, I[p])] = (uint16_t)p;
        {
            // zero the tile's first m rows (16-byte stores; the tile starts 16-byte aligned)
            const int n16 = (int)((m * LDX * sizeof(C) + 15) / 16);
            for (int t = lane; t < n16; t += 32) reinterpret_cast<int4*>(X)[t] = make_int4(0, 0, 0, 0);
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
        const int rk = hr[hset_find(hk, hmask, hshift, (int)k)];  // row of e_k
        if (lane == 0) X[rk * LDX + nj] = C(1);
        __syncwarp();
        // ---- 2. Householder QR of X (each lane its own rows)
        const int steps = nj < m ? nj : m;
        for (int c = 0; c < steps; c++) {
            C v[R];
#pragma unroll
            for (int i = 0; i < R; i++) {
                const int row = lane + 32 * i;
                v[i] = row < m ? X[row * LDX + c] : C(0);
            }
            const C xl = v[0];
            if (lane < c) v[0] = C(0);  // rows >= c only
            C sp = 0;
#pragma unroll
            for (int i = 0; i < R; i++) sp = fma(v[i], v[i], sp);
            const C sig2 = warp_sum(sp);
            const C x0 = __shfl_sync(FULL, xl, c);
            const C nrm = rnd<S>(sqrt(sig2));
            if (nrm != C(0)) {
                const C alpha = x0 >= C(0) ? -nrm : nrm;
                const C v0 = rnd<S>(x0 - alpha);
                const C vtv = C(2) * nrm * (nrm + fabs(x0));
                // the later columns and e_k (column nj), two at a time
                for (int t = c + 1; t <= nj; t += 2) {
                    const bool two = t + 1 <= nj;
                    C xa[R], xb[R];
                    C ga = 0, gb = 0;
#pragma unroll
                    for (int i = 0; i < R; i++) {
                        const int row = lane + 32 * i;
                        xa[i] = row < m ? X[row * LDX + t] : C(0);
                        xb[i] = (two && row < m) ? X[row * LDX + t + 1] : C(0);
                    }
#pragma unroll
                    for (int i = 0; i < R; i++) {
                        ga = fma(v[i], xa[i], ga);
                        gb = fma(v[i], xb[i], gb);
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        ga += __shfl_xor_sync(FULL, ga, o);
                        gb += __shfl_xor_sync(FULL, gb, o);
                    }
                    const C acta = __shfl_sync(FULL, xa[0], c);
                    const C actb = __shfl_sync(FULL, xb[0], c);
                    const C sva = ga + (v0 - x0) * acta, svb = gb + (v0 - x0) * actb;
                    const C fa = rnd<S>((sva + sva) / vtv), fb = rnd<S>((svb + svb) / vtv);
#pragma unroll
                    for (int i = 0; i < R; i++) {
                        const int row = lane + 32 * i;
                        if (row < m && row > c) {
                            X[row * LDX + t] = rnd<S>(xa[i] - fa * v[i]);
                            if (two) X[row * LDX + t + 1] = rnd<S>(xb[i] - fb * v[i]);
                        } else if (row == c) {
                            X[row * LDX + t] = rnd<S>(acta - fa * v0);
                            if (two) X[row * LDX + t + 1] = rnd<S>(actb - fb * v0);
                        }
                    }
                }
                if (lane == c) X[c * LDX + c] = alpha;
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
            const C sp = rnd<S>(rnd<S>(sres[p]) - (p == rk ? C(1) : C(0)));
            s2p = fma(sp, sp, s2p);
        }
        const C snorm = rnd<S>(sqrt(warp_sum(s2p)));
        if (!isfinite((double)snorm)) fl |= CF_NONFINITE;
        if (snorm <= (C)a.eps) fl |= CF_CONVERGED;
        // ---- outputs: row k of P = mbar_k * d(J_k)
        if (lane < F) {
            const bool in = lane < nj;
            a.Jidx[k * F + lane] = in ? jl : -1;
            ((S*)a.mval)[k * F + lane] = from_d<S>(in ? (double)mv : 0.0);
            a.Praw[k * F + lane] = in ? (double)mv * a.d[jl] : 0.0;
            if (in && !isfinite((double)mv)) fl |= CF_NONFINITE;
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
    const size_t smem = Cfg::bytes() * Cfg::WPB;
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

// bins 2..7 of spai_bin (bin 7 at u_f = double: the 16-warp CTA kernel)
template <class S>
int launch_spai_cta_nw16(const SpaiArgs& a0, int num_sms, size_t smem_cap, cudaStream_t s);

template <class S>
int launch_spai_mid_bin(const SpaiArgs& a, int bin, int num_sms, size_t smem_cap, cudaStream_t s)
{
    switch (bin) {
    case 2: return launch_spai_mid<S, 4, 16>(a, num_sms, smem_cap, s);
    case 3: return launch_spai_mid<S, 8, 16>(a, num_sms, smem_cap, s);
    case 4: return launch_spai_mid<S, 4, 32>(a, num_sms, smem_cap, s);
    case 5: return launch_spai_mid<S, 8, 32>(a, num_sms, smem_cap, s);
    case 6: return launch_spai_mid<S, 16, 16>(a, num_sms, smem_cap, s);
    case 7:
        if constexpr (std::is_same<S, double>::value) return launch_spai_cta_nw16<S>(a, num_sms, smem_cap, s);
        else return launch_spai_mid<S, 16, 32>(a, num_sms, smem_cap, s);
    default: return SPAI_ERR_INTERNAL;
    }
}

}  // namespace spai
