// SPAI column kernel for mid-size shadows of fixed patterns: one warp per
// column, 64 < |I_k| <= 32 R rows and |J_k| <= NC columns.
//
// The warp and CTA kernels keep one tile column per lane, so a column of
// ~150 shadow rows and ~12 pattern columns either does not fit a warp's
// registers or needs a CTA of 8 warps that synchronises at every
// Householder step.  Here the tile is held by rows: lane l keeps rows
// l, l + 32, ..., l + 32 (R-1) of [B(I_k,J_k) | e_k(I_k)] in registers
// (R (NC + 1) values), and every inner product of a step is a lane-local
// sum over its R rows followed by a warp sum; the column loop is unrolled at
// compile time so that every register index is static.
//
// Per column:
//   1. gather: each lane l < |J_k| walks row J_k[l] of A (the u_f values of
//      B = A^T D) and inserts its row indices into a shared-memory hash set
//      (new keys appended to I in arrival order); I_k is sorted (warp
//      bitonic sort), each hash slot records its key's rank, and the second
//      walk scatters every value to its rank's row of the zeroed tile W
//      (shared memory, kept unmodified for step 4, stored in u_f: its
//      entries are u_f values);
//   2. Householder QR of the register tile: per step c the norm of the
//      pivot column below row c, then for every later column its inner
//      product with the reflector (a warp sum each) and the update of every
//      lane's rows, rounded to u_f as stored (the arithmetic of the warp and
//      CTA kernels: v = x - alpha e_1 with alpha = -sign(x_0) ||x||,
//      v^T v = 2 ||x|| (||x|| + |x_0|));
//   3. back substitution m_c = (y_c - sum_{t>c} R(c,t) m_t) / R(c,c): row
//      c of R is lane c's first register row;
//   4. explicit residual s = B(I,J) m - e_k from W and ||s||_2.
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
    static constexpr int LDW = NC + 1;     // row stride of W (odd in 4-byte words for float)
    static constexpr int WPB = 2;          // warps per block
    static constexpr size_t bytes()
    {
        return ((size_t)HS * 4 + (size_t)HS * 2 + (size_t)MM * 4 + (size_t)MM * LDW * sizeof(S) + 15) & ~size_t(15);
    }
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
    constexpr int MM = Cfg::MM, HS = Cfg::HS, LDW = Cfg::LDW, WPB = Cfg::WPB;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned char* base = smem + (size_t)wib * Cfg::bytes();
    int32_t* hk = (int32_t*)base;
    uint16_t* hr = (uint16_t*)(base + (size_t)HS * 4);
    int32_t* I = (int32_t*)(base + (size_t)HS * 6);
    S* W = (S*)(base + (size_t)HS * 6 + (size_t)MM * 4);
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
        __syncwarp();
        int64_t q0 = 0;
        int len = 0;
        if (lane < nj) {
            q0 = a.rp[jl];
            len = (int)(a.rp[jl + 1] - q0);
        } else if (lane == nj) {
            len = 1;  // the list {k}: e_k
        }
        const int maxlen = warp_max(len);
        int m = 0;
        for (int t0 = 0; t0 < maxlen; t0 += 4) {
            int key[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                key[u] = -1;
                if (t0 + u < len) {
                    if (lane < nj) {
                        if (!bmarked<S>(bv[q0 + t0 + u])) key[u] = a.col[q0 + t0 + u];
                    } else {
                        key[u] = (int)k;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const bool isnew = key[u] >= 0 && hset_insert(hk, hmask, hshift, key[u]);
                const unsigned bal = __ballot_sync(FULL, isnew);
                if (isnew) {
                    const int pos = m + __popc(bal & ((1u << lane) - 1u));
                    if (pos < MM) I[pos] = key[u];
                }
                m += __popc(bal);
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
            const int n16 = (int)((m * LDW * sizeof(S) + 15) / 16);
            for (int t = lane; t < n16; t += 32) reinterpret_cast<int4*>(W)[t] = make_int4(0, 0, 0, 0);
        }
        __syncwarp();
        for (int t0 = 0; t0 < maxlen; t0 += 4) {
            if (lane < nj) {
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    if (t0 + u < len) {
                        const S b = bv[q0 + t0 + u];
                        if (!bmarked<S>(b)) W[(int)hr[hset_find(hk, hmask, hshift, a.col[q0 + t0 + u])] * LDW + lane] = b;
                    }
                }
            }
        }
        const int rk = hr[hset_find(hk, hmask, hshift, (int)k)];  // row of e_k
        __syncwarp();
        // ---- 2. Householder QR, rows in registers
        // X[i][0..NC): row lane + 32 i of B(I,J); X[i][NC]: of e_k
        C X[R][NC + 1];
#pragma unroll
        for (int i = 0; i < R; i++) {
            const int row = lane + 32 * i;
#pragma unroll
            for (int t = 0; t < NC; t++) X[i][t] = row < m ? (C)to_c(W[row * LDW + t]) : C(0);
            X[i][NC] = row == rk ? C(1) : C(0);
        }
        const int steps = nj < m ? nj : m;
#pragma unroll
        for (int c = 0; c < NC; c++) {
            if (c < steps) {
                // rows >= c: every slot but the first, and the first from lane c on
                C sp = 0;
#pragma unroll
                for (int i = 0; i < R; i++) {
                    const C x = (i > 0 || lane >= c) ? X[i][c] : C(0);
                    sp = fma(x, x, sp);
                }
                const C sig2 = warp_sum(sp);
                const C x0 = __shfl_sync(FULL, X[0][c], c);
                const C nrm = rnd<S>(sqrt(sig2));
                if (nrm != C(0)) {
                    const C alpha = x0 >= C(0) ? -nrm : nrm;
                    const C v0 = rnd<S>(x0 - alpha);
                    const C vtv = C(2) * nrm * (nrm + fabs(x0));
                    // the later columns, then the right-hand side e_k
#pragma unroll
                    for (int t = c + 1; t <= NC; t++) {
                        if (t < nj || t == NC) {
                            C gp = 0;
#pragma unroll
                            for (int i = 0; i < R; i++) {
                                const C v = (i > 0 || lane >= c) ? X[i][c] : C(0);
                                gp = fma(v, X[i][t], gp);
                            }
                            const C g = warp_sum(gp);
                            const C act = __shfl_sync(FULL, X[0][t], c);
                            const C sv = g + (v0 - x0) * act;
                            const C f = rnd<S>((sv + sv) / vtv);
#pragma unroll
                            for (int i = 0; i < R; i++) {
                                const int row = lane + 32 * i;
                                if (row > c) X[i][t] = rnd<S>(X[i][t] - f * X[i][c]);
                                else if (row == c) X[i][t] = rnd<S>(act - f * v0);
                            }
                        }
                    }
                    if (lane == c) X[0][c] = alpha;
                }
            }
        }
        // ---- 3. back substitution: row c of R is lane c's X[0][0..NC), y_c its X[0][NC]
        C mreg[NC];
        int fl = 0;
#pragma unroll
        for (int c = NC - 1; c >= 0; c--) {
            mreg[c] = C(0);
            if (c < nj) {
                C part = 0;
#pragma unroll
                for (int t = c + 1; t < NC; t++)
                    if (t < nj) part = fma(X[0][t], mreg[t], part);
                const C rcc = __shfl_sync(FULL, X[0][c], c);
                C mc = 0;
                if (c < m && rcc != C(0)) mc = rnd<S>(rnd<S>(X[0][NC] - part) / rcc);
                else fl = CF_SINGULAR;
                mreg[c] = __shfl_sync(FULL, mc, c);
            }
        }
        // ---- 4. explicit residual from W
        C s2p = 0;
#pragma unroll
        for (int i = 0; i < R; i++) {
            const int row = lane + 32 * i;
            if (row < m) {
                C acc = 0;
#pragma unroll
                for (int t = 0; t < NC; t++)
                    if (t < nj) acc = fma((C)to_c(W[row * LDW + t]), mreg[t], acc);
                const C sp = rnd<S>(rnd<S>(acc) - (row == rk ? C(1) : C(0)));
                s2p = fma(sp, sp, s2p);
            }
        }
        const C snorm = rnd<S>(sqrt(warp_sum(s2p)));
        if (!isfinite((double)snorm)) fl |= CF_NONFINITE;
        if (snorm <= (C)a.eps) fl |= CF_CONVERGED;
        // ---- outputs: row k of P = mbar_k * d(J_k)
        if (lane < F) {
            C mv = 0;
#pragma unroll
            for (int t = 0; t < NC; t++)
                if (t == lane) mv = mreg[t];
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

// bins 2..4 of spai_bin
template <class S>
int launch_spai_mid_bin(const SpaiArgs& a, int bin, int num_sms, size_t smem_cap, cudaStream_t s)
{
    if (bin == 2) return launch_spai_mid<S, 4, 16>(a, num_sms, smem_cap, s);
    if constexpr (!std::is_same<S, double>::value) {
        if (bin == 3) return launch_spai_mid<S, 8, 16>(a, num_sms, smem_cap, s);
        if (bin == 4) return launch_spai_mid<S, 4, 32>(a, num_sms, smem_cap, s);
    }
    return SPAI_ERR_INTERNAL;
}

}  // namespace spai
