// SPAI column kernel for large shadows: one CTA of NW warps per column.
//
// The same steps as the warp kernel (spai_column.cuh) for tiles of up to
// 32*NW rows:
//   - gather: the warps take the rows j in J_k of A, collect their row
//     indices (plus k) in a shared-memory hash set, sort them into I_k and
//     write the tile [B(I_k,J_k) | e_k(I_k)] (row-major, shared memory, kept
//     unmodified); the hash set then gives the position of a row in I_k for
//     rho's inner products;
//   - Householder QR with the tile in registers: warp w holds rows
//     [32w, 32w+32), lane t holds column t.  Each step the lanes holding the
//     pivot column publish it to shared memory together with the pivot row;
//     every lane forms its warp's partial dot product, the NW partials of a
//     column are summed in warp order by every thread, and the trailing
//     lanes apply the reflector to their registers;
//   - back substitution in warp 0 (R has at most 31 rows, all in warp 0);
//   - explicit residual, candidate sets (all L_k rows in parallel, a block
//     scan places their column lists), a block bitonic sort and compaction,
//     rho_j for every candidate in parallel, the mean as a fixed-order block
//     sum, and up to beta block arg-min selections.
// Arithmetic and readings are those of the warp kernel.
#pragma once

#include "spai_column.cuh"

namespace spai {

template <int NW>
struct CtaSmem {
    static constexpr int MM = 32 * NW;
};

// block-wide exclusive scan of one int per thread; returns the prefix, *total
// gets the sum.  tmp: 32 ints of shared memory.
__device__ __forceinline__ int block_excl_scan(int v, int* tmp, int* total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = lane < nw ? tmp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) tmp[lane] = t;
    }
    __syncthreads();
    const int pre = (wid > 0 ? tmp[wid - 1] : 0) + x - v;
    *total = tmp[nw - 1];
    __syncthreads();
    return pre;
}

// block bitonic sort of a[0..len2), len2 a power of two
__device__ inline void block_bitonic_sort(int32_t* a, int len2)
{
    for (int size = 2; size <= len2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < len2 / 2; t += blockDim.x) {
                const int i = 2 * t - (t & (stride - 1));
                const int j = i + stride;
                const bool up = ((i & size) == 0);
                const int32_t x = a[i], y = a[j];
                if ((x > y) == up) { a[i] = y; a[j] = x; }
            }
            __syncthreads();
        }
    }
}

template <class C>
struct CtaTile {
    int32_t* hk;     // 2 mm: hash set of the shadow's row indices
    uint16_t* hr;    // 2 mm: each key's position in the sorted I_k
    int32_t* I;      // mm
    C* W;            // mm * LD (original tile)
    C* v;            // mm: pivot column, then the residual
    C* P;            // NW * 33: per-warp partial dot products
    C* arow;         // 32: the pivot row
    C* mb;           // 32
    int32_t* J;      // 32
    int32_t* lcnt;   // 32
    int32_t* tmp;    // 64
    int32_t* lcol;   // 32 * rl
    C* lval;         // 32 * rl
    int32_t* cand;   // cmax
    C* rho;          // cmax
    C* red;          // 33
    int* sc;         // 8 scalars
};

template <class C>
__host__ __device__ inline size_t cta_tile_bytes(int mm, int nw, int rl, int cmax)
{
    size_t b = align16((size_t)2 * mm * 4) + align16((size_t)2 * mm * 2);
    b += align16((size_t)mm * 4);
    b += align16((size_t)mm * SPAI_LD * sizeof(C));
    b += align16((size_t)mm * sizeof(C));
    b += align16((size_t)nw * 33 * sizeof(C));
    b += align16(32 * sizeof(C)) * 2;
    b += 2 * 32 * 4 + 64 * 4;
    b += align16((size_t)32 * rl * 4) + align16((size_t)32 * rl * sizeof(C));
    b += align16((size_t)cmax * 4) + align16((size_t)cmax * sizeof(C));
    b += align16(33 * sizeof(C)) + 8 * 4;
    return align16(b);
}

template <class C>
__device__ inline CtaTile<C> cta_carve(unsigned char* base, int mm, int nw, int rl, int cmax)
{
    CtaTile<C> t;
    size_t off = 0;
    t.hk = (int32_t*)(base + off); off += align16((size_t)2 * mm * 4);
    t.hr = (uint16_t*)(base + off); off += align16((size_t)2 * mm * 2);
    t.I = (int32_t*)(base + off); off += align16((size_t)mm * 4);
    t.W = (C*)(base + off); off += align16((size_t)mm * SPAI_LD * sizeof(C));
    t.v = (C*)(base + off); off += align16((size_t)mm * sizeof(C));
    t.P = (C*)(base + off); off += align16((size_t)nw * 33 * sizeof(C));
    t.arow = (C*)(base + off); off += align16(32 * sizeof(C));
    t.mb = (C*)(base + off); off += align16(32 * sizeof(C));
    t.J = (int32_t*)(base + off); off += 32 * 4;
    t.lcnt = (int32_t*)(base + off); off += 32 * 4;
    t.tmp = (int32_t*)(base + off); off += 64 * 4;
    t.lcol = (int32_t*)(base + off); off += align16((size_t)32 * rl * 4);
    t.lval = (C*)(base + off); off += align16((size_t)32 * rl * sizeof(C));
    t.cand = (int32_t*)(base + off); off += align16((size_t)cmax * 4);
    t.rho = (C*)(base + off); off += align16((size_t)cmax * sizeof(C));
    t.red = (C*)(base + off); off += align16(33 * sizeof(C));
    t.sc = (int*)(base + off);
    return t;
}

// deterministic block sum (warp sums in warp order); every thread gets it
template <class C>
__device__ __forceinline__ C block_sum_det(C v, C* red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        C t = lane < nw ? red[lane] : C(0);
        t = warp_sum(t);
        if (lane == 0) red[32] = t;
    }
    __syncthreads();
    const C r = red[32];
    __syncthreads();
    return r;
}

// position of key in the sorted shadow through the hash set (-1: not in I_k)
__device__ __forceinline__ int cta_find(const int32_t* hk, const uint16_t* hr, unsigned mask, int shift, int key)
{
    unsigned h = hset_slot(key, shift);
    for (unsigned probe = 0; probe <= mask; probe++) {
        const int v = hk[h];
        if (v == key) return hr[h];
        if (v == -1) return -1;
        h = (h + 1u) & mask;
    }
    return -1;
}

// Steps 1-2 block-parallel: every warp takes rows J[t] of A (t = warp, warp + NW, ...), its
// lanes the entries, and inserts the row indices into a hash set of 2 MM slots (new keys
// appended to I in arrival order, plus k); I is then sorted (block bitonic sort), each slot
// records its key's position, and the entries are written to their rows of the zeroed tile
// [B(I,J) | e_k].  The same sorted I_k and tile as the sorted merge.  Returns |I_k| (beyond
// MM: nothing written past the tile).
template <class S, class C, int NW>
__device__ int cta_gather_hash(const SpaiArgs& a, const CtaTile<C>& T, int64_t k, int nj, int* cnt)
{
    constexpr int MM = 32 * NW, HS = 2 * MM;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, BT = blockDim.x;
    const unsigned mask = HS - 1;
    const int shift = 32 - (31 - __clz(HS));
    const S* bv = (const S*)a.bval;
    for (int t = tid; t < HS; t += BT) T.hk[t] = -1;
    if (tid == 0) *cnt = 0;
    __syncthreads();
    auto add = [&](int key) {
        if (hset_insert(T.hk, mask, shift, key)) {
            const int pos = atomicAdd(cnt, 1);
            if (pos < MM) T.I[pos] = key;
        }
    };
    if (tid == 0) add((int)k);
    for (int t = wid; t < nj; t += NW) {
        const int j = T.J[t];
        const int64_t b = a.rp[j], e = a.rp[j + 1];
        for (int64_t q = b + lane; q < e; q += 32)
            if (!bmarked<S>(bv[q])) add(a.col[q]);
    }
    __syncthreads();
    const int m = *cnt;
    if (m > MM) return m;
    int len2 = 1;
    while (len2 < m) len2 <<= 1;
    for (int t = m + tid; t < len2; t += BT) T.I[t] = INT_MAX;
    __syncthreads();
    block_bitonic_sort(T.I, len2);
    for (int p = tid; p < m; p += BT) {
        const int key = T.I[p];
        unsigned h = hset_slot(key, shift);
        for (unsigned probe = 0; probe <= mask && T.hk[h] != key; probe++) h = (h + 1u) & mask;
        T.hr[h] = (uint16_t)p;
    }
    for (int t = tid; t < m * SPAI_LD; t += BT) T.W[t] = C(0);
    __syncthreads();
    for (int t = wid; t < nj; t += NW) {
        const int j = T.J[t];
        const int64_t b = a.rp[j], e = a.rp[j + 1];
        for (int64_t q = b + lane; q < e; q += 32) {
            const S v = bv[q];
            if (!bmarked<S>(v)) T.W[cta_find(T.hk, T.hr, mask, shift, a.col[q]) * SPAI_LD + t] = to_c(v);
        }
    }
    if (tid == 0) T.W[cta_find(T.hk, T.hr, mask, shift, (int)k) * SPAI_LD + nj] = C(1);
    __syncthreads();
    return m;
}

template <class S, bool ADAPTIVE, int NW>
__global__ void __launch_bounds__(32 * NW, NW <= 8 ? 2 : 1) k_spai_cta(SpaiArgs a)
{
    typedef typename Compute<S>::T C;
    constexpr int MM = 32 * NW;
    extern __shared__ __align__(16) unsigned char smem[];
    const CtaTile<C> T = cta_carve<C>(smem, MM, NW, a.rl, a.cmax);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, BT = blockDim.x;
    const unsigned FULL = 0xffffffffu;
    const int F = a.F;
    int* sc = T.sc;  // [0] nj, [1] m, [2] flags from warp 0, [3] nadd, [4] the gather's count

    const int64_t ncols = a.list ? a.nlist : a.n;
    for (int64_t idx = blockIdx.x; idx < ncols; idx += gridDim.x) {
        const int64_t k = a.list ? (int64_t)a.list[idx] : idx;
        if (tid == 0) { sc[0] = a.Jcnt[k]; sc[2] = 0; }
        __syncthreads();
        int nj = sc[0];
        if (tid < nj) T.J[tid] = a.Jidx[k * F + tid];
        __syncthreads();
        int m = 0, ns = 0, fl = 0;
        bool deferred = false;
        C snorm = 0;
        // the column outgrew the tile or the candidate list: the large-shadow
        // kernel resumes it at `step` with the pattern in T.J
        auto defer = [&](int step) {
            if (tid < nj) a.Jidx[k * F + tid] = T.J[tid];
            if (tid == 0) {
                a.Jcnt[k] = nj;
                a.nsolve[k] = step;
                a.flags[k] = fl | sc[2];
                if (a.big) a.big[atomicAdd(a.nbig, 1)] = (int32_t)k;
                else atomicCAS(a.err, 0, SPAI_ERR_INTERNAL);
            }
            deferred = true;
            __syncthreads();
        };
        for (int step = 0;; step++) {
            // ---- gather (every warp)
            m = cta_gather_hash<S, C, NW>(a, T, k, nj, &sc[4]);
            if (m > MM) { defer(step); break; }
            // ---- Householder QR, tile in registers: warp w rows [32w, 32w+32), lane t column t.
            // Warps whose rows all lie beyond |I_k| hold zeros: they skip the
            // arithmetic and only take part in the barriers.
            const int nwa = (m + 31) >> 5;
            const bool wact = wid < nwa;
            C col[32];
#pragma unroll
            for (int r = 0; r < 32; r++) {
                const int row = 32 * wid + r;
                col[r] = (row < m && lane <= nj) ? T.W[row * SPAI_LD + lane] : C(0);
            }
            const int steps = nj < m ? nj : m;
            for (int c = 0; c < steps; c++) {
                // publish the pivot column (rows >= c) and the pivot row
                if (wact) {
#pragma unroll
                    for (int r = 0; r < 32; r++) {
                        const int row = 32 * wid + r;
                        if (lane == c) T.v[row] = row >= c ? col[r] : C(0);
                        if (wid == 0 && r == c && lane <= nj) T.arow[lane] = col[r];
                    }
                }
                __syncthreads();
                if (wact) {
                    C g0 = 0, g1 = 0;
#pragma unroll
                    for (int r = 0; r < 32; r += 2) {
                        g0 = fma(T.v[32 * wid + r], col[r], g0);
                        g1 = fma(T.v[32 * wid + r + 1], col[r + 1], g1);
                    }
                    T.P[wid * 33 + lane] = g0 + g1;
                }
                __syncthreads();
                C g = 0, sig2 = 0;
                for (int w = 0; w < nwa; w++) {
                    g += T.P[w * 33 + lane];
                    sig2 += T.P[w * 33 + c];
                }
                const C x0 = T.v[c];
                const C nrm = rnd<S>(sqrt(sig2));
                if (nrm != C(0)) {
                    const C alpha = x0 >= C(0) ? -nrm : nrm;
                    const C v0 = rnd<S>(x0 - alpha);
                    const C vtv = C(2) * nrm * (nrm + fabs(x0));
                    if (wact && lane > c && lane <= nj) {
                        const C act = T.arow[lane];
                        const C sv = g + (v0 - x0) * act;
                        const C f = rnd<S>((sv + sv) / vtv);
#pragma unroll
                        for (int r = 0; r < 32; r++) {
                            const int row = 32 * wid + r;
                            if (row > c) col[r] = rnd<S>(col[r] - f * T.v[row]);
                            else if (row == c) col[r] = rnd<S>(act - f * v0);
                        }
                    }
                    if (wid == 0 && lane == c) {
#pragma unroll
                        for (int r = 0; r < 32; r++)
                            if (r == c) col[r] = alpha;
                    }
                }
                __syncthreads();
            }
            // ---- back substitution (warp 0 holds R): m_c = (y_c - sum_t R(c,t) m_t) / R(c,c)
            if (wid == 0) {
                int f0 = 0;
                C mv = 0;
                for (int c = nj - 1; c >= 0; c--) {
                    C rc = 0;
#pragma unroll
                    for (int r = 0; r < 32; r++)
                        if (r == c) rc = col[r];
                    C part = (lane > c && lane < nj) ? rc * mv : C(0);
                    part = warp_sum(part);
                    const C yc = __shfl_sync(FULL, rc, nj);
                    const C rcc = __shfl_sync(FULL, rc, c);
                    C mc = 0;
                    if (c < m && rcc != C(0)) mc = rnd<S>(rnd<S>(yc - part) / rcc);
                    else f0 = CF_SINGULAR;
                    if (lane == c) mv = mc;
                }
                if (lane < nj) T.mb[lane] = mv;
                if (lane == 0 && f0) sc[2] |= f0;
            }
            __syncthreads();
            // ---- explicit residual from the original tile
            C part = 0;
            for (int p = tid; p < m; p += BT) {
                C acc = 0;
                for (int c = 0; c < nj; c++) acc = fma(T.W[p * SPAI_LD + c], T.mb[c], acc);
                const C sp = rnd<S>(rnd<S>(acc) - T.W[p * SPAI_LD + nj]);
                T.v[p] = sp;
                part = fma(sp, sp, part);
            }
            const C s2 = block_sum_det(part, T.red);
            snorm = rnd<S>(sqrt(s2));
            ns++;
            if (!isfinite((double)snorm)) fl |= CF_NONFINITE;
            if (snorm <= (C)a.eps) { fl |= CF_CONVERGED; break; }
            if (!ADAPTIVE) break;
            if (step >= a.alpha) { fl |= CF_ALPHA; break; }
            if (nj >= F) { fl |= CF_FILLCAP; break; }
            // ---- candidates: the column lists of A for the rows l of I with s_l != 0
            int cntp = 0, l = 0;
            if (tid < m && T.v[tid] != C(0)) {
                l = T.I[tid];
                cntp = (int)(a.cp[l + 1] - a.cp[l]);
            }
            int total = 0;
            const int off = block_excl_scan(cntp, T.tmp, &total);
            if (total > a.cmax) { defer(step); break; }  // redone from this step's solve
            for (int q = 0; q < cntp; q++) {
                if (off + q >= a.cmax) break;
                const int j = a.ri[a.cp[l] + q];
                T.cand[off + q] = bsearch_smem(T.J, nj, j) < 0 ? j : INT_MAX;
            }
            const int cnt = total < a.cmax ? total : a.cmax;
            int len2 = 1;
            while (len2 < cnt) len2 <<= 1;
            for (int t = cnt + tid; t < len2; t += BT) T.cand[t] = INT_MAX;
            __syncthreads();
            block_bitonic_sort(T.cand, len2);
            // unique (sorted, INT_MAX dropped), compacted into rho's storage, then back
            int32_t* uniq = reinterpret_cast<int32_t*>(T.rho);
            int u = 0;
            for (int base = 0; base < cnt; base += BT) {
                const int t = base + tid;
                const int v = t < cnt ? T.cand[t] : INT_MAX;
                const int keep = (t < cnt && v != INT_MAX && (t == 0 || T.cand[t - 1] != v)) ? 1 : 0;
                int tot = 0;
                const int pos = block_excl_scan(keep, T.tmp, &tot);
                if (keep) uniq[u + pos] = v;
                u += tot;
            }
            __syncthreads();
            for (int t = tid; t < u; t += BT) T.cand[t] = uniq[t];
            __syncthreads();
            if (u == 0) { fl |= CF_NOCAND; break; }
            // ---- rho_j for every candidate
            for (int t = tid; t < u; t += BT) {
                const int j = T.cand[t];
                C num = 0, den = 0;
                for (int64_t q = a.rp[j]; q < a.rp[j + 1]; q++) {
                    const C bij = bvalue<S>(((const S*)a.bval)[q]);
                    const int p = cta_find(T.hk, T.hr, 2 * MM - 1, 32 - (31 - __clz(2 * MM)), a.col[q]);
                    if (p >= 0) num = fma(T.v[p], bij, num);
                    if (!a.rho_restricted || p >= 0) den = fma(bij, bij, den);
                }
                C r2 = s2;
                if (den > C(0)) r2 = s2 - num * num / den;
                T.rho[t] = sqrt(r2 > C(0) ? r2 : C(0));
            }
            __syncthreads();
            C rs = 0;
            for (int t = tid; t < u; t += BT) rs += T.rho[t];
            const C mean = block_sum_det(rs, T.red) / (C)u;
            // ---- up to min(beta, F - nj) acceptable indices with the smallest rho
            const int room = F - nj;
            const int want = a.beta < room ? a.beta : room;
            if (tid == 0) sc[3] = 0;
            __syncthreads();
            for (int itr = 0; itr < want; itr++) {
                C br = C(0);
                int bj = INT_MAX, bt = -1;
                for (int t = tid; t < u; t += BT) {
                    const C rr = T.rho[t];
                    const int j = T.cand[t];
                    if (j < 0 || !(rr <= mean)) continue;
                    if (bt < 0 || rr < br || (rr == br && j < bj)) { br = rr; bj = j; bt = t; }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const C ob = __shfl_xor_sync(FULL, br, o);
                    const int oj = __shfl_xor_sync(FULL, bj, o);
                    const int ot = __shfl_xor_sync(FULL, bt, o);
                    const bool take = ot >= 0 && (bt < 0 || ob < br || (ob == br && oj < bj));
                    if (take) { br = ob; bj = oj; bt = ot; }
                }
                if (lane == 0) { T.P[wid * 3] = br; T.tmp[wid] = bj; T.tmp[32 + wid] = bt; }
                __syncthreads();
                if (tid == 0) {
                    C b2 = C(0);
                    int j2 = INT_MAX, t2 = -1;
                    for (int w = 0; w < NW; w++) {
                        const int ow = T.tmp[32 + w];
                        if (ow < 0) continue;
                        const C ob = T.P[w * 3];
                        const int oj = T.tmp[w];
                        if (t2 < 0 || ob < b2 || (ob == b2 && oj < j2)) { b2 = ob; j2 = oj; t2 = ow; }
                    }
                    if (t2 >= 0) {
                        T.cand[t2] = -1;
                        const int nn = nj + sc[3];
                        int pos = nn;
                        while (pos > 0 && T.J[pos - 1] > j2) { T.J[pos] = T.J[pos - 1]; pos--; }
                        T.J[pos] = j2;
                        sc[3] = sc[3] + 1;
                    }
                }
                __syncthreads();
                if (sc[3] <= itr) break;  // nothing was acceptable
            }
            const int nadd = sc[3];
            __syncthreads();
            if (nadd == 0) { fl |= CF_NOCAND; break; }
            nj += nadd;
        }
        if (deferred) continue;
        fl |= sc[2];
        // ---- outputs: row k of P = mbar_k * d(J_k) (entries past |J_k| are never read)
        for (int t = tid; t < nj; t += BT) {
            const int j = T.J[t];
            const C mv = T.mb[t];
            a.Jidx[k * F + t] = j;
            a.Praw[k * F + t] = (double)mv * a.d[j];
            if (!isfinite((double)mv)) atomicOr(&sc[2], CF_NONFINITE);
        }
        __syncthreads();
        if (tid == 0) {
            a.Jcnt[k] = nj;
            a.colres[k] = (double)snorm;
            a.flags[k] = fl | sc[2];
            a.Icnt[k] = m;
            a.nsolve[k] = ns;
        }
        __syncthreads();
    }
}

template <class S, int NW>
int launch_spai_cta_nw(const SpaiArgs& a0, bool adaptive, int num_sms, size_t smem_cap, cudaStream_t s)
{
    typedef typename Compute<S>::T C;
    SpaiArgs a = a0;
    if (!adaptive) a.cmax = 0;
    a.mmax = 32 * NW;
    while (adaptive && a.cmax > 512 && cta_tile_bytes<C>(a.mmax, NW, a.rl, a.cmax) > smem_cap) a.cmax >>= 1;
    const size_t smem = cta_tile_bytes<C>(a.mmax, NW, a.rl, a.cmax);
    if (smem > smem_cap) return SPAI_ERR_UNSUPPORTED;
    a.warp_bytes = (int)smem;
    void (*kern)(SpaiArgs) = adaptive ? k_spai_cta<S, true, NW> : k_spai_cta<S, false, NW>;
    SPAI_CUDA_TRY(allow_max_dynamic_smem(kern));
    int occ = 0;
    SPAI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * NW, smem));
    if (occ < 1) return SPAI_ERR_UNSUPPORTED;
    int64_t blocks = std::min<int64_t>(a.list ? a.nlist : a.n, (int64_t)num_sms * occ);
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, 32 * NW, smem, s>>>(a);
    SPAI_CUDA_TRY(cudaGetLastError());
    return 0;
}

// Adaptive patterns grow, so they run 16 warps per column (tiles of 512
// rows).  Fixed patterns: bins 5 (8 warps per column, up to 256 rows, which
// fits two CTAs per SM) and 6 (16 warps, up to 512 rows) of spai_bin.
template <class S>
int launch_spai_cta_t(const SpaiArgs& a0, bool adaptive, int num_sms, size_t smem_cap, cudaStream_t s)
{
    return launch_spai_cta_nw<S, 16>(a0, adaptive, num_sms, smem_cap, s);
}

template <class S>
int launch_spai_cta_nw8(const SpaiArgs& a0, int num_sms, size_t smem_cap, cudaStream_t s)
{
    return launch_spai_cta_nw<S, 8>(a0, false, num_sms, smem_cap, s);
}

template <class S>
int launch_spai_cta_nw16(const SpaiArgs& a0, int num_sms, size_t smem_cap, cudaStream_t s)
{
    return launch_spai_cta_nw<S, 16>(a0, false, num_sms, smem_cap, s);
}

}  // namespace spai
