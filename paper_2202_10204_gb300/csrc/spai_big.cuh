// SPAI column kernel for shadows beyond the CTA kernel's register tile.
//
// Algorithm 1 for the columns that the warp kernel (spai_column.cuh) and the
// CTA kernel (spai_cta.cuh) cannot hold: fixed patterns whose shadow |I_k|
// exceeds 512 rows (listed by k_pattern), and adaptive columns whose shadow or
// candidate list outgrew those kernels' shared memory at some Grote-Huckle
// step (they write their current pattern J_k and the step to resume at, and
// append k to the same list).  Since the QR of every step is computed from
// scratch, resuming at that step with that pattern continues the column
// exactly where the smaller kernel left it.
//
// One CTA of 16 warps per column; the tile [B(I_k,J_k) | e_k(I_k)], its
// working copy, the pivot column / residual, the row lists and the candidate
// arrays live in a per-CTA slab of global memory sized from the largest shadow
// the matrix allows (max_fill times the longest row of A, plus one), so there
// is no row limit.  The steps and their arithmetic are those of the CTA
// kernel: Householder reflectors with v = x - alpha e_1, alpha = -sign(x_1)
// ||x|| (sign(0) = +1); every stored value rounded to u_f, inner products in
// the compute type, the partial sums of the 16 warps added in warp order.
#pragma once

#include "spai_cta.cuh"

namespace spai {

constexpr int BIG_NW = 16;

template <class C>
struct BigSlab {
    int32_t* I;     // mcap: the sorted shadow
    C* W;           // mcap * SPAI_LD: the gathered tile, unmodified
    C* X;           // mcap * SPAI_LD: the working copy the reflectors overwrite
    C* v;           // mcap: pivot column, then the residual
    int32_t* lcol;  // 32 * rl: row lists of the gather
    C* lval;        // 32 * rl
    int32_t* cand;  // ccap: candidate indices
    C* rho;         // ccap
    int32_t* uniq;  // ccap: compaction buffer
};

template <class C>
__host__ __device__ inline size_t big_slab_bytes(int mcap, int rl, int ccap)
{
    size_t b = align16((size_t)mcap * 4);
    b += 2 * align16((size_t)mcap * SPAI_LD * sizeof(C));
    b += align16((size_t)mcap * sizeof(C));
    b += align16((size_t)32 * rl * 4) + align16((size_t)32 * rl * sizeof(C));
    b += align16((size_t)ccap * 4) + align16((size_t)ccap * sizeof(C)) + align16((size_t)ccap * 4);
    return (b + 255) & ~size_t(255);
}

template <class C>
__device__ inline BigSlab<C> big_carve(unsigned char* base, int mcap, int rl, int ccap)
{
    BigSlab<C> t;
    size_t off = 0;
    t.I = (int32_t*)(base + off); off += align16((size_t)mcap * 4);
    t.W = (C*)(base + off); off += align16((size_t)mcap * SPAI_LD * sizeof(C));
    t.X = (C*)(base + off); off += align16((size_t)mcap * SPAI_LD * sizeof(C));
    t.v = (C*)(base + off); off += align16((size_t)mcap * sizeof(C));
    t.lcol = (int32_t*)(base + off); off += align16((size_t)32 * rl * 4);
    t.lval = (C*)(base + off); off += align16((size_t)32 * rl * sizeof(C));
    t.cand = (int32_t*)(base + off); off += align16((size_t)ccap * 4);
    t.rho = (C*)(base + off); off += align16((size_t)ccap * sizeof(C));
    t.uniq = (int32_t*)(base + off);
    return t;
}

// list[0 .. *count) holds the columns to process.  ADAPTIVE: each resumes at
// step nsolve[k] with the pattern Jcnt[k], Jidx[k*F ..] and the flags flags[k]
// its first kernel recorded; fixed patterns start at step 0.
template <class S, bool ADAPTIVE>
__global__ void __launch_bounds__(32 * BIG_NW, 1)
    k_spai_big(SpaiArgs a, const int32_t* __restrict__ list, const int* __restrict__ count, unsigned char* slab,
               size_t slab_bytes, int mcap, int ccap)
{
    typedef typename Compute<S>::T C;
    constexpr int NW = BIG_NW;
    __shared__ C Ps[NW * 33];
    __shared__ C arow[32], mb[32], red[33];
    __shared__ int32_t J[32], lcnt[32], tmp[64];
    __shared__ int sc[4];  // [0] |I_k| from the gather, [1] singular flag, [2] selections
    const BigSlab<C> T = big_carve<C>(slab + (size_t)blockIdx.x * slab_bytes, mcap, a.rl, ccap);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, BT = blockDim.x;
    const unsigned FULL = 0xffffffffu;
    const int F = a.F;
    const int total = *count;

    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int64_t k = list[item];
        int nj = a.Jcnt[k];
        if (tid < nj) J[tid] = a.Jidx[k * F + tid];
        if (tid == 0) sc[1] = 0;
        int step0 = 0, fl = 0;
        if (ADAPTIVE) {
            step0 = a.nsolve[k];
            fl = a.flags[k];
        }
        __syncthreads();
        int m = 0, ns = step0;
        C snorm = 0;
        for (int step = step0;; step++) {
            // ---- gather (warp 0): I_k sorted and the tile, into the slab
            if (wid == 0) {
                const int mg = gather_ptrs<S, C>(a, T.I, T.W, J, T.lcol, T.lval, lcnt, k, nj, mcap);
                if (lane == 0) sc[0] = mg;
            }
            __syncthreads();
            m = sc[0];
            if (m > mcap) {  // cannot happen: mcap bounds every shadow of this matrix
                if (tid == 0) atomicCAS(a.err, 0, SPAI_ERR_INTERNAL);
                __syncthreads();
                break;
            }
            for (int q = tid; q < m * SPAI_LD; q += BT) T.X[q] = T.W[q];
            __syncthreads();
            // ---- Householder QR of X (rows [0, m), columns [0, nj], column nj = e_k)
            const int steps = nj < m ? nj : m;
            for (int c = 0; c < steps; c++) {
                for (int r = tid; r < m; r += BT) T.v[r] = r >= c ? T.X[r * SPAI_LD + c] : C(0);
                if (tid <= nj) arow[tid] = T.X[c * SPAI_LD + tid];
                __syncthreads();
                C g0 = 0, g1 = 0;
                if (lane <= nj) {
                    int r = c + wid;
                    for (; r + NW < m; r += 2 * NW) {
                        g0 = fma(T.v[r], T.X[r * SPAI_LD + lane], g0);
                        g1 = fma(T.v[r + NW], T.X[(r + NW) * SPAI_LD + lane], g1);
                    }
                    if (r < m) g0 = fma(T.v[r], T.X[r * SPAI_LD + lane], g0);
                }
                Ps[wid * 33 + lane] = g0 + g1;
                __syncthreads();
                C g = 0, sig2 = 0;
                for (int w = 0; w < NW; w++) {
                    g += Ps[w * 33 + lane];
                    sig2 += Ps[w * 33 + c];
                }
                const C x0 = arow[c];
                const C nrm = rnd<S>(sqrt(sig2));
                if (nrm != C(0)) {
                    const C alpha = x0 >= C(0) ? -nrm : nrm;
                    const C v0 = rnd<S>(x0 - alpha);
                    const C vtv = C(2) * nrm * (nrm + fabs(x0));
                    if (lane > c && lane <= nj) {
                        const C act = arow[lane];
                        const C sv = g + (v0 - x0) * act;
                        const C f = rnd<S>((sv + sv) / vtv);
                        for (int r = c + wid; r < m; r += NW) {
                            if (r > c) T.X[r * SPAI_LD + lane] = rnd<S>(T.X[r * SPAI_LD + lane] - f * T.v[r]);
                            else T.X[r * SPAI_LD + lane] = rnd<S>(act - f * v0);
                        }
                    }
                    if (tid == 0) T.X[c * SPAI_LD + c] = alpha;
                }
                __syncthreads();
            }
            // ---- back substitution (warp 0; R is rows 0..nj-1 of X)
            if (wid == 0) {
                int f0 = 0;
                C mv = 0;
                for (int c = nj - 1; c >= 0; c--) {
                    const C rc = lane <= nj ? T.X[c * SPAI_LD + lane] : C(0);
                    C part = (lane > c && lane < nj) ? rc * mv : C(0);
                    part = warp_sum(part);
                    const C yc = __shfl_sync(FULL, rc, nj);
                    const C rcc = __shfl_sync(FULL, rc, c);
                    C mc = 0;
                    if (c < m && rcc != C(0)) mc = rnd<S>(rnd<S>(yc - part) / rcc);
                    else f0 = CF_SINGULAR;
                    if (lane == c) mv = mc;
                }
                if (lane < nj) mb[lane] = mv;
                if (lane == 0 && f0) sc[1] |= f0;
            }
            __syncthreads();
            // ---- explicit residual from the unmodified tile
            C part = 0;
            for (int p = tid; p < m; p += BT) {
                C acc = 0;
                for (int c = 0; c < nj; c++) acc = fma(T.W[p * SPAI_LD + c], mb[c], acc);
                const C sp = rnd<S>(rnd<S>(acc) - T.W[p * SPAI_LD + nj]);
                T.v[p] = sp;
                part = fma(sp, sp, part);
            }
            const C s2 = block_sum_det(part, red);
            snorm = rnd<S>(sqrt(s2));
            ns++;
            if (!isfinite((double)snorm)) fl |= CF_NONFINITE;
            if (snorm <= (C)a.eps) { fl |= CF_CONVERGED; break; }
            if (!ADAPTIVE) break;
            if (step >= a.alpha) { fl |= CF_ALPHA; break; }
            if (nj >= F) { fl |= CF_FILLCAP; break; }
            // ---- candidates: the column lists of A for the rows l of I with s_l != 0,
            // minus J, placed by block scans over chunks of BT rows (at most m * maxcol)
            int cnt = 0;
            for (int base = 0; base < m; base += BT) {
                const int p = base + tid;
                int cntp = 0, l = 0;
                if (p < m && T.v[p] != C(0)) {
                    l = T.I[p];
                    cntp = (int)(a.cp[l + 1] - a.cp[l]);
                }
                int tot = 0;
                const int off = cnt + block_excl_scan(cntp, tmp, &tot);
                for (int q = 0; q < cntp; q++) {
                    const int j = a.ri[a.cp[l] + q];
                    if (off + q < ccap) T.cand[off + q] = bsearch_smem(J, nj, j) < 0 ? j : INT_MAX;
                }
                cnt += tot;
            }
            if (cnt > ccap) {  // cannot happen: ccap >= mcap * (longest column of A)
                if (tid == 0) atomicCAS(a.err, 0, SPAI_ERR_INTERNAL);
                cnt = ccap;
            }
            int len2 = 1;
            while (len2 < cnt) len2 <<= 1;
            for (int t = cnt + tid; t < len2; t += BT) T.cand[t] = INT_MAX;
            __syncthreads();
            block_bitonic_sort(T.cand, len2);
            int u = 0;
            for (int base = 0; base < cnt; base += BT) {
                const int t = base + tid;
                const int v = t < cnt ? T.cand[t] : INT_MAX;
                const int keep = (t < cnt && v != INT_MAX && (t == 0 || T.cand[t - 1] != v)) ? 1 : 0;
                int tot = 0;
                const int pos = block_excl_scan(keep, tmp, &tot);
                if (keep) T.uniq[u + pos] = v;
                u += tot;
            }
            __syncthreads();
            for (int t = tid; t < u; t += BT) T.cand[t] = T.uniq[t];
            __syncthreads();
            if (u == 0) { fl |= CF_NOCAND; break; }
            // ---- rho_j for every candidate
            for (int t = tid; t < u; t += BT) {
                const int j = T.cand[t];
                C num = 0, den = 0;
                for (int64_t q = a.rp[j]; q < a.rp[j + 1]; q++) {
                    const C bij = bvalue<S>(((const S*)a.bval)[q]);
                    const int p = bsearch_smem(T.I, m, a.col[q]);
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
            const C mean = block_sum_det(rs, red) / (C)u;
            // ---- up to min(beta, F - nj) acceptable indices with the smallest rho
            const int room = F - nj;
            const int want = a.beta < room ? a.beta : room;
            if (tid == 0) sc[2] = 0;
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
                if (lane == 0) { Ps[wid * 3] = br; tmp[wid] = bj; tmp[32 + wid] = bt; }
                __syncthreads();
                if (tid == 0) {
                    C b2 = C(0);
                    int j2 = INT_MAX, t2 = -1;
                    for (int w = 0; w < NW; w++) {
                        const int ow = tmp[32 + w];
                        if (ow < 0) continue;
                        const C ob = Ps[w * 3];
                        const int oj = tmp[w];
                        if (t2 < 0 || ob < b2 || (ob == b2 && oj < j2)) { b2 = ob; j2 = oj; t2 = ow; }
                    }
                    if (t2 >= 0) {
                        T.cand[t2] = -1;
                        int pos = nj + sc[2];
                        while (pos > 0 && J[pos - 1] > j2) { J[pos] = J[pos - 1]; pos--; }
                        J[pos] = j2;
                        sc[2] = sc[2] + 1;
                    }
                }
                __syncthreads();
                if (sc[2] <= itr) break;  // nothing was acceptable
            }
            const int nadd = sc[2];
            __syncthreads();
            if (nadd == 0) { fl |= CF_NOCAND; break; }
            nj += nadd;
        }
        fl |= sc[1];
        // ---- outputs: row k of P = mbar_k * d(J_k) (entries past |J_k| are never read)
        int nf = 0;
        for (int t = tid; t < nj; t += BT) {
            const int j = J[t];
            const C mv = mb[t];
            a.Jidx[k * F + t] = j;
            a.Praw[k * F + t] = (double)mv * a.d[j];
            if (!isfinite((double)mv)) nf = CF_NONFINITE;
        }
        if (nf) atomicOr(&sc[1], nf);
        __syncthreads();
        if (tid == 0) {
            a.Jcnt[k] = nj;
            a.colres[k] = (double)snorm;
            a.flags[k] = fl | sc[1];
            a.Icnt[k] = m;
            a.nsolve[k] = ns;
        }
        __syncthreads();
    }
}

// Bytes of one CTA's slab for a matrix whose shadows have at most mcap rows
// and whose candidate lists have at most ccap entries.
template <class S>
size_t spai_big_slab_bytes(int mcap, int rl, int ccap)
{
    return big_slab_bytes<typename Compute<S>::T>(mcap, rl, ccap);
}

template <class S>
int launch_spai_big_t(const SpaiArgs& a, bool adaptive, const int32_t* list, const int* count, int grid,
                      unsigned char* slab, size_t slab_bytes, int mcap, int ccap, cudaStream_t s)
{
    void (*kern)(SpaiArgs, const int32_t*, const int*, unsigned char*, size_t, int, int) =
        adaptive ? k_spai_big<S, true> : k_spai_big<S, false>;
    if (grid < 1) return 0;
    kern<<<(unsigned)grid, 32 * BIG_NW, 0, s>>>(a, list, count, slab, slab_bytes, mcap, ccap);
    SPAI_CUDA_TRY(cudaGetLastError());
    return 0;
}

}  // namespace spai
