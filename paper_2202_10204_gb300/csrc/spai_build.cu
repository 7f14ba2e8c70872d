// SPAI construction on the GPU: Algorithm 1 (Grote-Huckle / Sedlacek variant)
// run on B = A^T D (Section 4 scaling), giving the left preconditioner
// P = M^T D (Section 3: run on A^T, transpose).
//
// Steps (each a kernel):
//   k_scale        d_j = 1 / max_i |a_ji|: every column of A^T (row of A) to max-abs 1
//   k_col_count / k_col_fill / k_col_sort
//                  structure of A^T (column lists of A) for pattern(A), pattern(A^2)
//                  and the candidate sets N_l of the adaptive step
//   k_pattern      initial J_k (identity, pattern(A), pattern(A^2)) with the fill cap
//   k_shadow_count |I_k| for sizing the per-column tiles
//   k_spai         one warp per column: gather B(I_k, J_k) (sorted warp merge of the
//                  rows j in J_k), Householder QR, back substitution, explicit
//                  residual s = B(I,J) m - e_k and ||s||, and (adaptive) the rho_jk
//                  scores, mean acceptance and up-to-beta augmentation, looping
//   k_assemble     P row k = m_k * d(J_k) in CSR (column k of M is row k of P)
#include <climits>
#include <cstdio>
#include <cstring>

#include "common.cuh"
#include "internal.h"

using namespace spai;

namespace {

constexpr int LD = 33;          // row stride of the per-column tile (32 columns + pad)
constexpr int MAX_FILL = 31;    // |J_k| <= 31 so that [B(I,J) | e] fits 32 lanes
constexpr int MMAX_LIMIT = 512; // largest |I_k| handled by the warp kernel

// ---------------------------------------------------------------- scaling

__global__ void k_scale(int64_t n, const int64_t* __restrict__ rp, const double* __restrict__ val,
                        int scale, double* __restrict__ d, int* __restrict__ err)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double mx = 0.0;
        bool fin = true;
        for (int64_t q = rp[i]; q < rp[i + 1]; q++) {
            double a = val[q];
            if (!isfinite(a)) fin = false;
            mx = fmax(mx, fabs(a));
        }
        if (!fin) atomicCAS(err, 0, SPAI_ERR_NONFINITE);
        if (mx == 0.0) atomicCAS(err, 0, SPAI_ERR_ZERO_ROW);
        d[i] = scale ? (mx > 0.0 ? 1.0 / mx : 1.0) : 1.0;
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

int scan_counts(int64_t n, const int32_t* in, int64_t* out, cudaStream_t s)
{
    const int64_t chunk = 1 << 16;
    int nb = (int)((n + chunk - 1) / chunk);
    if (nb < 1) nb = 1;
    int64_t* sums = nullptr;
    int rc = dev_alloc((void**)&sums, sizeof(int64_t) * (nb + 1), s);
    if (rc) return rc;
    k_block_sums<<<nb, 256, 0, s>>>(n, in, sums, chunk);
    k_scan_sums<<<1, 32, 0, s>>>(nb, sums);
    k_scan_chunks<<<nb, 256, 0, s>>>(n, in, sums, out, chunk);
    dev_free(sums, s);
    SPAI_CUDA_TRY(cudaGetLastError());
    return 0;
}

// ---------------------------------------------------------------- warp merge
// Sorted union of up to 32 sorted index lists, one per lane.  Each lane
// holds the head of its list; the warp repeatedly takes the minimum head
// (one REDUX), and every lane whose head equals it advances.  `emit(p, idx,
// has)` runs on all lanes for output position p.

struct ListCursor {
    int64_t q, e;
    int head;
};

__device__ __forceinline__ void cursor_load(ListCursor& c, const int32_t* __restrict__ idx,
                                            const double* __restrict__ val)
{
    // skip stored zeros when values are given (the shadow counts |a_ij| != 0)
    if (val) while (c.q < c.e && val[c.q] == 0.0) c.q++;
    c.head = c.q < c.e ? idx[c.q] : INT_MAX;
}

// ---------------------------------------------------------------- pattern

// Initial pattern J_k, capped at F keeping k and then the nearest indices
// (ties to the smaller index).  One warp per column; `buf` is a per-warp
// shared buffer of `cap` ints for the uncapped union.
__global__ void k_pattern(int64_t n, int init, int F, const int64_t* __restrict__ cp, const int32_t* __restrict__ ri,
                          int32_t* __restrict__ Jidx, int32_t* __restrict__ Jcnt, int cap, int* __restrict__ err)
{
    extern __shared__ int32_t pbuf[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    int32_t* buf = pbuf + wib * cap;
    for (int64_t k = blockIdx.x * (int64_t)wpb + wib; k < n; k += (int64_t)gridDim.x * wpb) {
        int cnt = 0;
        if (init == SPAI_PAT_IDENTITY) {
            if (lane == 0) buf[0] = (int32_t)k;
            cnt = 1;
        } else if (init == SPAI_PAT_A) {
            int64_t b = cp[k], e = cp[k + 1];
            cnt = (int)(e - b);
            if (cnt > cap) { if (lane == 0) atomicCAS(err, 0, SPAI_ERR_UNSUPPORTED); cnt = cap; }
            for (int t = lane; t < cnt; t += 32) buf[t] = ri[b + t];
        } else {
            // union over i in column k of A of column i of A (column k of A^2)
            int64_t b = cp[k], e = cp[k + 1];
            if (e - b > 32) { if (lane == 0) atomicCAS(err, 0, SPAI_ERR_UNSUPPORTED); e = b + 32; }
            ListCursor c;
            if (lane < e - b) {
                int i = ri[b + lane];
                c.q = cp[i]; c.e = cp[i + 1];
            } else { c.q = 0; c.e = 0; }
            cursor_load(c, ri, nullptr);
            while (true) {
                int mn = __reduce_min_sync(0xffffffffu, c.head);
                if (mn == INT_MAX) break;
                if (lane == 0 && cnt < cap) buf[cnt] = mn;
                cnt++;
                if (c.head == mn) { c.q++; cursor_load(c, ri, nullptr); }
            }
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
                    bool can_l = lo > 0, can_r = hi < cnt;
                    if (can_l && can_r) {
                        long dl = (long)k - buf[lo - 1], dr = (long)buf[hi] - k;
                        if (dl <= dr) lo--; else hi++;
                    } else if (can_l) lo--;
                    else hi++;
                }
            }
            lo = __shfl_sync(0xffffffffu, lo, 0);
            hi = __shfl_sync(0xffffffffu, hi, 0);
        }
        int nj = hi - lo;
        for (int t = lane; t < F; t += 32) Jidx[k * F + t] = t < nj ? buf[lo + t] : -1;
        if (lane == 0) Jcnt[k] = nj;
        __syncwarp();
    }
}

// |I_k| = |union of the nonzero columns of rows j in J_k, plus k|
__global__ void k_shadow_count(int64_t n, int F, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                               const double* __restrict__ val, const int32_t* __restrict__ Jidx,
                               const int32_t* __restrict__ Jcnt, int32_t* __restrict__ Icnt, int* __restrict__ maxI)
{
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    for (int64_t k = blockIdx.x * (int64_t)wpb + wib; k < n; k += (int64_t)gridDim.x * wpb) {
        int nj = Jcnt[k];
        ListCursor c;
        if (lane < nj) {
            int j = Jidx[k * F + lane];
            c.q = rp[j]; c.e = rp[j + 1];
            cursor_load(c, col, val);
        } else if (lane == nj) {
            c.q = 0; c.e = 1; c.head = (int)k;
        } else {
            c.q = 0; c.e = 0; c.head = INT_MAX;
        }
        int cnt = 0;
        while (true) {
            int mn = __reduce_min_sync(0xffffffffu, c.head);
            if (mn == INT_MAX) break;
            cnt++;
            if (c.head == mn) {
                c.q++;
                if (lane < nj) cursor_load(c, col, val);
                else c.head = INT_MAX;
            }
        }
        if (lane == 0) {
            Icnt[k] = cnt;
            atomicMax(maxI, cnt);
        }
    }
}

// ---------------------------------------------------------------- the column kernel

struct SpaiArgs {
    int64_t n;
    int F;
    const int64_t* rp;
    const int32_t* col;
    const double* val;
    const int64_t* cp;   // A^T structure (adaptive)
    const int32_t* ri;
    const double* d;
    int32_t* Jidx;       // n * F, in: initial pattern, out: final pattern
    int32_t* Jcnt;       // n
    double* Praw;        // n * F: mbar * d(J)
    void* mval;          // n * F in storage precision
    double* colres;      // n
    int32_t* flags;      // n
    int32_t* Icnt;       // n
    int32_t* nsolve;     // n
    double eps;
    int alpha, beta, rho_restricted;
    int mmax, cmax;      // per-warp tile rows and candidate capacity
    int warp_bytes;
    int* err;
};

__device__ __forceinline__ int bsearch_smem(const int32_t* a, int len, int key)
{
    int lo = 0, hi = len - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int v = a[mid];
        if (v == key) return mid;
        if (v < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

// warp bitonic sort of a[0..len2) in shared memory, len2 a power of two
__device__ void warp_bitonic_sort(int32_t* a, int len2)
{
    const int lane = threadIdx.x & 31;
    for (int size = 2; size <= len2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = lane; t < len2 / 2; t += 32) {
                int i = 2 * t - (t & (stride - 1));
                int j = i + stride;
                bool up = ((i & size) == 0);
                int32_t x = a[i], y = a[j];
                if ((x > y) == up) { a[i] = y; a[j] = x; }
            }
            __syncwarp();
        }
    }
}

#define CF_CONVERGED 1
#define CF_FILLCAP 2
#define CF_ALPHA 4
#define CF_NOCAND 8
#define CF_SINGULAR 16
#define CF_NONFINITE 32
#define CF_TOOBIG 64   // the augmented shadow exceeded the tile: previous solve kept

template <class S, bool ADAPTIVE>
__global__ void __launch_bounds__(256) k_spai(SpaiArgs a)
{
    typedef typename Compute<S>::T C;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int MM = a.mmax;
    unsigned char* base = smem + (size_t)wib * a.warp_bytes;
    int32_t* Iidx = (int32_t*)base;
    size_t off = ((size_t)MM * 4 + 15) & ~size_t(15);
    C* W = (C*)(base + off);
    off += ((size_t)MM * LD * sizeof(C) + 15) & ~size_t(15);
    C* s = (C*)(base + off);
    off += ((size_t)MM * sizeof(C) + 15) & ~size_t(15);
    C* mb = (C*)(base + off);
    off += 32 * sizeof(C);
    int32_t* Jl = (int32_t*)(base + off);
    off += 32 * 4;
    int32_t* Jprev = (int32_t*)(base + off);
    off += 32 * 4;
    int32_t* cand = (int32_t*)(base + off);
    off += (size_t)a.cmax * 4;
    C* rho = (C*)(base + off);
    const unsigned FULL = 0xffffffffu;
    const int F = a.F;

    for (int64_t k = blockIdx.x * (int64_t)wpb + wib; k < a.n; k += (int64_t)gridDim.x * wpb) {
        int nj = a.Jcnt[k];
        if (lane < nj) Jl[lane] = a.Jidx[k * F + lane];
        __syncwarp();
        int fl = 0, m = 0, ns = 0, nj_prev = nj, m_prev = 0;
        C snorm = 0;
        for (int step = 0;; step++) {
            // ---- gather Abar = B(I_k, J_k), ebar = e_k(I_k) by a sorted merge
            ListCursor cur;
            double dj = 0.0;
            if (lane < nj) {
                int j = Jl[lane];
                dj = a.d[j];
                cur.q = a.rp[j]; cur.e = a.rp[j + 1];
                cursor_load(cur, a.col, a.val);
            } else if (lane == nj) {
                cur.q = 0; cur.e = 1; cur.head = (int)k;
            } else {
                cur.q = 0; cur.e = 0; cur.head = INT_MAX;
            }
            m = 0;
            while (true) {
                int mn = __reduce_min_sync(FULL, cur.head);
                if (mn == INT_MAX) break;
                bool has = cur.head == mn;
                if (m < MM) {
                    if (lane == 0) Iidx[m] = mn;
                    if (lane <= nj) {
                        C v = C(0);
                        if (has) v = lane < nj ? to_c(from_d<S>(a.val[cur.q] * dj)) : C(1);
                        W[m * LD + lane] = v;
                    }
                }
                m++;
                if (has) {
                    cur.q++;
                    if (lane < nj) cursor_load(cur, a.col, a.val);
                    else cur.head = INT_MAX;
                }
            }
            __syncwarp();
            if (m > MM) {
                fl |= CF_TOOBIG;
                if (step == 0) {
                    if (lane == 0) atomicCAS(a.err, 0, SPAI_ERR_UNSUPPORTED);
                } else {
                    // the augmented shadow does not fit the tile: keep the previous solve
                    nj = nj_prev;
                    m = m_prev;
                    if (lane < nj) Jl[lane] = Jprev[lane];
                    __syncwarp();
                }
                break;
            }
            // ---- Householder QR of [Abar | ebar]; lane t owns column t
            const int steps = nj < m ? nj : m;
            for (int c = 0; c < steps; c++) {
                C g0 = 0, g1 = 0;
                if (lane <= nj) {
                    int i = c;
                    for (; i + 1 < m; i += 2) {
                        g0 = fma(W[i * LD + c], W[i * LD + lane], g0);
                        g1 = fma(W[(i + 1) * LD + c], W[(i + 1) * LD + lane], g1);
                    }
                    if (i < m) g0 = fma(W[i * LD + c], W[i * LD + lane], g0);
                }
                C g = g0 + g1;
                C sig2 = __shfl_sync(FULL, g, c);
                C nrm = rnd<S>(sqrt(sig2));
                if (nrm == C(0)) continue;
                C x0 = W[c * LD + c];
                C alpha = x0 >= C(0) ? -nrm : nrm;
                C v0 = rnd<S>(x0 - alpha);
                C vtv = C(2) * nrm * (nrm + fabs(x0));
                __syncwarp();
                if (lane > c && lane <= nj) {
                    C act = W[c * LD + lane];
                    C sv = g + (v0 - x0) * act;
                    C f = rnd<S>((sv + sv) / vtv);
                    W[c * LD + lane] = rnd<S>(act - f * v0);
                    for (int i = c + 1; i < m; i++) W[i * LD + lane] = rnd<S>(W[i * LD + lane] - f * W[i * LD + c]);
                }
                __syncwarp();
                if (lane == c) W[c * LD + c] = alpha;
                __syncwarp();
            }
            // ---- back substitution R mbar = (Q^T ebar)(1:nj); lane t ends with mbar_t
            {
                C y = lane < nj ? W[lane * LD + nj] : C(0);
                C mv = 0;
                for (int c = nj - 1; c >= 0; c--) {
                    C mc = 0;
                    if (lane == c) {
                        C rcc = c < m ? W[c * LD + c] : C(0);
                        if (rcc != C(0)) mc = rnd<S>(rnd<S>(y) / rcc);
                        else fl |= CF_SINGULAR;
                        mv = mc;
                    }
                    mc = __shfl_sync(FULL, mc, c);
                    if (lane < c) y = y - W[lane * LD + c] * mc;
                }
                fl = (int)__reduce_or_sync(FULL, (unsigned)fl);
                if (lane < nj) mb[lane] = mv;
            }
            __syncwarp();
            // ---- explicit residual s = Abar mbar - ebar, re-gathered from A
            for (int p = lane; p < m; p += 32) s[p] = C(0);
            __syncwarp();
            for (int c = 0; c < nj; c++) {
                int j = Jl[c];
                double djc = a.d[j];
                C mc = mb[c];
                for (int64_t q = a.rp[j] + lane; q < a.rp[j + 1]; q += 32) {
                    double av = a.val[q];
                    if (av != 0.0) {
                        int p = bsearch_smem(Iidx, m, a.col[q]);
                        s[p] = fma(to_c(from_d<S>(av * djc)), mc, s[p]);
                    }
                }
                __syncwarp();
            }
            C part = 0;
            for (int p = lane; p < m; p += 32) {
                C e = Iidx[p] == (int)k ? C(1) : C(0);
                C sp = rnd<S>(rnd<S>(s[p]) - e);
                s[p] = sp;
                part = fma(sp, sp, part);
            }
            C s2 = warp_sum(part);
            snorm = rnd<S>(sqrt(s2));
            ns++;
            __syncwarp();
            if (!isfinite((double)snorm)) fl |= CF_NONFINITE;
            if (snorm <= (C)a.eps) { fl |= CF_CONVERGED; break; }
            if (!ADAPTIVE) break;
            if (step >= a.alpha) { fl |= CF_ALPHA; break; }
            if (nj >= F) { fl |= CF_FILLCAP; break; }
            // ---- candidates: J~ = union over l in I with s_l != 0 of {j : a_jl != 0} \ J
            int cnt = 0;
            bool over = false;
            for (int p = 0; p < m; p++) {
                if (s[p] == C(0)) continue;
                int l = Iidx[p];
                int64_t b = a.cp[l], e = a.cp[l + 1];
                for (int64_t q0 = b; q0 < e; q0 += 32) {
                    int64_t q = q0 + lane;
                    bool ok = false;
                    int j = 0;
                    if (q < e) {
                        j = a.ri[q];
                        ok = bsearch_smem(Jl, nj, j) < 0;
                    }
                    unsigned bal = __ballot_sync(FULL, ok);
                    int pos = cnt + __popc(bal & ((1u << lane) - 1u));
                    if (ok && pos < a.cmax) cand[pos] = j;
                    cnt += __popc(bal);
                }
            }
            if (cnt > a.cmax) { over = true; cnt = a.cmax; }
            if (over && lane == 0) atomicCAS(a.err, 0, SPAI_ERR_INTERNAL);
            int len2 = 1;
            while (len2 < cnt) len2 <<= 1;
            if (len2 > a.cmax) len2 = a.cmax; // cmax is a power of two
            for (int t = cnt + lane; t < len2; t += 32) cand[t] = INT_MAX;
            __syncwarp();
            warp_bitonic_sort(cand, len2);
            // unique, in order
            int u = 0;
            for (int t0 = 0; t0 < cnt; t0 += 32) {
                int t = t0 + lane;
                int v = t < cnt ? cand[t] : INT_MAX;
                bool keep = t < cnt && (t == 0 || cand[t - 1] != v);
                unsigned bal = __ballot_sync(FULL, keep);
                __syncwarp();
                if (keep) cand[u + __popc(bal & ((1u << lane) - 1u))] = v;
                u += __popc(bal);
                __syncwarp();
            }
            if (u == 0) { fl |= CF_NOCAND; break; }
            // ---- rho_j^2 = ||s||^2 - (s^T b_j)^2 / ||b_j||^2 (statistics in float, or double)
            for (int t = lane; t < u; t += 32) {
                int j = cand[t];
                double djj = a.d[j];
                C num = 0, den = 0;
                for (int64_t q = a.rp[j]; q < a.rp[j + 1]; q++) {
                    C bij = to_c(from_d<S>(a.val[q] * djj));
                    int p = bsearch_smem(Iidx, m, a.col[q]);
                    if (p >= 0) num = fma(s[p], bij, num);
                    if (!a.rho_restricted || p >= 0) den = fma(bij, bij, den);
                }
                C r2 = s2;
                if (den > C(0)) r2 = s2 - num * num / den;
                rho[t] = sqrt(r2 > C(0) ? r2 : C(0));
            }
            __syncwarp();
            C rs = 0;
            for (int t = lane; t < u; t += 32) rs += rho[t];
            C mean = warp_sum(rs) / (C)u;
            // ---- take up to min(beta, F - nj) acceptable indices with the smallest rho
            if (lane < nj) Jprev[lane] = Jl[lane];
            __syncwarp();
            int room = F - nj;
            int want = a.beta < room ? a.beta : room;
            int nadd = 0;
            for (int it = 0; it < want; it++) {
                C br = C(0);
                int bj = INT_MAX, bt = -1;
                for (int t = lane; t < u; t += 32) {
                    C r = rho[t];
                    int j = cand[t];
                    if (j < 0 || !(r <= mean)) continue;
                    if (bt < 0 || r < br || (r == br && j < bj)) { br = r; bj = j; bt = t; }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    C ob = __shfl_xor_sync(FULL, br, o);
                    int oj = __shfl_xor_sync(FULL, bj, o);
                    int ot = __shfl_xor_sync(FULL, bt, o);
                    bool take = ot >= 0 && (bt < 0 || ob < br || (ob == br && oj < bj));
                    if (take) { br = ob; bj = oj; bt = ot; }
                }
                if (bt < 0) break;
                if (lane == 0) {
                    cand[bt] = -1;
                    // sorted insert into J
                    int pos = nj + nadd;
                    while (pos > 0 && Jl[pos - 1] > bj) { Jl[pos] = Jl[pos - 1]; pos--; }
                    Jl[pos] = bj;
                }
                nadd++;
                __syncwarp();
            }
            if (nadd == 0) { fl |= CF_NOCAND; break; }
            nj_prev = nj;
            m_prev = m;
            nj += nadd;
            __syncwarp();
        }
        fl = (int)__reduce_or_sync(FULL, (unsigned)fl);
        // ---- outputs: row k of P = mbar_k * d(J_k)
        for (int t = lane; t < F; t += 32) {
            bool in = t < nj;
            int j = in ? Jl[t] : -1;
            C mv = in ? mb[t] : C(0);
            a.Jidx[k * F + t] = j;
            ((S*)a.mval)[k * F + t] = from_d<S>((double)mv);
            a.Praw[k * F + t] = in ? (double)mv * a.d[j] : 0.0;
            if (in && !isfinite((double)mv)) fl |= CF_NONFINITE;
        }
        fl = (int)__reduce_or_sync(FULL, (unsigned)fl);
        if (lane == 0) {
            a.Jcnt[k] = nj;
            a.colres[k] = (double)snorm;
            a.flags[k] = fl;
            a.Icnt[k] = m;
            a.nsolve[k] = ns;
        }
        __syncwarp();
    }
}

// P in CSR from the padded per-column results
template <class S>
__global__ void k_assemble(int64_t n, int F, const int32_t* __restrict__ Jidx, const int32_t* __restrict__ Jcnt,
                           const double* __restrict__ Praw, const int64_t* __restrict__ prp,
                           int32_t* __restrict__ pcol, double* __restrict__ pval, S* __restrict__ pval_uf)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        int64_t o = prp[k];
        int nj = Jcnt[k];
        for (int c = 0; c < nj; c++) {
            double v = Praw[k * F + c];
            pcol[o + c] = Jidx[k * F + c];
            pval[o + c] = v;
            pval_uf[o + c] = from_d<S>(v);
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

__global__ void k_max_row(int64_t n, const int64_t* __restrict__ rp, int* __restrict__ out)
{
    int mx = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        mx = max(mx, (int)(rp[i + 1] - rp[i]));
#pragma unroll
    for (int q = 16; q > 0; q >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, q));
    if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}

template <class S>
size_t warp_bytes_for(int mmax, int cmax)
{
    typedef typename Compute<S>::T C;
    size_t b = ((size_t)mmax * 4 + 15) & ~size_t(15);
    b += ((size_t)mmax * LD * sizeof(C) + 15) & ~size_t(15);
    b += ((size_t)mmax * sizeof(C) + 15) & ~size_t(15);
    b += 32 * sizeof(C) + 64 * 4;
    b += (size_t)cmax * 4 + (size_t)cmax * sizeof(C);
    return (b + 15) & ~size_t(15);
}

template <class S>
int launch_spai(const SpaiArgs& a0, bool adaptive, int num_sms, size_t smem_cap, cudaStream_t s)
{
    SpaiArgs a = a0;
    if (!adaptive) a.cmax = 0;
    // candidate capacity: halve until one warp's tile fits
    while (adaptive && a.cmax > 256 && warp_bytes_for<S>(a.mmax, a.cmax) > smem_cap) a.cmax >>= 1;
    size_t wb = warp_bytes_for<S>(a.mmax, a.cmax);
    a.warp_bytes = (int)wb;
    int wpb = (int)(smem_cap / wb);
    if (wpb > 8) wpb = 8;
    if (wpb < 1) return SPAI_ERR_UNSUPPORTED;
    size_t smem = wb * wpb;
    auto kern = adaptive ? k_spai<S, true> : k_spai<S, false>;
    SPAI_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int64_t blocks = (a.n + wpb - 1) / wpb;
    int64_t cap = (int64_t)num_sms * 64;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, wpb * 32, smem, s>>>(a);
    SPAI_CUDA_TRY(cudaGetLastError());
    return 0;
}

}  // namespace

int spai_build_dev(int device, int num_sms, cudaStream_t s, const DevCsr& A, const spai_opts* o,
                   spai_precond* P_out, spai_stats* st)
{
    (void)device;
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
    int* err = nullptr;      // [0] error code, [1] max |I|, [2] max |J|
    int32_t* ccount = nullptr;
    int64_t* cp = nullptr;
    int32_t* ri = nullptr;
    int32_t *Jidx = nullptr, *Jcnt = nullptr, *Icnt = nullptr, *flags = nullptr, *nsolve = nullptr;
    double *Praw = nullptr, *colres = nullptr;
    void* mval = nullptr;
    unsigned long long* fstat = nullptr;
    size_t ssz = o->uf == SPAI_HALF ? 2 : (o->uf == SPAI_SINGLE ? 4 : 8);
    spai_precond P = nullptr;
    int h_err[3] = {0, 0, 0};
    unsigned long long h_fstat[3] = {0, 0, 0};
    int maxrow = 0, maxcol = 0;
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    const size_t smem_cap = optin > 0 ? (size_t)optin : (size_t)(100 * 1024);

#define TRY(x) do { rc = (x); if (rc) goto done; } while (0)
    TRY(dev_alloc((void**)&d, sizeof(double) * n, s));
    TRY(dev_alloc((void**)&err, sizeof(int) * 5, s));
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
    TRY(dev_alloc(&mval, ssz * n * F, s));
    TRY(dev_alloc((void**)&fstat, sizeof(unsigned long long) * 3, s));
    if (cudaMemsetAsync(err, 0, sizeof(int) * 5, s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
    if (cudaMemsetAsync(ccount, 0, sizeof(int32_t) * (n + 1), s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
    if (cudaMemsetAsync(fstat, 0, sizeof(unsigned long long) * 3, s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
    {
        int tb = 256;
        int gb = (int)std::min<int64_t>((n + tb - 1) / tb, (int64_t)num_sms * 32);
        if (gb < 1) gb = 1;
        k_scale<<<gb, tb, 0, s>>>(n, A.rowptr, A.val, o->scale, d, err);
        nl++;
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
        // the pattern: buffer for the uncapped union of pattern(A^2)
        const int cap = 1024;
        const int wpb = 4;
        size_t sm = (size_t)cap * 4 * wpb;
        SPAI_CUDA_TRY(cudaFuncSetAttribute(k_pattern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        int64_t blocks = std::min<int64_t>((n + wpb - 1) / wpb, (int64_t)num_sms * 64);
        if (blocks < 1) blocks = 1;
        k_pattern<<<(unsigned)blocks, wpb * 32, sm, s>>>(n, o->init, F, cp, ri, Jidx, Jcnt, cap, err);
        k_shadow_count<<<(unsigned)std::min<int64_t>((n + 7) / 8, (int64_t)num_sms * 64), 256, 0, s>>>(
            n, F, A.rowptr, A.col, A.val, Jidx, Jcnt, Icnt, err + 1);
        nl += 2;
        if (cudaGetLastError() != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
        if (cudaMemcpyAsync(h_err, err, sizeof(int) * 2, cudaMemcpyDeviceToHost, s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
        if (cudaStreamSynchronize(s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
        if (h_err[0]) { rc = h_err[0]; goto done; }
    }
    {
        // largest row nonzero count: bounds |I_k| <= max_fill * maxrow + 1 when adaptive
        int* mr = err + 3;
        k_max_row<<<(unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * 8) + 1, 256, 0, s>>>(n, A.rowptr, mr);
        k_max_row<<<(unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * 8) + 1, 256, 0, s>>>(n, cp, mr + 1);
        nl += 2;
        if (cudaMemcpyAsync(&maxrow, mr, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
        if (cudaMemcpyAsync(&maxcol, mr + 1, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
        if (cudaStreamSynchronize(s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
    }
    {
        SpaiArgs a;
        memset(&a, 0, sizeof(a));
        a.n = n; a.F = F; a.rp = A.rowptr; a.col = A.col; a.val = A.val; a.cp = cp; a.ri = ri; a.d = d;
        a.Jidx = Jidx; a.Jcnt = Jcnt; a.Praw = Praw; a.mval = mval; a.colres = colres; a.flags = flags;
        a.Icnt = Icnt; a.nsolve = nsolve; a.eps = o->eps;
        a.alpha = o->alpha < 0 ? (int)((n + o->beta - 1) / std::max(o->beta, 1)) : o->alpha;
        a.beta = o->beta; a.rho_restricted = o->rho_restricted; a.err = err;
        // adaptive: the tile holds up to MMAX_LIMIT shadow rows; a column whose
        // augmented shadow would exceed it keeps its previous solve (flag 64)
        int mneed = o->adaptive ? (int)std::min<int64_t>((int64_t)F * maxrow + 1, (int64_t)MMAX_LIMIT) : h_err[1];
        if (mneed < 1) mneed = 1;
        if (mneed > MMAX_LIMIT) { rc = SPAI_ERR_UNSUPPORTED; goto done; }
        a.mmax = (mneed + 31) & ~31;
        int cmax = 1;
        // raw candidate capacity: |I| * (largest column count of A); power of two
        while (cmax < (int64_t)a.mmax * maxcol) cmax <<= 1;
        a.cmax = cmax > 8192 ? 8192 : (cmax < 256 ? 256 : cmax);
        if (cudaEventRecord(ek0, s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
        if (o->uf == SPAI_HALF) TRY(launch_spai<__half>(a, o->adaptive != 0, num_sms, smem_cap, s));
        else if (o->uf == SPAI_SINGLE) TRY(launch_spai<float>(a, o->adaptive != 0, num_sms, smem_cap, s));
        else TRY(launch_spai<double>(a, o->adaptive != 0, num_sms, smem_cap, s));
        if (cudaEventRecord(ek1, s) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; }
        nl++;
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
    dev_free(d, s); dev_free(err, s); dev_free(ccount, s); dev_free(cp, s); dev_free(ri, s);
    dev_free(Jidx, s); dev_free(Jcnt, s); dev_free(Icnt, s); dev_free(flags, s); dev_free(nsolve, s);
    dev_free(Praw, s); dev_free(colres, s); dev_free(mval, s); dev_free(fstat, s);
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
