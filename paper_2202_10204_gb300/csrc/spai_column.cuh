// The SPAI column kernel: Algorithm 1 for one column k of M per warp,
// on B = A^T D (column j of B is row j of A times d_j).
//
// Per column:
//   1. load the rows j in J_k of A (nonzeros only, as the u_f values of
//      B = A^T D formed once per nonzero before the kernel) into shared
//      memory, one list per lane (all loads in flight);
//   2. gather: the union of those lists (plus the list {k}) is the shadow
//      I_k, sorted, and gives the dense tile [B(I_k,J_k) | e_k(I_k)]
//      (row-major, shared memory): through a hash set and a register sort
//      when the lists hold at most 256 entries, else a sorted warp merge;
//   3. Householder QR of the tile and back substitution with the tile in
//      registers (MM = 32/64 rows).  Single and double: lane t keeps column
//      t; each step the pivot lane writes its column to shared memory, every
//      lane forms its dot product with it (the pivot lane's own dot is
//      ||x||^2), and the trailing lanes apply the reflector to their
//      registers.  Half: the tile is held in the A-operand layout of
//      m16n8k16 MMAs and each step's 32 dot products are one tensor-core
//      matrix-vector product.  Back substitution, m_c = (y_c - sum_t R(c,t)
//      m_t) / R(c,c): row oriented for single and double (one warp sum per
//      row), column oriented at half (R in shared memory, lane t updating
//      y_t) (larger shadows: spai_cta.cuh);
//   4. explicit residual s = B(I,J) m - e and ||s||_2 from the original tile;
//   5. adaptive: candidates J~ (column lists of A for l in I with s_l != 0,
//      minus J), rho_j, mean acceptance, up to beta additions, loop.
// Arithmetic: values are stored in u_f (S) and every inner product and
// update runs in the compute type (float for half/single, double for
// double) with each stored result rounded to S -- the FP16-storage /
// FP32-accumulate model at u_f = half.
#pragma once

#include <climits>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace spai {

constexpr int SPAI_LD = 33;       // row stride of the tile (32 columns + pad)
constexpr int SPAI_MAX_FILL = 31; // |J_k| <= 31 so that [B(I,J) | e] fits 32 lanes
constexpr int SPAI_MMAX_LIMIT = 512;
constexpr int SPAI_LDR = 40;      // column stride of R (rows 0..31) in shared memory, half path
constexpr int SPAI_HASH = 512;    // slots of the gather's hash set (at most 256 keys)
constexpr int SPAI_AUX_BYTES = 2560;  // per warp: the hash set and its ranks, later R (half path)
static_assert(SPAI_HASH * 5 <= SPAI_AUX_BYTES && 32 * SPAI_LDR * 2 <= SPAI_AUX_BYTES, "aux region");

#define CF_CONVERGED 1
#define CF_FILLCAP 2
#define CF_ALPHA 4
#define CF_NOCAND 8
#define CF_SINGULAR 16
#define CF_NONFINITE 32

struct SpaiArgs {
    int64_t n;
    int F;
    const int64_t* rp;
    const int32_t* col;
    const double* val;
    const int64_t* cp;   // A^T structure (adaptive)
    const int32_t* ri;
    const double* d;
    const void* bval;    // nnz of A in u_f: b = fl(a_ij d_j), explicit zeros marked (bmark)
    int32_t* Jidx;       // n * F, in: initial pattern, out: final pattern
    int32_t* Jcnt;       // n
    double* Praw;        // n * F: mbar * d(J) (entries 0 .. |J_k|-1 of row k)
    double* colres;      // n
    int32_t* flags;      // n
    int32_t* Icnt;       // n
    int32_t* nsolve;     // n
    double eps;
    int alpha, beta, rho_restricted;
    int mmax, cmax;      // per-warp tile rows and candidate capacity
    int rl;              // longest row of A (list capacity per lane)
    int warp_bytes;
    // fixed patterns: the kernel of a bin takes the nlist columns of list
    // (null: all n columns, adaptive); the host side holds every bin's list
    // (bin b: bcnt[b] columns from blist + boff[b], see spai_bin)
    const int32_t* list;
    int64_t nlist;
    const int32_t* blist;
    int64_t boff[16], bcnt[16];  // at least SPAI_NBINS
    int* err;
    // columns for the large-shadow kernel (spai_big.cuh): fixed patterns whose
    // shadow exceeds the CTA tile (k_pattern), and adaptive columns that outgrew
    // the warp or CTA kernel's tile or candidate list (those kernels write the
    // current J_k to Jidx/Jcnt, the step to resume at to nsolve and the flags so
    // far to flags, then append k)
    int32_t* big;
    int* nbig;
};

// Fixed patterns: the column kernel of a column with shadow size m = |I_k|
// (at most SPAI_MMAX_LIMIT; larger shadows go to the large-shadow kernel)
// and nj = |J_k| columns:
//   0: warp kernel, 32-row register tile       1: warp kernel, 64 rows
//   2..13: warp kernel with the tile in shared memory (spai_mid.cuh), 32 R
//   rows by NC columns: up to 16 columns R = ceil(m/32) for R <= 8 (bins
//   2..7), then R = 10, 12, 16 (bins 8..10); 17..31 columns R = 4, 8, 16
//   (bins 11..13; at u_f = double bin 13 runs the 16-warp CTA kernel)
constexpr int SPAI_NBINS = 14;
__host__ __device__ inline int spai_bin(int m, int nj)
{
    if (m <= 32) return 0;
    if (m <= 64) return 1;
    const int R = (m + 31) / 32;
    if (nj <= 16) {
        if (R <= 8) return R - 1;
        return R <= 10 ? 8 : (R <= 12 ? 9 : 10);
    }
    return R <= 4 ? 11 : (R <= 8 ? 12 : 13);
}

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
__device__ inline void warp_bitonic_sort(int32_t* a, int len2)
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

// The entries of B = A^T D in the storage precision S, one per nonzero of A
// in its CSR order: b = fl_S(a_ij d_j), rounded once from the exact double
// product.  An explicit zero of A is stored as the all-ones bit pattern (a
// NaN, which no finite product rounds to), so the structural test a_ij != 0
// of the shadow needs no second array.
template <class S> __device__ __forceinline__ bool bmarked(S v);
template <> __device__ __forceinline__ bool bmarked<__half>(__half v) { return __half_as_ushort(v) == 0xffffu; }
template <> __device__ __forceinline__ bool bmarked<float>(float v) { return __float_as_uint(v) == 0xffffffffu; }
template <> __device__ __forceinline__ bool bmarked<double>(double v) { return __double_as_longlong(v) == -1LL; }
template <class S> __device__ __forceinline__ S bmark();
template <> __device__ __forceinline__ __half bmark<__half>() { return __ushort_as_half((unsigned short)0xffffu); }
template <> __device__ __forceinline__ float bmark<float>() { return __uint_as_float(0xffffffffu); }
template <> __device__ __forceinline__ double bmark<double>() { return __longlong_as_double(-1LL); }
// b as a compute-type value, explicit zeros as 0
template <class S> __device__ __forceinline__ typename Compute<S>::T bvalue(S v)
{
    typedef typename Compute<S>::T C;
    return bmarked<S>(v) ? C(0) : (C)to_c(v);
}

// per-warp shared-memory layout; the original tile W is kept in WT (u_f
// itself at half: its entries are half values, and the smaller tile lets more
// warps share an SM)
template <class C, class WT = C>
struct Tile {
    int32_t* I;     // mm
    WT* W;          // mm * LD: [B(I,J) | e]
    C* v;           // mm: pivot column / residual
    C* mb;          // 32
    int32_t* J;     // 32
    int32_t* lcol;  // 32 * rl
    C* lval;        // 32 * rl
    int32_t* lcnt;  // 32
    int32_t* cand;  // cmax
    C* rho;         // cmax
    WT* R;          // aux: 32 * SPAI_LDR, column-major R(0:31, 0:31) (half path, after the QR)
    int32_t* hkey;  // aux: SPAI_HASH keys of the gather's hash set (during the gather)
    unsigned char* hrank;  // aux: the rank in I_k of each slot's key
};

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

template <class C, class WT = C>
__host__ __device__ inline size_t tile_bytes(int mm, int rl, int cmax)
{
    size_t b = align16((size_t)mm * 4);
    b += align16((size_t)mm * SPAI_LD * sizeof(WT));
    b += align16((size_t)mm * sizeof(C));
    b += align16(32 * sizeof(C)) + 2 * 32 * 4;
    b += align16((size_t)32 * rl * 4) + align16((size_t)32 * rl * sizeof(C));
    b += align16((size_t)cmax * 4) + align16((size_t)cmax * sizeof(C));
    b += SPAI_AUX_BYTES;
    return align16(b);
}

template <class C, class WT = C>
__device__ inline Tile<C, WT> carve(unsigned char* base, int mm, int rl, int cmax)
{
    Tile<C, WT> t;
    size_t off = 0;
    t.I = (int32_t*)(base + off); off += align16((size_t)mm * 4);
    t.W = (WT*)(base + off); off += align16((size_t)mm * SPAI_LD * sizeof(WT));
    t.v = (C*)(base + off); off += align16((size_t)mm * sizeof(C));
    t.mb = (C*)(base + off); off += align16(32 * sizeof(C));
    t.J = (int32_t*)(base + off); off += 32 * 4;
    t.lcnt = (int32_t*)(base + off); off += 32 * 4;
    t.lcol = (int32_t*)(base + off); off += align16((size_t)32 * rl * 4);
    t.lval = (C*)(base + off); off += align16((size_t)32 * rl * sizeof(C));
    t.cand = (int32_t*)(base + off); off += align16((size_t)cmax * 4);
    t.rho = (C*)(base + off); off += align16((size_t)cmax * sizeof(C));
    t.R = std::is_same<WT, __half>::value ? (WT*)(base + off) : nullptr;
    t.hkey = (int32_t*)(base + off);
    t.hrank = (unsigned char*)(base + off + SPAI_HASH * 4);
    return t;
}

// Steps 1-2: lists of the rows in J, then the sorted merge.  Returns |I_k|
// (which may exceed mm; then only the first mm rows were written).
template <class WT> __device__ __forceinline__ WT to_w(float v);
template <> __device__ __forceinline__ __half to_w<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ float to_w<float>(float v) { return v; }
template <class WT> __device__ __forceinline__ WT to_w(double v) { return (WT)v; }

// Step 1: lane l < nj copies the nonzeros of row J[l] of A (column of B) to
// its list in shared memory; returns the list's length.
template <class S, class C>
__device__ __forceinline__ int load_lists(const SpaiArgs& a, const int32_t* TJ, int32_t* tlcol, C* tlval, int nj)
{
    const int lane = threadIdx.x & 31;
    int len = 0;
    if (lane < nj) {
        const int j = TJ[lane];
        const S* bv = (const S*)a.bval;
        const int64_t b = a.rp[j], e = a.rp[j + 1];
        int32_t* lc = tlcol + lane * a.rl;
        C* lv = tlval + lane * a.rl;
        for (int64_t q = b; q < e; q += 4) {
            S vv[4];
            int cc[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                vv[u] = q + u < e ? bv[q + u] : bmark<S>();
                cc[u] = q + u < e ? a.col[q + u] : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                if (!bmarked<S>(vv[u])) {  // the shadow counts |a_ij| != 0
                    lc[len] = cc[u];
                    lv[len] = to_c(vv[u]);
                    len++;
                }
            }
        }
    }
    return len;
}

template <class S, class C, class WT>
__device__ __forceinline__ int gather_ptrs(const SpaiArgs& a, int32_t* TI, WT* TW, const int32_t* TJ, int32_t* tlcol,
                                           C* tlval, int32_t* tlcnt, int64_t k, int nj, int mm)
{
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const int len = load_lists<S, C>(a, TJ, tlcol, tlval, nj);
    tlcnt[lane] = len;
    __syncwarp();
    // merge; lane nj carries the list {k} with value 1 (the e_k column)
    int q = 0;
    const int32_t* lc = tlcol + lane * a.rl;
    const C* lv = tlval + lane * a.rl;
    int head = lane < nj ? (len > 0 ? lc[0] : INT_MAX) : (lane == nj ? (int)k : INT_MAX);
    int m = 0;
    while (true) {
        const int mn = __reduce_min_sync(FULL, head);
        if (mn == INT_MAX) break;
        const bool has = head == mn;
        if (m < mm) {
            if (lane == 0) TI[m] = mn;
            if (lane <= nj) TW[m * SPAI_LD + lane] = to_w<WT>(has ? (lane < nj ? lv[q] : C(1)) : C(0));
        }
        m++;
        if (has) {
            q++;
            head = (lane < nj && q < len) ? lc[q] : INT_MAX;
        }
    }
    __syncwarp();
    return m;
}

// A shared-memory hash set of int keys >= 0: 2^(32 - shift) slots (mask =
// slots - 1), empty = -1, linear probing from the top bits of Knuth's
// multiplicative hash.  Callers keep the load at most one half, so every
// probe sequence ends.
__device__ __forceinline__ unsigned hset_slot(int key, int shift) { return ((unsigned)key * 2654435761u) >> shift; }
// inserts key; returns 1 if it was not there yet
__device__ __forceinline__ int hset_insert(int32_t* tab, unsigned mask, int shift, int key)
{
    unsigned h = hset_slot(key, shift);
    for (unsigned probe = 0; probe <= mask; probe++) {
        const int old = atomicCAS(&tab[h], -1, key);
        if (old == -1) return 1;
        if (old == key) return 0;
        h = (h + 1u) & mask;
    }
    return 0;
}
// slot of a key that is in the set
__device__ __forceinline__ unsigned hset_find(const int32_t* tab, unsigned mask, int shift, int key)
{
    unsigned h = hset_slot(key, shift);
    for (unsigned probe = 0; probe <= mask; probe++) {
        if (tab[h] == key) break;
        h = (h + 1u) & mask;
    }
    return h;
}

// bitonic sort of 64 keys held two per lane (element 2 lane + i in x_i),
// ascending
__device__ __forceinline__ void warp_sort64(int& x0, int& x1)
{
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
#pragma unroll
    for (int k = 2; k <= 64; k <<= 1) {
        const bool asc = ((2 * lane) & k) == 0;
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j == 1) {
                const int lo = min(x0, x1), hi = max(x0, x1);
                x0 = asc ? lo : hi;
                x1 = asc ? hi : lo;
            } else {
                const int lm = j >> 1;
                const int y0 = __shfl_xor_sync(FULL, x0, lm), y1 = __shfl_xor_sync(FULL, x1, lm);
                const bool keep_min = ((lane & lm) == 0) == asc;
                x0 = keep_min ? min(x0, y0) : max(x0, y0);
                x1 = keep_min ? min(x1, y1) : max(x1, y1);
            }
        }
    }
}

// Steps 1-2 with a hash set (warp kernel, mm <= 64, at most 256 keys): the
// distinct row indices of the lists and k are collected in the hash set
// (new keys appended to I in arrival order), I is sorted in registers, each
// slot records its key's rank, and every list entry is written to its rank's
// row of the zeroed tile.  Same I_k and tile as the sorted merge.
template <class S, class C, class WT>
__device__ __forceinline__ int gather_hash(const SpaiArgs& a, const Tile<C, WT>& T, int64_t k, int nj, int mm)
{
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    constexpr unsigned mask = SPAI_HASH - 1;
    constexpr int shift = 23;  // 32 - log2(SPAI_HASH)
    static_assert((1 << (32 - shift)) == SPAI_HASH, "hash set size");
    int32_t* hk = T.hkey;
    for (int t = lane; t < SPAI_HASH / 4; t += 32) reinterpret_cast<int4*>(hk)[t] = make_int4(-1, -1, -1, -1);
    const int len = load_lists<S, C>(a, T.J, T.lcol, T.lval, nj);
    __syncwarp();
    const int32_t* lc = T.lcol + lane * a.rl;
    const C* lv = T.lval + lane * a.rl;
    // lane nj carries the list {k} (the e_k column)
    const int mylen = lane < nj ? len : (lane == nj ? 1 : 0);
    const int maxlen = (int)__reduce_max_sync(FULL, (unsigned)mylen);
    int m = 0;
    for (int t = 0; t < maxlen; t++) {
        int key = -1;
        if (t < mylen) key = lane < nj ? lc[t] : (int)k;
        const bool isnew = key >= 0 && hset_insert(hk, mask, shift, key);
        const unsigned bal = __ballot_sync(FULL, isnew);
        if (isnew) {
            const int pos = m + __popc(bal & ((1u << lane) - 1u));
            if (pos < mm) T.I[pos] = key;
        }
        m += __popc(bal);
    }
    __syncwarp();
    if (m > mm) return m;
    int x0 = 2 * lane < m ? T.I[2 * lane] : INT_MAX;
    int x1 = 2 * lane + 1 < m ? T.I[2 * lane + 1] : INT_MAX;
    warp_sort64(x0, x1);
    __syncwarp();
    if (2 * lane < m) {
        T.I[2 * lane] = x0;
        T.hrank[hset_find(hk, mask, shift, x0)] = (unsigned char)(2 * lane);
    }
    if (2 * lane + 1 < m) {
        T.I[2 * lane + 1] = x1;
        T.hrank[hset_find(hk, mask, shift, x1)] = (unsigned char)(2 * lane + 1);
    }
    const int n16 = (int)((m * SPAI_LD * sizeof(WT) + 15) / 16);
    for (int t = lane; t < n16; t += 32) reinterpret_cast<int4*>(T.W)[t] = make_int4(0, 0, 0, 0);
    __syncwarp();
    for (int t = 0; t < mylen; t++) {
        const int key = lane < nj ? lc[t] : (int)k;
        const int r = T.hrank[hset_find(hk, mask, shift, key)];
        T.W[r * SPAI_LD + lane] = to_w<WT>(lane < nj ? lv[t] : C(1));
    }
    __syncwarp();
    return m;
}

template <class S, class C, class WT>
__device__ __forceinline__ int gather(const SpaiArgs& a, const Tile<C, WT>& T, int64_t k, int nj, int mm)
{
    if (nj * a.rl < SPAI_HASH / 2) return gather_hash<S, C, WT>(a, T, k, nj, mm);
    return gather_ptrs<S, C, WT>(a, T.I, T.W, T.J, T.lcol, T.lval, T.lcnt, k, nj, mm);
}

// Step 3, register path.  Returns flags (CF_SINGULAR); writes mbar to T.mb.
template <class S, class C, int MM>
__device__ __forceinline__ int qr_solve_reg(const Tile<C>& T, int m, int nj)
{
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    C col[MM];
#pragma unroll
    for (int i = 0; i < MM; i++) col[i] = (i < m && lane <= nj) ? T.W[i * SPAI_LD + lane] : C(0);
    const int steps = nj < m ? nj : m;
#pragma unroll
    for (int c = 0; c < SPAI_MAX_FILL; c++) {
        if (c < steps) {
            // the pivot lane publishes x = column c, rows >= c
            if (lane == c) {
#pragma unroll
                for (int i = 0; i < MM; i++) T.v[i] = i >= c ? col[i] : C(0);
            }
            __syncwarp();
            C g0 = 0, g1 = 0;
#pragma unroll
            for (int i = 0; i < MM; i += 2) {
                if (i + 1 >= c) {
                    g0 = fma(T.v[i], col[i], g0);
                    g1 = fma(T.v[i + 1], col[i + 1], g1);
                }
            }
            const C g = g0 + g1;
            const C sig2 = __shfl_sync(FULL, g, c);
            const C x0 = __shfl_sync(FULL, col[c], c);
            const C nrm = rnd<S>(sqrt(sig2));
            if (nrm != C(0)) {
                const C alpha = x0 >= C(0) ? -nrm : nrm;
                const C v0 = rnd<S>(x0 - alpha);
                const C vtv = C(2) * nrm * (nrm + fabs(x0));
                if (lane > c && lane <= nj) {
                    const C act = col[c];
                    const C sv = g + (v0 - x0) * act;
                    const C f = rnd<S>((sv + sv) / vtv);
                    col[c] = rnd<S>(act - f * v0);
#pragma unroll
                    for (int i = c + 1; i < MM; i++) col[i] = rnd<S>(col[i] - f * T.v[i]);
                }
                if (lane == c) col[c] = alpha;
            }
            __syncwarp();
        }
    }
    // back substitution, row oriented: R(c, t) is lane t's col[c]
    int fl = 0;
    C mv = 0;
#pragma unroll
    for (int c = SPAI_MAX_FILL - 1; c >= 0; c--) {
        if (c < nj) {
            C part = (lane > c && lane < nj) ? col[c] * mv : C(0);
            part = warp_sum(part);
            const C yc = __shfl_sync(FULL, col[c], nj);
            const C rcc = __shfl_sync(FULL, col[c], c);
            C mc = 0;
            if (c < m && rcc != C(0)) mc = rnd<S>(rnd<S>(yc - part) / rcc);
            else fl = CF_SINGULAR;
            if (lane == c) mv = mc;
        }
    }
    if (lane < nj) T.mb[lane] = mv;
    __syncwarp();
    return fl;
}

// d += a b on the tensor cores: one m16n8k16 tile, f16 operands, f32
// accumulators (a: 16 x 16 row-major fragment, b: 16 x 8 column-major)
__device__ __forceinline__ void mma_f16_f32(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned h2_bits(__half2 v) { return *reinterpret_cast<unsigned*>(&v); }
__device__ __forceinline__ __half2 bits_h2(unsigned v) { return *reinterpret_cast<__half2*>(&v); }
// element h (0 = low = the even row, 1 = high) of a packed pair
__device__ __forceinline__ float pair_elem(unsigned v, int h)
{
    return __half2float(__ushort_as_half((unsigned short)(h ? v >> 16 : v & 0xffffu)));
}
__device__ __forceinline__ unsigned pair_set(unsigned v, int h, __half x)
{
    const unsigned b = __half_as_ushort(x);
    return h ? ((v & 0xffffu) | (b << 16)) : ((v & 0xffff0000u) | b);
}

// Step 3, register path for u_f = half, on the tensor cores.  The tile X
// (rows r < MM, columns t < 32) is held in the A-operand layout of
// m16n8k16 MMAs that compute X^T v: with g = lane / 4 and q = lane % 4, the
// lane holds columns t = g + 8s (slots s = 0..3) at rows 16 ks + 2q + {0, 1,
// 8, 9} as packed half pairs, X[ks][s / 2][s % 2 (+ 2 for rows 8, 9)].  Per
// reflector step the pivot column is shuffled into the B operand (every
// lane q needs the rows its A fragment holds, from the lane of the pivot's
// group with the same q), and the MMAs give all 32 dot products v^T x_t
// with f16 x f16 products accumulated in f32; the lane of slot q then
// forms the reflector scalar f of column g + 8q, the quad exchanges them,
// and the update a - f v is one packed f16 FMA per row pair (the exact
// value rounded once to half: the trailing matrix is stored in u_f).
template <int MM>
__device__ __forceinline__ int qr_solve_reg_half(const Tile<float, __half>& T, int m, int nj)
{
    static_assert(MM % 16 == 0, "tile height is a multiple of the MMA k-step");
    constexpr int KS = MM / 16;
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, q = lane & 3;
    const unsigned FULL = 0xffffffffu;
    unsigned X[KS][2][4];
#pragma unroll
    for (int ks = 0; ks < KS; ks++)
#pragma unroll
        for (int mt = 0; mt < 2; mt++)
#pragma unroll
            for (int rg = 0; rg < 4; rg++) {
                const int t = 16 * mt + g + ((rg & 1) ? 8 : 0);
                const int r0 = 16 * ks + 2 * q + ((rg & 2) ? 8 : 0);
                const __half zero = __float2half_rn(0.f);
                const __half a0 = (r0 < m && t <= nj) ? T.W[r0 * SPAI_LD + t] : zero;
                const __half a1 = (r0 + 1 < m && t <= nj) ? T.W[(r0 + 1) * SPAI_LD + t] : zero;
                X[ks][mt][rg] = h2_bits(__halves2half2(a0, a1));
            }
    const int steps = nj < m ? nj : m;
    // Pivot steps c = 8 sc + (0..7).  The slot sc of column c and the k-step
    // and register pair of row c are fixed within a slot: the loop over the
    // four slots is unrolled (register indices are compile-time), the steps
    // within a slot are not (the kernel's code stays small enough for the
    // instruction caches).
#pragma unroll
    for (int sc = 0; sc < 4; sc++) {
        const int ksc = sc >> 1;              // k-step of rows 8 sc .. 8 sc + 7
        const int rh = (sc & 1) ? 2 : 0;      // register pair of those rows (+0 or +2)
        const int mt0 = sc >= 2 ? 1 : 0;      // columns below 16 mt0 are done
        const int cend = steps < 8 * sc + 8 ? steps : 8 * sc + 8;
#pragma unroll 1
        for (int c = 8 * sc; c < cend; c++) {
            const int gc = c & 7;                        // group of column c
            const int qc = (c & 7) >> 1, hc = c & 1;     // lane q and half of row c
            const unsigned hsel = hc ? 0x7632u : 0x5410u;  // byte_perm: element hc of two pairs
            // B operand: the pivot column with rows above c zeroed
            unsigned Bv[KS][2];
#pragma unroll
            for (int ks = 0; ks < KS; ks++) {
                if (ks < ksc) continue;
#pragma unroll
                for (int u = 0; u < 2; u++) {
                    unsigned v = __shfl_sync(FULL, X[ks][sc >> 1][(sc & 1) + 2 * u], gc * 4 + q);
                    if (ks == ksc) {
                        const int r = 16 * ks + 2 * q + 8 * u;
                        if (r + 1 < c) v = 0u;
                        else if (r < c) v &= 0xffff0000u;
                    }
                    Bv[ks][u] = v;
                }
            }
            float D[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; mt++) {
#pragma unroll
                for (int e = 0; e < 4; e++) D[mt][e] = 0.f;
                if (mt < mt0) continue;
#pragma unroll
                for (int ks = 0; ks < KS; ks++)
                    if (ks >= ksc) mma_f16_f32(D[mt], X[ks][mt], Bv[ks][0], Bv[ks][1]);
            }
            // slot s's dot product: D[s / 2][2 (s % 2)] (every column of B is v)
            const float sig2 = __shfl_sync(FULL, D[sc >> 1][2 * (sc & 1)], gc * 4);
            // row c of this lane's four columns (meaningful in the lanes q == qc)
            const unsigned rc01 = __byte_perm(X[ksc][0][rh], X[ksc][0][rh + 1], hsel);
            const unsigned rc23 = __byte_perm(X[ksc][1][rh], X[ksc][1][rh + 1], hsel);
            const float x0 = __shfl_sync(FULL, pair_elem(sc < 2 ? rc01 : rc23, sc & 1), gc * 4 + qc);
            const float nrm = rnd<__half>(sqrtf(sig2));
            if (nrm != 0.f) {
                const float alpha = x0 >= 0.f ? -nrm : nrm;
                const float v0 = rnd<__half>(x0 - alpha);
                const float vtv = 2.f * nrm * (nrm + fabsf(x0));
                // the lane of slot q forms f for column g + 8q
                const unsigned a01 = __shfl_sync(FULL, rc01, g * 4 + qc);
                const unsigned a23 = __shfl_sync(FULL, rc23, g * 4 + qc);
                const int tq = g + 8 * q;
                const float gq = q == 0 ? D[0][0] : q == 1 ? D[0][2] : q == 2 ? D[1][0] : D[1][2];
                const float act = pair_elem(q < 2 ? a01 : a23, q & 1);
                __half f = __float2half_rn(0.f);
                if (tq > c && tq <= nj) {
                    const float sv = gq + (v0 - x0) * act;
                    f = __float2half_rn((sv + sv) / vtv);
                }
                // quad exchange: pair (f of slots 0, 1) and pair (slots 2, 3)
                const unsigned fb = __half_as_ushort(f);
                const unsigned fo = __shfl_xor_sync(FULL, fb, 1);
                const unsigned pr = (q & 1) ? (fo | (fb << 16)) : (fb | (fo << 16));
                const unsigned po = __shfl_xor_sync(FULL, pr, 2);
                const unsigned f01 = (q & 2) ? po : pr, f23 = (q & 2) ? pr : po;
                // update operand: v with row c = v0
                if (q == qc) Bv[ksc][rh >> 1] = pair_set(Bv[ksc][rh >> 1], hc, __float2half_rn(v0));
                // without branches: columns that take no update (t <= c, t > nj) get
                // f = 0, i.e. x + (+-0) = x (at most the sign of a zero changes)
#pragma unroll
                for (int s = 0; s < 4; s++) {
                    const int t = g + 8 * s;
                    if (s < sc) continue;  // every column of this slot is final
                    const unsigned fp = s < 2 ? f01 : f23;
                    const unsigned fs = (s & 1) ? (fp >> 16) : (fp & 0xffffu);
                    const unsigned nfb = (t > c && t <= nj) ? ((fs | (fs << 16)) ^ 0x80008000u) : 0u;
                    const __half2 nf = bits_h2(nfb);
#pragma unroll
                    for (int ks = 0; ks < KS; ks++) {
                        if (ks < ksc) continue;
#pragma unroll
                        for (int u = 0; u < 2; u++) {
                            unsigned& x = X[ks][s >> 1][(s & 1) + 2 * u];
                            x = h2_bits(__hfma2(nf, bits_h2(Bv[ks][u]), bits_h2(x)));
                        }
                    }
                }
                // the pivot column's row c becomes alpha
                if (g == gc && q == qc) {
                    unsigned& x = X[ksc][sc >> 1][(sc & 1) + rh];
                    x = pair_set(x, hc, __float2half_rn(alpha));
                }
            }
        }
    }
    // back substitution, column oriented: R (rows and columns 0..31) goes to
    // shared memory column-major; lane t keeps y_t = R(t, nj) minus the
    // products R(t, c) m_c of the solved rows (f32 FMAs), and m_c =
    // fl_h(fl_h(y_c) / R(c, c)) leaves a chain of one shuffle and one division
    // per row
    __half* Rs = T.R;
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
        for (int ks = 0; ks < (KS < 2 ? KS : 2); ks++)
#pragma unroll
            for (int u = 0; u < 2; u++)
                *reinterpret_cast<unsigned*>(Rs + (g + 8 * s) * SPAI_LDR + 16 * ks + 2 * q + 8 * u) = X[ks][s >> 1][(s & 1) + 2 * u];
    __syncwarp();
    int fl = 0;
    float y = lane < nj ? __half2float(Rs[nj * SPAI_LDR + lane]) : 0.f;
    float mv = 0.f;
#pragma unroll 1
    for (int c = nj - 1; c >= 0; c--) {
        const float rcc = __half2float(Rs[c * SPAI_LDR + c]);
        const float rtc = __half2float(Rs[c * SPAI_LDR + lane]);
        const float yc = __shfl_sync(FULL, y, c);
        float mc = 0.f;
        if (c < m && rcc != 0.f) mc = rnd<__half>(rnd<__half>(yc) / rcc);
        else fl = CF_SINGULAR;
        if (lane == c) mv = mc;
        if (lane < c) y = fmaf(-rtc, mc, y);
    }
    if (lane < nj) T.mb[lane] = mv;
    __syncwarp();
    return fl;
}

// Step 4: s = B(I,J) mbar - e from the unmodified tile
template <class S, class C, class WT>
__device__ __forceinline__ C residual(const Tile<C, WT>& T, int m, int nj)
{
    const int lane = threadIdx.x & 31;
    C part = 0;
    for (int p = lane; p < m; p += 32) {
        C acc = 0;
        for (int c = 0; c < nj; c++) acc = fma((C)to_c(T.W[p * SPAI_LD + c]), T.mb[c], acc);
        const C sp = rnd<S>(rnd<S>(acc) - (C)to_c(T.W[p * SPAI_LD + nj]));
        T.v[p] = sp;
        part = fma(sp, sp, part);
    }
    __syncwarp();
    return warp_sum(part);
}

template <class S>
struct TileStore {
    typedef typename std::conditional<std::is_same<S, __half>::value, __half, typename Compute<S>::T>::type T;
};

// Launched with 64-thread blocks (two columns).  At u_f = half the bound lets
// ten blocks share an SM (92-95 registers, no spills); single and double tiles
// need more registers per lane and keep the compiler's choice.
template <class S>
constexpr int spai_min_blocks() { return std::is_same<S, __half>::value ? 10 : 1; }

template <class S, bool ADAPTIVE, int MM>
__global__ void __launch_bounds__(64, spai_min_blocks<S>()) k_spai(SpaiArgs a)
{
    typedef typename Compute<S>::T C;
    typedef typename TileStore<S>::T WT;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const Tile<C, WT> T = carve<C, WT>(smem + (size_t)wib * a.warp_bytes, a.mmax, a.rl, a.cmax);
    const unsigned FULL = 0xffffffffu;
    const int F = a.F;
    const int mm = a.mmax;

    const int64_t ncols = a.list ? a.nlist : a.n;
    for (int64_t idx = blockIdx.x * (int64_t)wpb + wib; idx < ncols; idx += (int64_t)gridDim.x * wpb) {
        const int64_t k = a.list ? (int64_t)a.list[idx] : idx;
        int nj = a.Jcnt[k];
        if (lane < nj) T.J[lane] = a.Jidx[k * F + lane];
        __syncwarp();
        int fl = 0, m = 0, ns = 0;
        bool deferred = false;
        C snorm = 0;
        // the column outgrew this kernel's tile or candidate list: the
        // large-shadow kernel resumes it at `step` with the pattern in T.J
        auto defer = [&](int step) {
            fl = (int)__reduce_or_sync(FULL, (unsigned)fl);
            if (lane < nj) a.Jidx[k * F + lane] = T.J[lane];
            if (lane == 0) {
                a.Jcnt[k] = nj;
                a.nsolve[k] = step;
                a.flags[k] = fl;
                if (a.big) a.big[atomicAdd(a.nbig, 1)] = (int32_t)k;
                else atomicCAS(a.err, 0, SPAI_ERR_INTERNAL);
            }
            deferred = true;
            __syncwarp();
        };
        for (int step = 0;; step++) {
            m = gather<S, C, WT>(a, T, k, nj, mm);
            if (m > mm) { defer(step); break; }
            if constexpr (std::is_same<S, __half>::value) fl |= qr_solve_reg_half<MM>(T, m, nj);
            else fl |= qr_solve_reg<S, C, MM>(T, m, nj);
            const C s2 = residual<S, C, WT>(T, m, nj);
            snorm = rnd<S>(sqrt(s2));
            ns++;
            if (!isfinite((double)snorm)) fl |= CF_NONFINITE;
            if (snorm <= (C)a.eps) { fl |= CF_CONVERGED; break; }
            if (!ADAPTIVE) break;
            if (step >= a.alpha) { fl |= CF_ALPHA; break; }
            if (nj >= F) { fl |= CF_FILLCAP; break; }
            // ---- candidates: J~ = union over l in I with s_l != 0 of {j : a_jl != 0} \ J
            int cnt = 0;
            for (int p = 0; p < m; p++) {
                if (T.v[p] == C(0)) continue;
                const int l = T.I[p];
                const int64_t b = a.cp[l], e = a.cp[l + 1];
                for (int64_t q0 = b; q0 < e; q0 += 32) {
                    const int64_t q = q0 + lane;
                    bool ok = false;
                    int j = 0;
                    if (q < e) {
                        j = a.ri[q];
                        ok = bsearch_smem(T.J, nj, j) < 0;
                    }
                    const unsigned bal = __ballot_sync(FULL, ok);
                    const int pos = cnt + __popc(bal & ((1u << lane) - 1u));
                    if (ok && pos < a.cmax) T.cand[pos] = j;
                    cnt += __popc(bal);
                }
            }
            if (cnt > a.cmax) { defer(step); break; }  // redone from this step's solve
            int len2 = 1;
            while (len2 < cnt) len2 <<= 1;
            for (int t = cnt + lane; t < len2; t += 32) T.cand[t] = INT_MAX;
            __syncwarp();
            warp_bitonic_sort(T.cand, len2);
            int u = 0;
            for (int t0 = 0; t0 < cnt; t0 += 32) {
                const int t = t0 + lane;
                const int v = t < cnt ? T.cand[t] : INT_MAX;
                const bool keep = t < cnt && (t == 0 || T.cand[t - 1] != v);
                const unsigned bal = __ballot_sync(FULL, keep);
                __syncwarp();
                if (keep) T.cand[u + __popc(bal & ((1u << lane) - 1u))] = v;
                u += __popc(bal);
                __syncwarp();
            }
            if (u == 0) { fl |= CF_NOCAND; break; }
            // ---- rho_j^2 = ||s||^2 - (s^T b_j)^2 / ||b_j||^2
            for (int t = lane; t < u; t += 32) {
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
            __syncwarp();
            C rs = 0;
            for (int t = lane; t < u; t += 32) rs += T.rho[t];
            const C mean = warp_sum(rs) / (C)u;
            // ---- up to min(beta, F - nj) acceptable indices with the smallest rho
            const int room = F - nj;
            const int want = a.beta < room ? a.beta : room;
            int nadd = 0;
            for (int it = 0; it < want; it++) {
                C br = C(0);
                int bj = INT_MAX, bt = -1;
                for (int t = lane; t < u; t += 32) {
                    const C r = T.rho[t];
                    const int j = T.cand[t];
                    if (j < 0 || !(r <= mean)) continue;
                    if (bt < 0 || r < br || (r == br && j < bj)) { br = r; bj = j; bt = t; }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const C ob = __shfl_xor_sync(FULL, br, o);
                    const int oj = __shfl_xor_sync(FULL, bj, o);
                    const int ot = __shfl_xor_sync(FULL, bt, o);
                    const bool take = ot >= 0 && (bt < 0 || ob < br || (ob == br && oj < bj));
                    if (take) { br = ob; bj = oj; bt = ot; }
                }
                if (bt < 0) break;
                if (lane == 0) {
                    T.cand[bt] = -1;
                    int pos = nj + nadd;
                    while (pos > 0 && T.J[pos - 1] > bj) { T.J[pos] = T.J[pos - 1]; pos--; }
                    T.J[pos] = bj;
                }
                nadd++;
                __syncwarp();
            }
            if (nadd == 0) { fl |= CF_NOCAND; break; }
            nj += nadd;
            __syncwarp();
        }
        if (deferred) continue;
        fl = (int)__reduce_or_sync(FULL, (unsigned)fl);
        // ---- outputs: row k of P = mbar_k * d(J_k) (entries past |J_k| are never read)
        for (int t = lane; t < nj; t += 32) {
            const int j = T.J[t];
            const C mv = T.mb[t];
            a.Jidx[k * F + t] = j;
            a.Praw[k * F + t] = (double)mv * a.d[j];
            if (!isfinite((double)mv)) fl |= CF_NONFINITE;
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

template <class S>
int launch_spai_cta_t(const SpaiArgs& a0, bool adaptive, int num_sms, size_t smem_cap, cudaStream_t s);

template <class S>
int launch_spai_cta_nw8(const SpaiArgs& a0, int num_sms, size_t smem_cap, cudaStream_t s);
template <class S>
int launch_spai_cta_nw16(const SpaiArgs& a0, int num_sms, size_t smem_cap, cudaStream_t s);
// the tile tuner's choices (capi.cu)
int mid_tune_get(int device, int uf, int bin);
void mid_tune_put(int device, int uf, int bin, int variant);
// the shared-memory tile kernel (spai_mid.cuh), compiled in spai_mid_<u_f>.cu
int launch_spai_mid_bin_half(const SpaiArgs& a, int bin, int num_sms, size_t smem_cap, cudaStream_t s);
int launch_spai_mid_bin_single(const SpaiArgs& a, int bin, int num_sms, size_t smem_cap, cudaStream_t s);
int launch_spai_mid_bin_double(const SpaiArgs& a, int bin, int num_sms, size_t smem_cap, cudaStream_t s);
template <class S>
inline int launch_spai_mid_bin(const SpaiArgs& a, int bin, int num_sms, size_t smem_cap, cudaStream_t s)
{
    if constexpr (std::is_same<S, __half>::value) return launch_spai_mid_bin_half(a, bin, num_sms, smem_cap, s);
    else if constexpr (std::is_same<S, float>::value) return launch_spai_mid_bin_single(a, bin, num_sms, smem_cap, s);
    else return launch_spai_mid_bin_double(a, bin, num_sms, smem_cap, s);
}

// The warp kernel with a register tile of MMsel rows (over a.list when set).
template <class S>
int launch_spai_warp(const SpaiArgs& a0, bool adaptive, int MMsel, int num_sms, size_t smem_cap, cudaStream_t s);

// Launch for storage type S.  Fixed patterns run every bin's columns (from
// k_bin_place) in the bin's kernel (spai_bin), so that a column is computed
// the same way whatever matrix or batch it belongs to.  Adaptive patterns
// grow, so they run in the warp kernel when no shadow can exceed 64 rows and
// in the 16-warp CTA kernel otherwise.
template <class S>
int launch_spai_t(const SpaiArgs& a0, bool adaptive, int num_sms, size_t smem_cap, cudaStream_t s)
{
    if (adaptive) {
        SpaiArgs a = a0;
        a.list = nullptr;
        if (a.mmax > 64) return launch_spai_cta_t<S>(a, true, num_sms, smem_cap, s);
        return launch_spai_warp<S>(a, true, a.mmax <= 32 ? 32 : 64, num_sms, smem_cap, s);
    }
    for (int b = 0; b < SPAI_NBINS; b++) {
        if (a0.bcnt[b] == 0) continue;
        SpaiArgs a = a0;
        a.list = a0.blist + a0.boff[b];
        a.nlist = a0.bcnt[b];
        int rc;
        if (b <= 1) rc = launch_spai_warp<S>(a, false, b == 0 ? 32 : 64, num_sms, smem_cap, s);
        else if (b == 13 && std::is_same<S, double>::value) rc = launch_spai_cta_nw16<S>(a, num_sms, smem_cap, s);
        else rc = launch_spai_mid_bin<S>(a, b, num_sms, smem_cap, s);
        if (rc) return rc;
    }
    return 0;
}

template <class S>
int launch_spai_warp(const SpaiArgs& a0, bool adaptive, int MMsel, int num_sms, size_t smem_cap, cudaStream_t s)
{
    typedef typename Compute<S>::T C;
    typedef typename TileStore<S>::T WT;
    SpaiArgs a = a0;
    if (!adaptive) a.cmax = 0;
    a.mmax = MMsel;
    while (adaptive && a.cmax > 256 && tile_bytes<C, WT>(a.mmax, a.rl, a.cmax) > smem_cap) a.cmax >>= 1;
    const size_t wb = tile_bytes<C, WT>(a.mmax, a.rl, a.cmax);
    a.warp_bytes = (int)wb;
    // two warps (columns) per block: register-tile warps gain nothing from
    // sharing a larger block, and small blocks keep the occupancy granularity fine
    const int wpb = 2;
    if (wb * wpb > smem_cap) return SPAI_ERR_UNSUPPORTED;
    const size_t smem = wb * wpb;
    void (*kern)(SpaiArgs) = nullptr;
    if (adaptive) kern = MMsel == 32 ? k_spai<S, true, 32> : k_spai<S, true, 64>;
    else kern = MMsel == 32 ? k_spai<S, false, 32> : k_spai<S, false, 64>;
    SPAI_CUDA_TRY(allow_max_dynamic_smem(kern));
    int64_t blocks = ((a.list ? a.nlist : a.n) + wpb - 1) / wpb;
    const int64_t cap = (int64_t)num_sms * 64;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, wpb * 32, smem, s>>>(a);
    SPAI_CUDA_TRY(cudaGetLastError());
    return 0;
}

}  // namespace spai

int launch_spai_half(const spai::SpaiArgs& a, bool adaptive, int num_sms, size_t smem_cap, cudaStream_t s);
int launch_spai_single(const spai::SpaiArgs& a, bool adaptive, int num_sms, size_t smem_cap, cudaStream_t s);
int launch_spai_double(const spai::SpaiArgs& a, bool adaptive, int num_sms, size_t smem_cap, cudaStream_t s);
// the large-shadow kernel (spai_big.cuh) over list[0 .. *count), grid CTAs,
// each with slab_bytes of the slab
int launch_spai_big_half(const spai::SpaiArgs& a, bool adaptive, const int32_t* list, const int* count, int grid,
                         unsigned char* slab, size_t slab_bytes, int mcap, int ccap, cudaStream_t s);
int launch_spai_big_single(const spai::SpaiArgs& a, bool adaptive, const int32_t* list, const int* count, int grid,
                           unsigned char* slab, size_t slab_bytes, int mcap, int ccap, cudaStream_t s);
int launch_spai_big_double(const spai::SpaiArgs& a, bool adaptive, const int32_t* list, const int* count, int grid,
                           unsigned char* slab, size_t slab_bytes, int mcap, int ccap, cudaStream_t s);
