// The refinement kernel of Algorithm 3 (SPAI-GMRES-IR): device code shared
// by the per-precision instantiation units (gmres_ir_k_*.cu) and the host
// code in gmres_ir.cu.  The whole refinement loop of one system is ONE
// persistent cooperative kernel (k_ir); k_ir_batch runs many systems, one
// team of blocks per system at a time.  Each block owns a contiguous slice of
// rows, keeps its slice of the Arnoldi vector w in shared memory, and meets
// the other blocks only at bounded grid-wide exchanges: every grid-wide dot
// product is a fixed-order tree (block partials in slots, every block sums
// the slots in the same order), so all blocks hold bit-identical scalars and
// take identical control-flow decisions (GMRES convergence, refinement stop)
// without another barrier.  The Givens rotations, H, g and y are double
// precision in every block.
//
// Template parameters: TU, TG, TP the storage types of u, u_g, u_p (u_g and u_p
// may be half, for the one-reduction MGS only: vectors and matrix values are
// stored in half, every operation on them is binary32); RM = 2
// for the double-double residual (u_r = quad); LS selects the one-reduction
// MGS (orth 2), compiled as its own kernel so that the MGS / CGS2 kernel
// keeps its register allocation.
#pragma once

#include <algorithm>
#include <climits>
#include <cstring>

#include "common.cuh"
#include "internal.h"

namespace spai {


constexpr int IR_THREADS = 1024;
constexpr int KMAX_LIMIT = 1024;
constexpr int MAX_GRID = 160;   // exchange slots are polled by one warp, SPL slots per lane
constexpr int SPL = (MAX_GRID + 31) / 32;
constexpr int SLOT_WORDS = 16;  // one 128-byte line per block and parity (up to 4 words used)
constexpr int PF = 4;           // rows per thread whose next basis entries are prefetched
constexpr int MGS_GROUP_MIN_GRID = 64;  // grids from this size run the Gram-Schmidt rounds in a group
// one-reduction MGS: from this many partials (2 (j + 1) values x blocks) the sums over blocks are
// split among the blocks (one more exchange round) instead of every block reading all of them
constexpr int IR_DIST_MIN = 32768;

// SELL-32: rows in slices of 32; slice s stores its entries column-major
// (entry c of row 32s+l at off[s] + 32c + l), padded to the slice's longest
// row with (col = own row, val = 0).  Loads of one entry slot by a warp are
// one contiguous 128-byte line.
struct Sell {
    const int64_t* off;  // nslices + 1 element offsets
    const int32_t* col;
    const void* val;     // precision u_p
};

struct IrArgs {
    int64_t n;
    int64_t rb;                 // rows per block (multiple of 32)
    Sell A, P;                  // P.off == nullptr: P = I
    const int64_t* arp;         // A in CSR, float64 (residual)
    const int32_t* aci;
    const double* aval;
    const double* b;
    void* x;                    // n, precision u
    void* r;                    // n, precision u
    void* wbuf;                 // n, precision u_g: published w (or z)
    void* tbuf;                 // n, precision u_p: t = A v
    void* V;                    // ldv x (kmax + 1), precision u_g; a block reads back only its own rows
    int64_t ldv;
    double* R;                  // (kmax + 1) x kmax column-major, written by block 0
    unsigned long long* msg;    // [2 parities][gridDim.x][SLOT_WORDS] epoch-tagged words
    unsigned long long* msg2;   // the same for the Gram-Schmidt group's rounds
    int g2;                     // Gram-Schmidt group: blocks 0..g2-1, each over the rows of two
                                // blocks (0: every block runs the rounds on its own rows)
    int* err;
    long long limit;            // clock64 cycles a wait may take
    double anorm, bnorm, tau, stop_tol;
    int kmax, imax, stop_rule;
    int* its;                   // imax
    double* nbe;                // imax + 1
    int* out;                   // [0] steps, [1] flags
    int orth;                   // 0 modified Gram-Schmidt, 1 classical Gram-Schmidt twice (CGS2)
    int side;                   // 0 left preconditioning (P A d = P r), 1 right (A P u = r, d = P u)
    int G;                      // blocks of this system
    int block0;                 // its first block in a batched launch (0 alone)
    void* pvec;                 // CGS2: 2 parities x gridDim.x x (kmax + 1) partial dot products (u_g);
                                // one-reduction MGS: [value][block], 2 (kmax + 1) values
    unsigned* gcount;           // CGS2 / one-reduction MGS: counter of the barrier that publishes them (zeroed)
    void* L;                    // one-reduction MGS: the rows of T = (I + L)^{-1}, L the strictly
                                // lower part of Q^T Q (row i: its i entries left of the unit
                                // diagonal, packed at i (i - 1) / 2), u_g; block 0 writes them
    int jl;                     // rows 0 .. jl-1 of T are also kept in each block's shared memory
    int sblock;                 // one-reduction MGS: 1 = the system's last block owns no rows and
                                // runs the Givens rotations alone, publishing R, g (gpub) and the
                                // residual estimate of column c (R's unused entry (kmax, c))
    double* gpub;               // kmax + 2: g as that block leaves it
};

// Bytes of a Krylov-part scalar for sg = sizeof(u_g): binary32 when the
// vectors are stored in half.
inline int ir_scalar_bytes(int sg) { return sg == 2 ? 4 : sg; }

// Dynamic shared memory of the refinement kernel (ir_body's layout), sg =
// sizeof(u_g): five double arrays of kmax + 2 (Givens, g, the current column,
// y), the slice offsets of A and P, the block's rows of w (two blocks' rows
// with a Gram-Schmidt group), and for the one-reduction MGS (orth 2) the rows
// of w next to those of u, the reduced inner products, b, row j of L, the
// unit partials (reused for row j of T and h), rows 0 .. jl-1 of T and the
// table of segments per vector.
inline size_t ir_smem_bytes(int64_t rb, int kmax, int g2, int orth, int jl, int sg)
{
    const int64_t nsl = (rb + 31) >> 5;
    size_t b = sizeof(double) * 5 * (kmax + 2) + sizeof(int64_t) * 2 * (nsl + 1) + (g2 ? 2 : 1) * rb * sg + 64;
    if (orth == 2)
        b += (size_t)sg * rb +
             (size_t)ir_scalar_bytes(sg) * (2 * (kmax + 1) + 2 * (kmax + 1) + 2 * (kmax + 1 + 32) +
                                            (size_t)jl * (jl - 1) / 2) +
             sizeof(int) * (kmax + 2) + 16 +  // the unit-count table
             (size_t)ir_scalar_bytes(sg) * IR_THREADS + 16;  // the T row's group partials
    return b;
}

// rows of T kept in shared memory: as many as fit beside the rest, at most
// kmax + 1, within 64 KiB
inline int ir_pick_jl(int64_t rb, int kmax, size_t dyn_max, int sg)
{
    const size_t base = ir_smem_bytes(rb, kmax, 0, 2, 0, sg);
    if (base + 1024 > dyn_max) return 0;
    const size_t room = std::min<size_t>(dyn_max - base - 1024, 64 << 10) / ir_scalar_bytes(sg);
    int jl = 0;
    while (jl < kmax + 1 && (size_t)(jl + 1) * jl / 2 <= room) jl++;
    return jl;
}

struct IrShared {
    int bid;          // the block's rank within its system
    int G;            // the system's block count
    unsigned epoch;
    unsigned epoch2;  // rounds of the Gram-Schmidt group
    unsigned gepoch;  // CGS2 barrier count
    int ok;
    double bcast[3];
    double resid;
    double dmax;   // this block's largest |d| of the last correction (as added to x, in u)
    double qprev;  // ||d_{i-2}|| / ||x_{i-1}|| (the stagnation test of the stop rules)
};

__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// One exchange round among all blocks of the co-resident grid.  Thread 0
// publishes NW 32-bit payload words, each tagged with the round's epoch in
// the upper 32 bits (one single-copy-atomic 64-bit store per word) after a
// fence that orders everything the block wrote before the preceding
// __syncthreads.  Each block's slot is a 128-byte line of its own: blocks
// sharing a line made every round measurably slower (the polls of all blocks
// and the stores of the line's owners queue on the same L2 line), while more
// polling warps or a denser layout made it slower still.  Warp 0 then polls every block's words of that epoch (lane
// l owns blocks l, l+32, ...), feeding them to `acc` in that fixed order,
// until one pass sees every word carry the epoch; it then fences (acquire)
// and `acc.finish` combines the lanes and publishes to shared memory.  Slots
// alternate between two parities, so a block can only overwrite a slot after
// every block has read it.  The wait is bounded: on expiry SPAI_ERR_TIMEOUT
// goes to *err and every block leaves.  Must be called by all threads after
// a __syncthreads that follows the block's writes.
struct NoWork {
    __device__ void operator()() const {}
};

// `work` runs on thread 0 after it has published the block's words and before
// warp 0 starts polling: the other blocks' words take about a microsecond to
// arrive, which hides short serial work there.
template <int NW, bool DATA, class Acc, bool GRP = false, class Work = NoWork>
__device__ __forceinline__ bool exchange(const IrArgs& a, IrShared* sh, const uint32_t* pay, Acc& acc,
                                         const Work& work = Work())
{
    // GRP: a round of the Gram-Schmidt group (blocks 0..g2-1), with its own
    // slots and epoch; only the group's blocks may call it
    const unsigned G = GRP ? (unsigned)a.g2 : (unsigned)sh->G;
    unsigned* epoch = GRP ? &sh->epoch2 : &sh->epoch;
    if (threadIdx.x < 32) {
        const unsigned ep = *epoch + 1u;
        unsigned long long* base = (GRP ? a.msg2 : a.msg) + (size_t)(ep & 1u) * G * SLOT_WORDS;
        if (threadIdx.x == 0) {
            if (DATA) __threadfence();
#pragma unroll
            for (int k = 0; k < NW; k++)
                st_relaxed_u64(base + (size_t)sh->bid * SLOT_WORDS + k, ((unsigned long long)ep << 32) | pay[k]);
            work();
        }
        const unsigned lane = threadIdx.x;
        const long long t0 = clock64();
        int ok = 1;
        for (unsigned spins = 1;; spins++) {
            bool all = true;
            acc.reset();
#pragma unroll
            for (int u = 0; u < SPL; u++) {
                const unsigned i = lane + 32u * u;
                if (i < G) {
                    uint32_t wv[NW];
#pragma unroll
                    for (int k = 0; k < NW; k++) {
                        unsigned long long w = ld_relaxed_u64(base + (size_t)i * SLOT_WORDS + k);
                        all = all && (unsigned)(w >> 32) == ep;
                        wv[k] = (uint32_t)w;
                    }
                    acc.add(wv);
                }
            }
            if (__all_sync(0xffffffffu, all)) break;
            if ((spins & 31u) == 0u) {
                int bad = 0;
                if (lane == 0) {
                    if (ld_relaxed_i32(a.err) != 0) bad = 1;
                    else if (clock64() - t0 > a.limit) { atomicCAS(a.err, 0, SPAI_ERR_TIMEOUT); bad = 1; }
                }
                if (__shfl_sync(0xffffffffu, bad, 0)) { ok = 0; break; }
            }
        }
        if (DATA) __threadfence();
        if (ok) acc.finish(lane, sh);
        __syncwarp();
        if (lane == 0) { sh->ok = ok; *epoch = ep; }
    }
    __syncthreads();
    return sh->ok != 0;
}

template <class T> struct SumAcc {
    T v;
    __device__ void reset() { v = T(0); }
    __device__ void add(const uint32_t* w)
    {
        if (sizeof(T) == 8) v += (T)__longlong_as_double((long long)(((unsigned long long)w[0] << 32) | w[1]));
        else v += (T)__uint_as_float(w[0]);
    }
    __device__ void finish(unsigned lane, IrShared* sh)
    {
        T t = warp_sum(v);
        if (lane == 0) sh->bcast[0] = (double)t;
    }
};

struct Max3Acc {
    double m[3];
    __device__ void reset() { m[0] = m[1] = m[2] = 0.0; }
    __device__ void add(const uint32_t* w)
    {
#pragma unroll
        for (int k = 0; k < 3; k++)
            m[k] = fmax(m[k], __longlong_as_double((long long)(((unsigned long long)w[2 * k] << 32) | w[2 * k + 1])));
    }
    __device__ void finish(unsigned lane, IrShared* sh)
    {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const double t = warp_max(m[k]);
            if (lane == 0) sh->bcast[k] = t;
        }
    }
};

struct NoAcc {
    __device__ void reset() {}
    __device__ void add(const uint32_t*) {}
    __device__ void finish(unsigned, IrShared*) {}
};

// Sum over all blocks of a per-thread value, in a fixed order; the result
// is identical in every block.  DATA: the round also publishes the global
// writes made before it (release/acquire); without it only the scalar
// travels, in the same single-copy-atomic word as its epoch.
template <bool DATA, class T, bool GRP = false, class Work = NoWork>
__device__ inline bool xsum(const IrArgs& a, IrShared* sh, T* red, T v, T& out, const Work& work = Work())
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    constexpr int NW = sizeof(T) == 8 ? 2 : 1;
    uint32_t pay[2] = {0u, 0u};
    if (wid == 0) {
        T t = lane < nw ? red[lane] : T(0);
        t = warp_sum(t);
        if (sizeof(T) == 8) {
            unsigned long long u = (unsigned long long)__double_as_longlong((double)t);
            pay[0] = (uint32_t)(u >> 32);
            pay[1] = (uint32_t)u;
        } else {
            pay[0] = __float_as_uint((float)t);
        }
    }
    SumAcc<T> acc;
    bool good = exchange<NW, DATA, SumAcc<T>, GRP>(a, sh, pay, acc, work);
    out = (T)sh->bcast[0];
    return good;
}

// Max of three non-negative doubles over all blocks; red holds 96 doubles.
__device__ inline bool xmax3(const IrArgs& a, IrShared* sh, double* red, const double (&v)[3], double (&o)[3])
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const double t = warp_max(v[k]);
        if (lane == 0) red[32 * k + wid] = t;
    }
    __syncthreads();
    uint32_t pay[6] = {0u, 0u, 0u, 0u, 0u, 0u};
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const double t = warp_max(lane < nw ? red[32 * k + lane] : 0.0);
            const unsigned long long u = (unsigned long long)__double_as_longlong(t);
            pay[2 * k] = (uint32_t)(u >> 32);
            pay[2 * k + 1] = (uint32_t)u;
        }
    }
    Max3Acc acc;
    bool good = exchange<6, true>(a, sh, pay, acc);
#pragma unroll
    for (int k = 0; k < 3; k++) o[k] = sh->bcast[k];
    return good;
}

// plain barrier (no payload)
__device__ inline bool xbar(const IrArgs& a, IrShared* sh)
{
    __syncthreads();
    uint32_t pay[1] = {0u};
    NoAcc acc;
    return exchange<1, true>(a, sh, pay, acc);
}

// y = M x for the block's rows (SELL-32), two rows per thread per pass with
// their loads interleaved; `store(row, value)` receives each result.  The
// slice offsets of the block live in shared memory (soff[0..nsl]).  Products
// and sums in the compute type of TP (binary32 for half values and inputs).
template <class TP, class Load, class Store>
__device__ __forceinline__ void sell_rows(int64_t r0, int64_t r1, const int64_t* soff, const int32_t* __restrict__ col,
                                          const TP* __restrict__ val, Load load, Store store)
{
    typedef typename Compute<TP>::T C;
    const int tid = threadIdx.x, BT = blockDim.x, lane = tid & 31;
    constexpr int U = 4;
    for (int64_t base = r0; base < r1; base += 2 * BT) {
        const int64_t ra = base + tid, rb = base + BT + tid;
        const bool va = ra < r1, vb = rb < r1;
        const int sa = (int)((ra - r0) >> 5), sb = (int)((rb - r0) >> 5);
        const int64_t oa = va ? soff[sa] + lane : 0, ob = vb ? soff[sb] + lane : 0;
        const int wa = va ? (int)((soff[sa + 1] - soff[sa]) >> 5) : 0;
        const int wb = vb ? (int)((soff[sb + 1] - soff[sb]) >> 5) : 0;
        C acc_a = C(0), acc_b = C(0);
        const int wmax = wa > wb ? wa : wb;
        // software pipeline: the entries of chunk c+1 load while chunk c gathers
        int ca[U], cb[U];
        TP xa[U], xb[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            ca[u] = u < wa ? __ldg(col + oa + 32 * u) : -1;
            xa[u] = u < wa ? __ldg(val + oa + 32 * u) : TP(0);
            cb[u] = u < wb ? __ldg(col + ob + 32 * u) : -1;
            xb[u] = u < wb ? __ldg(val + ob + 32 * u) : TP(0);
        }
        for (int c0 = 0; c0 < wmax; c0 += U) {
            C ga[U], gb[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                ga[u] = ca[u] >= 0 ? (C)load(ca[u]) : C(0);
                gb[u] = cb[u] >= 0 ? (C)load(cb[u]) : C(0);
            }
            C ya[U], yb[U];
#pragma unroll
            for (int u = 0; u < U; u++) { ya[u] = to_c(xa[u]); yb[u] = to_c(xb[u]); }
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int c = c0 + U + u;
                ca[u] = c < wa ? __ldg(col + oa + 32 * c) : -1;
                xa[u] = c < wa ? __ldg(val + oa + 32 * c) : TP(0);
                cb[u] = c < wb ? __ldg(col + ob + 32 * c) : -1;
                xb[u] = c < wb ? __ldg(val + ob + 32 * c) : TP(0);
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                acc_a = fma(ya[u], ga[u], acc_a);
                acc_b = fma(yb[u], gb[u], acc_b);
            }
        }
        if (va) store(ra, acc_a);
        if (vb) store(rb, acc_b);
    }
}

// max(m, |v|) with a NaN taken as infinite: fmax drops NaNs, and a non-finite
// residual or iterate must not pass for a small one in the stopping rule
__device__ __forceinline__ double max_abs(double m, double v) { return v != v ? INFINITY : fmax(m, fabs(v)); }

// v 2^e, exact (reading R17: the residual scaling of half-precision Krylov
// parts); the identity when HK is false
template <bool HK, class T> __device__ __forceinline__ T scale2(T v, int e)
{
    if constexpr (HK) return (T)ldexp((double)v, e);
    else return v;
}

// Threads per block of the refinement kernel: 896 (72 registers a thread)
// when the basis and the preconditioner products are single or half
// precision, which lets the one-reduction inner products keep four basis
// loads in flight per lane (1024 threads at 64 registers kept two); 512 when
// either is double, because the larger builds of those spill registers,
// which puts the basis prefetch behind HBM latency every Gram-Schmidt round.
template <class TG, class TP>
constexpr int ir_threads()
{
    return (sizeof(TG) == 8 || sizeof(TP) == 8) ? IR_THREADS / 2 : 896;
}

// The refinement of one system by its G blocks; `bid` is this block's rank.  BK: inside
// the batched kernel, whose claim loop holds more registers (fewer loads in flight).
template <class TU, class TG, class TP, int RM, bool LS, bool BK = false>
__device__ __forceinline__ void ir_body(const IrArgs& a, const int bid, const int G)
{
    // AG, AP: the arithmetic types of u_g and u_p (binary32 for half storage)
    typedef typename Compute<TG>::T AG;
    typedef typename Compute<TP>::T AP;
    // half storage in the Krylov part: the residual is scaled (reading R17)
    constexpr bool HK = sizeof(TG) == 2 || sizeof(TP) == 2;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ IrShared shs;
    __shared__ AG redg[33];
    __shared__ double redd[96];
    IrShared* sh = &shs;
    const int kmax = a.kmax;
    const int tid = threadIdx.x, BT = blockDim.x;
    // the Givens thread: thread 0, which also publishes the block's words, so that
    // the rotations of the Gram-Schmidt rounds run while its warp waits for the
    // other blocks
    const int GT = 0;
    const int64_t r0 = min(a.n, (int64_t)bid * a.rb);  // a block past the last row owns none
    const int64_t r1 = min(a.n, r0 + a.rb);
    // modified Gram-Schmidt rows [m0, m1): the block's own rows, or with a
    // Gram-Schmidt group the rows of blocks 2b and 2b+1 (empty outside it)
    const bool sub = a.g2 > 0;
    const bool gs = !sub || (int)bid < a.g2;
    const int64_t m0 = sub ? min(a.n, (int64_t)bid * 2 * a.rb) : r0;
    const int64_t m1 = sub ? (gs ? min(a.n, m0 + 2 * a.rb) : m0) : r1;
    const int nsl = (int)((a.rb + 31) >> 5);
    double* cs = (double*)smem;            // kmax + 2
    double* sn = cs + (kmax + 2);          // kmax + 2
    double* g = sn + (kmax + 2);           // kmax + 2
    double* hc = g + (kmax + 2);           // kmax + 2
    double* yv = hc + (kmax + 2);          // kmax + 2
    int64_t* soa = (int64_t*)(yv + (kmax + 2));  // nsl + 1 slice offsets of A
    int64_t* sop = soa + (nsl + 1);        // nsl + 1 slice offsets of P
    // w for rows [m0, m1) (rb, or 2 rb with a group), 16-byte aligned
    TG* ws = (TG*)(((uintptr_t)(sop + (nsl + 1)) + 15) & ~(uintptr_t)15);
    // Gram-Schmidt rows of this thread: PF rows as UV vectors of VN consecutive
    // rows, vector u = rows [vrow(u), vrow(u) + VN), then rows m0 + PF BT + tid
    // (step BT); the group's load, the first partial and every round use it
    constexpr int VN = 16 / (int)sizeof(TG);
    constexpr int UV = PF / VN;
    typedef typename std::conditional<sizeof(TG) == 8, double2, float4>::type TV;  // 16 bytes
    auto vrow = [&](int u) -> int64_t { return m0 + (int64_t)VN * (tid + u * BT); };
    // the prefetch set of basis vector Vb: out[u VN + e] = Vb[vrow(u) + e] (0 beyond m1)
    auto vload = [&](const TG* Vb, TG* out) {
#pragma unroll
        for (int u = 0; u < UV; u++) {
            const int64_t s0 = vrow(u);
            if (s0 + VN <= m1) {
                const TV t = __ldcg(reinterpret_cast<const TV*>(Vb + s0));
                memcpy(out + u * VN, &t, sizeof(TV));
            } else {
#pragma unroll
                for (int e = 0; e < VN; e++) out[u * VN + e] = s0 + e < m1 ? ldcg(&Vb[s0 + e]) : TG(0);
            }
        }
    };
    TU* x = (TU*)a.x;
    TU* r = (TU*)a.r;
    TG* wbuf = (TG*)a.wbuf;
    TP* tbuf = (TP*)a.tbuf;
    TG* V = (TG*)a.V;
    const TP* av = (const TP*)a.A.val;
    const TP* pv = (const TP*)a.P.val;
    const bool hasP = a.P.off != nullptr;
    // the Arnoldi product w = second(first(v)): left P (A v), right A (P v)
    const bool rightP = hasP && a.side == 1;
    const int64_t s0 = r0 >> 5;
    const int64_t nslg = (a.n + 31) >> 5;
    for (int i = tid; i <= nsl; i += BT) {
        int64_t sg = min(s0 + i, nslg);
        soa[i] = a.A.off[sg];
        sop[i] = hasP ? a.P.off[sg] : 0;
    }
    if (tid == 0) {
        sh->bid = bid; sh->G = G; sh->epoch = 0; sh->epoch2 = 0; sh->gepoch = 0; sh->ok = 1;
        sh->dmax = 0.0; sh->qprev = 0.0;
    }
    __syncthreads();
    const GridBarrier gbar{a.gcount, a.err, a.limit, (unsigned)G};
    unsigned vx = 0;  // CGS2 exchanges so far (identical in every block)

    int steps = 0, flags = 0;
    for (int it = 0; it <= a.imax; it++) {
        // ---------------- residual r = b - A x in u_r, stored in u
        double rmax = 0.0, xmax = 0.0;
        for (int64_t row = r0 + tid; row < r1; row += BT) {
            double hi = a.b[row], lo = 0.0;
            for (int64_t q = a.arp[row]; q < a.arp[row + 1]; q++) {
                double xv = (double)ldcg(&x[a.aci[q]]);
                if (RM == 2) dd_sub_prod(hi, lo, a.aval[q], xv);
                else hi = fma(-a.aval[q], xv, hi);
            }
            TU rv = (TU)(hi + lo);
            r[row] = rv;
            rmax = max_abs(rmax, (double)rv);
            xmax = max_abs(xmax, (double)x[row]);
        }
        double mx[3];
        if (!xmax3(a, sh, redd, {rmax, xmax, sh->dmax}, mx)) return;
        const double rn = mx[0], xn = mx[1], dn = mx[2];
        const double den = a.anorm * xn + a.bnorm;
        const double nb = den > 0.0 ? rn / den : 0.0;
        if (bid == 0 && tid == 0) a.nbe[it] = nb;
        if (!isfinite(nb)) { flags |= 8; break; }
        // the stopping rules (identical decisions in every block: the maxima are exchanged)
        const double q = xn > 0.0 ? dn / xn : (dn > 0.0 ? INFINITY : 0.0);
        if (a.stop_rule == IR_STOP_BACKWARD && nb <= a.stop_tol) { flags |= 1; break; }
        if (a.stop_rule == IR_STOP_CORRECTION && it >= 1 && q <= a.stop_tol) { flags |= 1; break; }
        if (it == a.imax) { flags |= 2; break; }
        if (a.stop_rule != IR_STOP_FIXED && it >= 2 && q >= 0.5 * sh->qprev) { flags |= 16; break; }
        __syncthreads();  // every thread has read sh->qprev and sh->dmax
        if (tid == 0) { sh->qprev = q; sh->dmax = 0.0; }
        // R17: GMRES takes r 2^-esc with ||r||_inf = m 2^esc, m in [0.5, 1), and the
        // correction is scaled back (half storage only)
        int esc = 0;
        if (HK && rn > 0.0) frexp(rn, &esc);

        // ---------------- z = P r (left) or r (right) in u_p, stored in u_g; beta = ||z||
        AG part = AG(0);
        if (hasP && !rightP) {
            sell_rows<TP>(r0, r1, sop, a.P.col, pv, [&](int c) { return (TP)scale2<HK>(ldcg(&r[c]), -esc); },
                          [&](int64_t row, AP v) {
                              TG z = (TG)(TP)v;
                              ws[row - r0] = z;
                              wbuf[row] = z;
                              part = fma((AG)z, (AG)z, part);
                          });
        } else {
            for (int64_t row = r0 + tid; row < r1; row += BT) {
                TG z = (TG)(TP)scale2<HK>(r[row], -esc);
                ws[row - r0] = z;
                wbuf[row] = z;
                part = fma((AG)z, (AG)z, part);
            }
        }
        AG bsq;
        if (!xsum<true>(a, sh, redg, part, bsq)) return;
        const AG beta = sqrt(bsq);
        int k = 0;
        if constexpr (LS) {
        if (beta > AG(0)) {
            // ---- GMRES with MGS in its one-reduction form (inverse compact WY, lagged
            // normalisation; Swirydowicz et al. 2020): one vector reduction per
            // iteration gives Q_j^T u_j, ||u_j||^2, Q_j^T w and u_j^T w for the not yet
            // normalised u_j and w = op(u_j); then r = ||u_j|| is h_{j,j-1}, q_j = u_j / r,
            // row j of L = (q_i^T q_k)_{i>k} is Q_j^T u_j / r, and the MGS coefficients of
            // column j are h = (I + L)^{-1} [Q_j^T w / r ; u_j^T w / r^2].  Three grid-wide
            // waits per iteration (after the first product, the reduction, and the
            // update that publishes u_{j+1}) instead of j + 3.
            //
            // The Givens rotations of column c (complete once iteration c+1 has
            // r_{c+1} = h_{c+1,c}) run on thread GT during iteration c+2's inner
            // products, which the other warps compute; the stop test follows them, so a
            // solve that converges at column c has done one more product and inner-
            // product pass than it uses.  The columns alternate between two buffers
            // (hc, and yv until the back substitution).
            const int nwp = BT >> 5, lane = tid & 31, wid = tid >> 5;
            const int64_t rbl = r1 - r0;
            // (rows in u_g; the scalars, partials and T in its arithmetic type)
            TG* wsm = ws + a.rb;                 // w for the block's rows
            AG* sred = (AG*)(wsm + a.rb);        // 2 (kmax + 1) inner products, summed over blocks
            AG* hv = sred + 2 * (kmax + 1);      // the right-hand side b, then h (kmax + 1)
            AG* lrow = hv + (kmax + 1);          // row j of L (kmax + 1)
            AG* upa = lrow + (kmax + 1);         // unit partials (kmax + 33 each)
            AG* upc = upa + (kmax + 33);
            AG* ttri = upc + (kmax + 33);        // rows 0 .. jl-1 of T = (I + L)^{-1}, packed
            AG* Tg = (AG*)a.L;                   // every row of T, packed (block 0 writes)
            AG* pv2 = (AG*)a.pvec;               // [value][block] block partials
            double* colb[2] = {hc, yv};          // column c of H (entries 0..c+1) in colb[c & 1]
            auto tri = [](int i) -> int64_t { return (int64_t)i * (i - 1) / 2; };
            // T(i, m) for m < i (row i of T, written in iteration i)
            auto tget = [&](int i, int m) -> AG { return i < a.jl ? ttri[tri(i) + m] : ldcg(&Tg[tri(i) + m]); };
            // rotations 0..c-1 and the new rotation c on column c; g, the residual estimate
            // (the entry that rotation q carries to rotation q+1 stays in a register: one
            // dependent FP64 FMA per rotation; the rotated entries go to R from block 0)
            auto givens = [&](int c) {
                const double* h = colb[c & 1];
                double x = h[0];
#pragma unroll 4
                for (int q = 0; q < c; q++) {
                    const double csq = cs[q], snq = sn[q], hq1 = h[q + 1];
                    const double out = fma(csq, x, snq * hq1);
                    x = fma(-snq, x, csq * hq1);
                    if (bid == 0 || a.sblock) a.R[(size_t)c * (kmax + 1) + q] = out;
                }
                const double hs = h[c + 1];
                const double dn = sqrt(x * x + hs * hs);
                if (dn == 0.0) { cs[c] = 1.0; sn[c] = 0.0; }
                else { cs[c] = x / dn; sn[c] = hs / dn; }
                g[c + 1] = -sn[c] * g[c];
                g[c] = cs[c] * g[c];
                sh->resid = fabs(g[c + 1]) / (double)beta;
                if (bid == 0) a.R[(size_t)c * (kmax + 1) + c] = dn;
                if (a.sblock) {
                    // the rotating block publishes: the other blocks read these after the
                    // next exchange round
                    a.R[(size_t)c * (kmax + 1) + c] = dn;
                    a.gpub[c] = g[c];
                    a.gpub[c + 1] = g[c + 1];
                    a.R[(size_t)c * (kmax + 1) + kmax] = sh->resid;
                }
            };
            // with a rotating block (sblock) only it runs the rotations, and the row blocks'
            // warp 0 joins the inner products
            const bool rotates = !a.sblock || bid == G - 1;
            if (tid == GT) g[0] = (double)beta;
            // units of the inner products: S row segments per vector, whole multiples of 32 VN
            // rows (chunks), S chosen so that the busiest of the nwu warps finishes first, a
            // unit costing its chunks plus about four chunks for its two warp reductions (at
            // most kmax + 33 units: the partials' storage).  stab[nv] for nv = 1..kmax+1
            // vectors, made once per solve (32-bit arithmetic; 64-bit division is slow here).
            int* stab = reinterpret_cast<int*>(ttri + (size_t)a.jl * (a.jl - 1) / 2);
            // partial sums of the T row's column groups (BT values)
            AG* tpart = reinterpret_cast<AG*>(((uintptr_t)(stab + kmax + 2) + 15) & ~(uintptr_t)15);
            {
                const int nwu = a.sblock ? nwp : nwp - 1;
                const int ck = 32 * VN;
                const int rows = (int)rbl;
                const int smax = rows > 0 ? (rows + ck - 1) / ck : 1;
                for (int nv = 1 + tid; nv <= kmax + 1; nv += BT) {
                    int best = INT_MAX, sb = 1;
                    for (int s2 = 1; s2 <= smax && nv * s2 <= kmax + 33; s2++) {
                        const int segc = ((rows + s2 - 1) / s2 + ck - 1) / ck;
                        const int cost = ((nv * s2 + nwu - 1) / nwu) * (segc + 4);
                        if (cost < best) { best = cost; sb = s2; }
                    }
                    stab[nv] = sb;
                }
                __syncthreads();
            }
            for (int j = 0; j <= kmax; j++) {
                const bool prod = j < kmax;
                // w = P (A u_j) (left) or A (P u_j) (right) in u_p, stored in u_g; u_j is read
                // from the published wbuf (the first u_0 is z).  (Running the second product
                // on warps 1.. beside the rotations of thread GT slowed both: the FP64
                // instructions hold up their sub-partition.)
                if (prod) {
                    if (hasP) {
                        sell_rows<TP>(r0, r1, rightP ? sop : soa, rightP ? a.P.col : a.A.col, rightP ? pv : av,
                                      [&](int c) { return (TP)ldcg(&wbuf[c]); },
                                      [&](int64_t row, AP v) { tbuf[row] = (TP)v; });
                        if (!xbar(a, sh)) return;
                        sell_rows<TP>(r0, r1, rightP ? soa : sop, rightP ? a.A.col : a.P.col, rightP ? av : pv,
                                      [&](int c) { return ldcg(&tbuf[c]); },
                                      [&](int64_t row, AP v) { wsm[row - r0] = (TG)(TP)v; });
                    } else {
                        sell_rows<TP>(r0, r1, soa, a.A.col, av, [&](int c) { return (TP)ldcg(&wbuf[c]); },
                                      [&](int64_t row, AP v) { wsm[row - r0] = (TG)(TP)v; });
                    }
                }
                __syncthreads();
                const int nv = j + 1, nwu = a.sblock ? nwp : nwp - 1;
                const int64_t chunk = 32 * VN;
                const int S = stab[nv];
                if (!a.sblock && wid == 0) {
                    if (tid == GT && j >= 2) givens(j - 2);
                } else {
                    if (tid == GT && j >= 2 && rotates) givens(j - 2);
                    // ---- block partials: units (vector i, row segment), vector j being u_j
                    // itself; a_i = q_i . u_j (a_j = ||u_j||^2), c_i = q_i . w (c_j = u_j . w).
                    // Each lane reads VN consecutive rows per 16-byte load
                    const int64_t segr = (((rbl + S - 1) / S) + chunk - 1) / chunk * chunk;
                    for (int unit = wid - (a.sblock ? 0 : 1); unit < nv * S; unit += nwu) {
                        const int i = unit / S, sg = unit - i * S;
                        const int64_t m0 = r0 + sg * segr, m1 = min(r1, m0 + segr);
                        const TG* q = V + (int64_t)i * a.ldv;
                        AG sa = AG(0), sc = AG(0);
                        if (i < j) {
                            // IQ 16-byte loads of q issued together, then consumed in row order
                            // (the sums keep the order of a row-by-row loop); rows relative to r0
                            // (the double build has 128 registers a thread, the others 72)
                            constexpr int IQ = sizeof(TG) == 8 ? (BK ? 4 : 8) : (BK ? 2 : 4);
                            constexpr int CK = 32 * VN;
                            const TG* qb = q + r0;
                            const int e0 = (int)(m0 - r0), e1 = (int)(m1 - r0);
                            for (int rq = e0 + VN * lane; rq < e1; rq += IQ * CK) {
                                TV q4[IQ];
#pragma unroll
                                for (int uu = 0; uu < IQ; uu++) {
                                    const int row = rq + uu * CK;
                                    if (row + VN <= e1) q4[uu] = __ldcg(reinterpret_cast<const TV*>(qb + row));
                                }
#pragma unroll
                                for (int uu = 0; uu < IQ; uu++) {
                                    const int row = rq + uu * CK;
                                    if (row + VN <= e1) {
                                        const TV u4 = *reinterpret_cast<const TV*>(ws + row);
                                        const TV w4 = *reinterpret_cast<const TV*>(wsm + row);
                                        TG qe[VN], ue[VN], we[VN];
                                        memcpy(qe, &q4[uu], sizeof(TV));
                                        memcpy(ue, &u4, sizeof(TV));
                                        memcpy(we, &w4, sizeof(TV));
#pragma unroll
                                        for (int e = 0; e < VN; e++) {
                                            sa = fma((AG)qe[e], (AG)ue[e], sa);
                                            sc = fma((AG)qe[e], (AG)we[e], sc);
                                        }
                                    } else if (row < e1) {
                                        for (int e = 0; e < VN && row + e < e1; e++) {
                                            const AG qv = (AG)ldcg(qb + row + e);
                                            sa = fma(qv, (AG)ws[row + e], sa);
                                            sc = fma(qv, (AG)wsm[row + e], sc);
                                        }
                                    }
                                }
                            }
                        } else {
                            for (int64_t row = m0 + VN * lane; row < m1; row += chunk) {
                                for (int e = 0; e < VN && row + e < m1; e++) {
                                    const AG uv = (AG)ws[row + e - r0];
                                    sa = fma(uv, uv, sa);
                                    sc = fma(uv, (AG)wsm[row + e - r0], sc);
                                }
                            }
                        }
                        sa = warp_sum(sa);
                        sc = warp_sum(sc);
                        if (lane == 0) { upa[unit] = sa; upc[unit] = sc; }
                    }
                }
                __syncthreads();
                // column j-2 converged: k = j-1 columns (this iteration's products are unused);
                // with a rotating block the estimate is read after the exchange round below
                if (!a.sblock && j >= 2 && sh->resid <= a.tau) { k = j - 1; break; }
                for (int v = tid; v < 2 * nv; v += BT) {
                    const AG* src = v < nv ? upa : upc;
                    const int i = v < nv ? v : v - nv;
                    AG acc = AG(0);
                    for (int sg = 0; sg < S; sg++) acc += src[i * S + sg];
                    pv2[(size_t)v * G + bid] = acc;
                }
                // ---- the reduction over blocks (the partials published by an exchange round)
                if (!xbar(a, sh)) return;
                if (a.sblock && j >= 2 && __ldcg(&a.R[(size_t)(j - 2) * (kmax + 1) + kmax]) <= a.tau) {
                    k = j - 1;
                    break;
                }
                // the sums over blocks of the 2 nv partials, each in the same order (lanes over
                // blocks, then the warp's tree): every block sums them all, or, when that
                // would read many partials (2 nv G >= IR_DIST_MIN), block b sums the values
                // b, b + G, ... and publishes them for one more exchange round
                if (2 * nv * G < IR_DIST_MIN) {
                    for (int v0 = wid; v0 < 2 * nv; v0 += 2 * nwp) {
                        const int v1 = v0 + nwp;
                        const bool two = v1 < 2 * nv;
                        // every block's partial loaded first (all loads in flight), then summed
                        // in block order
                        AG x0[SPL], x1[SPL];
#pragma unroll
                        for (int q = 0; q < SPL; q++) {
                            const int b = lane + 32 * q;
                            x0[q] = b < G ? ldcg(&pv2[(size_t)v0 * G + b]) : AG(0);
                            x1[q] = (two && b < G) ? ldcg(&pv2[(size_t)v1 * G + b]) : AG(0);
                        }
                        AG acc0 = AG(0), acc1 = AG(0);
#pragma unroll
                        for (int q = 0; q < SPL; q++) {
                            if (lane + 32 * q < G) {
                                acc0 += x0[q];
                                acc1 += x1[q];
                            }
                        }
                        acc0 = warp_sum(acc0);
                        acc1 = warp_sum(acc1);
                        if (lane == 0) {
                            sred[v0] = acc0;
                            if (two) sred[v1] = acc1;
                        }
                    }
                    __syncthreads();
                } else {
                    AG* tot = (AG*)a.pvec + (size_t)2 * MAX_GRID * (kmax + 1);
                    for (int t = wid; bid + t * G < 2 * nv; t += nwp) {
                        const int v0 = bid + t * G;
                        AG x0[SPL];
#pragma unroll
                        for (int q = 0; q < SPL; q++) {
                            const int b = lane + 32 * q;
                            x0[q] = b < G ? ldcg(&pv2[(size_t)v0 * G + b]) : AG(0);
                        }
                        AG acc0 = AG(0);
#pragma unroll
                        for (int q = 0; q < SPL; q++)
                            if (lane + 32 * q < G) acc0 += x0[q];
                        acc0 = warp_sum(acc0);
                        if (lane == 0) tot[v0] = acc0;
                    }
                    if (!xbar(a, sh)) return;
                    for (int v = tid; v < 2 * nv; v += BT) sred[v] = ldcg(&tot[v]);
                    __syncthreads();
                }
                const AG rr = j == 0 ? beta : sqrt(sred[j]);
                if (j >= 1 && tid == GT) colb[(j - 1) & 1][j] = (double)rr;  // h_{j,j-1}
                if (j >= 1 && (rr == AG(0) || !prod)) {
                    // breakdown or the iteration cap: column j-1 is the last one
                    if (tid == GT && rotates) givens(j - 1);
                    __syncthreads();
                    k = j;
                    if (rr == AG(0)) flags |= 4;
                    break;
                }
                if (!prod) break;  // kmax = 0
                // ---- row j of L and b = [c / r ; (u_j . w / r) / r]; h = (I + L)^{-1} b, the same
                // in every block.  T = (I + L)^{-1} grows by one row per iteration, t_j =
                // -l_j^T T (row j of (I + L) T = I), so h = T b is a matrix-vector product (one
                // warp per entry) instead of a forward substitution; both give MGS's
                // coefficients.  trow = t_j, hout = h (the unit partials' storage, free here).
                AG* trow = upa;
                AG* hout = upc;
                for (int i = tid; i < j; i += BT) {
                    lrow[i] = sred[i] / rr;
                    hv[i] = sred[nv + i] / rr;
                }
                if (tid == 0) hv[j] = (sred[2 * nv - 1] / rr) / rr;
                __syncthreads();
                // t_{j,m} = -(l_{j,m} + sum_{m < k < j} l_{j,k} T(k, m)) (T(m, m) = 1), column by
                // column: thread m of group g sums the rows k of the g-th chunk of (m, j), so the
                // reads T(k, m) of one row k are consecutive over the threads (coalesced from
                // global memory, where rows jl.. live), UQ of them in flight per thread; the
                // groups' partials are added in group order.  Beside it, h_i = b_i + sum_{m < i}
                // T(i, m) b_m for i < j, a warp per row (lanes over m, four loads in flight).
                if (j > 0) {
                    const int JP = (j + 31) & ~31;
                    const int NG = JP <= BT ? min(BT / JP, 8) : 1;
                    const int kc = (j + NG - 1) / NG;
                    constexpr int UQ = 8;
                    for (int t = tid; t < (JP <= BT ? NG * JP : j); t += BT) {
                        const int m = JP <= BT ? t % JP : t;
                        const int g = JP <= BT ? t / JP : 0;
                        AG acc = AG(0);
                        if (m < j) {
                            const int kb = max(m + 1, g * kc), ke = min(j, (g + 1) * kc);
                            int k = kb;
                            for (; k + UQ <= ke; k += UQ) {
                                AG tv[UQ];
#pragma unroll
                                for (int u = 0; u < UQ; u++) tv[u] = tget(k + u, m);
#pragma unroll
                                for (int u = 0; u < UQ; u++) acc = fma(lrow[k + u], tv[u], acc);
                            }
                            for (; k < ke; k++) acc = fma(lrow[k], tget(k, m), acc);
                        }
                        if (JP <= BT) tpart[t] = acc;
                        else trow[m] = -(lrow[m] + acc);
                    }
                    for (int i = wid; i < j; i += nwp) {
                        AG acc = AG(0);
                        int m = lane;
                        for (; m + 96 < i; m += 128) {
                            const AG t0 = tget(i, m), t1 = tget(i, m + 32), t2 = tget(i, m + 64), t3 = tget(i, m + 96);
                            acc = fma(t0, hv[m], acc);
                            acc = fma(t1, hv[m + 32], acc);
                            acc = fma(t2, hv[m + 64], acc);
                            acc = fma(t3, hv[m + 96], acc);
                        }
                        for (; m < i; m += 32) acc = fma(tget(i, m), hv[m], acc);
                        acc = warp_sum(acc);
                        if (lane == 0) hout[i] = hv[i] + acc;
                    }
                    __syncthreads();
                    if (JP <= BT) {
                        for (int m = tid; m < j; m += BT) {
                            AG acc = AG(0);
                            for (int g = 0; g < NG; g++) acc += tpart[g * JP + m];
                            trow[m] = -(lrow[m] + acc);
                        }
                        __syncthreads();
                    }
                    for (int m = tid; m < j; m += BT) {
                        if (j < a.jl) ttri[tri(j) + m] = trow[m];
                        if (bid == 0) Tg[tri(j) + m] = trow[m];
                    }
                }
                if (wid == 0) {
                    AG acc = AG(0);
                    for (int m = lane; m < j; m += 32) acc = fma(trow[m], hv[m], acc);
                    acc = warp_sum(acc);
                    if (lane == 0) hout[j] = hv[j] + acc;
                }
                __syncthreads();
                {
                    double* hj = colb[j & 1];
                    for (int i = tid; i <= j; i += BT) hj[i] = (double)hout[i];
                }
                // ---- q_j = u_j / r into V, and u_{j+1} = w / r - Q_{j+1} h (the block's rows,
                // published for the next product)
                // (a thread's two rows share the loop over the basis: twice the loads in flight)
                TG* Vj = V + (int64_t)j * a.ldv;
                for (int64_t ra = r0 + tid; ra < r1; ra += 2 * BT) {
                    const int64_t rb2 = ra + BT;
                    const bool hb = rb2 < r1;
                    // q_j as stored (in u_g) is the vector the update subtracts
                    const TG qsa = (TG)((AG)ws[ra - r0] / rr);
                    const TG qsb = hb ? (TG)((AG)ws[rb2 - r0] / rr) : TG(0);
                    Vj[ra] = qsa;
                    if (hb) Vj[rb2] = qsb;
                    const AG qa = (AG)qsa, qb = (AG)qsb;
                    AG acca = (AG)wsm[ra - r0] / rr;
                    AG accb = hb ? (AG)wsm[rb2 - r0] / rr : AG(0);
                    const int64_t rbx = hb ? rb2 : ra;  // an in-range row for the second load
                    // (16 basis vectors unrolled: 32 loads of the two rows in flight)
#pragma unroll 16
                    for (int i = 0; i < j; i++) {
                        const TG* Vi = V + (int64_t)i * a.ldv;
                        const AG h = hout[i];
                        acca = fma(-h, (AG)ldcg(Vi + ra), acca);
                        accb = fma(-h, (AG)ldcg(Vi + rbx), accb);
                    }
                    acca = fma(-hout[j], qa, acca);
                    ws[ra - r0] = (TG)acca;
                    wbuf[ra] = (TG)acca;
                    if (hb) {
                        accb = fma(-hout[j], qb, accb);
                        ws[rb2 - r0] = (TG)accb;
                        wbuf[rb2] = (TG)accb;
                    }
                }
                if (!xbar(a, sh)) return;
            }
        }
        } else {
        if (beta > TG(0)) {
            for (int64_t row = r0 + tid; row < r1; row += BT) V[row] = ws[row - r0] / beta;
            if (tid == GT) g[0] = (double)beta;
            TG hdiv = beta;
            bool done = false;
            for (int j = 0; j < kmax && !done; j++) {
                // ---- t = A v_j (left) or P v_j (right) in u_p; v_j formed from the
                // published w: fl(w / h)
                sell_rows<TP>(r0, r1, rightP ? sop : soa, rightP ? a.P.col : a.A.col, rightP ? pv : av,
                              [&](int c) { return (TP)(ldcg(&wbuf[c]) / hdiv); },
                              [&](int64_t row, TP v) { tbuf[row] = v; });
                // prefetch v_0 for the first Gram-Schmidt dot while the barrier runs
                // (with a group the range holds other blocks' rows of v_0, which are
                // published by this barrier when j = 0: the load waits for it)
                TG vc[PF];
                if (!sub) vload(V, vc);
                if (!xbar(a, sh)) return;
                if (sub) vload(V, vc);
                // ---- w = P t (left) or A t (right) in u_p, stored in u_g (own rows, shared
                // memory); first MGS partial
                part = TG(0);
                if (sub) {
                    // publish w = P t; the group's blocks then read their double range
                    if (hasP) {
                        sell_rows<TP>(r0, r1, rightP ? soa : sop, rightP ? a.A.col : a.P.col, rightP ? av : pv,
                                      [&](int c) { return ldcg(&tbuf[c]); },
                                      [&](int64_t row, TP v) { wbuf[row] = (TG)v; });
                    } else {
                        for (int64_t row = r0 + tid; row < r1; row += BT) wbuf[row] = (TG)ldcg(&tbuf[row]);
                    }
                    if (!xbar(a, sh)) return;
#pragma unroll
                    for (int u = 0; u < UV; u++) {
                        const int64_t s0 = vrow(u);
                        if (s0 + VN <= m1) {
                            *reinterpret_cast<TV*>(ws + (s0 - m0)) = __ldcg(reinterpret_cast<const TV*>(wbuf + s0));
                        } else {
#pragma unroll
                            for (int e = 0; e < VN; e++)
                                if (s0 + e < m1) ws[s0 + e - m0] = ldcg(&wbuf[s0 + e]);
                        }
                    }
                    for (int64_t row = m0 + (int64_t)PF * BT + tid; row < m1; row += BT) ws[row - m0] = ldcg(&wbuf[row]);
                } else if (hasP) {
                    sell_rows<TP>(r0, r1, rightP ? soa : sop, rightP ? a.A.col : a.P.col, rightP ? av : pv,
                                  [&](int c) { return ldcg(&tbuf[c]); },
                                  [&](int64_t row, TP v) { ws[row - r0] = (TG)v; });
                } else {
                    for (int64_t row = r0 + tid; row < r1; row += BT) ws[row - r0] = (TG)ldcg(&tbuf[row]);
                }
                if (a.orth) {
                    // ---- classical Gram-Schmidt applied twice in u_g: each pass forms all
                    // j+1 projections of the same w (one vector exchange), then subtracts them
                    TG* cvec = reinterpret_cast<TG*>(yv);  // free until the back substitution
                    const int lane = tid & 31, wid = tid >> 5, nwp = BT >> 5;
                    __syncthreads();
                    for (int pass = 0; pass < 2; pass++) {
                        TG* pbase = (TG*)a.pvec + (size_t)(vx & 1u) * G * (kmax + 1);
                        for (int i = wid; i <= j; i += nwp) {
                            const TG* Vi = V + (int64_t)i * a.ldv;
                            TG acc = TG(0);
                            for (int64_t row = r0 + lane; row < r1; row += 32) acc = fma(Vi[row], ws[row - r0], acc);
                            acc = warp_sum(acc);
                            if (lane == 0) pbase[(size_t)bid * (kmax + 1) + i] = acc;
                        }
                        if (!grid_sync(gbar, &sh->gepoch, &sh->ok)) return;
                        for (int i = wid; i <= j; i += nwp) {
                            TG acc = TG(0);
                            for (unsigned b = lane; b < G; b += 32) acc += ldcg(&pbase[(size_t)b * (kmax + 1) + i]);
                            acc = warp_sum(acc);
                            if (lane == 0) cvec[i] = acc;
                        }
                        vx++;
                        __syncthreads();
                        if (tid == GT)
                            for (int i = 0; i <= j; i++) hc[i] = pass == 0 ? (double)cvec[i] : (double)((TG)hc[i] + cvec[i]);
                        for (int64_t row = r0 + tid; row < r1; row += BT) {
                            TG acc = ws[row - r0];
                            for (int i = 0; i <= j; i++) acc = fma(-cvec[i], V[(int64_t)i * a.ldv + row], acc);
                            ws[row - r0] = acc;
                        }
                        __syncthreads();
                    }
                    part = TG(0);
                    for (int64_t row = r0 + tid; row < r1; row += BT) {
                        const TG wv = ws[row - r0];
                        wbuf[row] = wv;
                        part = fma(wv, wv, part);
                    }
                    if (tid == GT) {
                        // rotations 0..j-1 on the new column
                        for (int q = 0; q < j; q++) {
                            const double t0 = cs[q] * hc[q] + sn[q] * hc[q + 1];
                            hc[q + 1] = -sn[q] * hc[q] + cs[q] * hc[q + 1];
                            hc[q] = t0;
                            if (bid == 0) a.R[(size_t)j * (kmax + 1) + q] = hc[q];
                        }
                    }
                } else {
                // the group's load gives each thread its Gram-Schmidt rows; without a
                // group sell_rows wrote w in its own row order.  Basis entries are read
                // through L2 (ld.cg): with a group they include rows that other blocks
                // wrote
                if (!sub) __syncthreads();
#pragma unroll
                for (int u = 0; u < UV; u++) {
                    const int64_t s0 = vrow(u);
#pragma unroll
                    for (int e = 0; e < VN; e++)
                        if (s0 + e < m1) part = fma(vc[u * VN + e], ws[s0 + e - m0], part);
                }
                for (int64_t row = m0 + (int64_t)PF * BT + tid; row < m1; row += BT) part = fma(ldcg(&V[row]), ws[row - m0], part);
                // ---- modified Gram-Schmidt in u_g (blocks outside the group skip it)
                for (int i = 0; i <= j && gs; i++) {
                    // prefetch v_{i+1} (rows [m0, m1)) before waiting for h_{i,j}
                    const TG* Vn = V + (int64_t)(i + 1) * a.ldv;
                    TG vn[PF];
                    if (i < j) vload(Vn, vn);
                    TG h;
                    // Givens, pipelined with the rounds: rotation q needs h_{q+1}, known
                    // after round q+1; thread 0 applies it during round q+2, between
                    // publishing and polling
                    const int pq = i - 2;
                    auto rot = [&]() {
                        if (pq >= 0) {
                            const double t0 = cs[pq] * hc[pq] + sn[pq] * hc[pq + 1];
                            hc[pq + 1] = -sn[pq] * hc[pq] + cs[pq] * hc[pq + 1];
                            hc[pq] = t0;
                            if (bid == 0) a.R[(size_t)j * (kmax + 1) + pq] = hc[pq];
                        }
                    };
                    if (sub ? !xsum<false, TG, true>(a, sh, redg, part, h, rot)
                            : !xsum<false, TG, false>(a, sh, redg, part, h, rot))
                        return;
                    if (tid == GT) hc[i] = (double)h;
                    const TG* Vi = V + (int64_t)i * a.ldv;
                    part = TG(0);
                    if (i < j) {
#pragma unroll
                        for (int u = 0; u < UV; u++) {
                            const int64_t s0 = vrow(u);
                            TG* wp = ws + (s0 - m0);
                            if (s0 + VN <= m1) {
                                TV t = *reinterpret_cast<const TV*>(wp);
                                TG wv[VN];
                                memcpy(wv, &t, sizeof(TV));
#pragma unroll
                                for (int e = 0; e < VN; e++) {
                                    wv[e] = fma(-h, vc[u * VN + e], wv[e]);
                                    part = fma(vn[u * VN + e], wv[e], part);
                                }
                                memcpy(&t, wv, sizeof(TV));
                                *reinterpret_cast<TV*>(wp) = t;
                            } else {
#pragma unroll
                                for (int e = 0; e < VN; e++)
                                    if (s0 + e < m1) {
                                        const TG wv = fma(-h, vc[u * VN + e], wp[e]);
                                        wp[e] = wv;
                                        part = fma(vn[u * VN + e], wv, part);
                                    }
                            }
                        }
#pragma unroll
                        for (int e = 0; e < PF; e++) vc[e] = vn[e];
                        for (int64_t row = m0 + (int64_t)PF * BT + tid; row < m1; row += BT) {
                            TG wv = fma(-h, ldcg(&Vi[row]), ws[row - m0]);
                            ws[row - m0] = wv;
                            part = fma(ldcg(&Vn[row]), wv, part);
                        }
                    } else {
#pragma unroll
                        for (int u = 0; u < UV; u++) {
                            const int64_t s0 = vrow(u);
                            TG* wp = ws + (s0 - m0);
                            if (s0 + VN <= m1) {
                                TV t = *reinterpret_cast<const TV*>(wp);
                                TG wv[VN];
                                memcpy(wv, &t, sizeof(TV));
#pragma unroll
                                for (int e = 0; e < VN; e++) {
                                    wv[e] = fma(-h, vc[u * VN + e], wv[e]);
                                    part = fma(wv[e], wv[e], part);
                                }
                                memcpy(&t, wv, sizeof(TV));
                                *reinterpret_cast<TV*>(wp) = t;
                                *reinterpret_cast<TV*>(wbuf + s0) = t;
                            } else {
#pragma unroll
                                for (int e = 0; e < VN; e++)
                                    if (s0 + e < m1) {
                                        const TG wv = fma(-h, vc[u * VN + e], wp[e]);
                                        wp[e] = wv;
                                        wbuf[s0 + e] = wv;
                                        part = fma(wv, wv, part);
                                    }
                            }
                        }
                        for (int64_t row = m0 + (int64_t)PF * BT + tid; row < m1; row += BT) {
                            TG wv = fma(-h, ldcg(&Vi[row]), ws[row - m0]);
                            ws[row - m0] = wv;
                            wbuf[row] = wv;
                            part = fma(wv, wv, part);
                        }
                    }
                }
                }
                // the last rotation of the rounds, j-1 (the CGS2 branch applied all)
                if (!a.orth && gs && tid == GT && j >= 1) {
                    const int q = j - 1;
                    const double t0 = cs[q] * hc[q] + sn[q] * hc[q + 1];
                    hc[q + 1] = -sn[q] * hc[q] + cs[q] * hc[q + 1];
                    hc[q] = t0;
                    if (bid == 0) a.R[(size_t)j * (kmax + 1) + q] = hc[q];
                }
                // outside the group part is 0; block 0 stores the rotated diagonal
                // entry h_jj (rotations 0..j-1 applied) in the unused last row of R's
                // column j for the blocks outside the group
                if (!gs) part = TG(0);
                if (sub && !a.orth && bid == 0 && tid == GT) a.R[(size_t)j * (kmax + 1) + kmax] = hc[j];
                TG hsq;
                if (!xsum<true>(a, sh, redg, part, hsq)) return;
                const TG hn = sqrt(hsq);
                if (sub && !a.orth && !gs && tid == GT) hc[j] = __ldcg(&a.R[(size_t)j * (kmax + 1) + kmax]);
                // ---- v_{j+1} = w / h_{j+1,j} (own rows; with a group from the published w)
                if (hn > TG(0)) {
                    TG* Vn = V + (int64_t)(j + 1) * a.ldv;
                    if (sub) {
                        for (int64_t row = r0 + tid; row < r1; row += BT) Vn[row] = ldcg(&wbuf[row]) / hn;
                    } else {
                        for (int64_t row = r0 + tid; row < r1; row += BT) Vn[row] = ws[row - r0] / hn;
                    }
                }
                // ---- the new Givens rotation in double (identical in every block);
                // rotations 0..j-1 were applied to this column during the rounds
                if (tid == GT) {
                    hc[j + 1] = (double)hn;
                    double dn = sqrt(hc[j] * hc[j] + hc[j + 1] * hc[j + 1]);
                    if (dn == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
                    else { cs[j] = hc[j] / dn; sn[j] = hc[j + 1] / dn; }
                    hc[j] = dn;
                    g[j + 1] = -sn[j] * g[j];
                    g[j] = cs[j] * g[j];
                    sh->resid = fabs(g[j + 1]) / (double)beta;
                    if (bid == 0) a.R[(size_t)j * (kmax + 1) + j] = hc[j];
                }
                __syncthreads();
                k = j + 1;
                hdiv = hn;
                if (hn == TG(0)) { flags |= 4; done = true; }
                else if (sh->resid <= a.tau) done = true;
            }
        }
        }
        if (beta > AG(0)) {
            // ---- y = R^{-1} g (double), d = V y in u_g, x = x + d in u
            if (!xbar(a, sh)) return;  // R columns from block 0 (or the rotating block)
            if (LS && a.sblock)
                for (int t = tid; t <= k; t += BT) g[t] = __ldcg(&a.gpub[t]);
            __syncthreads();
            if (tid < 32) {
                for (int t = tid; t < k; t += 32) yv[t] = g[t];
                __syncwarp();
                for (int c = k - 1; c >= 0; c--) {
                    if (tid == 0) {
                        double rcc = __ldcg(&a.R[(size_t)c * (kmax + 1) + c]);
                        yv[c] = rcc != 0.0 ? yv[c] / rcc : 0.0;
                    }
                    __syncwarp();
                    double yc = yv[c];
                    for (int t = tid; t < c; t += 32) yv[t] -= __ldcg(&a.R[(size_t)c * (kmax + 1) + t]) * yc;
                    __syncwarp();
                }
            }
            __syncthreads();
            double dmax = 0.0;  // this thread's largest |d| (as added to x, in u)
            if (rightP) {
                // right preconditioning: d = P (V_k y), the product in u_p stored in u_g
                for (int64_t row = r0 + tid; row < r1; row += BT) {
                    AG dsum = AG(0);
                    for (int i = 0; i < k; i++) dsum = fma((AG)V[(int64_t)i * a.ldv + row], (AG)yv[i], dsum);
                    wbuf[row] = (TG)dsum;
                }
                if (!xbar(a, sh)) return;
                sell_rows<TP>(r0, r1, sop, a.P.col, pv, [&](int c) { return (TP)ldcg(&wbuf[c]); },
                              [&](int64_t row, AP v) {
                                  const TU du = scale2<HK>((TU)(TG)(TP)v, esc);
                                  dmax = max_abs(dmax, (double)du);
                                  x[row] = (TU)((TU)x[row] + du);
                              });
            } else {
                for (int64_t row = r0 + tid; row < r1; row += BT) {
                    AG dsum = AG(0);
                    for (int i = 0; i < k; i++) dsum = fma((AG)V[(int64_t)i * a.ldv + row], (AG)yv[i], dsum);
                    const TU du = scale2<HK>((TU)dsum, esc);
                    dmax = max_abs(dmax, (double)du);
                    x[row] = (TU)((TU)x[row] + du);
                }
            }
            dmax = block_max(dmax, redd);
            if (tid == 0) sh->dmax = dmax;
        }
        if (bid == 0 && tid == 0) a.its[it] = k;
        steps = it + 1;
        // x must be complete before the next residual
        if (!xbar(a, sh)) return;
    }
    if (bid == 0 && tid == 0) {
        a.out[0] = steps;
        a.out[1] = flags;
    }
}

template <class TU, class TG, class TP, int RM, bool LS>
__global__ void __launch_bounds__(ir_threads<TG, TP>(), 1) k_ir(IrArgs a)
{
    ir_body<TU, TG, TP, RM, LS>(a, (int)blockIdx.x, (int)gridDim.x);
}

// Many systems in one cooperative launch (gmres_ir_solve_batch).  The grid
// is cut into teams of contiguous blocks; teams of one class have the same
// size and solve the systems of that class (args[cs[c] .. cs[c+1]), each
// prepared for that team size), one after another, taking the next from the
// class's counter as soon as they are done, so a system with many iterations
// holds only its own team's SMs.  Classes are in decreasing team size; a
// team whose class has no system left takes one of a later class (smaller
// teams), which its first a.G blocks solve exactly as a team of that size
// would.  Team j: blocks tb[j] .. tb[j+1]-1, class tc[j].  Waits are bounded
// like every other wait of the refinement: a team that gives up leaves.
struct BatchPlan {
    const int* tb;   // nteams + 1 first blocks
    const int* tc;   // nteams classes
    const int* cs;   // nclasses + 1 offsets into args
    int nteams, ncls;
};

template <class TU, class TG, class TP, int RM, bool LS>
__global__ void __launch_bounds__(ir_threads<TG, TP>(), 1) k_ir_batch(const IrArgs* __restrict__ args, BatchPlan plan,
                                                                     unsigned* next, unsigned long long* claim,
                                                                     long long limit)
{
    __shared__ int s_sys, s_team;
    if (threadIdx.x == 0) {
        // this block's team: the last j with tb[j] <= blockIdx.x
        int lo = 0, hi = plan.nteams - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (plan.tb[mid] <= (int)blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        s_team = lo;
    }
    __syncthreads();
    const int team = s_team;
    const int rank = (int)blockIdx.x - plan.tb[team];
    const int c = plan.tc[team];
    for (unsigned round = 1;; round++) {
        if (threadIdx.x == 0) {
            int sys = -1;
            if (rank == 0) {
                for (int cc = c; cc < plan.ncls && sys < 0; cc++) {
                    const int q = (int)atomicAdd(&next[cc], 1u);
                    if (q < plan.cs[cc + 1] - plan.cs[cc]) sys = plan.cs[cc] + q;
                }
                st_relaxed_u64(&claim[team], ((unsigned long long)round << 32) | (unsigned)sys);
            } else {
                const long long t0 = clock64();
                for (;;) {
                    const unsigned long long w = ld_relaxed_u64(&claim[team]);
                    if ((unsigned)(w >> 32) == round) { sys = (int)(unsigned)w; break; }
                    if (clock64() - t0 > limit) break;  // the leader is gone: leave
                }
            }
            s_sys = sys;
        }
        __syncthreads();
        const int sys = s_sys;
        __syncthreads();
        if (sys < 0) return;
        const int G = args[sys].G;  // T, or a smaller class's team size
        if (rank < G) ir_body<TU, TG, TP, RM, LS, true>(args[sys], rank, G);
        __syncthreads();
    }
}

// The kernels of one precision tuple, for run-time dispatch: `one` is
// k_ir, `batch` k_ir_batch, `threads` their block size.
struct IrKernels {
    const void* one = nullptr;
    const void* batch = nullptr;
    int threads = 0;
};

template <class TU, class TG, class TP, int RM, bool LS>
void ir_kernels_set(IrKernels* k)
{
    k->one = (const void*)k_ir<TU, TG, TP, RM, LS>;
    k->batch = (const void*)k_ir_batch<TU, TG, TP, RM, LS>;
    k->threads = ir_threads<TG, TP>();
}

template <class TU, class TG, class TP>
void ir_kernels_t(int rm, bool ls, IrKernels* k)
{
    if (rm == 2) {
        if (ls) ir_kernels_set<TU, TG, TP, 2, true>(k);
        else ir_kernels_set<TU, TG, TP, 2, false>(k);
    } else {
        if (ls) ir_kernels_set<TU, TG, TP, 1, true>(k);
        else ir_kernels_set<TU, TG, TP, 1, false>(k);
    }
}

// Half Krylov storage (u_g or u_p = half): the one-reduction MGS only; the
// other forms are not instantiated (k->one stays null).
template <class TU, class TG, class TP>
void ir_kernels_ls(int rm, bool ls, IrKernels* k)
{
    if (!ls) return;
    if (rm == 2) ir_kernels_set<TU, TG, TP, 2, true>(k);
    else ir_kernels_set<TU, TG, TP, 1, true>(k);
}

// defined one per (u, u_g, u_p) in gmres_ir_k_<u><u_g><u_p>.cu (f single, d double)
void ir_kernels_fff(int rm, bool ls, IrKernels* k);
void ir_kernels_ffd(int rm, bool ls, IrKernels* k);
void ir_kernels_fdf(int rm, bool ls, IrKernels* k);
void ir_kernels_fdd(int rm, bool ls, IrKernels* k);
void ir_kernels_dff(int rm, bool ls, IrKernels* k);
void ir_kernels_dfd(int rm, bool ls, IrKernels* k);
void ir_kernels_ddf(int rm, bool ls, IrKernels* k);
void ir_kernels_ddd(int rm, bool ls, IrKernels* k);
// half (h) u_g and/or u_p: gmres_ir_k_x<u_g><u_p>.cu, both u in one unit
void ir_kernels_fhh(int rm, bool ls, IrKernels* k);
void ir_kernels_dhh(int rm, bool ls, IrKernels* k);
void ir_kernels_fhf(int rm, bool ls, IrKernels* k);
void ir_kernels_dhf(int rm, bool ls, IrKernels* k);
void ir_kernels_ffh(int rm, bool ls, IrKernels* k);
void ir_kernels_dfh(int rm, bool ls, IrKernels* k);

}  // namespace spai
