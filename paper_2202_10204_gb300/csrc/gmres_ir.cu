// SPAI-GMRES-IR on the GPU: Algorithm 3 of the paper.
//
//   x0 = P b in u_f, stored in u                     (k_x0)
//   for i = 0 .. i_max-1:
//       r_i = b - A x_i in u_r, stored in u          (residual phase)
//       solve P A d_i = P r_i by left-preconditioned
//       MGS-GMRES in u_g, products with A, P in u_p  (Arnoldi phases)
//       x_{i+1} = x_i + d_i in u                      (update phase)
//
// The whole refinement loop is ONE persistent cooperative kernel (k_ir):
// each block owns a contiguous slice of rows, keeps its slice of the
// Arnoldi vector w in shared memory, and meets the other blocks only at
// bounded grid barriers (common.cuh).  Every grid-wide dot product is a
// fixed-order tree: block partials are written to a slot, and after the
// barrier every block sums the slots in the same order, so all blocks hold
// bit-identical scalars and take identical control-flow decisions (GMRES
// convergence, refinement stop) without another barrier.  The Givens
// rotations, H, g and y are double precision in every block.
//
// Per Arnoldi iteration j: barrier after t = A v_j, j+1 barriers for the
// MGS dots, one for ||w||.  v_{j+1} = w / h_{j+1,j} is never re-published:
// readers form fl(w_c / h) from the published w themselves, which is the
// same correctly rounded quotient the owner stores into V.
#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>
#include <vector>

#include "common.cuh"
#include "internal.h"

using namespace spai;

namespace {

constexpr int IR_THREADS = 1024;
constexpr int KMAX_LIMIT = 1024;
constexpr int MAX_GRID = 160;   // exchange slots are polled by one warp, SPL slots per lane
constexpr int SPL = (MAX_GRID + 31) / 32;
constexpr int SLOT_WORDS = 16;  // one 128-byte line per block and parity (up to 4 words used)
constexpr int PF = 4;           // rows per thread whose next basis entries are prefetched
constexpr int MGS_GROUP_MIN_GRID = 64;  // grids from this size run the Gram-Schmidt rounds in a group

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
    void* pvec;                 // CGS2: 2 parities x gridDim.x x (kmax + 1) partial dot products (u_g)
    unsigned* gcount;           // CGS2: counter of the barrier that publishes them (zeroed)
};

struct IrShared {
    int bid;          // the block's rank within its system
    int G;            // the system's block count
    unsigned epoch;
    unsigned epoch2;  // rounds of the Gram-Schmidt group
    unsigned gepoch;  // CGS2 barrier count
    int ok;
    double bcast[3];
    double resid;
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
__device__ bool xsum(const IrArgs& a, IrShared* sh, T* red, T v, T& out, const Work& work = Work())
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
__device__ bool xmax3(const IrArgs& a, IrShared* sh, double* red, const double (&v)[3], double (&o)[3])
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
__device__ bool xbar(const IrArgs& a, IrShared* sh)
{
    __syncthreads();
    uint32_t pay[1] = {0u};
    NoAcc acc;
    return exchange<1, true>(a, sh, pay, acc);
}

// y = M x for the block's rows (SELL-32), two rows per thread per pass with
// their loads interleaved; `store(row, value)` receives each result.  The
// slice offsets of the block live in shared memory (soff[0..nsl]).
template <class TP, class Load, class Store>
__device__ __forceinline__ void sell_rows(int64_t r0, int64_t r1, const int64_t* soff, const int32_t* __restrict__ col,
                                          const TP* __restrict__ val, Load load, Store store)
{
    const int tid = threadIdx.x, BT = blockDim.x, lane = tid & 31;
    constexpr int U = 4;
    for (int64_t base = r0; base < r1; base += 2 * BT) {
        const int64_t ra = base + tid, rb = base + BT + tid;
        const bool va = ra < r1, vb = rb < r1;
        const int sa = (int)((ra - r0) >> 5), sb = (int)((rb - r0) >> 5);
        const int64_t oa = va ? soff[sa] + lane : 0, ob = vb ? soff[sb] + lane : 0;
        const int wa = va ? (int)((soff[sa + 1] - soff[sa]) >> 5) : 0;
        const int wb = vb ? (int)((soff[sb + 1] - soff[sb]) >> 5) : 0;
        TP acc_a = TP(0), acc_b = TP(0);
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
            TP ga[U], gb[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                ga[u] = ca[u] >= 0 ? (TP)load(ca[u]) : TP(0);
                gb[u] = cb[u] >= 0 ? (TP)load(cb[u]) : TP(0);
            }
            TP ya[U], yb[U];
#pragma unroll
            for (int u = 0; u < U; u++) { ya[u] = xa[u]; yb[u] = xb[u]; }
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

// Threads per block of the refinement kernel: 1024 when the basis and the
// preconditioner products are single precision; 512 when either is double,
// because the 1024-thread build of those spills registers (64 per thread),
// which puts the basis prefetch behind HBM latency every Gram-Schmidt round.
template <class TG, class TP>
constexpr int ir_threads()
{
    return (sizeof(TG) == 8 || sizeof(TP) == 8) ? IR_THREADS / 2 : IR_THREADS;
}

// The refinement of one system by its G blocks; `bid` is this block's rank.
template <class TU, class TG, class TP, int RM>
__device__ __forceinline__ void ir_body(const IrArgs& a, const int bid, const int G)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ IrShared shs;
    __shared__ TG redg[33];
    __shared__ double redd[96];
    IrShared* sh = &shs;
    const int kmax = a.kmax;
    const int tid = threadIdx.x, BT = blockDim.x;
    // the Givens thread: thread 0, which also publishes the block's words, so that
    // the rotations of the Gram-Schmidt rounds run while its warp waits for the
    // other blocks
    const int GT = 0;
    const int64_t r0 = (int64_t)bid * a.rb;
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
    typedef typename std::conditional<sizeof(TG) == 4, float4, double2>::type TV;
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
    if (tid == 0) { sh->bid = bid; sh->G = G; sh->epoch = 0; sh->epoch2 = 0; sh->gepoch = 0; sh->ok = 1; }
    __syncthreads();
    const GridBarrier gbar{a.gcount, a.err, a.limit, (unsigned)G};
    unsigned vx = 0;  // CGS2 exchanges so far (identical in every block)

    int steps = 0, flags = 0;
    double dmax = 0.0;   // this thread's largest |d| of the last correction (as added to x, in u)
    double qprev = 0.0;  // ||d_{i-2}|| / ||x_{i-1}|| (the stagnation test)
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
            rmax = fmax(rmax, fabs((double)rv));
            xmax = fmax(xmax, fabs((double)x[row]));
        }
        double mx[3];
        if (!xmax3(a, sh, redd, {rmax, xmax, dmax}, mx)) return;
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
        if (a.stop_rule != IR_STOP_FIXED && it >= 2 && q >= 0.5 * qprev) { flags |= 16; break; }
        qprev = q;
        dmax = 0.0;

        // ---------------- z = P r (left) or r (right) in u_p, stored in u_g; beta = ||z||
        TG part = TG(0);
        if (hasP && !rightP) {
            sell_rows<TP>(r0, r1, sop, a.P.col, pv, [&](int c) { return (TP)ldcg(&r[c]); },
                          [&](int64_t row, TP v) { TG z = (TG)v; ws[row - r0] = z; wbuf[row] = z; part = fma(z, z, part); });
        } else {
            for (int64_t row = r0 + tid; row < r1; row += BT) {
                TG z = (TG)(TP)r[row];
                ws[row - r0] = z;
                wbuf[row] = z;
                part = fma(z, z, part);
            }
        }
        TG bsq;
        if (!xsum<true>(a, sh, redg, part, bsq)) return;
        const TG beta = sqrt(bsq);
        int k = 0;
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
            // ---- y = R^{-1} g (double), d = V y in u_g, x = x + d in u
            if (!xbar(a, sh)) return;  // R columns from block 0
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
            if (rightP) {
                // right preconditioning: d = P (V_k y), the product in u_p stored in u_g
                for (int64_t row = r0 + tid; row < r1; row += BT) {
                    TG dsum = TG(0);
                    for (int i = 0; i < k; i++) dsum = fma(V[(int64_t)i * a.ldv + row], (TG)yv[i], dsum);
                    wbuf[row] = dsum;
                }
                if (!xbar(a, sh)) return;
                sell_rows<TP>(r0, r1, sop, a.P.col, pv, [&](int c) { return (TP)ldcg(&wbuf[c]); },
                              [&](int64_t row, TP v) {
                                  const TU du = (TU)(TG)v;
                                  dmax = fmax(dmax, fabs((double)du));
                                  x[row] = (TU)((TU)x[row] + du);
                              });
            } else {
                for (int64_t row = r0 + tid; row < r1; row += BT) {
                    TG dsum = TG(0);
                    for (int i = 0; i < k; i++) dsum = fma(V[(int64_t)i * a.ldv + row], (TG)yv[i], dsum);
                    const TU du = (TU)dsum;
                    dmax = fmax(dmax, fabs((double)du));
                    x[row] = (TU)((TU)x[row] + du);
                }
            }
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

template <class TU, class TG, class TP, int RM>
__global__ void __launch_bounds__(ir_threads<TG, TP>(), 1) k_ir(IrArgs a)
{
    ir_body<TU, TG, TP, RM>(a, (int)blockIdx.x, (int)gridDim.x);
}

// Many systems in one cooperative launch, scheduled dynamically: the grid is
// split into teams of T blocks; the first block of a team claims the next
// system from *next (an atomic counter) and hands its index to the team
// through the team's word in `claim`, tagged with the team's claim count, and
// the team runs that system (with its own arguments, exchange slots and error
// word) as a grid of T blocks.  Teams never wait on one another, so a system
// with many iterations holds only its own team's SMs.  Waits are bounded like
// every other wait of the refinement: a team that gives up leaves.
template <class TU, class TG, class TP, int RM>
__global__ void __launch_bounds__(ir_threads<TG, TP>(), 1) k_ir_batch(const IrArgs* __restrict__ args, int count,
                                                                     int T, unsigned* next,
                                                                     unsigned long long* claim, long long limit)
{
    __shared__ int s_sys;
    const int team = (int)blockIdx.x / T, rank = (int)blockIdx.x % T;
    for (unsigned round = 1;; round++) {
        if (threadIdx.x == 0) {
            int sys = -1;
            if (rank == 0) {
                sys = (int)atomicAdd(next, 1u);
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
        if (sys < 0 || sys >= count) return;
        ir_body<TU, TG, TP, RM>(args[sys], rank, T);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- SELL-32 conversion

// width of each 32-row slice (longest row), times 32
__global__ void k_sell_width(int64_t n, const int64_t* __restrict__ rp, int32_t* __restrict__ w32)
{
    const int lane = threadIdx.x & 31;
    const int64_t nsl = (n + 31) >> 5;
    for (int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; s < nsl;
         s += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        int64_t row = s * 32 + lane;
        int len = row < n ? (int)(rp[row + 1] - rp[row]) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
        if (lane == 0) w32[s] = len * 32;
    }
}

template <class TP>
__global__ void k_sell_fill(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const double* __restrict__ val, const int64_t* __restrict__ off, int32_t* __restrict__ scol,
                            TP* __restrict__ sval)
{
    const int lane = threadIdx.x & 31;
    const int64_t nsl = (n + 31) >> 5;
    for (int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; s < nsl;
         s += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t row = s * 32 + lane;
        const int w = (int)((off[s + 1] - off[s]) >> 5);
        const int64_t b = row < n ? rp[row] : 0;
        const int len = row < n ? (int)(rp[row + 1] - b) : 0;
        for (int c = 0; c < w; c++) {
            int64_t o = off[s] + 32 * c + lane;
            if (c < len) { scol[o] = ci[b + c]; sval[o] = (TP)val[b + c]; }
            else { scol[o] = row < n ? (int32_t)row : 0; sval[o] = TP(0); }
        }
    }
}

// x0 = P_f b in u_f (FP16 storage / FP32 accumulation at half), stored in u
template <class S, class TU>
__global__ void k_x0(int64_t n, const int64_t* __restrict__ prp, const int32_t* __restrict__ pci,
                     const S* __restrict__ pv, const double* __restrict__ b, TU* __restrict__ x)
{
    typedef typename Compute<S>::T C;
    for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < n; row += (int64_t)gridDim.x * blockDim.x) {
        C acc = C(0);
        if (prp) {
            for (int64_t q = prp[row]; q < prp[row + 1]; q++)
                acc = fma(to_c(pv[q]), to_c(from_d<S>(b[pci[q]])), acc);
        } else {
            acc = to_c(from_d<S>(b[row]));
        }
        x[row] = (TU)to_c(from_d<S>((double)acc));
    }
}

template <class TU>
__global__ void k_to_double(int64_t n, const TU* __restrict__ x, double* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)x[i];
}


// ||A||_inf, ||b||_inf, and the largest row count q: per-block maxima, then
// one atomic per block and value
__global__ void k_norms(int64_t n, const int64_t* __restrict__ rp, const double* __restrict__ val,
                        const double* __restrict__ b, unsigned long long* __restrict__ out)
{
    __shared__ double sa[32], sb[32];
    __shared__ int sq[32];
    double an = 0.0, bn = 0.0;
    int q = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; p++) s += fabs(val[p]);
        an = fmax(an, s);
        bn = fmax(bn, fabs(b[i]));
        q = max(q, (int)(rp[i + 1] - rp[i]));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    an = warp_max(an);
    bn = warp_max(bn);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q = max(q, __shfl_xor_sync(0xffffffffu, q, o));
    if (lane == 0) { sa[wid] = an; sb[wid] = bn; sq[wid] = q; }
    __syncthreads();
    if (wid == 0) {
        an = lane < nw ? sa[lane] : 0.0;
        bn = lane < nw ? sb[lane] : 0.0;
        q = lane < nw ? sq[lane] : 0;
        an = warp_max(an);
        bn = warp_max(bn);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) q = max(q, __shfl_xor_sync(0xffffffffu, q, o));
        if (lane == 0) {
            // non-negative doubles order like their bit patterns
            atomicMax(&out[0], (unsigned long long)__double_as_longlong(an));
            atomicMax(&out[1], (unsigned long long)__double_as_longlong(bn));
            atomicMax(&out[2], (unsigned long long)q);
        }
    }
}

template <class TU, class TG, class TP, int RM>
int launch_ir(IrArgs& a, int num_sms, cudaStream_t s, int* grid_out)
{
    auto kern = k_ir<TU, TG, TP, RM>;
    // one block per SM, at least 256 rows per block, rows per
    // block a multiple of 32 so that blocks own whole SELL slices
    int64_t G = std::min<int64_t>((a.n + 255) / 256, std::min(num_sms, MAX_GRID));
    if (G < 1) G = 1;
    a.rb = ((a.n + G - 1) / G + 31) & ~int64_t(31);
    G = (a.n + a.rb - 1) / a.rb;
    const int64_t nsl = (a.rb + 31) >> 5;
    // Gram-Schmidt group: on large grids the scalar rounds run among half the
    // blocks (each over two blocks' rows); a round among 76 blocks took
    // ~1.2 us against ~1.7 us among 152, which outweighs the extra barrier
    // that publishes w once per iteration.  CGS2 has no scalar rounds.
    a.g2 = (!a.orth && G >= MGS_GROUP_MIN_GRID) ? (int)((G + 1) / 2) : 0;
    auto smem_for = [&](int g2) {
        return sizeof(double) * 5 * (a.kmax + 2) + sizeof(int64_t) * 2 * (nsl + 1) + (g2 ? 2 : 1) * a.rb * sizeof(TG) + 64;
    };
    size_t dyn_max = 0;
    SPAI_CUDA_TRY(allow_max_dynamic_smem(kern, &dyn_max));
    if (a.g2 && smem_for(a.g2) > dyn_max) a.g2 = 0;  // the doubled row range does not fit
    const size_t smem = smem_for(a.g2);
    if (smem > dyn_max) return SPAI_ERR_UNSUPPORTED;
    int occ = 0;
    constexpr int threads = ir_threads<TG, TP>();
    SPAI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem));
    if ((int64_t)occ * num_sms < G) return SPAI_ERR_UNSUPPORTED;
    void* args[] = {(void*)&a};
    SPAI_CUDA_TRY(cudaLaunchCooperativeKernel((void*)kern, dim3((unsigned)G), dim3(threads), args, smem, s));
    *grid_out = (int)G;
    return 0;
}

template <class TU, class TG, class TP>
int launch_ir_rm(IrArgs& a, int rm, int num_sms, cudaStream_t s, int* grid)
{
    if (rm == 2) return launch_ir<TU, TG, TP, 2>(a, num_sms, s, grid);
    return launch_ir<TU, TG, TP, 1>(a, num_sms, s, grid);
}

int prec_bytes(int p) { return p == SPAI_HALF ? 2 : (p == SPAI_SINGLE ? 4 : 8); }

}  // namespace

// SELL-32 copy of a CSR matrix with values rounded to `prec` (single or double),
// in two halves: sell_begin computes the slice offsets (the entry count stays
// on the device at off[nslices]); sell_finish allocates and fills once that
// count is known on the host.
int sell_begin(int64_t n, const int64_t* rp, int num_sms, cudaStream_t s, SellMat* out, int* launches)
{
    const int64_t nsl = (n + 31) >> 5;
    int32_t* w32 = nullptr;
    int rc = dev_alloc((void**)&w32, sizeof(int32_t) * nsl, s);
    if (rc) return rc;
    rc = dev_alloc((void**)&out->off, sizeof(int64_t) * (nsl + 1), s);
    if (rc) { dev_free(w32, s); return rc; }
    const int tb = 256;
    const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((nsl * 32 + tb - 1) / tb, (int64_t)num_sms * 16));
    k_sell_width<<<gb, tb, 0, s>>>(n, rp, w32);
    rc = scan_counts(nsl, w32, out->off, s);
    *launches += 4;
    dev_free(w32, s);
    return rc;
}

int sell_finish(int64_t n, const int64_t* rp, const int32_t* ci, const double* val, int prec, int num_sms,
                cudaStream_t s, SellMat* out, int64_t total, int* launches)
{
    const int64_t nsl = (n + 31) >> 5;
    const int tb = 256;
    const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((nsl * 32 + tb - 1) / tb, (int64_t)num_sms * 16));
    int rc;
    out->prec = prec;
    out->nnz = total;
    if ((rc = dev_alloc((void**)&out->col, sizeof(int32_t) * std::max<int64_t>(total, 1), s))) return rc;
    if ((rc = dev_alloc(&out->val, (size_t)prec_bytes(prec) * std::max<int64_t>(total, 1), s))) return rc;
    if (prec == SPAI_SINGLE) k_sell_fill<float><<<gb, tb, 0, s>>>(n, rp, ci, val, out->off, out->col, (float*)out->val);
    else k_sell_fill<double><<<gb, tb, 0, s>>>(n, rp, ci, val, out->off, out->col, (double*)out->val);
    *launches += 1;
    SPAI_CUDA_TRY(cudaGetLastError());
    return 0;
}

int sell_build(int64_t n, const int64_t* rp, const int32_t* ci, const double* val, int prec, int num_sms,
               cudaStream_t s, SellMat* out, int* launches)
{
    int rc = sell_begin(n, rp, num_sms, s, out, launches);
    if (rc) return rc;
    const int64_t nsl = (n + 31) >> 5;
    int64_t total = 0;
    if (cudaMemcpyAsync(&total, out->off + nsl, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SPAI_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SPAI_ERR_CUDA;
    return sell_finish(n, rp, ci, val, prec, num_sms, s, out, total, launches);
}

void sell_free(SellMat* m, cudaStream_t s)
{
    dev_free(m->off, s);
    dev_free(m->col, s);
    dev_free(m->val, s);
    m->off = nullptr;
    m->col = nullptr;
    m->val = nullptr;
}

namespace {

// One system's refinement: buffers, the host copies of its results, and the
// kernel arguments.  gmres_ir_dev runs one job; gmres_ir_batch_dev runs many
// jobs per cooperative launch.
struct IrJob {
    const DevCsr* A = nullptr;
    spai_precond P = nullptr;
    const double* b = nullptr;
    double* xout = nullptr;
    int64_t n = 0;
    int kmax = 0, imax = 0;
    void *x = nullptr, *r = nullptr, *wbuf = nullptr, *tbuf = nullptr, *V = nullptr;
    double *R = nullptr, *nbe = nullptr;
    int *its = nullptr, *outv = nullptr, *err = nullptr;
    unsigned long long* msg = nullptr;
    unsigned long long* norms = nullptr;
    void* pvec = nullptr;
    unsigned* gcount = nullptr;
    SellMat As;
    const SellMat* Ps = nullptr;
    unsigned long long h_norms[3] = {0, 0, 0};
    int h_out[2] = {0, 0}, h_err = 0;
    int h_its[SPAI_IR_MAX_STEPS + 1] = {0};
    double h_nbe[SPAI_IR_MAX_STEPS + 1] = {0.0};
    IrArgs a;
};

int ir_check_opts(const ir_opts* o)
{
    if (!o) return SPAI_ERR_INVALID_ARG;
    if (o->u != SPAI_SINGLE && o->u != SPAI_DOUBLE) return SPAI_ERR_UNSUPPORTED;
    if (o->ug != SPAI_SINGLE && o->ug != SPAI_DOUBLE) return SPAI_ERR_UNSUPPORTED;
    if (o->up != SPAI_SINGLE && o->up != SPAI_DOUBLE) return SPAI_ERR_UNSUPPORTED;
    if (o->ur != SPAI_DOUBLE && o->ur != SPAI_QUAD) return SPAI_ERR_UNSUPPORTED;
    if (o->uf != SPAI_HALF && o->uf != SPAI_SINGLE && o->uf != SPAI_DOUBLE) return SPAI_ERR_UNSUPPORTED;
    if (o->ir_max_steps < 1 || o->ir_max_steps > SPAI_IR_MAX_STEPS) return SPAI_ERR_INVALID_ARG;
    if (!(o->tau >= 0.0)) return SPAI_ERR_INVALID_ARG;
    if (o->orth != 0 && o->orth != 1) return SPAI_ERR_INVALID_ARG;
    if (o->side != 0 && o->side != 1) return SPAI_ERR_INVALID_ARG;
    if (o->stop != IR_STOP_BACKWARD && o->stop != IR_STOP_FIXED && o->stop != IR_STOP_CORRECTION)
        return SPAI_ERR_INVALID_ARG;
    return 0;
}

// The stopping threshold (reading R8): the caller's, else q u for the
// backward-error rule (q the longest row of A, the limit of Theorem 2) and u
// for the correction rule.
double ir_stop_tol(const ir_opts* o, int q)
{
    const double uu = o->u == SPAI_SINGLE ? 5.9604644775390625e-08 : 1.1102230246251565e-16;
    if (o->stop_tol > 0) return o->stop_tol;
    return o->stop == IR_STOP_CORRECTION ? uu : q * uu;
}

int ir_job_kmax(int64_t n, const ir_opts* o, int* kmax)
{
    int k = o->gmres_max_it > 0 ? o->gmres_max_it : (int)std::min<int64_t>(n, 500);
    if (k > n) k = (int)n;
    if (k > KMAX_LIMIT) return SPAI_ERR_UNSUPPORTED;
    if (k < 1) k = 1;
    *kmax = k;
    return 0;
}

// The job's buffers (allocated and cleared on s).
int ir_job_alloc(IrJob& J, cudaStream_t s, const ir_opts* o)
{
#define TRY(x) do { int rc_ = (x); if (rc_) return rc_; } while (0)
#define CTRY(x) do { if ((x) != cudaSuccess) return SPAI_ERR_CUDA; } while (0)
    const int64_t n = J.n;
    const int su = prec_bytes(o->u), sg = prec_bytes(o->ug), sp = prec_bytes(o->up);
    const int64_t ldv = (n + 31) & ~int64_t(31);
    const int kmax = J.kmax, imax = J.imax;
    TRY(dev_alloc(&J.x, (size_t)su * n, s));
    TRY(dev_alloc(&J.r, (size_t)su * n, s));
    TRY(dev_alloc(&J.wbuf, (size_t)sg * n, s));
    TRY(dev_alloc(&J.tbuf, (size_t)sp * n, s));
    TRY(dev_alloc(&J.V, (size_t)sg * ldv * (kmax + 1), s));
    TRY(dev_alloc((void**)&J.R, sizeof(double) * (size_t)(kmax + 1) * kmax, s));
    TRY(dev_alloc((void**)&J.msg, sizeof(unsigned long long) * 4 * MAX_GRID * SLOT_WORDS, s));
    TRY(dev_alloc((void**)&J.nbe, sizeof(double) * (imax + 1), s));
    TRY(dev_alloc((void**)&J.its, sizeof(int) * (imax + 1), s));
    TRY(dev_alloc((void**)&J.outv, sizeof(int) * 2, s));
    TRY(dev_alloc((void**)&J.err, sizeof(int) * 2, s));
    // [0..2] the norms and the longest row, [3] [4] SELL entry counts of A and P
    TRY(dev_alloc((void**)&J.norms, sizeof(unsigned long long) * 5, s));
    CTRY(cudaMemsetAsync(J.norms, 0, sizeof(unsigned long long) * 5, s));
    if (o->orth) {
        TRY(dev_alloc(&J.pvec, (size_t)sg * 2 * MAX_GRID * (kmax + 1), s));
        TRY(dev_alloc((void**)&J.gcount, sizeof(unsigned), s));
        CTRY(cudaMemsetAsync(J.gcount, 0, sizeof(unsigned), s));
    }
    CTRY(cudaMemsetAsync(J.its, 0, sizeof(int) * (imax + 1), s));
    CTRY(cudaMemsetAsync(J.outv, 0, sizeof(int) * 2, s));
    CTRY(cudaMemsetAsync(J.err, 0, sizeof(int) * 2, s));
    CTRY(cudaMemsetAsync(J.msg, 0, sizeof(unsigned long long) * 4 * MAX_GRID * SLOT_WORDS, s));
    return 0;
#undef TRY
#undef CTRY
}

// ||A||_inf, ||b||_inf, the longest row into J.norms, and x0 = P b in u_f
// stored in u, enqueued on s.
int ir_job_norms_x0(IrJob& J, int num_sms, cudaStream_t s, const ir_opts* o, int* nl)
{
    const int64_t n = J.n;
    const int tb = 256;
    const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((n + tb - 1) / tb, (int64_t)num_sms * 32));
    const DevCsr& A = *J.A;
    spai_precond P = J.P;
    k_norms<<<gb, tb, 0, s>>>(n, A.rowptr, A.val, J.b, J.norms);
    (*nl)++;
    // x0 = P b in u_f, stored in u
    const int64_t* prp = P ? P->rowptr : nullptr;
    const int32_t* pci = P ? P->col : nullptr;
    const void* pvf = P ? P->val_uf : nullptr;
#define X0(S, TU) k_x0<S, TU><<<gb, tb, 0, s>>>(n, prp, pci, (const S*)pvf, J.b, (TU*)J.x)
    if (o->u == SPAI_SINGLE) {
        if (o->uf == SPAI_HALF) X0(__half, float);
        else if (o->uf == SPAI_SINGLE) X0(float, float);
        else X0(double, float);
    } else {
        if (o->uf == SPAI_HALF) X0(__half, double);
        else if (o->uf == SPAI_SINGLE) X0(float, double);
        else X0(double, double);
    }
#undef X0
    (*nl)++;
    if (cudaGetLastError() != cudaSuccess) return SPAI_ERR_CUDA;
    return 0;
}

// Allocations, SELL-32 copies of A (and of P, cached on the handle), the norms
// and x0 = P b, enqueued on s with one synchronisation (for the SELL entry
// counts and the norms, which are on the host when it returns).
int ir_job_prepare(IrJob& J, int num_sms, cudaStream_t s, const ir_opts* o, int* nl)
{
    int rc = ir_job_alloc(J, s, o);
    if (rc) return rc;
    const DevCsr& A = *J.A;
    spai_precond P = J.P;
    // one host synchronisation for the SELL entry counts and the norms: the
    // counts join the norms on the device, and one copy brings all five
    const int64_t nsl = (J.n + 31) >> 5;
    SellMat* cache = nullptr;
    rc = sell_begin(J.n, A.rowptr, num_sms, s, &J.As, nl);
    if (rc) return rc;
    if (cudaMemcpyAsync(J.norms + 3, J.As.off + nsl, 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return SPAI_ERR_CUDA;
    if (P) {
        cache = o->up == SPAI_SINGLE ? &P->sell_f32 : &P->sell_f64;
        if (!cache->off) {
            rc = sell_begin(J.n, P->rowptr, num_sms, s, cache, nl);
            if (rc) return rc;
            if (cudaMemcpyAsync(J.norms + 4, cache->off + nsl, 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                return SPAI_ERR_CUDA;
        } else {
            cache = nullptr;  // already made
        }
        J.Ps = o->up == SPAI_SINGLE ? &P->sell_f32 : &P->sell_f64;
    }
    rc = ir_job_norms_x0(J, num_sms, s, o, nl);
    if (rc) return rc;
    unsigned long long h[5] = {0, 0, 0, 0, 0};
    if (cudaMemcpyAsync(h, J.norms, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SPAI_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SPAI_ERR_CUDA;
    for (int k = 0; k < 3; k++) J.h_norms[k] = h[k];
    const int64_t tot[2] = {(int64_t)h[3], (int64_t)h[4]};
    rc = sell_finish(J.n, A.rowptr, A.col, A.val, o->up, num_sms, s, &J.As, tot[0], nl);
    if (rc) return rc;
    if (cache) rc = sell_finish(J.n, P->rowptr, P->col, P->val, o->up, num_sms, s, cache, tot[1], nl);
    return rc;
}

// The kernel arguments, once the norms have reached the host (after a sync).
void ir_job_args(IrJob& J, int device, const ir_opts* o)
{
    IrArgs& a = J.a;
    memset(&a, 0, sizeof(a));
    double anorm, bnorm;
    long long t0 = (long long)J.h_norms[0], t1 = (long long)J.h_norms[1];
    memcpy(&anorm, &t0, 8);
    memcpy(&bnorm, &t1, 8);
    const int q = (int)J.h_norms[2];
    const DevCsr& A = *J.A;
    a.n = J.n;
    a.A.off = J.As.off; a.A.col = J.As.col; a.A.val = J.As.val;
    if (J.Ps) { a.P.off = J.Ps->off; a.P.col = J.Ps->col; a.P.val = J.Ps->val; }
    a.arp = A.rowptr; a.aci = A.col; a.aval = A.val;
    a.b = J.b; a.x = J.x; a.r = J.r; a.wbuf = J.wbuf; a.tbuf = J.tbuf; a.V = J.V;
    a.ldv = (J.n + 31) & ~int64_t(31); a.R = J.R; a.msg = J.msg;
    a.msg2 = J.msg + 2 * MAX_GRID * SLOT_WORDS;
    a.err = J.err;
    int clk_khz = device_attr_cached(cudaDevAttrClockRate, device);
    if (clk_khz <= 0) clk_khz = 2000000;
    a.limit = (long long)clk_khz * 1000LL * 4;  // about four seconds per wait
    a.anorm = anorm; a.bnorm = bnorm; a.tau = o->tau;
    a.stop_tol = ir_stop_tol(o, q);
    a.kmax = J.kmax; a.imax = J.imax; a.stop_rule = o->stop;
    a.its = J.its; a.nbe = J.nbe; a.out = J.outv;
    a.orth = o->orth; a.pvec = J.pvec; a.gcount = J.gcount; a.side = o->side;
}

// x in double and the result copies, enqueued on s.
int ir_job_collect(IrJob& J, int num_sms, cudaStream_t s, const ir_opts* o, int* nl)
{
    const int tb = 256;
    const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((J.n + tb - 1) / tb, (int64_t)num_sms * 32));
    if (o->u == SPAI_SINGLE) k_to_double<float><<<gb, tb, 0, s>>>(J.n, (const float*)J.x, J.xout);
    else k_to_double<double><<<gb, tb, 0, s>>>(J.n, (const double*)J.x, J.xout);
    (*nl)++;
    if (cudaGetLastError() != cudaSuccess) return SPAI_ERR_CUDA;
    if (cudaMemcpyAsync(J.h_out, J.outv, sizeof(J.h_out), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SPAI_ERR_CUDA;
    if (cudaMemcpyAsync(&J.h_err, J.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SPAI_ERR_CUDA;
    if (cudaMemcpyAsync(J.h_its, J.its, sizeof(int) * J.imax, cudaMemcpyDeviceToHost, s) != cudaSuccess) return SPAI_ERR_CUDA;
    if (cudaMemcpyAsync(J.h_nbe, J.nbe, sizeof(double) * (J.imax + 1), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SPAI_ERR_CUDA;
    return 0;
}

// After a sync: the statistics (timings and launch counts are the caller's)
// and the return code of the job.
int ir_job_result(const IrJob& J, const ir_opts* o, ir_stats* st)
{
    if (J.h_err) return J.h_err;
    if (st) {
        memset(st->its, 0, sizeof(st->its));
        for (int i = 0; i < J.imax; i++) st->its[i] = J.h_its[i];
        for (int i = 0; i <= SPAI_IR_MAX_STEPS; i++) st->nbe[i] = 0.0;
        st->steps = J.h_out[0];
        st->flags = J.h_out[1];
        for (int i = 0; i <= st->steps && i <= J.imax; i++) st->nbe[i] = J.h_nbe[i];
        st->total_its = 0;
        for (int i = 0; i < st->steps; i++) st->total_its += st->its[i];
        st->final_nbe = st->nbe[st->steps];
        st->nnz_P = J.P ? J.P->nnz : 0;
    }
    if (J.h_out[1] & 8) return SPAI_ERR_NONFINITE;
    if (!(J.h_out[1] & 1) && o->stop != IR_STOP_FIXED) return SPAI_WARN_NOT_CONVERGED;
    return 0;
}

void ir_job_free(IrJob& J, cudaStream_t s)
{
    sell_free(&J.As, s);
    dev_free(J.x, s); dev_free(J.r, s); dev_free(J.wbuf, s); dev_free(J.tbuf, s); dev_free(J.V, s);
    dev_free(J.R, s); dev_free(J.msg, s); dev_free(J.nbe, s); dev_free(J.its, s); dev_free(J.outv, s);
    dev_free(J.err, s); dev_free(J.norms, s); dev_free(J.pvec, s); dev_free(J.gcount, s);
    J.x = J.r = J.wbuf = J.tbuf = J.V = J.pvec = nullptr;
    J.R = J.nbe = nullptr;
    J.its = J.outv = J.err = nullptr;
    J.msg = J.norms = nullptr;
    J.gcount = nullptr;
}

// Instantiate F<TU, TG, TP> for the run-time precisions and call it.
template <class F>
int dispatch_tuple(const ir_opts* o, F&& f)
{
    if (o->u == SPAI_DOUBLE) {
        if (o->ug == SPAI_DOUBLE) {
            if (o->up == SPAI_DOUBLE) return f.template run<double, double, double>();
            return f.template run<double, double, float>();
        }
        if (o->up == SPAI_DOUBLE) return f.template run<double, float, double>();
        return f.template run<double, float, float>();
    }
    if (o->ug == SPAI_DOUBLE) {
        if (o->up == SPAI_DOUBLE) return f.template run<float, double, double>();
        return f.template run<float, double, float>();
    }
    if (o->up == SPAI_DOUBLE) return f.template run<float, float, double>();
    return f.template run<float, float, float>();
}

struct LaunchOne {
    IrArgs* a;
    int rm, num_sms;
    cudaStream_t s;
    int* grid;
    template <class TU, class TG, class TP>
    int run() { return launch_ir_rm<TU, TG, TP>(*a, rm, num_sms, s, grid); }
};

}  // namespace

int gmres_ir_dev(int device, int num_sms, cudaStream_t s, const DevCsr& A, spai_precond P,
                 const double* b, double* xout, const ir_opts* o, ir_stats* st)
{
    int rc = ir_check_opts(o);
    if (rc) return rc;
    if (P && P->uf != o->uf) return SPAI_ERR_INVALID_ARG;
    IrJob J;
    J.A = &A; J.P = P; J.b = b; J.xout = xout; J.n = A.n; J.imax = o->ir_max_steps;
    rc = ir_job_kmax(A.n, o, &J.kmax);
    if (rc) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr, ek0 = nullptr, ek1 = nullptr;
    SPAI_CUDA_TRY(cudaEventCreate(&e0));
    SPAI_CUDA_TRY(cudaEventCreate(&e1));
    SPAI_CUDA_TRY(cudaEventCreate(&ek0));
    SPAI_CUDA_TRY(cudaEventCreate(&ek1));
    int nl = 0;  // kernels launched
    int grid = 0;
#define TRY(x) do { rc = (x); if (rc) goto done; } while (0)
#define CTRY(x) do { if ((x) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; } } while (0)
    CTRY(cudaEventRecord(e0, s));
    TRY(ir_job_prepare(J, num_sms, s, o, &nl));  // the norms are on the host when it returns
    ir_job_args(J, device, o);
    CTRY(cudaEventRecord(ek0, s));
    {
        LaunchOne L{&J.a, o->ur == SPAI_QUAD ? 2 : 1, num_sms, s, &grid};
        TRY(dispatch_tuple(o, L));
    }
    CTRY(cudaEventRecord(ek1, s));
    nl++;
    TRY(ir_job_collect(J, num_sms, s, o, &nl));
    CTRY(cudaEventRecord(e1, s));
    CTRY(cudaStreamSynchronize(s));
    rc = ir_job_result(J, o, st);
    if (rc >= 0 && st) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        st->ms_ir = ms;
        cudaEventElapsedTime(&ms, ek0, ek1);
        st->ms_kernel = ms;
        st->launches += nl;
        st->grid = grid;
    }
done:
#undef TRY
#undef CTRY
    ir_job_free(J, s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (ek0) cudaEventDestroy(ek0);
    if (ek1) cudaEventDestroy(ek1);
    if (rc < 0) cudaStreamSynchronize(s);
    return rc;
}

// ====================================================================
// Self-test of the bounded device waits (spai_selftest_wait_timeout): the
// blocks of a small launch run one exchange round (mode 0) or one counter
// barrier (mode 1) that counts one block more than the grid holds, so they
// wait for a word or an arrival that nothing provides.  Each wait gives up
// after a.limit clock cycles, records SPAI_ERR_TIMEOUT and returns, exactly as
// in the refinement kernels.
// ====================================================================

namespace {

__global__ void k_wait_probe(IrArgs a, int mode)
{
    __shared__ IrShared shs;
    if (threadIdx.x == 0) {
        shs.bid = (int)blockIdx.x;
        shs.G = (int)gridDim.x + 1;  // a block that does not exist
        shs.epoch = 0;
        shs.epoch2 = 0;
        shs.gepoch = 0;
        shs.ok = 1;
    }
    __syncthreads();
    if (mode == 0) {
        uint32_t pay[1] = {0u};
        NoAcc acc;
        exchange<1, true>(a, &shs, pay, acc);
    } else {
        const GridBarrier gb{a.gcount, a.err, a.limit, gridDim.x + 1};
        grid_sync(gb, &shs.gepoch, &shs.ok);
    }
}

}  // namespace

extern "C" int spai_selftest_wait_timeout(int device, int mode, double limit_ms)
{
    if (mode != 0 && mode != 1) return SPAI_ERR_INVALID_ARG;
    if (!(limit_ms > 0.0) || limit_ms > 10000.0) return SPAI_ERR_INVALID_ARG;
    SPAI_CUDA_TRY(cudaSetDevice(device));
    constexpr int grid = 4;
    unsigned long long* msg = nullptr;
    int* err = nullptr;
    unsigned* gcount = nullptr;
    const size_t msg_bytes = sizeof(unsigned long long) * 2 * (grid + 1) * SLOT_WORDS;
    int rc = 0;
    if (cudaMalloc((void**)&msg, msg_bytes) != cudaSuccess || cudaMalloc((void**)&err, sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&gcount, sizeof(unsigned)) != cudaSuccess)
        rc = SPAI_ERR_NO_MEMORY;
    if (!rc && (cudaMemset(msg, 0, msg_bytes) != cudaSuccess || cudaMemset(err, 0, sizeof(int)) != cudaSuccess ||
                cudaMemset(gcount, 0, sizeof(unsigned)) != cudaSuccess))
        rc = SPAI_ERR_CUDA;
    if (!rc) {
        IrArgs a;
        memset(&a, 0, sizeof(a));
        a.msg = msg;
        a.err = err;
        a.gcount = gcount;
        int clk_khz = device_attr_cached(cudaDevAttrClockRate, device);
        if (clk_khz <= 0) clk_khz = 2000000;
        a.limit = (long long)((double)clk_khz * limit_ms);
        k_wait_probe<<<grid, 32>>>(a, mode);
        int h = 0;
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = SPAI_ERR_CUDA;
        else
            rc = h;  // SPAI_ERR_TIMEOUT when every wait gave up as designed
    }
    cudaFree(msg);
    cudaFree(err);
    cudaFree(gcount);
    return rc;
}

// ====================================================================
// Batched refinement (gmres_ir_solve_batch): many independent systems in one
// persistent cooperative launch.  Cooperative launches of separate systems
// hardly overlap on the GPU (16 solves of an n = 4096 system: 111 ms one
// after another, 66-70 ms from 2 or 4 host threads), while one such system
// keeps only 16 of 152 SMs busy.  The batch splits the co-resident grid into
// teams of T blocks (T from the median order, about BATCH_ROWS_PER_BLOCK rows
// per block, at most 16); each team takes the next system (larger first) as
// soon as it is done with its last one, so systems with many GMRES iterations
// do not hold up the others' SMs.  All systems are prepared before the launch
// (their buffers coexist).
// ====================================================================

namespace {

constexpr int64_t BATCH_ROWS_PER_BLOCK = 2048;

template <class TU, class TG, class TP, int RM>
struct BatchRun {
    int device, num_sms;
    cudaStream_t s;
    const ir_opts* o;
    std::vector<IrJob>* jobs;
    std::vector<int>* order;   // systems by decreasing order n
    int* nl;
    float* ms_kernel;
    int* team_size;

    size_t smem_for(const IrArgs& a) const
    {
        const int64_t nsl = (a.rb + 31) >> 5;
        return sizeof(double) * 5 * (a.kmax + 2) + sizeof(int64_t) * 2 * (nsl + 1) + (a.g2 ? 2 : 1) * a.rb * sizeof(TG) + 64;
    }

    int run()
    {
        auto kern = k_ir_batch<TU, TG, TP, RM>;
        constexpr int threads = ir_threads<TG, TP>();
        size_t dyn_max = 0;
        SPAI_CUDA_TRY(allow_max_dynamic_smem(kern, &dyn_max));
        std::vector<IrJob>& J = *jobs;
        const int count = (int)J.size();
        // team size from the median order: about BATCH_ROWS_PER_BLOCK rows per block
        std::vector<int64_t> ns(count);
        for (int i = 0; i < count; i++) ns[i] = J[i].n;
        std::nth_element(ns.begin(), ns.begin() + count / 2, ns.end());
        const int64_t med = ns[count / 2];
        const int T = (int)std::max<int64_t>(1, std::min<int64_t>(16, (med + BATCH_ROWS_PER_BLOCK / 2) / BATCH_ROWS_PER_BLOCK));
        int rc = 0;
        // preparation without a wait per system: buffers, SELL offsets, norms and x0
        // for all systems, then one copy of every SELL size and norm to the host,
        // then the SELL fills
        std::vector<char> pbuild(count, 0);
        std::set<spai_precond> building;
        unsigned long long* d_slots = nullptr;
        rc = dev_alloc((void**)&d_slots, sizeof(unsigned long long) * 5 * count, s);
        if (rc) return rc;
        for (int i : *order) {
            IrJob& jb = J[i];
            if (!rc) rc = ir_job_alloc(jb, s, o);
            if (!rc) rc = sell_begin(jb.n, jb.A->rowptr, num_sms, s, &jb.As, nl);
            const int64_t nsl = (jb.n + 31) >> 5;
            unsigned long long* slot = d_slots + 5 * (size_t)i;
            if (!rc && jb.P) {
                SellMat* cache = o->up == SPAI_SINGLE ? &jb.P->sell_f32 : &jb.P->sell_f64;
                if (!cache->off && !building.count(jb.P)) {
                    rc = sell_begin(jb.n, jb.P->rowptr, num_sms, s, cache, nl);
                    building.insert(jb.P);
                    pbuild[i] = 1;
                    if (!rc && cudaMemcpyAsync(slot + 4, cache->off + nsl, 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                        rc = SPAI_ERR_CUDA;
                }
                jb.Ps = cache;
            }
            if (!rc) rc = ir_job_norms_x0(jb, num_sms, s, o, nl);
            if (!rc && cudaMemcpyAsync(slot, jb.norms, 24, cudaMemcpyDeviceToDevice, s) != cudaSuccess) rc = SPAI_ERR_CUDA;
            if (!rc && cudaMemcpyAsync(slot + 3, jb.As.off + nsl, 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                rc = SPAI_ERR_CUDA;
        }
        // a preconditioner's SELL copy counts as built once its offsets exist: on
        // failure the copies this batch started are dropped again
        auto drop_started = [&]() {
            for (spai_precond P : building) sell_free(o->up == SPAI_SINGLE ? &P->sell_f32 : &P->sell_f64, s);
        };
        std::vector<unsigned long long> hs(5 * (size_t)count, 0);
        if (!rc && cudaMemcpyAsync(hs.data(), d_slots, sizeof(unsigned long long) * hs.size(), cudaMemcpyDeviceToHost, s) !=
                       cudaSuccess)
            rc = SPAI_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess && !rc) rc = SPAI_ERR_CUDA;
        dev_free(d_slots, s);
        if (rc) { drop_started(); return rc; }
        for (int i : *order) {
            IrJob& jb = J[i];
            const unsigned long long* h = hs.data() + 5 * (size_t)i;
            for (int k = 0; k < 3; k++) jb.h_norms[k] = h[k];
            rc = sell_finish(jb.n, jb.A->rowptr, jb.A->col, jb.A->val, o->up, num_sms, s, &jb.As, (int64_t)h[3], nl);
            if (!rc && pbuild[i])
                rc = sell_finish(jb.n, jb.P->rowptr, jb.P->col, jb.P->val, o->up, num_sms, s,
                                 o->up == SPAI_SINGLE ? &jb.P->sell_f32 : &jb.P->sell_f64, (int64_t)h[4], nl);
            if (rc) { drop_started(); return rc; }
        }
        // arguments in claim order (larger systems first), every system on T blocks
        std::vector<IrArgs> h(count);
        size_t smem = 0;
        for (int q = 0; q < count; q++) {
            IrJob& jb = J[(*order)[q]];
            ir_job_args(jb, device, o);
            IrArgs& a = jb.a;
            a.G = T;
            a.rb = std::max<int64_t>(32, ((jb.n + T - 1) / T + 31) & ~int64_t(31));
            a.g2 = 0;
            a.block0 = 0;
            smem = std::max(smem, smem_for(a));
            h[q] = a;
        }
        if (smem > dyn_max) return SPAI_ERR_UNSUPPORTED;
        int occ = 0;
        SPAI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem));
        const int teams = (occ * num_sms) / T;
        if (teams < 1) return SPAI_ERR_UNSUPPORTED;
        *team_size = T;
        IrArgs* d_args = nullptr;
        unsigned* d_next = nullptr;
        unsigned long long* d_claim = nullptr;
        rc = dev_alloc((void**)&d_args, sizeof(IrArgs) * count, s);
        if (!rc) rc = dev_alloc((void**)&d_next, sizeof(unsigned), s);
        if (!rc) rc = dev_alloc((void**)&d_claim, sizeof(unsigned long long) * teams, s);
        if (!rc && cudaMemcpyAsync(d_args, h.data(), sizeof(IrArgs) * count, cudaMemcpyHostToDevice, s) != cudaSuccess)
            rc = SPAI_ERR_CUDA;
        if (!rc && cudaMemsetAsync(d_next, 0, sizeof(unsigned), s) != cudaSuccess) rc = SPAI_ERR_CUDA;
        if (!rc && cudaMemsetAsync(d_claim, 0, sizeof(unsigned long long) * teams, s) != cudaSuccess) rc = SPAI_ERR_CUDA;
        cudaEvent_t k0 = nullptr, k1 = nullptr;
        if (!rc && (cudaEventCreate(&k0) != cudaSuccess || cudaEventCreate(&k1) != cudaSuccess)) rc = SPAI_ERR_CUDA;
        if (!rc) {
            const IrArgs* pa = d_args;
            int cnt = count, tt = T;
            long long limit = h[0].limit;
            void* args[] = {(void*)&pa, (void*)&cnt, (void*)&tt, (void*)&d_next, (void*)&d_claim, (void*)&limit};
            cudaEventRecord(k0, s);
            if (cudaLaunchCooperativeKernel((void*)kern, dim3((unsigned)(teams * T)), dim3(threads), args, smem, s) !=
                cudaSuccess)
                rc = SPAI_ERR_CUDA;
            cudaEventRecord(k1, s);
            (*nl)++;
        }
        for (int i = 0; i < count; i++)
            if (!rc) rc = ir_job_collect(J[i], num_sms, s, o, nl);
        if (cudaStreamSynchronize(s) != cudaSuccess && !rc) rc = SPAI_ERR_CUDA;
        if (!rc) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, k0, k1);
            *ms_kernel += ms;
        }
        if (k0) cudaEventDestroy(k0);
        if (k1) cudaEventDestroy(k1);
        dev_free(d_args, s);
        dev_free(d_next, s);
        dev_free(d_claim, s);
        return rc;
    }
};

struct LaunchBatch {
    int device, num_sms;
    cudaStream_t s;
    const ir_opts* o;
    std::vector<IrJob>* jobs;
    std::vector<int>* order;
    int* nl;
    float* ms_kernel;
    int* team_size;
    template <class TU, class TG, class TP>
    int run()
    {
        if (o->ur == SPAI_QUAD)
            return BatchRun<TU, TG, TP, 2>{device, num_sms, s, o, jobs, order, nl, ms_kernel, team_size}.run();
        return BatchRun<TU, TG, TP, 1>{device, num_sms, s, o, jobs, order, nl, ms_kernel, team_size}.run();
    }
};

}  // namespace

int gmres_ir_batch_dev(int device, int num_sms, cudaStream_t s, int count, const DevCsr* A, const spai_precond* P,
                       const double* const* b, double* const* xout, const ir_opts* o, ir_stats* st, int* status)
{
    int rc = ir_check_opts(o);
    if (rc) return rc;
    if (count < 0 || (count > 0 && (!A || !b || !xout))) return SPAI_ERR_INVALID_ARG;
    std::vector<IrJob> jobs(count);
    for (int i = 0; i < count; i++) {
        spai_precond Pi = P ? P[i] : nullptr;
        if (Pi && (Pi->uf != o->uf || Pi->n != A[i].n)) return SPAI_ERR_INVALID_ARG;
        IrJob& J = jobs[i];
        J.A = &A[i]; J.P = Pi; J.b = b[i]; J.xout = xout[i]; J.n = A[i].n; J.imax = o->ir_max_steps;
        rc = ir_job_kmax(A[i].n, o, &J.kmax);
        if (rc) return rc;
    }
    std::vector<int> order(count);
    for (int i = 0; i < count; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return jobs[x].n > jobs[y].n; });
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SPAI_CUDA_TRY(cudaEventCreate(&e0));
    SPAI_CUDA_TRY(cudaEventCreate(&e1));
    int nl = 0;
    float ms_kernel = 0.f;
    cudaEventRecord(e0, s);
    int team = 0;
    LaunchBatch L{device, num_sms, s, o, &jobs, &order, &nl, &ms_kernel, &team};
    rc = dispatch_tuple(o, L);
    cudaEventRecord(e1, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && rc >= 0) rc = SPAI_ERR_CUDA;
    float ms_all = 0.f;
    if (rc >= 0) cudaEventElapsedTime(&ms_all, e0, e1);
    int worst = 0;
    for (int i = 0; i < count; i++) {
        int ri = rc < 0 ? rc : ir_job_result(jobs[i], o, st ? &st[i] : nullptr);
        if (status) status[i] = ri;
        if (ri < 0 && worst >= 0) worst = ri;
        else if (ri > 0 && worst == 0) worst = ri;
        if (st && rc >= 0) {
            st[i].ms_ir = ms_all;
            st[i].ms_kernel = ms_kernel;
            st[i].launches = nl;
            st[i].grid = team;
        }
        ir_job_free(jobs[i], s);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    return rc < 0 ? rc : worst;
}

// ====================================================================
// Allocation-free refinement solve (gmres_ir_solve_noalloc).
//
// For callers that must not allocate device memory: real-time loops (the
// allocator's latency is unbounded and cudaFree synchronises the device),
// hosts that own their memory budget exactly, or runtimes that forbid the
// CUDA allocator after start-up.  The refinement
// scratch (SELL copies of A and P, the Krylov basis, the residual and
// iterate, the exchange slots) lives in one file-scope device array of
// SPAI_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds
// until exit.  Host code never passes the array's name to a kernel (on the
// host it is only a stand-in symbol): its device address is looked up once
// per device with cudaGetSymbolAddress, on the first call made on that
// device.
// ====================================================================

static __device__ __align__(256) unsigned char g_noalloc_scratch[SPAI_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_noalloc_mu;
unsigned char* g_noalloc_base[128] = {nullptr};

int noalloc_base(int dev, unsigned char** out)
{
    if (dev < 0 || dev >= 128) return SPAI_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            spai_set_last_cuda_error(e);
            return SPAI_ERR_CUDA;
        }
        g_noalloc_base[dev] = (unsigned char*)p;
    }
    *out = g_noalloc_base[dev];
    return 0;
}

// exclusive scan of ns counts into out[0..ns], one block
__global__ void k_scan_one_block(int64_t ns, const int32_t* __restrict__ in, int64_t* __restrict__ out)
{
    __shared__ int64_t wsum[32];
    __shared__ int64_t carry;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < ns; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const int64_t v = i < ns ? in[i] : 0;
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
        const int64_t pre = carry + (w > 0 ? wsum[w - 1] : 0) + x - v;
        if (i < ns) out[i] = pre;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = pre + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) out[ns] = carry;
}

// x0 = P b in u_f with P's float64 values rounded to u_f on the fly
template <class S, class TU>
__global__ void k_x0_dbl(int64_t n, const int64_t* __restrict__ prp, const int32_t* __restrict__ pci,
                         const double* __restrict__ pv, const double* __restrict__ b, TU* __restrict__ x)
{
    typedef typename Compute<S>::T C;
    for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < n; row += (int64_t)gridDim.x * blockDim.x) {
        C acc = C(0);
        if (prp) {
            for (int64_t q = prp[row]; q < prp[row + 1]; q++)
                acc = fma(to_c(from_d<S>(pv[q])), to_c(from_d<S>(b[pci[q]])), acc);
        } else {
            acc = to_c(from_d<S>(b[row]));
        }
        x[row] = (TU)to_c(from_d<S>((double)acc));
    }
}

struct Carve {
    unsigned char* base;
    size_t off, cap;
    void* take(size_t bytes)
    {
        off = (off + 255) & ~size_t(255);
        if (off + bytes > cap) return nullptr;
        void* p = base + off;
        off += bytes;
        return p;
    }
};

}  // namespace

extern "C" int gmres_ir_solve_noalloc(const spai_csr* A, const spai_csr* P, const double* b, double* xout,
                                      const ir_opts* o, void* cuda_stream, ir_stats* st)
{
    if (!A || !b || !xout || !o) return SPAI_ERR_INVALID_ARG;
    if (!A->on_device || (P && !P->on_device)) return SPAI_ERR_INVALID_ARG;
    if (A->n < 1 || A->nnz < 0 || !A->rowptr || !A->col || !A->val) return SPAI_ERR_INVALID_ARG;
    if (o->side != 0 && o->side != 1) return SPAI_ERR_INVALID_ARG;
    if (P && (P->n != A->n || P->nnz < 0 || !P->rowptr || !P->col || !P->val)) return SPAI_ERR_INVALID_ARG;
    if (A->n > INT32_MAX) return SPAI_ERR_UNSUPPORTED;
    if (o->u != SPAI_SINGLE && o->u != SPAI_DOUBLE) return SPAI_ERR_UNSUPPORTED;
    if (o->ug != SPAI_SINGLE && o->ug != SPAI_DOUBLE) return SPAI_ERR_UNSUPPORTED;
    if (o->up != SPAI_SINGLE && o->up != SPAI_DOUBLE) return SPAI_ERR_UNSUPPORTED;
    if (o->ur != SPAI_DOUBLE && o->ur != SPAI_QUAD) return SPAI_ERR_UNSUPPORTED;
    if (o->uf != SPAI_HALF && o->uf != SPAI_SINGLE && o->uf != SPAI_DOUBLE) return SPAI_ERR_UNSUPPORTED;
    if (o->ir_max_steps < 1 || o->ir_max_steps > SPAI_IR_MAX_STEPS) return SPAI_ERR_INVALID_ARG;
    if (!(o->tau >= 0.0)) return SPAI_ERR_INVALID_ARG;
    if (o->orth != 0 && o->orth != 1) return SPAI_ERR_INVALID_ARG;
    if (o->stop != IR_STOP_BACKWARD && o->stop != IR_STOP_FIXED && o->stop != IR_STOP_CORRECTION)
        return SPAI_ERR_INVALID_ARG;
    const int64_t n = A->n;
    int kmax = o->gmres_max_it > 0 ? o->gmres_max_it : (int)std::min<int64_t>(n, 500);
    if (kmax > n) kmax = (int)n;
    if (kmax > KMAX_LIMIT) return SPAI_ERR_UNSUPPORTED;
    if (kmax < 1) kmax = 1;
    const int imax = o->ir_max_steps;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int device = 0, num_sms = 0;
    SPAI_CUDA_TRY(cudaGetDevice(&device));
    SPAI_CUDA_TRY(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device));
    unsigned char* base = nullptr;
    int rc = noalloc_base(device, &base);
    if (rc) return rc;

    const int su = prec_bytes(o->u), sg = prec_bytes(o->ug), sp = prec_bytes(o->up);
    const int64_t ldv = (n + 31) & ~int64_t(31);
    const int64_t nsl = (n + 31) >> 5;
    Carve cv{base, 0, (size_t)SPAI_NOALLOC_SCRATCH_BYTES};
    const size_t msg_bytes = sizeof(unsigned long long) * 4 * MAX_GRID * SLOT_WORDS;
    // control words: err[2], out[2], the CSR check flags, its[imax + 1], nbe[imax + 1], the norms
    const size_t ctrl_bytes = sizeof(int) * 6 + sizeof(int) * (imax + 1) + sizeof(double) * (imax + 1) +
                              sizeof(unsigned long long) * 3 + 64;
    unsigned long long* msg = (unsigned long long*)cv.take(msg_bytes);
    unsigned char* ctrl = (unsigned char*)cv.take(ctrl_bytes);
    void* x = cv.take((size_t)su * n);
    void* r = cv.take((size_t)su * n);
    void* wbuf = cv.take((size_t)sg * n);
    void* tbuf = cv.take((size_t)sp * n);
    void* V = cv.take((size_t)sg * ldv * (kmax + 1));
    double* R = (double*)cv.take(sizeof(double) * (size_t)(kmax + 1) * kmax);
    int64_t* aoff = (int64_t*)cv.take(sizeof(int64_t) * (nsl + 1));
    int32_t* aw = (int32_t*)cv.take(sizeof(int32_t) * nsl);
    int64_t* poff = P ? (int64_t*)cv.take(sizeof(int64_t) * (nsl + 1)) : nullptr;
    int32_t* pw = P ? (int32_t*)cv.take(sizeof(int32_t) * nsl) : nullptr;
    // CGS2: the partial dot products of every block and the counter of their barrier
    void* pvec = o->orth ? cv.take((size_t)sg * 2 * MAX_GRID * (kmax + 1)) : nullptr;
    if (!msg || !ctrl || !x || !r || !wbuf || !tbuf || !V || !R || !aoff || !aw || (P && (!poff || !pw)) ||
        (o->orth && !pvec))
        return SPAI_ERR_UNSUPPORTED;  // the problem does not fit the fixed scratch
    int* err = (int*)ctrl;
    int* outv = err + 2;
    int* csrf = outv + 2;                   // structural check flags of A and P
    unsigned* gcount = (unsigned*)(csrf + 1);
    int* its = csrf + 2;
    double* nbe = (double*)(((uintptr_t)(its + imax + 1) + 7) & ~uintptr_t(7));
    unsigned long long* norms = (unsigned long long*)(nbe + imax + 1);
    // the array keeps the previous call's contents: clear what must start at zero
    SPAI_CUDA_TRY(cudaMemsetAsync(msg, 0, msg_bytes, s));
    SPAI_CUDA_TRY(cudaMemsetAsync(ctrl, 0, ctrl_bytes, s));
    const int tb = 256;
    const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((n + tb - 1) / tb, (int64_t)num_sms * 32));
    const int gs = (int)std::max<int64_t>(1, std::min<int64_t>((nsl * 32 + tb - 1) / tb, (int64_t)num_sms * 16));
    int nl = 0;
    // the structural check of both device CSRs (rowptr order and range, columns in
    // [0, n) and ascending, no empty row of A) before any kernel indexes with them;
    // its flags come back with the SELL sizes below
    {
        const int gc = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * 8));
        k_csr_check<<<gc, 256, 0, s>>>(n, A->nnz, A->rowptr, A->col, csrf, 0);
        nl++;
        if (P) {
            // rows of P may be empty (a zero row of P is a valid preconditioner row)
            k_csr_check<<<gc, 256, 0, s>>>(n, P->nnz, P->rowptr, P->col, csrf, 1);
            nl++;
        }
        SPAI_CUDA_TRY(cudaGetLastError());
        int h_csr = 0;
        SPAI_CUDA_TRY(cudaMemcpyAsync(&h_csr, csrf, sizeof(int), cudaMemcpyDeviceToHost, s));
        SPAI_CUDA_TRY(cudaStreamSynchronize(s));
        if (h_csr & 1) return SPAI_ERR_INVALID_ARG;
        if (h_csr & 2) return SPAI_ERR_ZERO_ROW;
    }
    k_sell_width<<<gs, tb, 0, s>>>(n, A->rowptr, aw);
    k_scan_one_block<<<1, 1024, 0, s>>>(nsl, aw, aoff);
    nl += 2;
    if (P) {
        k_sell_width<<<gs, tb, 0, s>>>(n, P->rowptr, pw);
        k_scan_one_block<<<1, 1024, 0, s>>>(nsl, pw, poff);
        nl += 2;
    }
    int64_t tot[2] = {0, 0};
    SPAI_CUDA_TRY(cudaMemcpyAsync(&tot[0], aoff + nsl, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if (P) SPAI_CUDA_TRY(cudaMemcpyAsync(&tot[1], poff + nsl, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SPAI_CUDA_TRY(cudaStreamSynchronize(s));
    int32_t* acol = (int32_t*)cv.take(sizeof(int32_t) * std::max<int64_t>(tot[0], 1));
    void* aval = cv.take((size_t)sp * std::max<int64_t>(tot[0], 1));
    int32_t* pcol = P ? (int32_t*)cv.take(sizeof(int32_t) * std::max<int64_t>(tot[1], 1)) : nullptr;
    void* pval = P ? cv.take((size_t)sp * std::max<int64_t>(tot[1], 1)) : nullptr;
    if (!acol || !aval || (P && (!pcol || !pval))) return SPAI_ERR_UNSUPPORTED;
    if (o->up == SPAI_SINGLE) {
        k_sell_fill<float><<<gs, tb, 0, s>>>(n, A->rowptr, A->col, A->val, aoff, acol, (float*)aval);
        if (P) k_sell_fill<float><<<gs, tb, 0, s>>>(n, P->rowptr, P->col, P->val, poff, pcol, (float*)pval);
    } else {
        k_sell_fill<double><<<gs, tb, 0, s>>>(n, A->rowptr, A->col, A->val, aoff, acol, (double*)aval);
        if (P) k_sell_fill<double><<<gs, tb, 0, s>>>(n, P->rowptr, P->col, P->val, poff, pcol, (double*)pval);
    }
    nl += P ? 2 : 1;
    k_norms<<<gb, tb, 0, s>>>(n, A->rowptr, A->val, b, norms);
    nl++;
    {
        const int64_t* prp = P ? P->rowptr : nullptr;
        const int32_t* pci = P ? P->col : nullptr;
        const double* pvd = P ? P->val : nullptr;
#define X0D(S, TU) k_x0_dbl<S, TU><<<gb, tb, 0, s>>>(n, prp, pci, pvd, b, (TU*)x)
        if (o->u == SPAI_SINGLE) {
            if (o->uf == SPAI_HALF) X0D(__half, float);
            else if (o->uf == SPAI_SINGLE) X0D(float, float);
            else X0D(double, float);
        } else {
            if (o->uf == SPAI_HALF) X0D(__half, double);
            else if (o->uf == SPAI_SINGLE) X0D(float, double);
            else X0D(double, double);
        }
#undef X0D
        nl++;
    }
    SPAI_CUDA_TRY(cudaGetLastError());
    unsigned long long h_norms[3] = {0, 0, 0};
    SPAI_CUDA_TRY(cudaMemcpyAsync(h_norms, norms, sizeof(h_norms), cudaMemcpyDeviceToHost, s));
    SPAI_CUDA_TRY(cudaStreamSynchronize(s));
    IrArgs a;
    memset(&a, 0, sizeof(a));
    double anorm, bnorm;
    {
        long long t0 = (long long)h_norms[0], t1 = (long long)h_norms[1];
        memcpy(&anorm, &t0, 8);
        memcpy(&bnorm, &t1, 8);
    }
    const int q = (int)h_norms[2];
    a.n = n;
    a.A.off = aoff; a.A.col = acol; a.A.val = aval;
    if (P) { a.P.off = poff; a.P.col = pcol; a.P.val = pval; }
    a.arp = A->rowptr; a.aci = A->col; a.aval = A->val;
    a.b = b; a.x = x; a.r = r; a.wbuf = wbuf; a.tbuf = tbuf; a.V = V; a.ldv = ldv; a.R = R; a.msg = msg;
    a.msg2 = msg + 2 * MAX_GRID * SLOT_WORDS;
    a.err = err;
    int clk_khz = device_attr_cached(cudaDevAttrClockRate, device);
    if (clk_khz <= 0) clk_khz = 2000000;
    a.limit = (long long)clk_khz * 1000LL * 4;
    a.anorm = anorm; a.bnorm = bnorm; a.tau = o->tau;
    a.stop_tol = ir_stop_tol(o, q);
    a.kmax = kmax; a.imax = imax; a.stop_rule = o->stop;
    a.its = its; a.nbe = nbe; a.out = outv;
    a.side = o->side;
    a.orth = o->orth; a.pvec = pvec; a.gcount = gcount;
    const int rm = o->ur == SPAI_QUAD ? 2 : 1;
    int grid = 0;
    if (o->u == SPAI_DOUBLE) {
        if (o->ug == SPAI_DOUBLE) {
            if (o->up == SPAI_DOUBLE) rc = launch_ir_rm<double, double, double>(a, rm, num_sms, s, &grid);
            else rc = launch_ir_rm<double, double, float>(a, rm, num_sms, s, &grid);
        } else {
            if (o->up == SPAI_DOUBLE) rc = launch_ir_rm<double, float, double>(a, rm, num_sms, s, &grid);
            else rc = launch_ir_rm<double, float, float>(a, rm, num_sms, s, &grid);
        }
    } else {
        if (o->ug == SPAI_DOUBLE) {
            if (o->up == SPAI_DOUBLE) rc = launch_ir_rm<float, double, double>(a, rm, num_sms, s, &grid);
            else rc = launch_ir_rm<float, double, float>(a, rm, num_sms, s, &grid);
        } else {
            if (o->up == SPAI_DOUBLE) rc = launch_ir_rm<float, float, double>(a, rm, num_sms, s, &grid);
            else rc = launch_ir_rm<float, float, float>(a, rm, num_sms, s, &grid);
        }
    }
    if (rc) return rc;
    nl++;
    if (o->u == SPAI_SINGLE) k_to_double<float><<<gb, tb, 0, s>>>(n, (const float*)x, xout);
    else k_to_double<double><<<gb, tb, 0, s>>>(n, (const double*)x, xout);
    nl++;
    SPAI_CUDA_TRY(cudaGetLastError());
    int h_out[2] = {0, 0}, h_err = 0;
    SPAI_CUDA_TRY(cudaMemcpyAsync(h_out, outv, sizeof(h_out), cudaMemcpyDeviceToHost, s));
    SPAI_CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (st) {
        memset(st, 0, sizeof(*st));
        SPAI_CUDA_TRY(cudaMemcpyAsync(st->its, its, sizeof(int) * imax, cudaMemcpyDeviceToHost, s));
        SPAI_CUDA_TRY(cudaMemcpyAsync(st->nbe, nbe, sizeof(double) * (imax + 1), cudaMemcpyDeviceToHost, s));
    }
    SPAI_CUDA_TRY(cudaStreamSynchronize(s));
    if (h_err) return h_err;
    if (st) {
        st->steps = h_out[0];
        st->flags = h_out[1];
        for (int i = 0; i < st->steps; i++) st->total_its += st->its[i];
        for (int i = st->steps + 1; i <= SPAI_IR_MAX_STEPS; i++) st->nbe[i] = 0.0;
        st->final_nbe = st->nbe[st->steps];
        st->launches = nl;
        st->grid = grid;
        st->nnz_P = P ? P->nnz : 0;
    }
    if (h_out[1] & 8) return SPAI_ERR_NONFINITE;
    if (!(h_out[1] & 1) && o->stop != IR_STOP_FIXED) return SPAI_WARN_NOT_CONVERGED;
    return 0;
}
