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
#include <climits>
#include <cstdio>
#include <cstring>

#include "common.cuh"
#include "internal.h"

using namespace spai;

namespace {

constexpr int IR_THREADS = 1024;
constexpr int KMAX_LIMIT = 1024;

struct IrArgs {
    int64_t n;
    int64_t rb;                 // rows per block
    const int64_t* arp;
    const int32_t* aci;
    const double* aval;         // A in double (residual)
    const void* aval_p;         // A in u_p
    const int64_t* prp;         // P (may be null: P = I)
    const int32_t* pci;
    const void* pval_p;         // P in u_p
    const double* b;
    void* x;                    // n, precision u
    void* r;                    // n, precision u
    void* wbuf;                 // n, precision u_g: published w (or z)
    void* tbuf;                 // n, precision u_p: t = A v
    void* V;                    // ldv x (kmax + 1), precision u_g; only own rows are ever read back
    int64_t ldv;
    double* R;                  // (kmax + 1) x kmax column-major, written by block 0
    double* part;              // 2 slots x gridDim.x partials (two values each)
    GridBarrier gb;
    double anorm, bnorm, tau, stop_tol;
    int kmax, imax, stop_rule, la, lp;
    int* its;                   // imax
    double* nbe;                // imax + 1
    int* out;                   // [0] steps, [1] flags
};

struct IrShared {
    unsigned epoch;
    int flag;
    int slot;
    double bcast[2];
    double resid;
};

template <class T> __device__ __forceinline__ T ldv_(const T* p) { return ldcg(p); }

// Sum of a block-uniform value over all blocks; every block gets the same
// bits.  Returns false if the barrier failed.
// Lane-strided sum of the G partials of `slot`, all loads in flight at once
// (the partials live in L2; a dependent chain of loads would serialise their
// latency).  Fixed order: lane l adds l, l+32, l+64, ...
template <class T>
__device__ __forceinline__ T lane_partial_sum(const double* part, int slot, int comp)
{
    const unsigned G = gridDim.x, lane = threadIdx.x;
    const double* base = part + (size_t)slot * G * 2 + comp;
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; u++) {
        unsigned i = lane + 32u * u;
        v[u] = i < G ? __ldcg(base + (size_t)i * 2) : 0.0;
    }
    T acc = T(0);
#pragma unroll
    for (int u = 0; u < 8; u++) acc += (T)v[u];
    for (unsigned i = lane + 256u; i < G; i += 32) acc += (T)__ldcg(base + (size_t)i * 2);
    return acc;
}

template <class T>
__device__ bool gsum(const IrArgs& a, IrShared* sh, T v, T& out)
{
    const int slot = sh->slot;
    if (threadIdx.x == 0) a.part[(size_t)(slot * gridDim.x + blockIdx.x) * 2] = (double)v;
    if (!grid_sync(a.gb, &sh->epoch, &sh->flag)) return false;
    if (threadIdx.x < 32) {
        T acc = lane_partial_sum<T>(a.part, slot, 0);
        acc = warp_sum(acc);
        if (threadIdx.x == 0) { sh->bcast[0] = (double)acc; sh->slot = slot ^ 1; }
    }
    __syncthreads();
    out = (T)sh->bcast[0];
    return true;
}

// Max of two block-uniform values over all blocks.
__device__ bool gmax2(const IrArgs& a, IrShared* sh, double v0, double v1, double& o0, double& o1)
{
    const int slot = sh->slot;
    if (threadIdx.x == 0) {
        a.part[(size_t)(slot * gridDim.x + blockIdx.x) * 2] = v0;
        a.part[(size_t)(slot * gridDim.x + blockIdx.x) * 2 + 1] = v1;
    }
    if (!grid_sync(a.gb, &sh->epoch, &sh->flag)) return false;
    if (threadIdx.x < 32) {
        double m0 = 0.0, m1 = 0.0;
        for (unsigned i = threadIdx.x; i < gridDim.x; i += 32) {
            double p0 = __ldcg(&a.part[(size_t)(slot * gridDim.x + i) * 2]);
            double p1 = __ldcg(&a.part[(size_t)(slot * gridDim.x + i) * 2 + 1]);
            m0 = fmax(m0, p0);
            m1 = fmax(m1, p1);
        }
        m0 = warp_max(m0);
        m1 = warp_max(m1);
        if (threadIdx.x == 0) { sh->bcast[0] = m0; sh->bcast[1] = m1; sh->slot = slot ^ 1; }
    }
    __syncthreads();
    o0 = sh->bcast[0];
    o1 = sh->bcast[1];
    return true;
}

template <class T> __device__ __forceinline__ T to_t(double v) { return (T)v; }

// y[row] = sum_q M[row, q] * f(src[col]) with L lanes per row, for the
// block's rows; result handed to `store(row, value)`.
template <class TP, class Load, class Store>
__device__ __forceinline__ void spmv_rows(int64_t r0, int64_t r1, int L, const int64_t* __restrict__ rp,
                                          const int32_t* __restrict__ ci, const TP* __restrict__ mv, Load load,
                                          Store store)
{
    const int per = blockDim.x / L;
    const int g = threadIdx.x / L, l = threadIdx.x % L;
    for (int64_t base = r0; base < r1; base += per) {
        int64_t row = base + g;
        TP acc = TP(0);
        if (row < r1) {
            for (int64_t q = rp[row] + l; q < rp[row + 1]; q += L) acc = fma(mv[q], (TP)load(ci[q]), acc);
        }
        for (int o = L >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (row < r1 && l == 0) store(row, acc);
    }
}

template <class TU, class TG, class TP, int RM>
__global__ void __launch_bounds__(IR_THREADS, 1) k_ir(IrArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ IrShared shs;
    __shared__ TG redg[33];
    __shared__ double redd[33];
    IrShared* sh = &shs;
    const int kmax = a.kmax;
    double* cs = (double*)smem;           // kmax + 2
    double* sn = cs + (kmax + 2);          // kmax + 2
    double* g = sn + (kmax + 2);           // kmax + 2
    double* hc = g + (kmax + 2);           // kmax + 2
    double* yv = hc + (kmax + 2);          // kmax + 2
    TG* ws = (TG*)(yv + (kmax + 2));       // rb
    const int tid = threadIdx.x, BT = blockDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * a.rb;
    const int64_t r1 = min(a.n, r0 + a.rb);
    TU* x = (TU*)a.x;
    TU* r = (TU*)a.r;
    TG* wbuf = (TG*)a.wbuf;
    TP* tbuf = (TP*)a.tbuf;
    TG* V = (TG*)a.V;
    const TP* av = (const TP*)a.aval_p;
    const TP* pv = (const TP*)a.pval_p;
    if (tid == 0) { sh->epoch = 0; sh->slot = 0; sh->flag = 1; }
    __syncthreads();

    int steps = 0, flags = 0;
    // x (written by k_x0 before this launch) is visible to every block.
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
        rmax = block_max(rmax, redd);
        xmax = block_max(xmax, redd);
        double rn, xn;
        if (!gmax2(a, sh, rmax, xmax, rn, xn)) return;
        const double den = a.anorm * xn + a.bnorm;
        const double nb = den > 0.0 ? rn / den : 0.0;
        if (blockIdx.x == 0 && tid == 0) a.nbe[it] = nb;
        if (!isfinite(nb)) { flags |= 8; break; }
        if (a.stop_rule == IR_STOP_BACKWARD && nb <= a.stop_tol) { flags |= 1; break; }
        if (it == a.imax) { flags |= 2; break; }

        // ---------------- z = P r in u_p, stored in u_g; beta = ||z||
        TG part = TG(0);
        if (a.prp) {
            spmv_rows<TP>(r0, r1, a.lp, a.prp, a.pci, pv, [&](int c) { return (TP)ldcg(&r[c]); },
                          [&](int64_t row, TP v) { TG z = (TG)v; ws[row - r0] = z; wbuf[row] = z; });
        } else {
            for (int64_t row = r0 + tid; row < r1; row += BT) {
                TG z = (TG)(TP)r[row];
                ws[row - r0] = z;
                wbuf[row] = z;
            }
        }
        __syncthreads();
        for (int64_t row = r0 + tid; row < r1; row += BT) { TG z = ws[row - r0]; part = fma(z, z, part); }
        part = block_sum(part, redg);
        TG bsq;
        if (!gsum(a, sh, part, bsq)) return;
        const TG beta = sqrt(bsq);
        int k = 0;
        if (beta > TG(0)) {
            for (int64_t row = r0 + tid; row < r1; row += BT) V[row] = ws[row - r0] / beta;
            if (tid == 0) { g[0] = (double)beta; }
            TG hdiv = beta;
            bool done = false;
            for (int j = 0; j < kmax && !done; j++) {
                // ---- t = A v_j in u_p; v_j formed from the published w: fl(w / h)
                spmv_rows<TP>(r0, r1, a.la, a.arp, a.aci, av, [&](int c) { return (TP)(ldcg(&wbuf[c]) / hdiv); },
                              [&](int64_t row, TP v) { tbuf[row] = v; });
                if (!grid_sync(a.gb, &sh->epoch, &sh->flag)) return;
                // ---- w = P t in u_p, stored in u_g (own rows, shared memory)
                if (a.prp) {
                    spmv_rows<TP>(r0, r1, a.lp, a.prp, a.pci, pv, [&](int c) { return ldcg(&tbuf[c]); },
                                  [&](int64_t row, TP v) { ws[row - r0] = (TG)v; });
                } else {
                    for (int64_t row = r0 + tid; row < r1; row += BT) ws[row - r0] = (TG)ldcg(&tbuf[row]);
                }
                __syncthreads();
                // ---- modified Gram-Schmidt in u_g
                const TG* Vj = V + r0;  // column 0, own rows start
                part = TG(0);
                for (int64_t row = r0 + tid; row < r1; row += BT) part = fma(Vj[row - r0], ws[row - r0], part);
                for (int i = 0; i <= j; i++) {
                    part = block_sum(part, redg);
                    TG h;
                    if (!gsum(a, sh, part, h)) return;
                    if (tid == 0) hc[i] = (double)h;
                    const TG* Vi = V + (int64_t)i * a.ldv + r0;
                    const TG* Vn = V + (int64_t)(i + 1) * a.ldv + r0;
                    part = TG(0);
                    if (i < j) {
                        for (int64_t row = r0 + tid; row < r1; row += BT) {
                            TG wv = fma(-h, Vi[row - r0], ws[row - r0]);
                            ws[row - r0] = wv;
                            part = fma(Vn[row - r0], wv, part);
                        }
                    } else {
                        for (int64_t row = r0 + tid; row < r1; row += BT) {
                            TG wv = fma(-h, Vi[row - r0], ws[row - r0]);
                            ws[row - r0] = wv;
                            wbuf[row] = wv;
                            part = fma(wv, wv, part);
                        }
                    }
                }
                part = block_sum(part, redg);
                TG hsq;
                if (!gsum(a, sh, part, hsq)) return;
                const TG hn = sqrt(hsq);
                // ---- v_{j+1} = w / h_{j+1,j} (own rows)
                if (hn > TG(0)) {
                    TG* Vn = V + (int64_t)(j + 1) * a.ldv + r0;
                    for (int64_t row = r0 + tid; row < r1; row += BT) Vn[row - r0] = ws[row - r0] / hn;
                }
                // ---- Givens rotations in double (identical in every block)
                if (tid == 0) {
                    hc[j + 1] = (double)hn;
                    for (int i = 0; i < j; i++) {
                        double t0 = cs[i] * hc[i] + sn[i] * hc[i + 1];
                        hc[i + 1] = -sn[i] * hc[i] + cs[i] * hc[i + 1];
                        hc[i] = t0;
                    }
                    double dn = sqrt(hc[j] * hc[j] + hc[j + 1] * hc[j + 1]);
                    if (dn == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
                    else { cs[j] = hc[j] / dn; sn[j] = hc[j + 1] / dn; }
                    hc[j] = dn;
                    g[j + 1] = -sn[j] * g[j];
                    g[j] = cs[j] * g[j];
                    sh->resid = fabs(g[j + 1]) / (double)beta;
                    if (blockIdx.x == 0)
                        for (int i = 0; i <= j; i++) a.R[(size_t)j * (kmax + 1) + i] = hc[i];
                }
                __syncthreads();
                k = j + 1;
                hdiv = hn;
                if (hn == TG(0)) { flags |= 4; done = true; }
                else if (sh->resid <= a.tau) done = true;
            }
            // ---- y = R^{-1} g (double), d = V y in u_g, x = x + d in u
            if (!grid_sync(a.gb, &sh->epoch, &sh->flag)) return;  // R columns from block 0
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
            for (int64_t row = r0 + tid; row < r1; row += BT) {
                TG dsum = TG(0);
                for (int i = 0; i < k; i++) dsum = fma(V[(int64_t)i * a.ldv + row], (TG)yv[i], dsum);
                x[row] = (TU)((TU)x[row] + (TU)dsum);
            }
        }
        if (blockIdx.x == 0 && tid == 0) a.its[it] = k;
        steps = it + 1;
        // x must be complete before the next residual
        if (!grid_sync(a.gb, &sh->epoch, &sh->flag)) return;
    }
    if (blockIdx.x == 0 && tid == 0) {
        a.out[0] = steps;
        a.out[1] = flags;
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

__global__ void k_to_float(int64_t n, const double* __restrict__ x, float* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __double2float_rn(x[i]);
}

// ||A||_inf, ||b||_inf, and the largest row count q
__global__ void k_norms(int64_t n, const int64_t* __restrict__ rp, const double* __restrict__ val,
                        const double* __restrict__ b, unsigned long long* __restrict__ out)
{
    double an = 0.0, bn = 0.0;
    int q = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; p++) s += fabs(val[p]);
        an = fmax(an, s);
        bn = fmax(bn, fabs(b[i]));
        q = max(q, (int)(rp[i + 1] - rp[i]));
    }
    an = warp_max(an);
    bn = warp_max(bn);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q = max(q, __shfl_xor_sync(0xffffffffu, q, o));
    if ((threadIdx.x & 31) == 0) {
        // non-negative doubles order like their bit patterns
        atomicMax(&out[0], (unsigned long long)__double_as_longlong(an));
        atomicMax(&out[1], (unsigned long long)__double_as_longlong(bn));
        atomicMax(&out[2], (unsigned long long)q);
    }
}

int lanes_for(double avg)
{
    int L = 1;
    while (L < 32 && L < avg) L <<= 1;
    return L;
}

template <class TU, class TG, class TP, int RM>
int launch_ir(IrArgs& a, int num_sms, cudaStream_t s, size_t fixed_smem_per_row, int* grid_out)
{
    auto kern = k_ir<TU, TG, TP, RM>;
    int occ = 0;
    // choose the grid: at most the co-resident capacity, rows per block >= 256
    int64_t G = (a.n + 255) / 256;
    int maxg = 0;
    for (int attempt = 0; attempt < 2; attempt++) {
        int64_t g0 = G;
        size_t smem = 0;
        int64_t rb = (a.n + g0 - 1) / g0;
        smem = sizeof(double) * 5 * (a.kmax + 2) + rb * fixed_smem_per_row + 64;
        SPAI_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        SPAI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, IR_THREADS, smem));
        maxg = occ * num_sms;
        if (maxg < 1) return SPAI_ERR_UNSUPPORTED;
        if (G > maxg) G = maxg; else break;
    }
    if (G < 1) G = 1;
    a.rb = (a.n + G - 1) / G;
    G = (a.n + a.rb - 1) / a.rb;
    if (G < 1) G = 1;
    size_t smem = sizeof(double) * 5 * (a.kmax + 2) + a.rb * fixed_smem_per_row + 64;
    SPAI_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    SPAI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, IR_THREADS, smem));
    if ((int64_t)occ * num_sms < G) return SPAI_ERR_UNSUPPORTED;
    void* args[] = {(void*)&a};
    SPAI_CUDA_TRY(cudaLaunchCooperativeKernel((void*)kern, dim3((unsigned)G), dim3(IR_THREADS), args, smem, s));
    *grid_out = (int)G;
    return 0;
}

template <class TU, class TG, class TP>
int launch_ir_rm(IrArgs& a, int rm, int num_sms, cudaStream_t s, int* grid)
{
    size_t per_row = sizeof(TG);
    if (rm == 2) return launch_ir<TU, TG, TP, 2>(a, num_sms, s, per_row, grid);
    return launch_ir<TU, TG, TP, 1>(a, num_sms, s, per_row, grid);
}

int prec_bytes(int p) { return p == SPAI_HALF ? 2 : (p == SPAI_SINGLE ? 4 : 8); }

}  // namespace

int gmres_ir_dev(int device, int num_sms, cudaStream_t s, const DevCsr& A, spai_precond P,
                 const double* b, double* xout, const ir_opts* o, ir_stats* st)
{
    (void)device;
    const int64_t n = A.n;
    if (!o) return SPAI_ERR_INVALID_ARG;
    if (o->u != SPAI_SINGLE && o->u != SPAI_DOUBLE) return SPAI_ERR_UNSUPPORTED;
    if (o->ug != SPAI_SINGLE && o->ug != SPAI_DOUBLE) return SPAI_ERR_UNSUPPORTED;
    if (o->up != SPAI_SINGLE && o->up != SPAI_DOUBLE) return SPAI_ERR_UNSUPPORTED;
    if (o->ur != SPAI_DOUBLE && o->ur != SPAI_QUAD) return SPAI_ERR_UNSUPPORTED;
    if (o->uf != SPAI_HALF && o->uf != SPAI_SINGLE && o->uf != SPAI_DOUBLE) return SPAI_ERR_UNSUPPORTED;
    if (P && P->uf != o->uf) return SPAI_ERR_INVALID_ARG;
    if (o->ir_max_steps < 1 || o->ir_max_steps > SPAI_IR_MAX_STEPS) return SPAI_ERR_INVALID_ARG;
    if (!(o->tau >= 0.0)) return SPAI_ERR_INVALID_ARG;
    int kmax = o->gmres_max_it > 0 ? o->gmres_max_it : (int)std::min<int64_t>(n, 500);
    if (kmax > n) kmax = (int)n;
    if (kmax > KMAX_LIMIT) return SPAI_ERR_UNSUPPORTED;
    if (kmax < 1) kmax = 1;
    const int imax = o->ir_max_steps;

    int rc = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr, ek0 = nullptr, ek1 = nullptr;
    SPAI_CUDA_TRY(cudaEventCreate(&e0));
    SPAI_CUDA_TRY(cudaEventCreate(&e1));
    SPAI_CUDA_TRY(cudaEventCreate(&ek0));
    SPAI_CUDA_TRY(cudaEventCreate(&ek1));
    int nl = 0;  // kernels launched
    const int su = prec_bytes(o->u), sg = prec_bytes(o->ug), sp = prec_bytes(o->up);
    void *x = nullptr, *r = nullptr, *wbuf = nullptr, *tbuf = nullptr, *V = nullptr, *aval_p = nullptr;
    double *R = nullptr, *part = nullptr, *nbe = nullptr;
    int *its = nullptr, *outv = nullptr, *err = nullptr;
    unsigned* bar = nullptr;
    unsigned long long* norms = nullptr;
    unsigned long long h_norms[3] = {0, 0, 0};
    int h_out[2] = {0, 0}, h_err = 0;
    int grid = 0;
    const void* pval_p = nullptr;
    int64_t ldv = (n + 31) & ~int64_t(31);
    const int tb = 256;
    const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((n + tb - 1) / tb, (int64_t)num_sms * 32));
    IrArgs a;
    memset(&a, 0, sizeof(a));

#define TRY(x) do { rc = (x); if (rc) goto done; } while (0)
#define CTRY(x) do { if ((x) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; } } while (0)
    TRY(dev_alloc(&x, (size_t)su * n, s));
    TRY(dev_alloc(&r, (size_t)su * n, s));
    TRY(dev_alloc(&wbuf, (size_t)sg * n, s));
    TRY(dev_alloc(&tbuf, (size_t)sp * n, s));
    TRY(dev_alloc(&V, (size_t)sg * ldv * (kmax + 1), s));
    TRY(dev_alloc((void**)&R, sizeof(double) * (size_t)(kmax + 1) * kmax, s));
    TRY(dev_alloc((void**)&part, sizeof(double) * 2 * 2 * 4096, s));
    TRY(dev_alloc((void**)&nbe, sizeof(double) * (imax + 1), s));
    TRY(dev_alloc((void**)&its, sizeof(int) * (imax + 1), s));
    TRY(dev_alloc((void**)&outv, sizeof(int) * 2, s));
    TRY(dev_alloc((void**)&err, sizeof(int) * 2, s));
    TRY(dev_alloc((void**)&bar, sizeof(unsigned) * 2, s));
    TRY(dev_alloc((void**)&norms, sizeof(unsigned long long) * 3, s));
    CTRY(cudaMemsetAsync(norms, 0, sizeof(unsigned long long) * 3, s));
    CTRY(cudaMemsetAsync(its, 0, sizeof(int) * (imax + 1), s));
    CTRY(cudaMemsetAsync(outv, 0, sizeof(int) * 2, s));
    CTRY(cudaMemsetAsync(err, 0, sizeof(int) * 2, s));
    CTRY(cudaMemsetAsync(bar, 0, sizeof(unsigned) * 2, s));
    CTRY(cudaEventRecord(e0, s));
    // A in u_p
    if (o->up == SPAI_SINGLE) {
        TRY(dev_alloc(&aval_p, sizeof(float) * (A.nnz > 0 ? A.nnz : 1), s));
        k_to_float<<<gb, tb, 0, s>>>(A.nnz, A.val, (float*)aval_p);
        nl++;
    }
    // P in u_p
    if (P) {
        if (o->up == SPAI_SINGLE) {
            if (!P->val_f32) {
                TRY(dev_alloc((void**)&P->val_f32, sizeof(float) * (P->nnz > 0 ? P->nnz : 1), s));
                k_to_float<<<gb, tb, 0, s>>>(P->nnz, P->val, P->val_f32);
                nl++;
            }
            pval_p = P->val_f32;
        } else {
            pval_p = P->val;
        }
    }
    k_norms<<<gb, tb, 0, s>>>(n, A.rowptr, A.val, b, norms);
    nl++;
    CTRY(cudaMemcpyAsync(h_norms, norms, sizeof(h_norms), cudaMemcpyDeviceToHost, s));
    // x0 = P b in u_f, stored in u
    {
        const int64_t* prp = P ? P->rowptr : nullptr;
        const int32_t* pci = P ? P->col : nullptr;
        const void* pvf = P ? P->val_uf : nullptr;
#define X0(S, TU) k_x0<S, TU><<<gb, tb, 0, s>>>(n, prp, pci, (const S*)pvf, b, (TU*)x)
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
        nl++;
        CTRY(cudaGetLastError());
    }
    CTRY(cudaStreamSynchronize(s));
    {
        double anorm, bnorm;
        long long t0 = (long long)h_norms[0], t1 = (long long)h_norms[1];
        memcpy(&anorm, &t0, 8);
        memcpy(&bnorm, &t1, 8);
        const int q = (int)h_norms[2];
        const double uu = o->u == SPAI_SINGLE ? 5.9604644775390625e-08 : 1.1102230246251565e-16;
        a.n = n;
        a.arp = A.rowptr; a.aci = A.col; a.aval = A.val;
        a.aval_p = o->up == SPAI_SINGLE ? aval_p : (const void*)A.val;
        a.prp = P ? P->rowptr : nullptr;
        a.pci = P ? P->col : nullptr;
        a.pval_p = pval_p;
        a.b = b; a.x = x; a.r = r; a.wbuf = wbuf; a.tbuf = tbuf; a.V = V; a.ldv = ldv; a.R = R; a.part = part;
        a.gb.count = bar; a.gb.err = err;
        int clk_khz = 0;
        cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, device);
        if (clk_khz <= 0) clk_khz = 2000000;
        a.gb.limit = (long long)clk_khz * 1000LL * 4;  // about four seconds per wait
        a.anorm = anorm; a.bnorm = bnorm; a.tau = o->tau;
        a.stop_tol = o->stop_tol > 0 ? o->stop_tol : q * uu;
        a.kmax = kmax; a.imax = imax; a.stop_rule = o->stop;
        a.la = lanes_for(n > 0 ? (double)A.nnz / n : 1.0);
        a.lp = P ? lanes_for(n > 0 ? (double)P->nnz / n : 1.0) : 1;
        a.its = its; a.nbe = nbe; a.out = outv;
        const int rm = o->ur == SPAI_QUAD ? 2 : 1;
        CTRY(cudaEventRecord(ek0, s));
        if (o->u == SPAI_DOUBLE) {
            if (o->ug == SPAI_DOUBLE) {
                if (o->up == SPAI_DOUBLE) TRY((launch_ir_rm<double, double, double>(a, rm, num_sms, s, &grid)));
                else TRY((launch_ir_rm<double, double, float>(a, rm, num_sms, s, &grid)));
            } else {
                if (o->up == SPAI_DOUBLE) TRY((launch_ir_rm<double, float, double>(a, rm, num_sms, s, &grid)));
                else TRY((launch_ir_rm<double, float, float>(a, rm, num_sms, s, &grid)));
            }
        } else {
            if (o->ug == SPAI_DOUBLE) {
                if (o->up == SPAI_DOUBLE) TRY((launch_ir_rm<float, double, double>(a, rm, num_sms, s, &grid)));
                else TRY((launch_ir_rm<float, double, float>(a, rm, num_sms, s, &grid)));
            } else {
                if (o->up == SPAI_DOUBLE) TRY((launch_ir_rm<float, float, double>(a, rm, num_sms, s, &grid)));
                else TRY((launch_ir_rm<float, float, float>(a, rm, num_sms, s, &grid)));
            }
        }
    }
    CTRY(cudaEventRecord(ek1, s));
    nl++;
    if (o->u == SPAI_SINGLE) k_to_double<float><<<gb, tb, 0, s>>>(n, (const float*)x, xout);
    else k_to_double<double><<<gb, tb, 0, s>>>(n, (const double*)x, xout);
    nl++;
    CTRY(cudaGetLastError());
    CTRY(cudaEventRecord(e1, s));
    CTRY(cudaMemcpyAsync(h_out, outv, sizeof(h_out), cudaMemcpyDeviceToHost, s));
    CTRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (st) {
        memset(st->its, 0, sizeof(st->its));
        CTRY(cudaMemcpyAsync(st->its, its, sizeof(int) * imax, cudaMemcpyDeviceToHost, s));
        for (int i = 0; i <= SPAI_IR_MAX_STEPS; i++) st->nbe[i] = 0.0;
        CTRY(cudaMemcpyAsync(st->nbe, nbe, sizeof(double) * (imax + 1), cudaMemcpyDeviceToHost, s));
    }
    CTRY(cudaStreamSynchronize(s));
    if (h_err) { rc = h_err; goto done; }
    if (st) {
        st->steps = h_out[0];
        st->flags = h_out[1];
        st->total_its = 0;
        for (int i = 0; i < st->steps; i++) st->total_its += st->its[i];
        for (int i = st->steps + 1; i <= SPAI_IR_MAX_STEPS; i++) st->nbe[i] = 0.0;
        st->final_nbe = st->nbe[st->steps];
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        st->ms_ir = ms;
        cudaEventElapsedTime(&ms, ek0, ek1);
        st->ms_kernel = ms;
        st->launches += nl;
        st->grid = grid;
        st->nnz_P = P ? P->nnz : 0;
    }
    if (h_out[1] & 8) rc = SPAI_ERR_NONFINITE;
    else if (!(h_out[1] & 1) && o->stop == IR_STOP_BACKWARD) rc = SPAI_WARN_NOT_CONVERGED;
done:
#undef TRY
#undef CTRY
    dev_free(x, s); dev_free(r, s); dev_free(wbuf, s); dev_free(tbuf, s); dev_free(V, s); dev_free(aval_p, s);
    dev_free(R, s); dev_free(part, s); dev_free(nbe, s); dev_free(its, s); dev_free(outv, s); dev_free(err, s);
    dev_free(bar, s); dev_free(norms, s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (ek0) cudaEventDestroy(ek0);
    if (ek1) cudaEventDestroy(ek1);
    if (rc < 0) cudaStreamSynchronize(s);
    return rc;
}
