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
#include <map>
#include <set>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "ir_kernel.cuh"

using namespace spai;

namespace {

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
            if (c < len) { scol[o] = ci[b + c]; sval[o] = from_d<TP>(val[b + c]); }
            else { scol[o] = row < n ? (int32_t)row : 0; sval[o] = from_d<TP>(0.0); }
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

// the kernels of the run-time precision tuple (u, u_g, u_p), u_r and orth
int ir_kernels(int u, int ug, int up, int ur, int orth, IrKernels* k)
{
    const int rm = ur == SPAI_QUAD ? 2 : 1;
    const bool ls = orth == 2;
    const bool ud = u == SPAI_DOUBLE;
    if (ug == SPAI_HALF || up == SPAI_HALF) {
        k->one = nullptr;
        if (ug == SPAI_HALF && up == SPAI_HALF) (ud ? ir_kernels_dhh : ir_kernels_fhh)(rm, ls, k);
        else if (ug == SPAI_HALF && up == SPAI_SINGLE) (ud ? ir_kernels_dhf : ir_kernels_fhf)(rm, ls, k);
        else if (ug == SPAI_SINGLE && up == SPAI_HALF) (ud ? ir_kernels_dfh : ir_kernels_ffh)(rm, ls, k);
        return k->one ? 0 : SPAI_ERR_UNSUPPORTED;
    }
    const int key = (u == SPAI_DOUBLE) * 4 + (ug == SPAI_DOUBLE) * 2 + (up == SPAI_DOUBLE);
    switch (key) {
    case 0: ir_kernels_fff(rm, ls, k); break;
    case 1: ir_kernels_ffd(rm, ls, k); break;
    case 2: ir_kernels_fdf(rm, ls, k); break;
    case 3: ir_kernels_fdd(rm, ls, k); break;
    case 4: ir_kernels_dff(rm, ls, k); break;
    case 5: ir_kernels_dfd(rm, ls, k); break;
    case 6: ir_kernels_ddf(rm, ls, k); break;
    default: ir_kernels_ddd(rm, ls, k); break;
    }
    return k->one ? 0 : SPAI_ERR_UNSUPPORTED;
}

// One system on its own grid: one block per SM, at least 256 rows per
// block, rows per block a multiple of 32 so that blocks own whole SELL
// slices.  sg = sizeof(u_g).
int launch_ir(IrArgs& a, const IrKernels& K, int sg, int num_sms, cudaStream_t s, int* grid_out)
{
    // the one-reduction MGS on grids of 8 or more row blocks adds a block without
    // rows that runs the Givens rotations (FP64 work beside the other blocks'
    // inner products slowed both)
    const bool sblock = a.orth == 2 && a.gpub && std::min<int64_t>((a.n + 255) / 256, std::min(num_sms, MAX_GRID)) >= 9;
    int64_t G = std::min<int64_t>((a.n + 255) / 256, std::min(num_sms, MAX_GRID) - (sblock ? 1 : 0));
    if (G < 1) G = 1;
    a.rb = ((a.n + G - 1) / G + 31) & ~int64_t(31);
    G = (a.n + a.rb - 1) / a.rb;
    a.sblock = sblock ? 1 : 0;
    if (sblock) G += 1;
    // Gram-Schmidt group: on large grids the scalar rounds run among half the
    // blocks (each over two blocks' rows); a round among 76 blocks took
    // ~1.2 us against ~1.7 us among 152, which outweighs the extra barrier
    // that publishes w once per iteration.  CGS2 and the one-reduction MGS have
    // no scalar rounds.
    a.g2 = (!a.orth && G >= MGS_GROUP_MIN_GRID) ? (int)((G + 1) / 2) : 0;
    size_t dyn_max = 0;
    SPAI_CUDA_TRY(allow_max_dynamic_smem_ptr(K.one, &dyn_max));
    a.jl = a.orth == 2 ? ir_pick_jl(a.rb, a.kmax, dyn_max, sg) : 0;
    auto smem_for = [&](int g2) { return ir_smem_bytes(a.rb, a.kmax, g2, a.orth, a.jl, sg); };
    if (a.g2 && smem_for(a.g2) > dyn_max) a.g2 = 0;  // the doubled row range does not fit
    const size_t smem = smem_for(a.g2);
    if (smem > dyn_max) return SPAI_ERR_UNSUPPORTED;
    int occ = 0;
    SPAI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, K.one, K.threads, smem));
    if ((int64_t)occ * num_sms < G) return SPAI_ERR_UNSUPPORTED;
    void* args[] = {(void*)&a};
    SPAI_CUDA_TRY(cudaLaunchCooperativeKernel(K.one, dim3((unsigned)G), dim3(K.threads), args, smem, s));
    *grid_out = (int)G;
    return 0;
}

int prec_bytes(int p) { return p == SPAI_HALF ? 2 : (p == SPAI_SINGLE ? 4 : 8); }

// the preconditioner's cached SELL-32 copy in u_p
SellMat* sell_cache(spai_precond P, int up)
{
    return up == SPAI_HALF ? &P->sell_f16 : (up == SPAI_SINGLE ? &P->sell_f32 : &P->sell_f64);
}

}  // namespace

// SELL-32 copy of a CSR matrix with values rounded to `prec` (half, single or double),
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
    if (prec == SPAI_HALF) k_sell_fill<__half><<<gb, tb, 0, s>>>(n, rp, ci, val, out->off, out->col, (__half*)out->val);
    else if (prec == SPAI_SINGLE) k_sell_fill<float><<<gb, tb, 0, s>>>(n, rp, ci, val, out->off, out->col, (float*)out->val);
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
    void* L = nullptr;
    double* gpub = nullptr;
    void* arena = nullptr;  // one allocation holding all of the above
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
    if (o->ug != SPAI_HALF && o->ug != SPAI_SINGLE && o->ug != SPAI_DOUBLE) return SPAI_ERR_UNSUPPORTED;
    if (o->up != SPAI_HALF && o->up != SPAI_SINGLE && o->up != SPAI_DOUBLE) return SPAI_ERR_UNSUPPORTED;
    // half Krylov storage: with the one-reduction MGS, and beside single only
    if ((o->ug == SPAI_HALF || o->up == SPAI_HALF) &&
        (o->orth != 2 || o->ug == SPAI_DOUBLE || o->up == SPAI_DOUBLE))
        return SPAI_ERR_UNSUPPORTED;
    if (o->ur != SPAI_DOUBLE && o->ur != SPAI_QUAD) return SPAI_ERR_UNSUPPORTED;
    if (o->uf != SPAI_HALF && o->uf != SPAI_SINGLE && o->uf != SPAI_DOUBLE) return SPAI_ERR_UNSUPPORTED;
    if (o->ir_max_steps < 1 || o->ir_max_steps > SPAI_IR_MAX_STEPS) return SPAI_ERR_INVALID_ARG;
    if (!(o->tau >= 0.0)) return SPAI_ERR_INVALID_ARG;
    if (o->orth < 0 || o->orth > 2) return SPAI_ERR_INVALID_ARG;
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

// The job's buffers, carved from one allocation on s (one runtime call instead
// of one per buffer: a batch prepares hundreds of jobs); the control words
// (norms, exchange slots, step counts, flags, counters) come first and are
// cleared together.
int ir_job_alloc(IrJob& J, cudaStream_t s, const ir_opts* o)
{
    const int64_t n = J.n;
    const int su = prec_bytes(o->u), sg = prec_bytes(o->ug), sp = prec_bytes(o->up);
    const int64_t ldv = (n + 31) & ~int64_t(31);
    const int kmax = J.kmax, imax = J.imax;
    size_t off = 0;
    auto place = [&](size_t bytes) {
        off = (off + 255) & ~size_t(255);
        const size_t at = off;
        off += bytes;
        return at;
    };
    // [0..2] the norms and the longest row, [3] [4] SELL entry counts of A and P
    const size_t o_norms = place(sizeof(unsigned long long) * 5);
    const size_t o_msg = place(sizeof(unsigned long long) * 4 * MAX_GRID * SLOT_WORDS);
    const size_t o_its = place(sizeof(int) * (imax + 1));
    const size_t o_outv = place(sizeof(int) * 2);
    const size_t o_err = place(sizeof(int) * 2);
    const size_t o_gcount = o->orth ? place(sizeof(unsigned)) : 0;
    const size_t ctrl = off;
    const size_t o_x = place((size_t)su * n);
    const size_t o_r = place((size_t)su * n);
    const size_t o_wbuf = place((size_t)sg * n);
    const size_t o_tbuf = place((size_t)sp * n);
    const size_t o_V = place((size_t)sg * ldv * (kmax + 1));
    const size_t o_R = place(sizeof(double) * (size_t)(kmax + 1) * kmax);
    const size_t o_nbe = place(sizeof(double) * (imax + 1));
    // CGS2: 2 parities x blocks x (kmax + 1) partials; one-reduction MGS: 2 (kmax + 1) values
    // x blocks, then the 2 (kmax + 1) sums of the split reduction
    const size_t o_pvec = o->orth ? place((size_t)ir_scalar_bytes(sg) * (2 * MAX_GRID + (o->orth == 2 ? 2 : 0)) * (kmax + 1)) : 0;
    const size_t o_L = o->orth == 2 ? place((size_t)ir_scalar_bytes(sg) * ((size_t)(kmax + 1) * kmax / 2 + 1)) : 0;
    const size_t o_gpub = o->orth == 2 ? place(sizeof(double) * (kmax + 2)) : 0;
    int rc = dev_alloc(&J.arena, off, s);
    if (rc) return rc;
    unsigned char* base = (unsigned char*)J.arena;
    J.norms = (unsigned long long*)(base + o_norms);
    J.msg = (unsigned long long*)(base + o_msg);
    J.its = (int*)(base + o_its);
    J.outv = (int*)(base + o_outv);
    J.err = (int*)(base + o_err);
    J.gcount = o->orth ? (unsigned*)(base + o_gcount) : nullptr;
    J.x = base + o_x;
    J.r = base + o_r;
    J.wbuf = base + o_wbuf;
    J.tbuf = base + o_tbuf;
    J.V = base + o_V;
    J.R = (double*)(base + o_R);
    J.nbe = (double*)(base + o_nbe);
    J.pvec = o->orth ? base + o_pvec : nullptr;
    J.L = o->orth == 2 ? base + o_L : nullptr;
    J.gpub = o->orth == 2 ? (double*)(base + o_gpub) : nullptr;
    if (cudaMemsetAsync(base, 0, ctrl, s) != cudaSuccess) return SPAI_ERR_CUDA;
    return 0;
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
        cache = sell_cache(P, o->up);
        if (!cache->off) {
            rc = sell_begin(J.n, P->rowptr, num_sms, s, cache, nl);
            if (rc) return rc;
            if (cudaMemcpyAsync(J.norms + 4, cache->off + nsl, 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                return SPAI_ERR_CUDA;
        } else {
            cache = nullptr;  // already made
        }
        J.Ps = sell_cache(P, o->up);
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
    a.orth = o->orth; a.pvec = J.pvec; a.gcount = J.gcount; a.L = J.L; a.gpub = J.gpub; a.side = o->side;
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
    dev_free(J.arena, s);
    J.arena = nullptr;
    J.gpub = nullptr;
    J.x = J.r = J.wbuf = J.tbuf = J.V = J.pvec = J.L = nullptr;
    J.R = J.nbe = nullptr;
    J.its = J.outv = J.err = nullptr;
    J.msg = J.norms = nullptr;
    J.gcount = nullptr;
}

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
        IrKernels K;
        TRY(ir_kernels(o->u, o->ug, o->up, o->ur, o->orth, &K));
        TRY(launch_ir(J.a, K, prec_bytes(o->ug), num_sms, s, &grid));
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
// Batched refinement (gmres_ir_solve_batch): many independent systems in
// persistent cooperative launches.  Cooperative launches of separate systems
// hardly overlap on the GPU (16 solves of an n = 4096 system: 111 ms one
// after another, 66-70 ms from 2 or 4 host threads), while one such system
// keeps only 16 of 152 SMs busy.  One launch splits the co-resident grid
// into teams; each team takes the next system of its class (larger first) as
// soon as it is done with its last one, so systems with many GMRES
// iterations do not hold up the others' SMs.  A system's team size is a
// function of its order and options alone (batch_team: about
// BATCH_ROWS_PER_BLOCK rows per block, raised until a block's rows fit its
// shared memory, at most 16 blocks), so its result is the same whatever
// batch it is solved in; the systems of one team size form a class, and the classes'
// teams share the launch (one team per class, then teams given one at a time
// to the class with the most rows per team; a team whose class is done takes
// systems of classes with smaller teams).  Systems of more than
// BATCH_SOLO_N rows, which fill the GPU alone, run on a grid of their own
// (the single-system path).  All systems of a launch are prepared before it
// (their buffers coexist).
// ====================================================================

namespace {

// Rows per block of a batched system.  A batch is bound by the bytes each
// block streams per iteration, not by its grid-wide waits, so fewer and
// fuller blocks per system solve more systems at once: the refinement of the
// 512-system batch (n 2e3..5e4, one-reduction MGS) took 0.31 s of kernel
// time at 8192 rows per block against 0.41 s at 2048 and 0.69 s at 1024
// (the textbook MGS: 0.35 s, 0.76 s, 1.39 s).
constexpr int64_t BATCH_ROWS_PER_BLOCK = 8192;
constexpr int64_t BATCH_SOLO_N = 65536;

int batch_team(int64_t n)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>(16, (n + BATCH_ROWS_PER_BLOCK / 2) / BATCH_ROWS_PER_BLOCK));
}

struct BatchRun {
    int device, num_sms;
    cudaStream_t s;
    const ir_opts* o;
    std::vector<IrJob>* jobs;
    // classes of one launch: (team size, systems by decreasing order), larger teams first
    const std::vector<std::pair<int, std::vector<int>>>* classes;
    int* nl;
    float* ms_kernel;
    IrKernels K;
    int sg;                    // sizeof(u_g)

    size_t smem_for(const IrArgs& a) const { return ir_smem_bytes(a.rb, a.kmax, a.g2, a.orth, a.jl, sg); }

    int run()
    {
        const void* kern = K.batch;
        const int threads = K.threads;
        size_t dyn_max = 0;
        SPAI_CUDA_TRY(allow_max_dynamic_smem_ptr(kern, &dyn_max));
        std::vector<IrJob>& J = *jobs;
        const int ncls = (int)classes->size();
        std::vector<int> order;        // args order: class by class
        std::vector<int> cs(ncls + 1, 0);
        for (int c = 0; c < ncls; c++) {
            const auto& v = (*classes)[c].second;
            order.insert(order.end(), v.begin(), v.end());
            cs[c + 1] = (int)order.size();
        }
        const int count = (int)order.size();
        int rc = 0;
        // preparation without a wait per system: buffers, SELL offsets, norms and x0
        // for all systems, then one copy of every SELL size and norm to the host,
        // then the SELL fills
        std::vector<char> pbuild(count, 0);
        std::set<spai_precond> building;
        unsigned long long* d_slots = nullptr;
        rc = dev_alloc((void**)&d_slots, sizeof(unsigned long long) * 5 * count, s);
        if (rc) return rc;
        for (int i = 0; i < count; i++) {
            IrJob& jb = J[order[i]];
            if (!rc) rc = ir_job_alloc(jb, s, o);
            if (!rc) rc = sell_begin(jb.n, jb.A->rowptr, num_sms, s, &jb.As, nl);
            const int64_t nsl = (jb.n + 31) >> 5;
            unsigned long long* slot = d_slots + 5 * (size_t)i;
            if (!rc && jb.P) {
                SellMat* cache = sell_cache(jb.P, o->up);
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
            for (spai_precond P : building) sell_free(sell_cache(P, o->up), s);
        };
        std::vector<unsigned long long> hs(5 * (size_t)count, 0);
        if (!rc && cudaMemcpyAsync(hs.data(), d_slots, sizeof(unsigned long long) * hs.size(), cudaMemcpyDeviceToHost, s) !=
                       cudaSuccess)
            rc = SPAI_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess && !rc) rc = SPAI_ERR_CUDA;
        dev_free(d_slots, s);
        if (rc) { drop_started(); return rc; }
        for (int i = 0; i < count; i++) {
            IrJob& jb = J[order[i]];
            const unsigned long long* h = hs.data() + 5 * (size_t)i;
            for (int k = 0; k < 3; k++) jb.h_norms[k] = h[k];
            rc = sell_finish(jb.n, jb.A->rowptr, jb.A->col, jb.A->val, o->up, num_sms, s, &jb.As, (int64_t)h[3], nl);
            if (!rc && pbuild[i])
                rc = sell_finish(jb.n, jb.P->rowptr, jb.P->col, jb.P->val, o->up, num_sms, s,
                                 sell_cache(jb.P, o->up), (int64_t)h[4], nl);
            if (rc) { drop_started(); return rc; }
        }
        // arguments in claim order, every system prepared for its class's team size
        std::vector<IrArgs> h(count);
        size_t smem = 0;
        std::vector<double> work(ncls, 0.0);
        for (int c = 0; c < ncls; c++) {
            const int T = (*classes)[c].first;
            for (int q = cs[c]; q < cs[c + 1]; q++) {
                IrJob& jb = J[order[q]];
                ir_job_args(jb, device, o);
                IrArgs& a = jb.a;
                a.G = T;
                a.rb = std::max<int64_t>(32, ((jb.n + T - 1) / T + 31) & ~int64_t(31));
                a.g2 = 0;
                a.block0 = 0;
                a.jl = a.orth == 2 ? ir_pick_jl(a.rb, a.kmax, dyn_max, sg) : 0;
                smem = std::max(smem, smem_for(a));
                h[q] = a;
                work[c] += (double)jb.n;
            }
        }
        if (smem > dyn_max) return SPAI_ERR_UNSUPPORTED;
        int occ = 0;
        SPAI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem));
        // teams: one per class, then one more at a time to the class with the most
        // work per team (rows as the measure), while blocks are left
        const int gmax = occ * num_sms;
        std::vector<int> teams(ncls, 1);
        int used = 0;
        for (int c = 0; c < ncls; c++) used += (*classes)[c].first;
        if (used > gmax) return SPAI_ERR_UNSUPPORTED;
        for (;;) {
            int best = -1;
            double bw = 0.0;
            for (int c = 0; c < ncls; c++) {
                const int T = (*classes)[c].first;
                if (teams[c] >= cs[c + 1] - cs[c] || used + T > gmax) continue;
                const double w = work[c] / teams[c];
                if (best < 0 || w > bw) { best = c; bw = w; }
            }
            if (best < 0) break;
            teams[best]++;
            used += (*classes)[best].first;
        }
        std::vector<int> tb(1, 0), tc;
        for (int c = 0; c < ncls; c++)
            for (int t = 0; t < teams[c]; t++) {
                tb.push_back(tb.back() + (*classes)[c].first);
                tc.push_back(c);
            }
        const int nteams = (int)tc.size();
        IrArgs* d_args = nullptr;
        unsigned* d_next = nullptr;
        unsigned long long* d_claim = nullptr;
        int* d_plan = nullptr;
        const int plan_ints = (nteams + 1) + nteams + (ncls + 1);
        std::vector<int> hp;
        hp.insert(hp.end(), tb.begin(), tb.end());
        hp.insert(hp.end(), tc.begin(), tc.end());
        hp.insert(hp.end(), cs.begin(), cs.end());
        rc = dev_alloc((void**)&d_args, sizeof(IrArgs) * count, s);
        if (!rc) rc = dev_alloc((void**)&d_next, sizeof(unsigned) * ncls, s);
        if (!rc) rc = dev_alloc((void**)&d_claim, sizeof(unsigned long long) * nteams, s);
        if (!rc) rc = dev_alloc((void**)&d_plan, sizeof(int) * plan_ints, s);
        if (!rc && cudaMemcpyAsync(d_args, h.data(), sizeof(IrArgs) * count, cudaMemcpyHostToDevice, s) != cudaSuccess)
            rc = SPAI_ERR_CUDA;
        if (!rc && cudaMemcpyAsync(d_plan, hp.data(), sizeof(int) * plan_ints, cudaMemcpyHostToDevice, s) != cudaSuccess)
            rc = SPAI_ERR_CUDA;
        if (!rc && cudaMemsetAsync(d_next, 0, sizeof(unsigned) * ncls, s) != cudaSuccess) rc = SPAI_ERR_CUDA;
        if (!rc && cudaMemsetAsync(d_claim, 0, sizeof(unsigned long long) * nteams, s) != cudaSuccess) rc = SPAI_ERR_CUDA;
        cudaEvent_t k0 = nullptr, k1 = nullptr;
        if (!rc && (cudaEventCreate(&k0) != cudaSuccess || cudaEventCreate(&k1) != cudaSuccess)) rc = SPAI_ERR_CUDA;
        if (!rc) {
            const IrArgs* pa = d_args;
            BatchPlan plan{d_plan, d_plan + nteams + 1, d_plan + 2 * nteams + 1, nteams, ncls};
            long long limit = h[0].limit;
            void* args[] = {(void*)&pa, (void*)&plan, (void*)&d_next, (void*)&d_claim, (void*)&limit};
            cudaEventRecord(k0, s);
            if (cudaLaunchCooperativeKernel(kern, dim3((unsigned)tb.back()), dim3(threads), args, smem, s) != cudaSuccess)
                rc = SPAI_ERR_CUDA;
            cudaEventRecord(k1, s);
            (*nl)++;
        }
        for (int i = 0; i < count; i++)
            if (!rc) rc = ir_job_collect(J[order[i]], num_sms, s, o, nl);
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
        dev_free(d_plan, s);
        return rc;
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
    IrKernels K;
    rc = ir_kernels(o->u, o->ug, o->up, o->ur, o->orth, &K);
    if (rc) return rc;
    size_t dyn_max = 0;
    SPAI_CUDA_TRY(allow_max_dynamic_smem_ptr(K.batch, &dyn_max));
    // the team sizes (the batch_team of the order, raised until a block's rows fit its
    // shared memory), then the systems that run alone
    std::map<int, std::vector<int>> byteam;
    std::vector<int> solo;
    std::vector<int> grid_of(count, 0);
    const int sg = prec_bytes(o->ug);
    for (int i : order) {
        const IrJob& jb = jobs[i];
        int T = jb.n > BATCH_SOLO_N ? 17 : batch_team(jb.n);
        for (; T <= 16; T++) {
            const int64_t rb = std::max<int64_t>(32, ((jb.n + T - 1) / T + 31) & ~int64_t(31));
            const int jl = o->orth == 2 ? ir_pick_jl(rb, jb.kmax, dyn_max, sg) : 0;
            if (ir_smem_bytes(rb, jb.kmax, 0, o->orth, jl, sg) <= dyn_max) break;
        }
        if (T > 16) solo.push_back(i);
        else byteam[T].push_back(i);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SPAI_CUDA_TRY(cudaEventCreate(&e0));
    SPAI_CUDA_TRY(cudaEventCreate(&e1));
    int nl = 0;
    float ms_kernel = 0.f;
    cudaEventRecord(e0, s);
    if (!rc && !byteam.empty()) {
        // all team sizes in one launch, larger teams first
        std::vector<std::pair<int, std::vector<int>>> classes(byteam.rbegin(), byteam.rend());
        BatchRun B{device, num_sms, s, o, &jobs, &classes, &nl, &ms_kernel, K, prec_bytes(o->ug)};
        rc = B.run();
        for (const auto& c : classes)
            for (int i : c.second) grid_of[i] = c.first;
    }
    for (int i : solo) {
        if (rc) break;
        IrJob& J = jobs[i];
        rc = ir_job_prepare(J, num_sms, s, o, &nl);
        if (!rc) {
            ir_job_args(J, device, o);
            cudaEvent_t k0 = nullptr, k1 = nullptr;
            if (cudaEventCreate(&k0) != cudaSuccess || cudaEventCreate(&k1) != cudaSuccess) rc = SPAI_ERR_CUDA;
            if (!rc) cudaEventRecord(k0, s);
            if (!rc) rc = launch_ir(J.a, K, prec_bytes(o->ug), num_sms, s, &grid_of[i]);
            if (!rc) {
                cudaEventRecord(k1, s);
                nl++;
                rc = ir_job_collect(J, num_sms, s, o, &nl);
            }
            if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = SPAI_ERR_CUDA;
            if (!rc) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, k0, k1);
                ms_kernel += ms;
            }
            if (k0) cudaEventDestroy(k0);
            if (k1) cudaEventDestroy(k1);
        }
    }
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
            st[i].grid = grid_of[i];
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
    if (P && (P->n != A->n || P->nnz < 0 || !P->rowptr || !P->col || !P->val)) return SPAI_ERR_INVALID_ARG;
    if (A->n > INT32_MAX) return SPAI_ERR_UNSUPPORTED;
    // the options of gmres_ir_solve, less half Krylov storage
    if (o->ug == SPAI_HALF || o->up == SPAI_HALF) return SPAI_ERR_UNSUPPORTED;
    {
        const int rc = ir_check_opts(o);
        if (rc) return rc;
    }
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
    // (scalars in u_g's arithmetic type, as the allocating path sizes them)
    void* pvec = o->orth ? cv.take((size_t)ir_scalar_bytes(sg) * (2 * MAX_GRID + (o->orth == 2 ? 2 : 0)) * (kmax + 1))
                         : nullptr;
    void* Lrows = o->orth == 2 ? cv.take((size_t)ir_scalar_bytes(sg) * ((size_t)(kmax + 1) * kmax / 2 + 1)) : nullptr;
    double* gpub = o->orth == 2 ? (double*)cv.take(sizeof(double) * (kmax + 2)) : nullptr;
    if (!msg || !ctrl || !x || !r || !wbuf || !tbuf || !V || !R || !aoff || !aw || (P && (!poff || !pw)) ||
        (o->orth && !pvec) || (o->orth == 2 && (!Lrows || !gpub)))
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
    a.orth = o->orth; a.pvec = pvec; a.gcount = gcount; a.L = Lrows; a.gpub = gpub;
    int grid = 0;
    {
        IrKernels K;
        rc = ir_kernels(o->u, o->ug, o->up, o->ur, o->orth, &K);
        if (!rc) rc = launch_ir(a, K, prec_bytes(o->ug), num_sms, s, &grid);
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
