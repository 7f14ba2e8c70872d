// Host-side objects behind the C ABI (context, preconditioner, device CSR).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <thread>
#include <vector>

#include "../../include/spai_ir.h"

// A CSR matrix resident on the device.  When `owned` is false the pointers
// are borrowed from the caller for the duration of one call.
struct DevCsr {
    int64_t n = 0, nnz = 0;
    int64_t* rowptr = nullptr;
    int32_t* col = nullptr;
    double* val = nullptr;
    bool owned = false;
};

// A matrix in SELL-32 layout (see gmres_ir.cu) with values in one precision.
struct SellMat {
    int64_t* off = nullptr;   // slice offsets, (n + 31) / 32 + 1
    int32_t* col = nullptr;
    void* val = nullptr;
    int64_t nnz = 0;          // stored entries, padding included
    int prec = SPAI_DOUBLE;
};

struct spai_precond_s {
    int device = 0;
    int64_t n = 0, nnz = 0;
    int64_t* rowptr = nullptr;   // n + 1
    int32_t* col = nullptr;      // nnz
    double* val = nullptr;       // nnz, unrounded mbar_k * d(J_k)
    SellMat sell_f16, sell_f32, sell_f64;  // lazily made SELL-32 copies in u_p = half / single / double
    void* val_uf = nullptr;      // copy rounded to u_f (used by x0 = P b)
    int uf = SPAI_DOUBLE;
    cudaStream_t stream = nullptr;  // the building context's stream (the default stream once it is gone)
    spai_ctx_s* owner = nullptr;    // the context that built it through spai_build, while it lives
};

struct ServeRequest;

struct spai_ctx_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0;
    int num_sms = 0;
    std::mutex mu;  // serialises the synchronous entry points
    // serving engine (capi.cu): an admission thread that uploads and builds
    // the preconditioners of every admitted group, a refinement thread that
    // solves prepared groups in batched launches; each on a stream of its own
    std::mutex qmu;
    std::condition_variable qcv;               // admission: new requests, freed budget, stop
    std::condition_variable rcv;               // refinement: prepared groups, stop
    std::deque<ServeRequest*> pending;         // submitted, not admitted
    std::deque<std::vector<ServeRequest*>> ready;  // admitted and prepared, not solved
    std::map<uint64_t, ServeRequest*> tickets;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> worker_streams;
    size_t in_use = 0;                         // estimated bytes of the admitted requests
    uint64_t qgen = 0;                         // bumped at every submission and release
    uint64_t next_ticket = 1;
    bool stopping = false;
    std::set<spai_precond_s*> live;  // preconditioners built by spai_build and not yet freed
};

// cudaDeviceGetAttribute, asked once per process for each (attribute, device); 0 on failure
int device_attr_cached(cudaDeviceAttr attr, int device);

// Let `kernel` launch with as much dynamic shared memory as the device's
// opt-in limit leaves beside its static shared memory; *dyn gets that size.
// The attribute is global to the kernel, so it is set to the maximum (once
// per kernel and device) rather than to one launch's size: with serving
// workers launching the same kernel from several threads, a per-launch value
// set by one thread could be lowered by another between its
// cudaFuncSetAttribute and its launch.
cudaError_t allow_max_dynamic_smem_ptr(const void* kernel, size_t* dyn);
template <class K>
inline cudaError_t allow_max_dynamic_smem(K* kernel, size_t* dyn = nullptr)
{
    size_t d = 0;
    cudaError_t e = allow_max_dynamic_smem_ptr((const void*)kernel, &d);
    if (dyn) *dyn = d;
    return e;
}

// stream-ordered device allocation helpers
int dev_alloc(void** p, size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);

// upload or borrow a CSR
int csr_to_device(const spai_csr* A, DevCsr* out, cudaStream_t s);
void csr_release(DevCsr* d, cudaStream_t s);
int csr_validate_host(const spai_csr* A);

// A build over the block-diagonal union of several matrices (spai_build_batch):
// rows ro[i] .. ro[i+1]-1 belong to matrix i.  The build then also writes, per
// matrix, stats[6 i .. 6 i + 5] = columns converged, columns stopped at the
// fill cap above eps, non-finite columns, max |I_k|, max |J_k| and nnz(P).
struct SpaiSegments {
    int count = 0;
    const int64_t* ro = nullptr;          // device, count + 1
    unsigned long long* stats = nullptr;  // device, 6 * count, zeroed by the caller
};

// phase implementations (spai_build.cu / gmres_ir.cu)
int spai_build_dev(int device, int num_sms, cudaStream_t s, const DevCsr& A, const spai_opts* o,
                   spai_precond* P_out, spai_stats* st, const SpaiSegments* seg = nullptr);
int gmres_ir_dev(int device, int num_sms, cudaStream_t s, const DevCsr& A, spai_precond P,
                 const double* b_dev, double* x_dev, const ir_opts* o, ir_stats* st);
// Many systems with the same options (see gmres_ir_solve_batch); status[i]
// receives each system's code (may be NULL).
int gmres_ir_batch_dev(int device, int num_sms, cudaStream_t s, int count, const DevCsr* A, const spai_precond* P,
                       const double* const* b_dev, double* const* x_dev, const ir_opts* o, ir_stats* st,
                       int* status);

int scan_counts(int64_t n, const int32_t* in, int64_t* out, cudaStream_t s);
int sell_build(int64_t n, const int64_t* rp, const int32_t* ci, const double* val, int prec, int num_sms,
               cudaStream_t s, SellMat* out, int* launches);
void sell_free(SellMat* m, cudaStream_t s);

// bytes the solve of an n x n system with nnz nonzeros may hold on the device
size_t estimate_footprint(int64_t n, int64_t nnz, const spai_opts* so, const ir_opts* io);
