// The C ABI (include/spai_ir.h): contexts, preconditioner objects, host <->
// device marshalling and the serving queue.  All numerical work is done by
// the kernels in spai_build.cu and gmres_ir.cu.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "internal.h"

static thread_local cudaError_t g_last_cuda = cudaSuccess;
void spai_set_last_cuda_error(cudaError_t e) { g_last_cuda = e; }

// Device memory comes from one stream-ordered pool per device that keeps
// freed blocks for reuse (unlimited release threshold) instead of returning
// them to the driver at every synchronisation: re-mapping the Krylov basis
// and the SPAI work arrays on every solve cost about 2 ms per solve at
// n = 262144.  spai_ctx_destroy trims the pool back to what is in use.
constexpr int SPAI_BATCH_STREAMS = 8;  // concurrent builds in spai_build_batch

static std::mutex g_pool_mu;
static std::mutex g_live_mu;  // guards spai_ctx_s::live and spai_precond_s::owner / stream
static cudaMemPool_t g_pool[64];

static cudaMemPool_t device_pool(int dev)
{
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        unsigned long long thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        // no reuse across streams through inserted dependencies: concurrent
        // builds and serving requests on different streams would otherwise
        // wait on one another's frees
        int no = 0;
        cudaMemPoolSetAttribute(pool, cudaMemPoolReuseFollowEventDependencies, &no);
        cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
        g_pool[dev] = pool;
    }
    return g_pool[dev];
}

static void trim_device_pool(int dev)
{
    if (dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (g_pool[dev]) cudaMemPoolTrimTo(g_pool[dev], 0);
}

// Device attributes are fixed for the life of the process; some queries
// (the SM clock rate) cost ~0.6 ms each on this driver, so they are asked
// once per device and attribute.
int device_attr_cached(cudaDeviceAttr attr, int device)
{
    static std::mutex mu;
    static std::map<std::pair<int, int>, int> cache;
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_pair((int)attr, device);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int v = 0;
    if (cudaDeviceGetAttribute(&v, attr, device) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cache[key] = v;
    return v;
}

cudaError_t allow_max_dynamic_smem_ptr(const void* kernel, size_t* dyn)
{
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_pair(kernel, dev);
    auto it = done.find(key);
    if (it != done.end()) {
        *dyn = it->second;
        return cudaSuccess;
    }
    const int optin = device_attr_cached(cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    // static and dynamic shared memory together may not exceed the opt-in limit
    const int d = optin - (int)fa.sharedSizeBytes;
    if (d <= 0) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, d);
    if (e != cudaSuccess) return e;
    done[key] = (size_t)d;
    *dyn = (size_t)d;
    return cudaSuccess;
}

int dev_alloc(void** p, size_t bytes, cudaStream_t s)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SPAI_ERR_CUDA;
    cudaMemPool_t pool = device_pool(dev);
    cudaError_t e = pool ? cudaMallocFromPoolAsync(p, bytes, pool, s) : cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? SPAI_ERR_NO_MEMORY : SPAI_ERR_CUDA;
    }
    return 0;
}

void dev_free(void* p, cudaStream_t s)
{
    if (p) cudaFreeAsync(p, s);
}

int csr_validate_host(const spai_csr* A)
{
    if (!A || A->n < 1 || A->nnz < 0 || !A->rowptr || !A->col || !A->val) return SPAI_ERR_INVALID_ARG;
    if (A->n > INT32_MAX) return SPAI_ERR_UNSUPPORTED;
    if (A->on_device) return 0;  // device arrays: csr_check_device, before the kernels use them
    if (A->rowptr[0] != 0 || A->rowptr[A->n] != A->nnz) return SPAI_ERR_INVALID_ARG;
    for (int64_t i = 0; i < A->n; i++) {
        int64_t b = A->rowptr[i], e = A->rowptr[i + 1];
        if (e < b) return SPAI_ERR_INVALID_ARG;
        if (e == b) return SPAI_ERR_ZERO_ROW;
        for (int64_t q = b; q < e; q++) {
            int32_t c = A->col[q];
            if (c < 0 || c >= A->n) return SPAI_ERR_INVALID_ARG;
            if (q > b && A->col[q - 1] >= c) return SPAI_ERR_INVALID_ARG;
        }
    }
    return 0;
}

// The structural check of every row on the device (k_csr_check, common.cuh):
// for host inputs after the copy (the O(1) checks run on the host first; a
// host loop over a matrix of millions of entries cost milliseconds per call),
// for device inputs before any kernel indexes with them.
int csr_check_device(const DevCsr& A, int num_sms, cudaStream_t s)
{
    int* flags = nullptr;
    int rc = dev_alloc((void**)&flags, sizeof(int), s);
    if (rc) return rc;
    int h = 0;
    const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((A.n + 255) / 256, (int64_t)num_sms * 8));
    if (cudaMemsetAsync(flags, 0, sizeof(int), s) != cudaSuccess) rc = SPAI_ERR_CUDA;
    if (!rc) {
        k_csr_check<<<gb, 256, 0, s>>>(A.n, A.nnz, A.rowptr, A.col, flags, 0);
        if (cudaGetLastError() != cudaSuccess) rc = SPAI_ERR_CUDA;
    }
    if (!rc && cudaMemcpyAsync(&h, flags, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) rc = SPAI_ERR_CUDA;
    if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = SPAI_ERR_CUDA;
    dev_free(flags, s);
    if (rc) return rc;
    return (h & 1) ? SPAI_ERR_INVALID_ARG : ((h & 2) ? SPAI_ERR_ZERO_ROW : 0);
}

// csr_validate_host over many matrices on several host threads (a batch of
// hundreds of matrices holds ~1e8 entries); the error of the first failing
// matrix in index order.
int csr_validate_many(const spai_csr* A, int count)
{
    std::vector<int> rcs(count, 0);
    const unsigned hc = std::thread::hardware_concurrency();
    const int nt = std::max(1, std::min<int>(count, (int)std::min<unsigned>(hc ? hc : 1, 16)));
    std::atomic<int> next{0};
    std::vector<std::thread> th;
    for (int t = 0; t < nt; t++)
        th.emplace_back([&] {
            for (int i = next++; i < count; i = next++) rcs[i] = csr_validate_host(&A[i]);
        });
    for (auto& t : th) t.join();
    for (int i = 0; i < count; i++)
        if (rcs[i]) return rcs[i];
    return 0;
}

int csr_check_args(const spai_csr* A)
{
    if (!A || A->n < 1 || A->nnz < 0 || !A->rowptr || !A->col || !A->val) return SPAI_ERR_INVALID_ARG;
    if (A->n > INT32_MAX) return SPAI_ERR_UNSUPPORTED;
    if (A->on_device) return 0;
    if (A->rowptr[0] != 0 || A->rowptr[A->n] != A->nnz) return SPAI_ERR_INVALID_ARG;
    return 0;
}

int csr_to_device(const spai_csr* A, DevCsr* out, cudaStream_t s)
{
    out->n = A->n;
    out->nnz = A->nnz;
    if (A->on_device) {
        out->rowptr = const_cast<int64_t*>(A->rowptr);
        out->col = const_cast<int32_t*>(A->col);
        out->val = const_cast<double*>(A->val);
        out->owned = false;
        return 0;
    }
    int rc;
    if ((rc = dev_alloc((void**)&out->rowptr, sizeof(int64_t) * (A->n + 1), s))) return rc;
    if ((rc = dev_alloc((void**)&out->col, sizeof(int32_t) * std::max<int64_t>(A->nnz, 1), s))) return rc;
    if ((rc = dev_alloc((void**)&out->val, sizeof(double) * std::max<int64_t>(A->nnz, 1), s))) return rc;
    out->owned = true;
    SPAI_CUDA_TRY(cudaMemcpyAsync(out->rowptr, A->rowptr, sizeof(int64_t) * (A->n + 1), cudaMemcpyHostToDevice, s));
    SPAI_CUDA_TRY(cudaMemcpyAsync(out->col, A->col, sizeof(int32_t) * A->nnz, cudaMemcpyHostToDevice, s));
    SPAI_CUDA_TRY(cudaMemcpyAsync(out->val, A->val, sizeof(double) * A->nnz, cudaMemcpyHostToDevice, s));
    return 0;
}

void csr_release(DevCsr* d, cudaStream_t s)
{
    if (d->owned) {
        dev_free(d->rowptr, s);
        dev_free(d->col, s);
        dev_free(d->val, s);
    }
    d->rowptr = nullptr;
    d->col = nullptr;
    d->val = nullptr;
    d->owned = false;
}

size_t estimate_footprint(int64_t n, int64_t nnz, const spai_opts* so, const ir_opts* io)
{
    size_t F = so ? (size_t)so->max_fill : 1;
    size_t kmax = io && io->gmres_max_it > 0 ? (size_t)io->gmres_max_it : (size_t)std::min<int64_t>(n, 500);
    size_t N = (size_t)n;
    size_t a = (size_t)nnz * 12 + (N + 1) * 8;                         // A
    size_t spai = so ? N * F * 24 + N * 48 + (size_t)nnz * 4 : 0;    // SPAI scratch
    size_t p = so ? N * F * 24 + (N + 1) * 8 : 0;                     // P (double + u_f + f32 + col)
    size_t ir = N * 8 * (kmax + 1) + N * 48 + (kmax + 2) * (kmax + 1) * 8 + (size_t)nnz * 4;
    return a + std::max(spai + p, p + ir) + (1u << 20);
}

// ------------------------------------------------------------------ serving

// Continuous batching.  solver_submit queues a request and returns; the
// admission thread admits every waiting request whose estimated footprint
// fits what the budget has left (a request passed over for longer than
// SERVE_MAX_BYPASS_MS is then admitted before any later one), uploads the
// admitted group, builds its preconditioners (fixed patterns: one build over
// the block-diagonal union, as spai_build_batch) and hands the group to the
// refinement thread, which solves it with the batched refinement
// (gmres_ir_batch_dev: teams of blocks sized by each system's order, larger
// systems on a grid of their own).  Requests that arrive while a group is
// being solved are admitted and prepared meanwhile (the admission thread's
// kernels share the GPU with the running refinement) and are solved in the
// next launch; each request's A, P, b and x stay on the device until its
// group is done.  A request's result depends only on the request: the union
// build gives each matrix its single-build preconditioner, and a system's
// team size is a function of its order.
constexpr double SERVE_MAX_BYPASS_MS = 200.0;

struct ServeRequest {
    uint64_t ticket = 0;
    int64_t n = 0, nnz = 0;
    std::vector<int64_t> rowptr;
    std::vector<int32_t> col;
    std::vector<double> val, b, x;
    spai_opts so{};
    ir_opts io{};
    bool has_so = false;
    size_t bytes = 0;
    std::chrono::steady_clock::time_point t_submit;
    bool done = false;
    int status = 0;
    ir_stats st{};
    // device state while admitted
    DevCsr dA;
    double* db = nullptr;
    double* dx = nullptr;
    spai_precond P = nullptr;
    int spai_rc = 0;
};

static void serve_release(spai_ctx ctx, ServeRequest* r, cudaStream_t s)
{
    if (r->P) spai_precond_free(r->P);
    r->P = nullptr;
    dev_free(r->db, s);
    dev_free(r->dx, s);
    r->db = r->dx = nullptr;
    csr_release(&r->dA, s);
}

// requests of one group share their options (one batched launch)
static bool same_opts(const ServeRequest* a, const ServeRequest* b)
{
    if (a->has_so != b->has_so || memcmp(&a->io, &b->io, sizeof(ir_opts)) != 0) return false;
    return !a->has_so || memcmp(&a->so, &b->so, sizeof(spai_opts)) == 0;
}

static void serve_finish(spai_ctx ctx, const std::vector<ServeRequest*>& g, cudaStream_t s)
{
    cudaStreamSynchronize(s);
    for (ServeRequest* r : g) serve_release(ctx, r, s);
    cudaStreamSynchronize(s);
    {
        std::lock_guard<std::mutex> lk(ctx->qmu);
        for (ServeRequest* r : g) {
            ctx->in_use -= r->bytes;
            r->done = true;
        }
        ctx->qgen++;
    }
    ctx->qcv.notify_all();
}

static int spai_build_union(spai_ctx ctx, cudaStream_t s, int lo, int hi, const spai_csr* A, const spai_opts* opts,
                            spai_precond* P_out, spai_stats* st, int* rcs);

// Upload a group and build its preconditioners (admission thread).  Requests
// that fail are finished at once with their error; the rest go to the
// refinement thread.
static void serve_prepare(spai_ctx ctx, std::vector<ServeRequest*>& g, cudaStream_t s)
{
    std::vector<ServeRequest*> ok;
    for (ServeRequest* r : g) {
        spai_csr A{r->n, r->nnz, r->rowptr.data(), r->col.data(), r->val.data(), 0};
        int rc = csr_to_device(&A, &r->dA, s);
        if (!rc) rc = dev_alloc((void**)&r->db, sizeof(double) * r->n, s);
        if (!rc) rc = dev_alloc((void**)&r->dx, sizeof(double) * r->n, s);
        if (!rc && cudaMemcpyAsync(r->db, r->b.data(), sizeof(double) * r->n, cudaMemcpyHostToDevice, s) != cudaSuccess)
            rc = SPAI_ERR_CUDA;
        r->status = rc;
    }
    const ServeRequest* g0 = g.front();
    if (g0->has_so) {
        std::vector<ServeRequest*> todo;
        for (ServeRequest* r : g)
            if (r->status == 0) todo.push_back(r);
        const int cnt = (int)todo.size();
        std::vector<spai_csr> As(cnt);
        std::vector<spai_precond> Ps(cnt, nullptr);
        std::vector<spai_stats> sts(cnt);
        std::vector<int> rcs(cnt, 0);
        for (int i = 0; i < cnt; i++) {
            const DevCsr& d = todo[i]->dA;
            As[i] = spai_csr{d.n, d.nnz, d.rowptr, d.col, d.val, 1};
            memset(&sts[i], 0, sizeof(spai_stats));
        }
        bool built = false;
        if (cnt > 1 && !g0->so.adaptive && (g0->so.side == 0 || g0->so.side == 1))
            built = spai_build_union(ctx, s, 0, cnt, As.data(), &g0->so, Ps.data(), sts.data(), rcs.data()) == 0;
        if (!built) {
            for (int i = 0; i < cnt; i++) {
                if (Ps[i]) { spai_precond_free(Ps[i]); Ps[i] = nullptr; }
                memset(&sts[i], 0, sizeof(spai_stats));
                rcs[i] = spai_build_dev(ctx->device, ctx->num_sms, s, todo[i]->dA, &g0->so, &Ps[i], &sts[i]);
            }
        }
        for (int i = 0; i < cnt; i++) {
            ServeRequest* r = todo[i];
            r->P = Ps[i];
            r->st.ms_spai = sts[i].ms;
            r->st.launches = sts[i].launches;
            if (rcs[i] < 0) r->status = rcs[i];
            else r->spai_rc = rcs[i];
        }
    }
    cudaStreamSynchronize(s);
    std::vector<ServeRequest*> failed;
    for (ServeRequest* r : g) (r->status < 0 ? failed : ok).push_back(r);
    if (!failed.empty()) serve_finish(ctx, failed, s);
    if (!ok.empty()) {
        {
            std::lock_guard<std::mutex> lk(ctx->qmu);
            ctx->ready.push_back(std::move(ok));
        }
        ctx->rcv.notify_all();
    }
}

static void serve_admission_loop(spai_ctx ctx)
{
    cudaSetDevice(ctx->device);
    cudaStream_t s = ctx->worker_streams[0];
    uint64_t seen = 0;
    for (;;) {
        std::vector<ServeRequest*> take;
        {
            std::unique_lock<std::mutex> lk(ctx->qmu);
            ctx->qcv.wait(lk, [&] { return ctx->stopping || (!ctx->pending.empty() && ctx->qgen != seen); });
            if (ctx->stopping) return;
            seen = ctx->qgen;
            const auto now = std::chrono::steady_clock::now();
            bool head_only = false;
            for (auto it = ctx->pending.begin(); it != ctx->pending.end();) {
                ServeRequest* r = *it;
                if (r->bytes <= ctx->budget - ctx->in_use) {
                    ctx->in_use += r->bytes;
                    take.push_back(r);
                    it = ctx->pending.erase(it);
                    continue;
                }
                // the oldest request that does not fit: after waiting long enough it
                // keeps the freed budget for itself
                if (it == ctx->pending.begin() &&
                    std::chrono::duration<double, std::milli>(now - r->t_submit).count() > SERVE_MAX_BYPASS_MS)
                    head_only = true;
                if (head_only) break;
                ++it;
            }
        }
        // groups of requests with the same options, in arrival order
        while (!take.empty()) {
            std::vector<ServeRequest*> g, rest;
            for (ServeRequest* r : take) (same_opts(take.front(), r) ? g : rest).push_back(r);
            serve_prepare(ctx, g, s);
            take.swap(rest);
        }
    }
}

static void serve_refine_loop(spai_ctx ctx)
{
    cudaSetDevice(ctx->device);
    cudaStream_t s = ctx->worker_streams[1];
    for (;;) {
        std::vector<ServeRequest*> g;
        {
            std::unique_lock<std::mutex> lk(ctx->qmu);
            ctx->rcv.wait(lk, [&] { return ctx->stopping || !ctx->ready.empty(); });
            if (ctx->stopping) return;
            // every prepared group with the same options as the oldest joins its launch
            g = std::move(ctx->ready.front());
            ctx->ready.pop_front();
            for (auto it = ctx->ready.begin(); it != ctx->ready.end();) {
                if (same_opts(g.front(), it->front())) {
                    g.insert(g.end(), it->begin(), it->end());
                    it = ctx->ready.erase(it);
                } else {
                    ++it;
                }
            }
        }
        const int cnt = (int)g.size();
        std::vector<DevCsr> As(cnt);
        std::vector<spai_precond> Ps(cnt);
        std::vector<const double*> bs(cnt);
        std::vector<double*> xs(cnt);
        std::vector<ir_stats> sts(cnt);
        std::vector<int> status(cnt, 0);
        for (int i = 0; i < cnt; i++) {
            As[i] = g[i]->dA;
            As[i].owned = false;
            if (g[i]->P) g[i]->P->stream = s;  // its frees and SELL copies go to this thread's stream now
            Ps[i] = g[i]->P;
            bs[i] = g[i]->db;
            xs[i] = g[i]->dx;
            memset(&sts[i], 0, sizeof(ir_stats));
        }
        int rc = gmres_ir_batch_dev(ctx->device, ctx->num_sms, s, cnt, As.data(), Ps.data(), bs.data(), xs.data(),
                                    &g.front()->io, sts.data(), status.data());
        for (int i = 0; i < cnt; i++) {
            ServeRequest* r = g[i];
            int ri = rc < 0 ? rc : status[i];
            if (ri >= 0) {
                r->x.resize(r->n);
                if (cudaMemcpyAsync(r->x.data(), r->dx, sizeof(double) * r->n, cudaMemcpyDeviceToHost, s) != cudaSuccess)
                    ri = SPAI_ERR_CUDA;
            }
            const double ms_spai = r->st.ms_spai;
            const int nl = r->st.launches;
            r->st = sts[i];
            r->st.ms_spai = ms_spai;
            r->st.launches += nl;
            if (r->P) r->st.nnz_P = r->P->nnz;
            r->status = ri < 0 ? ri : (ri > 0 ? ri : r->spai_rc);
        }
        if (rc == SPAI_ERR_CUDA) {
            const cudaError_t e = cudaGetLastError();
            fprintf(stderr, "spai serving: a batch of %d requests failed: %s\n", cnt, cudaGetErrorString(e));
        }
        serve_finish(ctx, g, s);
    }
}

extern "C" {

int spai_ctx_create(spai_ctx* out, int device, void* cuda_stream, size_t hbm_budget_bytes)
{
    if (!out) return SPAI_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    SPAI_CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return SPAI_ERR_INVALID_ARG;
    SPAI_CUDA_TRY(cudaSetDevice(device));
    int coop = 0;
    SPAI_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device));
    if (!coop) return SPAI_ERR_UNSUPPORTED;
    spai_ctx c = new spai_ctx_s();
    c->device = device;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return SPAI_ERR_CUDA; }
        c->own_stream = true;
    }
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    c->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.9 * (double)fr);
    *out = c;
    return 0;
}

void spai_ctx_destroy(spai_ctx c)
{
    if (!c) return;
    {
        std::lock_guard<std::mutex> lk(c->qmu);
        c->stopping = true;
    }
    c->qcv.notify_all();
    c->rcv.notify_all();
    for (auto& t : c->workers) t.join();
    cudaSetDevice(c->device);
    for (auto& g : c->ready)
        for (ServeRequest* r : g) serve_release(c, r, c->stream);
    for (auto s : c->worker_streams) cudaStreamDestroy(s);
    for (auto& kv : c->tickets) delete kv.second;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    {
        // preconditioners that outlive the context are freed on the default stream
        std::lock_guard<std::mutex> lk(g_live_mu);
        for (spai_precond_s* P : c->live) {
            P->stream = 0;
            P->owner = nullptr;
        }
        c->live.clear();
    }
    if (c->own_stream) cudaStreamDestroy(c->stream);
    trim_device_pool(c->device);
    delete c;
}

int spai_build(spai_ctx ctx, const spai_csr* A, const spai_opts* opts, spai_precond* P_out, spai_stats* st)
{
    if (!ctx || !A || !opts || !P_out) return SPAI_ERR_INVALID_ARG;
    *P_out = nullptr;
    int rc = csr_check_args(A);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ctx->mu);
    SPAI_CUDA_TRY(cudaSetDevice(ctx->device));
    DevCsr dA;
    rc = csr_to_device(A, &dA, ctx->stream);
    if (!rc) rc = csr_check_device(dA, ctx->num_sms, ctx->stream);
    if (!rc) rc = spai_build_dev(ctx->device, ctx->num_sms, ctx->stream, dA, opts, P_out, st);
    csr_release(&dA, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    if (*P_out) {
        std::lock_guard<std::mutex> lk2(g_live_mu);
        (*P_out)->owner = ctx;
        ctx->live.insert(*P_out);
    }
    return rc;
}

}  // extern "C"

// ------------------------------------------------------------------ batched SPAI over a block-diagonal union

// the segment holding position g: the largest i with off[i] <= g
__device__ __forceinline__ int segment_of(const int64_t* __restrict__ off, int count, int64_t g)
{
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The matrices' rows were copied to their places in the union (rowptr without
// its last entry); shift row pointers by the matrix's first nonzero and
// column indices by its first row, and close the row pointers.
__global__ void k_union_shift(int count, const int64_t* __restrict__ ro, const int64_t* __restrict__ zo, int64_t N,
                              int64_t nnz, int64_t* __restrict__ rp, int32_t* __restrict__ col)
{
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = t0; g < N; g += st) rp[g] += zo[segment_of(ro, count, g)];
    for (int64_t q = t0; q < nnz; q += st) col[q] += (int32_t)ro[segment_of(zo, count, q)];
    if (t0 == 0) rp[N] = nnz;
}

struct PartPtrs {
    int64_t* rp;
    int32_t* col;
    double* val;
    void* vuf;
};

// P of the union, cut into the matrices' own preconditioners: rows of block
// i (rows ro[i] .. ro[i+1]-1, nonzeros pz[i] .. pz[i+1]-1) with columns
// shifted back by ro[i]
__global__ void k_split_rows(int count, const int64_t* __restrict__ ro, int64_t N, const int64_t* __restrict__ prp,
                             const PartPtrs* __restrict__ parts)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x) {
        const int i = segment_of(ro, count, g);
        const int64_t base = prp[ro[i]], r = g - ro[i];
        parts[i].rp[r] = prp[g] - base;
        if (g + 1 == ro[i + 1]) parts[i].rp[r + 1] = prp[g + 1] - base;
    }
}

template <class S>
__global__ void k_split_nz(int count, const int64_t* __restrict__ ro, const int64_t* __restrict__ pz, int64_t nnz,
                           const int32_t* __restrict__ col, const double* __restrict__ val, const S* __restrict__ vuf,
                           const PartPtrs* __restrict__ parts)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x) {
        const int i = segment_of(pz, count, q);
        const int64_t t = q - pz[i];
        parts[i].col[t] = col[q] - (int32_t)ro[i];
        parts[i].val[t] = val[q];
        ((S*)parts[i].vuf)[t] = vuf[q];
    }
}

// Bytes one union build of n rows and nnz nonzeros may hold: the union's A,
// the build's scratch and P (twice for the right construction's transposes)
// and the split copies of P.
static size_t union_footprint(int64_t n, int64_t nnz, const spai_opts* o)
{
    const size_t F = (size_t)o->max_fill, N = (size_t)n, Z = (size_t)nnz;
    size_t b = estimate_footprint(n, nnz, o, nullptr) + N * F * 24 + (N + 1) * 8;
    if (o->side == 1) b += Z * 12 + N * 8 + N * F * 16;
    return b;
}

// Matrices lo .. hi-1 built as one block-diagonal matrix: one pass of every
// kernel of the build instead of one per matrix.  Columns of a fixed pattern
// are independent and each is computed by the kernel its own shadow size
// selects, so every preconditioner is the one spai_build gives for its
// matrix, bit for bit.  Returns 0 with every handle set, or an error (the
// caller then builds these matrices one by one, which attributes it).
static int spai_build_union(spai_ctx ctx, cudaStream_t s, int lo, int hi, const spai_csr* A, const spai_opts* opts,
                            spai_precond* P_out, spai_stats* st, int* rcs)
{
    const int count = hi - lo;
    std::vector<int64_t> ro(count + 1, 0), zo(count + 1, 0);
    for (int i = 0; i < count; i++) {
        ro[i + 1] = ro[i] + A[lo + i].n;
        zo[i + 1] = zo[i] + A[lo + i].nnz;
    }
    const int64_t N = ro[count], Z = zo[count];
    int rc = 0;
    DevCsr U;
    U.n = N;
    U.nnz = Z;
    U.owned = true;
    int64_t *dro = nullptr, *dzo = nullptr, *dpz = nullptr;
    int* dflags = nullptr;
    unsigned long long* dstats = nullptr;
    PartPtrs* dparts = nullptr;
    spai_precond PU = nullptr;
    std::vector<spai_precond> parts(count, nullptr);
    std::vector<unsigned long long> hs(6 * (size_t)count, 0);
    std::vector<int> hflags(count, 0);
    spai_stats su;
    memset(&su, 0, sizeof(su));
    bool want_cols = false;
    std::vector<double> colres;
    std::vector<int32_t> nJ, nI, fl;
    const size_t ssz = opts->uf == SPAI_HALF ? 2 : (opts->uf == SPAI_SINGLE ? 4 : 8);
    const int tb = 256;
    int nl = 0;
#define TRYU(x) do { rc = (x); if (rc) goto done; } while (0)
#define CUDAU(x) do { if ((x) != cudaSuccess) { rc = SPAI_ERR_CUDA; goto done; } } while (0)
    TRYU(dev_alloc((void**)&dro, sizeof(int64_t) * (count + 1), s));
    TRYU(dev_alloc((void**)&dzo, sizeof(int64_t) * (count + 1), s));
    TRYU(dev_alloc((void**)&dpz, sizeof(int64_t) * (count + 1), s));
    TRYU(dev_alloc((void**)&dflags, sizeof(int) * count, s));
    TRYU(dev_alloc((void**)&dstats, sizeof(unsigned long long) * 6 * count, s));
    TRYU(dev_alloc((void**)&U.rowptr, sizeof(int64_t) * (N + 1), s));
    TRYU(dev_alloc((void**)&U.col, sizeof(int32_t) * std::max<int64_t>(Z, 1), s));
    TRYU(dev_alloc((void**)&U.val, sizeof(double) * std::max<int64_t>(Z, 1), s));
    CUDAU(cudaMemsetAsync(dflags, 0, sizeof(int) * count, s));
    CUDAU(cudaMemsetAsync(dstats, 0, sizeof(unsigned long long) * 6 * count, s));
    CUDAU(cudaMemcpyAsync(dro, ro.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s));
    CUDAU(cudaMemcpyAsync(dzo, zo.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s));
    {
        // device inputs are checked where they are, before anything reads them by index
        bool any_dev = false;
        for (int i = 0; i < count; i++) {
            const spai_csr& a = A[lo + i];
            if (!a.on_device) continue;
            any_dev = true;
            const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((a.n + 255) / 256, (int64_t)ctx->num_sms * 8));
            k_csr_check<<<gb, 256, 0, s>>>(a.n, a.nnz, a.rowptr, a.col, dflags + i, 0);
            nl++;
        }
        if (any_dev) {
            CUDAU(cudaGetLastError());
            CUDAU(cudaMemcpyAsync(hflags.data(), dflags, sizeof(int) * count, cudaMemcpyDeviceToHost, s));
            CUDAU(cudaStreamSynchronize(s));
            for (int i = 0; i < count; i++)
                if (hflags[i]) { rc = (hflags[i] & 1) ? SPAI_ERR_INVALID_ARG : SPAI_ERR_ZERO_ROW; goto done; }
        }
    }
    for (int i = 0; i < count; i++) {
        const spai_csr& a = A[lo + i];
        const cudaMemcpyKind kind = a.on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        CUDAU(cudaMemcpyAsync(U.rowptr + ro[i], a.rowptr, sizeof(int64_t) * a.n, kind, s));
        CUDAU(cudaMemcpyAsync(U.col + zo[i], a.col, sizeof(int32_t) * a.nnz, kind, s));
        CUDAU(cudaMemcpyAsync(U.val + zo[i], a.val, sizeof(double) * a.nnz, kind, s));
    }
    {
        const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((std::max(N, Z) + tb - 1) / tb, (int64_t)ctx->num_sms * 16));
        k_union_shift<<<gb, tb, 0, s>>>(count, dro, dzo, N, Z, U.rowptr, U.col);
        nl++;
        CUDAU(cudaGetLastError());
    }
    for (int i = 0; i < count && !want_cols; i++)
        want_cols = st && (st[lo + i].colres || st[lo + i].nJ || st[lo + i].nI || st[lo + i].flags);
    if (want_cols) {
        colres.resize(N); nJ.resize(N); nI.resize(N); fl.resize(N);
        su.colres = colres.data(); su.nJ = nJ.data(); su.nI = nI.data(); su.flags = fl.data();
    }
    {
        SpaiSegments seg;
        seg.count = count;
        seg.ro = dro;
        seg.stats = dstats;
        rc = spai_build_dev(ctx->device, ctx->num_sms, s, U, opts, &PU, &su, &seg);
        if (rc < 0) goto done;
        rc = 0;
    }
    CUDAU(cudaMemcpyAsync(hs.data(), dstats, sizeof(unsigned long long) * 6 * count, cudaMemcpyDeviceToHost, s));
    CUDAU(cudaStreamSynchronize(s));
    {
        std::vector<int64_t> pz(count + 1, 0);
        for (int i = 0; i < count; i++) pz[i + 1] = pz[i] + (int64_t)hs[6 * (size_t)i + 5];
        if (pz[count] != PU->nnz) { rc = SPAI_ERR_INTERNAL; goto done; }
        std::vector<PartPtrs> hp(count);
        for (int i = 0; i < count; i++) {
            spai_precond P = new spai_precond_s();
            parts[i] = P;
            P->n = A[lo + i].n;
            P->nnz = pz[i + 1] - pz[i];
            P->uf = opts->uf;
            P->stream = s;
            P->device = ctx->device;
            const int64_t z = std::max<int64_t>(P->nnz, 1);
            TRYU(dev_alloc((void**)&P->rowptr, sizeof(int64_t) * (P->n + 1), s));
            TRYU(dev_alloc((void**)&P->col, sizeof(int32_t) * z, s));
            TRYU(dev_alloc((void**)&P->val, sizeof(double) * z, s));
            TRYU(dev_alloc(&P->val_uf, ssz * z, s));
            hp[i] = PartPtrs{P->rowptr, P->col, P->val, P->val_uf};
        }
        TRYU(dev_alloc((void**)&dparts, sizeof(PartPtrs) * count, s));
        CUDAU(cudaMemcpyAsync(dparts, hp.data(), sizeof(PartPtrs) * count, cudaMemcpyHostToDevice, s));
        CUDAU(cudaMemcpyAsync(dpz, pz.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s));
        const int64_t ZP = PU->nnz;
        const int gr = (int)std::max<int64_t>(1, std::min<int64_t>((N + tb - 1) / tb, (int64_t)ctx->num_sms * 16));
        const int gz = (int)std::max<int64_t>(1, std::min<int64_t>((ZP + tb - 1) / tb, (int64_t)ctx->num_sms * 16));
        k_split_rows<<<gr, tb, 0, s>>>(count, dro, N, PU->rowptr, dparts);
        if (ZP > 0) {
            if (opts->uf == SPAI_HALF)
                k_split_nz<__half><<<gz, tb, 0, s>>>(count, dro, dpz, ZP, PU->col, PU->val, (const __half*)PU->val_uf, dparts);
            else if (opts->uf == SPAI_SINGLE)
                k_split_nz<float><<<gz, tb, 0, s>>>(count, dro, dpz, ZP, PU->col, PU->val, (const float*)PU->val_uf, dparts);
            else
                k_split_nz<double><<<gz, tb, 0, s>>>(count, dro, dpz, ZP, PU->col, PU->val, (const double*)PU->val_uf, dparts);
        }
        nl += 2;
        CUDAU(cudaGetLastError());
        CUDAU(cudaStreamSynchronize(s));
    }
    for (int i = 0; i < count; i++) {
        const unsigned long long* h = &hs[6 * (size_t)i];
        if (st) {
            spai_stats& o = st[lo + i];
            const int64_t r0 = ro[i], n = A[lo + i].n;
            if (o.colres) memcpy(o.colres, colres.data() + r0, sizeof(double) * n);
            if (o.nJ) memcpy(o.nJ, nJ.data() + r0, sizeof(int32_t) * n);
            if (o.nI) memcpy(o.nI, nI.data() + r0, sizeof(int32_t) * n);
            if (o.flags) memcpy(o.flags, fl.data() + r0, sizeof(int32_t) * n);
            o.n = n;
            o.nnz_P = (int64_t)h[5];
            o.cols_converged = (int64_t)h[0];
            o.cols_fillcap = (int64_t)h[1];
            o.cols_nonfinite = (int64_t)h[2];
            o.max_I = (int)h[3];
            o.max_J = (int)h[4];
            // one pass built them all: its time and launches
            o.ms = su.ms;
            o.ms_kernel = su.ms_kernel;
            o.launches = su.launches + nl;
        }
        rcs[lo + i] = h[2] > 0 ? SPAI_ERR_NONFINITE : (h[1] > 0 ? SPAI_WARN_FILLCAP : 0);
        P_out[lo + i] = parts[i];
        parts[i] = nullptr;
    }
done:
#undef TRYU
#undef CUDAU
    if (rc) cudaGetLastError();
    for (auto P : parts)
        if (P) spai_precond_free(P);
    if (PU) spai_precond_free(PU);
    csr_release(&U, s);
    dev_free(dro, s); dev_free(dzo, s); dev_free(dpz, s); dev_free(dflags, s); dev_free(dstats, s); dev_free(dparts, s);
    cudaStreamSynchronize(s);
    return rc;
}

extern "C" {

}  // extern "C"

// Matrices lo .. hi-1 built one by one: several at once, each on a stream of
// its own (builds of small matrices are bound by launch gaps and host
// synchronisations), after the work already queued on the context's stream.
static int spai_build_each(spai_ctx ctx, int lo, int hi, const spai_csr* A, const spai_opts* opts,
                           spai_precond* P_out, spai_stats* st, int* rcs)
{
    const int count = hi - lo;
    const int nt = std::min(count, SPAI_BATCH_STREAMS);
    cudaEvent_t ready = nullptr;
    SPAI_CUDA_TRY(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    std::vector<cudaStream_t> ss(nt, nullptr);
    int rc = 0;
    if (cudaEventRecord(ready, ctx->stream) != cudaSuccess) rc = SPAI_ERR_CUDA;
    for (int t = 0; t < nt && !rc; t++) {
        if (cudaStreamCreateWithFlags(&ss[t], cudaStreamNonBlocking) != cudaSuccess) rc = SPAI_ERR_CUDA;
        else if (cudaStreamWaitEvent(ss[t], ready, 0) != cudaSuccess) rc = SPAI_ERR_CUDA;  // after the caller's work
    }
    if (!rc) {
        std::atomic<int> next{lo};
        std::vector<std::thread> th;
        for (int t = 0; t < nt; t++) {
            th.emplace_back([&, t] {
                cudaSetDevice(ctx->device);
                cudaStream_t s = ss[t];
                for (int i = next++; i < hi; i = next++) {
                    DevCsr dA;
                    int r = csr_to_device(&A[i], &dA, s);
                    if (!r && A[i].on_device) r = csr_check_device(dA, ctx->num_sms, s);
                    if (!r) r = spai_build_dev(ctx->device, ctx->num_sms, s, dA, opts, &P_out[i], st ? &st[i] : nullptr);
                    csr_release(&dA, s);
                    if (cudaStreamSynchronize(s) != cudaSuccess && r >= 0) r = SPAI_ERR_CUDA;
                    rcs[i] = r;
                }
            });
        }
        for (auto& t : th) t.join();
        // the handles' frees go to the context's stream from now on
        for (int i = lo; i < hi; i++)
            if (P_out[i]) P_out[i]->stream = ctx->stream;
    }
    for (auto s : ss)
        if (s) cudaStreamDestroy(s);
    cudaEventDestroy(ready);
    return rc;
}

extern "C" {

int spai_build_batch(spai_ctx ctx, int count, const spai_csr* A, const spai_opts* opts, spai_precond* P_out,
                     spai_stats* st, int* status)
{
    if (!ctx || !opts || count < 0) return SPAI_ERR_INVALID_ARG;
    if (count == 0) return 0;
    if (!A || !P_out) return SPAI_ERR_INVALID_ARG;
    for (int i = 0; i < count; i++) P_out[i] = nullptr;
    {
        const int rc = csr_validate_many(A, count);
        if (rc) return rc;
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    SPAI_CUDA_TRY(cudaSetDevice(ctx->device));
    std::vector<int> rcs(count, 0);
    int rc = 0;
    if (!opts->adaptive && count > 1 && (opts->side == 0 || opts->side == 1)) {
        // fixed patterns: consecutive matrices are built together as one
        // block-diagonal matrix, in groups whose build fits half the free
        // device memory (64 GiB at most) and 2^31 - 1 rows; a group whose
        // build fails is built again matrix by matrix, which attributes the error
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { cudaGetLastError(); fr = 0; }
        const size_t cap = std::min<size_t>(fr / 2, (size_t)64 << 30);
        for (int lo = 0; lo < count && !rc;) {
            int hi = lo;
            int64_t n = 0, z = 0;
            while (hi < count) {
                const int64_t n2 = n + A[hi].n, z2 = z + A[hi].nnz;
                if (hi > lo && (n2 > INT32_MAX || union_footprint(n2, z2, opts) > cap)) break;
                n = n2;
                z = z2;
                hi++;
            }
            if (hi - lo < 2 || spai_build_union(ctx, ctx->stream, lo, hi, A, opts, P_out, st, rcs.data()) != 0)
                rc = spai_build_each(ctx, lo, hi, A, opts, P_out, st, rcs.data());
            lo = hi;
        }
    } else {
        rc = spai_build_each(ctx, 0, count, A, opts, P_out, st, rcs.data());
    }
    for (int i = 0; i < count; i++) {
        if (P_out[i]) {
            // the handle belongs to the context from now on
            std::lock_guard<std::mutex> lk2(g_live_mu);
            P_out[i]->stream = ctx->stream;
            P_out[i]->owner = ctx;
            ctx->live.insert(P_out[i]);
        }
        if (status) status[i] = rcs[i];
        if (!rc && rcs[i] < 0) rc = rcs[i];
    }
    if (!rc)
        for (int i = 0; i < count && !rc; i++)
            if (rcs[i] > 0) rc = rcs[i];
    return rc;
}

}  // extern "C"

// ------------------------------------------------------------------ the tile tuner's choices

static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int>, int> g_tune;

namespace spai {
int mid_tune_get(int device, int uf, int bin)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(std::make_tuple(device, uf, bin));
    return it == g_tune.end() ? -1 : it->second;
}
void mid_tune_put(int device, int uf, int bin, int variant)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (variant < 0) g_tune.erase(std::make_tuple(device, uf, bin));
    else g_tune[std::make_tuple(device, uf, bin)] = variant;
}
}  // namespace spai

extern "C" {

int spai_tune_get(int device, int uf, int bin)
{
    if (bin < 2 || bin > 13 || (uf != SPAI_HALF && uf != SPAI_SINGLE && uf != SPAI_DOUBLE)) return SPAI_ERR_INVALID_ARG;
    return spai::mid_tune_get(device, uf, bin);
}

int spai_tune_set(int device, int uf, int bin, int variant)
{
    if (bin < 2 || bin > 13 || (uf != SPAI_HALF && uf != SPAI_SINGLE && uf != SPAI_DOUBLE)) return SPAI_ERR_INVALID_ARG;
    if (variant < -1 || variant >= 4) return SPAI_ERR_INVALID_ARG;
    spai::mid_tune_put(device, uf, bin, variant);
    return 0;
}

int spai_precond_info(spai_precond P, int64_t* n, int64_t* nnz)
{
    if (!P) return SPAI_ERR_INVALID_ARG;
    if (n) *n = P->n;
    if (nnz) *nnz = P->nnz;
    return 0;
}

int spai_precond_export(spai_precond P, int64_t* rowptr, int32_t* col, double* val)
{
    if (!P) return SPAI_ERR_INVALID_ARG;
    SPAI_CUDA_TRY(cudaSetDevice(P->device));
    cudaStream_t s = P->stream;
    if (rowptr) SPAI_CUDA_TRY(cudaMemcpyAsync(rowptr, P->rowptr, sizeof(int64_t) * (P->n + 1), cudaMemcpyDeviceToHost, s));
    if (col) SPAI_CUDA_TRY(cudaMemcpyAsync(col, P->col, sizeof(int32_t) * P->nnz, cudaMemcpyDeviceToHost, s));
    if (val) SPAI_CUDA_TRY(cudaMemcpyAsync(val, P->val, sizeof(double) * P->nnz, cudaMemcpyDeviceToHost, s));
    SPAI_CUDA_TRY(cudaStreamSynchronize(s));
    return 0;
}

void spai_precond_free(spai_precond P)
{
    if (!P) return;
    cudaStream_t s;
    {
        std::lock_guard<std::mutex> lk(g_live_mu);
        if (P->owner) P->owner->live.erase(P);
        P->owner = nullptr;
        s = P->stream;
    }
    cudaSetDevice(P->device);
    dev_free(P->rowptr, s);
    dev_free(P->col, s);
    dev_free(P->val, s);
    sell_free(&P->sell_f16, s);
    sell_free(&P->sell_f32, s);
    sell_free(&P->sell_f64, s);
    dev_free(P->val_uf, s);
    cudaStreamSynchronize(s);
    delete P;
}

int gmres_ir_solve(spai_ctx ctx, const spai_csr* A, spai_precond P, const spai_opts* sopts, const double* b,
                   double* x, const ir_opts* opts, ir_stats* st)
{
    if (!ctx || !A || !b || !x || !opts) return SPAI_ERR_INVALID_ARG;
    int rc = csr_check_args(A);
    if (rc) return rc;
    if (P && P->n != A->n) return SPAI_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    SPAI_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    if (st) memset(st, 0, sizeof(*st));
    DevCsr dA;
    double *db = nullptr, *dx = nullptr;
    spai_precond own = nullptr;
    int wrc = 0;
    rc = csr_to_device(A, &dA, s);
    if (!rc) rc = csr_check_device(dA, ctx->num_sms, s);
    if (!rc) {
        if (A->on_device) {
            db = const_cast<double*>(b);
            dx = x;
        } else {
            rc = dev_alloc((void**)&db, sizeof(double) * A->n, s);
            if (!rc) rc = dev_alloc((void**)&dx, sizeof(double) * A->n, s);
            if (!rc && cudaMemcpyAsync(db, b, sizeof(double) * A->n, cudaMemcpyHostToDevice, s) != cudaSuccess) rc = SPAI_ERR_CUDA;
        }
    }
    if (!rc && !P && sopts) {
        spai_stats sst{};
        rc = spai_build_dev(ctx->device, ctx->num_sms, s, dA, sopts, &own, &sst);
        if (rc > 0) { wrc = rc; rc = 0; }
        if (st) { st->ms_spai = sst.ms; st->launches = sst.launches; }
        P = own;
    }
    if (!rc) {
        int rr = gmres_ir_dev(ctx->device, ctx->num_sms, s, dA, P, db, dx, opts, st);
        if (rr < 0) rc = rr; else if (rr > 0) wrc = rr;
    }
    if (!rc && !A->on_device) {
        if (cudaMemcpyAsync(x, dx, sizeof(double) * A->n, cudaMemcpyDeviceToHost, s) != cudaSuccess) rc = SPAI_ERR_CUDA;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess && !rc) rc = SPAI_ERR_CUDA;
    if (own) spai_precond_free(own);
    if (!A->on_device) {
        dev_free(db, s);
        dev_free(dx, s);
    }
    csr_release(&dA, s);
    cudaStreamSynchronize(s);
    return rc ? rc : wrc;
}

int gmres_ir_solve_batch(spai_ctx ctx, int count, const spai_csr* A, const spai_precond* P,
                         const double* const* b, double* const* x, const ir_opts* opts, ir_stats* st,
                         int* status)
{
    if (!ctx || !opts || count < 0) return SPAI_ERR_INVALID_ARG;
    if (count == 0) return 0;
    if (!A || !b || !x) return SPAI_ERR_INVALID_ARG;
    for (int i = 0; i < count; i++)
        if (!b[i] || !x[i]) return SPAI_ERR_INVALID_ARG;
    {
        const int rc = csr_validate_many(A, count);
        if (rc) return rc;
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    SPAI_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    if (st) memset(st, 0, sizeof(ir_stats) * (size_t)count);
    std::vector<DevCsr> dA(count);
    std::vector<const double*> db(count, nullptr);
    std::vector<double*> dx(count, nullptr);
    int rc = 0;
    for (int i = 0; i < count && !rc; i++) {
        rc = csr_to_device(&A[i], &dA[i], s);
        if (rc) break;
        if (A[i].on_device) {
            rc = csr_check_device(dA[i], ctx->num_sms, s);
            if (rc) break;
            db[i] = b[i];
            dx[i] = x[i];
        } else {
            double* t = nullptr;
            rc = dev_alloc((void**)&t, sizeof(double) * A[i].n, s);
            if (!rc && cudaMemcpyAsync(t, b[i], sizeof(double) * A[i].n, cudaMemcpyHostToDevice, s) != cudaSuccess)
                rc = SPAI_ERR_CUDA;
            db[i] = t;
            if (!rc) rc = dev_alloc((void**)&dx[i], sizeof(double) * A[i].n, s);
        }
    }
    if (!rc) rc = gmres_ir_batch_dev(ctx->device, ctx->num_sms, s, count, dA.data(), P, db.data(), dx.data(), opts,
                                     st, status);
    for (int i = 0; i < count; i++) {
        if (!A[i].on_device) {
            if (rc >= 0 && dx[i] &&
                cudaMemcpyAsync(x[i], dx[i], sizeof(double) * A[i].n, cudaMemcpyDeviceToHost, s) != cudaSuccess)
                rc = SPAI_ERR_CUDA;
            dev_free(const_cast<double*>(db[i]), s);
            dev_free(dx[i], s);
        }
        csr_release(&dA[i], s);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess && rc >= 0) rc = SPAI_ERR_CUDA;
    return rc;
}

int solver_submit(spai_ctx ctx, const spai_csr* A, const double* b, const spai_opts* sopts, const ir_opts* opts,
                  uint64_t* ticket)
{
    if (!ctx || !A || !b || !opts || !ticket) return SPAI_ERR_INVALID_ARG;
    int rc = csr_validate_host(A);
    if (rc) return rc;
    size_t bytes = estimate_footprint(A->n, A->nnz, sopts, opts);
    if (bytes > ctx->budget) return SPAI_ERR_ADMISSION;
    ServeRequest* r = new ServeRequest();
    r->n = A->n;
    r->nnz = A->nnz;
    r->rowptr.resize(A->n + 1);
    r->col.resize(A->nnz);
    r->val.resize(A->nnz);
    r->b.resize(A->n);
    if (A->on_device) {
        cudaSetDevice(ctx->device);
        if (cudaMemcpy(r->rowptr.data(), A->rowptr, sizeof(int64_t) * (A->n + 1), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(r->col.data(), A->col, sizeof(int32_t) * A->nnz, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(r->val.data(), A->val, sizeof(double) * A->nnz, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(r->b.data(), b, sizeof(double) * A->n, cudaMemcpyDeviceToHost) != cudaSuccess) {
            delete r;
            return SPAI_ERR_CUDA;
        }
        // the copy of a device input gets the host's structural check
        const spai_csr hc{r->n, r->nnz, r->rowptr.data(), r->col.data(), r->val.data(), 0};
        const int vr = csr_validate_host(&hc);
        if (vr) {
            delete r;
            return vr;
        }
    } else {
        memcpy(r->rowptr.data(), A->rowptr, sizeof(int64_t) * (A->n + 1));
        memcpy(r->col.data(), A->col, sizeof(int32_t) * A->nnz);
        memcpy(r->val.data(), A->val, sizeof(double) * A->nnz);
        memcpy(r->b.data(), b, sizeof(double) * A->n);
    }
    if (sopts) { r->so = *sopts; r->has_so = true; }
    r->io = *opts;
    r->bytes = bytes;
    r->t_submit = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(ctx->qmu);
        if (ctx->workers.empty()) {
            cudaSetDevice(ctx->device);
            cudaStream_t ws[2] = {nullptr, nullptr};
            for (int i = 0; i < 2; i++) {
                if (cudaStreamCreateWithFlags(&ws[i], cudaStreamNonBlocking) != cudaSuccess) {
                    for (int k = 0; k < i; k++) cudaStreamDestroy(ws[k]);  // a later submit starts afresh
                    delete r;
                    return SPAI_ERR_CUDA;
                }
            }
            ctx->worker_streams.assign(ws, ws + 2);
            ctx->workers.emplace_back(serve_admission_loop, ctx);
            ctx->workers.emplace_back(serve_refine_loop, ctx);
        }
        r->ticket = ctx->next_ticket++;
        ctx->tickets[r->ticket] = r;
        ctx->pending.push_back(r);
        ctx->qgen++;
        *ticket = r->ticket;
    }
    ctx->qcv.notify_all();
    return 0;
}

int solver_poll(spai_ctx ctx, uint64_t ticket, double* x, ir_stats* st)
{
    if (!ctx) return SPAI_ERR_INVALID_ARG;
    ServeRequest* r = nullptr;
    {
        std::lock_guard<std::mutex> lk(ctx->qmu);
        auto it = ctx->tickets.find(ticket);
        if (it == ctx->tickets.end()) return SPAI_ERR_NOT_FOUND;
        r = it->second;
        if (!r->done) return SPAI_PENDING;
        ctx->tickets.erase(it);
    }
    if (x && r->status >= 0) memcpy(x, r->x.data(), sizeof(double) * r->n);
    if (st) *st = r->st;
    int rc = r->status;
    delete r;
    return rc;
}

const char* spai_strerror(int code)
{
    switch (code) {
    case SPAI_OK: return "ok";
    case SPAI_WARN_NOT_CONVERGED: return "refinement stopped at i_max above the stop tolerance";
    case SPAI_WARN_FILLCAP: return "some SPAI columns stopped at the fill cap above eps";
    case SPAI_PENDING: return "request pending";
    case SPAI_ERR_INVALID_ARG: return "invalid argument";
    case SPAI_ERR_ZERO_ROW: return "a row of A has no nonzero entry (A is singular)";
    case SPAI_ERR_NONFINITE: return "non-finite value (input, overflow in u_f, or a non-finite refinement iterate)";
    case SPAI_ERR_NO_MEMORY: return "device memory allocation failed";
    case SPAI_ERR_ADMISSION: return "request exceeds the context's HBM budget";
    case SPAI_ERR_TIMEOUT: return "a bounded device-side wait expired";
    case SPAI_ERR_CUDA: {
        // the last CUDA error the library saw on the calling thread
        static thread_local char buf[160];
        if (g_last_cuda == cudaSuccess) return "CUDA runtime error";
        snprintf(buf, sizeof(buf), "CUDA runtime error (last on this thread: %s)", cudaGetErrorName(g_last_cuda));
        return buf;
    }
    case SPAI_ERR_UNSUPPORTED: return "precision tuple or size not supported";
    case SPAI_ERR_NOT_FOUND: return "unknown ticket";
    case SPAI_ERR_INTERNAL: return "device-side consistency check failed";
    default: return "unknown status";
    }
}

}  // extern "C"
