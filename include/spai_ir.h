/*
 * spai_ir.h -- C ABI of the GB300 SPAI-GMRES-IR library.
 *
 * Solves sparse nonsingular A x = b by GMRES-based iterative refinement left-
 * preconditioned by a Frobenius-norm sparse approximate inverse (Carson &
 * Khan, "Mixed precision iterative refinement with sparse approximate
 * inverse preconditioning", arXiv 2202.10204):
 *   - the preconditioner is Algorithm 1 (Grote-Huckle / Sedlacek SPAI) run on
 *     A^T D, D the diagonal that scales every column of A^T (every row of A)
 *     to max-abs 1, and P = M^T D (Section 3 and Section 4 set-up);
 *   - the solve is Algorithm 3 (SPAI-GMRES-IR) with the five precisions
 *     (u_f, u, u_g, u_p, u_r) of Section 3.1.
 *
 * Conventions for every entry point:
 *   - return value 0 is success, > 0 a warning, < 0 an error (SPAI_* codes);
 *     spai_strerror() names each code.  No entry point aborts the process.
 *   - the caller owns every buffer it passes; the library never frees a
 *     caller buffer nor keeps a caller pointer beyond the call (solver_submit
 *     copies its inputs before it returns, solver_poll writes x during its
 *     own call).
 *   - CSR arrays: rowptr[n+1] int64 (rowptr[0] = 0, non-decreasing), col[nnz]
 *     int32 in [0, n) sorted ascending within a row, val[nnz] float64.
 *     With on_device = 1 all three are device pointers on the context's
 *     device, otherwise host pointers.  Every input is checked in full
 *     (SPAI_ERR_INVALID_ARG for a structural error, which takes precedence
 *     over SPAI_ERR_ZERO_ROW for an empty row) before any kernel indexes
 *     with it: one pass over the rows on the device (for host inputs after
 *     the copy; solver_submit checks its host copy on the host).
 *   - all work runs on the context's CUDA stream on one GPU; every call
 *     returns after its results are complete.
 *   - calls on one context are serialised by the context; distinct contexts
 *     may be used from different threads.
 */
#ifndef SPAI_IR_H
#define SPAI_IR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define SPAI_OK 0
#define SPAI_WARN_NOT_CONVERGED 1  /* IR stopped (i_max or stagnation) unconverged  */
#define SPAI_WARN_FILLCAP 2        /* some SPAI columns stopped at the fill cap     */
#define SPAI_PENDING 3             /* solver_poll: request not finished yet          */
#define SPAI_ERR_INVALID_ARG (-1)  /* bad pointer, size, option or CSR structure     */
#define SPAI_ERR_ZERO_ROW (-2)     /* a row of A has no nonzero: A is singular       */
#define SPAI_ERR_NONFINITE (-3)    /* Inf/NaN in the input or overflow in u_f        */
#define SPAI_ERR_NO_MEMORY (-4)    /* device allocation failed                       */
#define SPAI_ERR_ADMISSION (-5)    /* request larger than the context's HBM budget   */
#define SPAI_ERR_TIMEOUT (-6)      /* a bounded device-side wait expired             */
#define SPAI_ERR_CUDA (-7)         /* a CUDA runtime call failed                     */
#define SPAI_ERR_UNSUPPORTED (-8)  /* precision tuple or size outside what is built  */
#define SPAI_ERR_NOT_FOUND (-9)    /* unknown ticket                                 */
#define SPAI_ERR_INTERNAL (-10)    /* device-side consistency check failed           */

/* ---- precisions (Table 1) -------------------------------------------- */
typedef enum {
    SPAI_HALF = 0,   /* IEEE binary16, u = 2^-11 */
    SPAI_SINGLE = 1, /* IEEE binary32, u = 2^-24 */
    SPAI_DOUBLE = 2, /* IEEE binary64, u = 2^-53 */
    SPAI_QUAD = 3    /* u_r only: the residual is computed in double-double */
} spai_prec;

/* initial pattern J of Algorithm 1 (Section 2.2: identity, or the pattern of
 * A or of a power of A).  Column k of the pattern is the nonzero rows of
 * column k of A (resp. A^2). */
typedef enum { SPAI_PAT_IDENTITY = 0, SPAI_PAT_A = 1, SPAI_PAT_A2 = 2 } spai_pattern_init;

/* refinement stopping rule (Algorithm 3 fixes only i_max) */
typedef enum {
    IR_STOP_BACKWARD = 0,  /* stop before step i once ||r_i||_inf/(||A||_inf||x_i||_inf+||b||_inf) <= stop_tol */
    IR_STOP_FIXED = 1,     /* always run ir_max_steps steps */
    IR_STOP_CORRECTION = 2 /* stop before step i >= 1 once ||d_{i-1}||_inf/||x_i||_inf <= stop_tol */
    /* With BACKWARD and CORRECTION the refinement also stops, without
     * convergence (flag 16, SPAI_WARN_NOT_CONVERGED), when it stagnates: before
     * step i >= 2, if ||d_{i-1}||_inf/||x_i||_inf >= (||d_{i-2}||_inf/||x_{i-1}||_inf)/2,
     * i.e. the last correction did not halve relative to the iterate.  The
     * convergence tests come first. */
} ir_stop_rule;

typedef struct {
    int64_t n, nnz;
    const int64_t* rowptr;
    const int32_t* col;
    const double* val;
    int on_device; /* 1: device pointers (borrowed for the call), 0: host */
} spai_csr;

/* Algorithm 1 parameters. */
typedef struct {
    spai_pattern_init init; /* initial pattern J                                  */
    int adaptive;           /* 0: fixed pattern, 1: Grote-Huckle augmentation     */
    double eps;             /* column tolerance: stop when ||s_k||_2 <= eps       */
    int alpha;              /* max augmentation steps per column; < 0: ceil(n/beta) */
    int beta;               /* max indices added per step (>= 1 when adaptive)    */
    int max_fill;           /* cap on |J_k|, 1..31; larger initial patterns keep k
                               and the indices nearest to k                        */
    spai_prec uf;           /* precision of the construction (half/single/double) */
    int scale;              /* 1: run on A^T D (recommended), 0: on A^T           */
    int rho_restricted;     /* 1: rho_jk uses ||b_j(I_k)|| (literal Algorithm 1)  */
    int side;               /* 0: left preconditioner P ~ A^{-1} with P A ~ I (the
                               paper's Section 3: Algorithm 1 on A^T D, P = M^T D);
                               1: right preconditioner with A P ~ I (Algorithm 1 on
                               A D, D scaling the columns of A, P = D M; the variant
                               the paper leaves as future work at the end of
                               Section 3).  Patterns then refer to A^T: pattern(A)
                               gives pattern(P) = pattern(A).  Per-column stats
                               describe the columns of M, i.e. the columns of P.  */
} spai_opts;

/* Algorithm 3 parameters: the five precisions, tau, i_max and the stop rule. */
typedef struct {
    spai_prec uf, u, ug, up, ur; /* u in {single,double}; ug,up in {single,double}, or
                                    half in one or both with single for the other and
                                    orth = 2 (half storage of the Krylov vectors and of
                                    the matrices' product copies, binary32 arithmetic;
                                    GMRES then solves for r scaled by the power of two
                                    nearest below ||r||_inf, and d is scaled back:
                                    values beyond half's range give a non-finite
                                    status); ur in {double,quad}, ur >= u        */
    double tau;                  /* GMRES relative tolerance on ||P(r - A d)||/||P r|| */
    int gmres_max_it;            /* iterations per GMRES solve (1..1024); <= 0: min(n, 500) */
    int ir_max_steps;            /* i_max (1..64)                                      */
    ir_stop_rule stop;
    double stop_tol;             /* <= 0: q*u (BACKWARD, q the largest row nonzero count of A,
                                    the limit of Theorem 2) or u (CORRECTION)          */
    int orth;                    /* Arnoldi orthogonalisation: 0 modified Gram-Schmidt (the
                                    paper's MGS-GMRES, j+1 scalar reductions in iteration j);
                                    1 classical Gram-Schmidt applied twice (CGS2: two vector
                                    reductions per iteration); 2 MGS in its inverse compact WY
                                    form with lagged normalisation (Swirydowicz, Langou,
                                    Ananthan, Yang and Thomas, "Low synchronization
                                    Gram-Schmidt and GMRES algorithms", 2020): one vector
                                    reduction per iteration, MGS in exact arithmetic and
                                    MGS-like loss of orthogonality */
    int side;                    /* 0: left preconditioning (Algorithm 3: GMRES on P A d = P r,
                                    tau bounds ||P(r - A d)||/||P r||); 1: right preconditioning
                                    (GMRES on A P u = r, d = P u, tau bounds ||r - A d||/||r||;
                                    future work in the paper's Section 3).  Ignored when P is
                                    NULL. */
} ir_opts;

#define SPAI_IR_MAX_STEPS 64

typedef struct {
    int64_t n;
    int64_t nnz_P;             /* nonzeros of P = sum_k |J_k|                        */
    int64_t cols_converged;    /* columns with ||s_k|| <= eps                         */
    int64_t cols_fillcap;      /* columns stopped at max_fill above eps               */
    int64_t cols_nonfinite;    /* columns with Inf/NaN (overflow in u_f)              */
    int max_I, max_J;          /* largest |I_k| and |J_k|                             */
    double ms;                 /* device time of the build, milliseconds              */
    double ms_kernel;          /* device time of the column kernel alone              */
    int launches;              /* kernels the build launched                          */
    /* optional per-column host outputs, filled when non-NULL (length n each): */
    double* colres;            /* ||s_k||_2 as computed in u_f                         */
    int32_t* nJ;               /* |J_k|                                                */
    int32_t* nI;               /* |I_k| of the final least-squares solve               */
    int32_t* flags;            /* bit 0 converged, 1 fill cap, 2 alpha, 3 no candidate,
                                  4 zero pivot, 5 non-finite                           */
} spai_stats;

typedef struct {
    int steps;                           /* GMRES solves performed                   */
    int total_its;                       /* sum of its[]                             */
    int its[SPAI_IR_MAX_STEPS];          /* GMRES iterations per refinement step     */
    double nbe[SPAI_IR_MAX_STEPS + 1];   /* normwise backward error before each step */
    double final_nbe;                    /* backward error of the returned x         */
    int flags;                           /* 1 converged, 2 max steps, 4 breakdown, 8 non-finite,
                                            16 stagnated (see ir_stop_rule)          */
    int64_t nnz_P;
    double ms_spai, ms_ir;               /* device time of the two phases            */
    double ms_kernel;                    /* device time of the refinement kernel alone */
    int launches;                        /* kernels launched (build included)        */
    int grid;                            /* blocks of the refinement kernel          */
} ir_stats;

typedef struct spai_ctx_s* spai_ctx;
typedef struct spai_precond_s* spai_precond;

/* Create a context on `device` that runs on `cuda_stream` (a cudaStream_t;
 * NULL: the context creates its own).  hbm_budget_bytes bounds the device
 * memory the serving queue admits (0: 90% of free memory at creation).
 * This call and every call given the context (or a preconditioner built on
 * it) make its device current on the calling thread (cudaSetDevice) and leave
 * it current when they return. */
int spai_ctx_create(spai_ctx* out, int device, void* cuda_stream, size_t hbm_budget_bytes);
/* Waits for the context's work, stops its serving workers and releases its
 * stream (if it created it).  Preconditioners it built stay valid and may be
 * freed later (on the default stream). */
void spai_ctx_destroy(spai_ctx ctx);

/* Algorithm 1 on A^T D (Section 2.2, Algorithm 1; Section 4 scaling), giving
 * the left preconditioner P = M^T D in CSR on the device.  *P_out is owned by
 * the caller and released with spai_precond_free.  st may be NULL. */
int spai_build(spai_ctx ctx, const spai_csr* A, const spai_opts* opts, spai_precond* P_out,
               spai_stats* st);

/* spai_build for `count` matrices with the same options, after the work
 * already queued on the context's stream.  Fixed patterns (adaptive = 0):
 * consecutive matrices are built together as one block-diagonal matrix, so
 * every kernel of the build runs once for the group instead of once per
 * matrix (groups are cut where the build would need more than half the free
 * device memory, 64 GiB at most, or more than 2^31 - 1 rows).  The columns of
 * Algorithm 1 are independent and each is computed by the kernel its own
 * shadow size selects, so each preconditioner is bit for bit the one
 * spai_build gives for its matrix.  A group whose build fails is built again
 * matrix by matrix, which attributes the error.  Adaptive patterns: the
 * builds run concurrently on streams of their own.  On return every
 * preconditioner belongs to the context's stream like one from spai_build.
 * P_out[count] receives the handles (NULL where a build failed); st (count
 * entries, may be NULL) and status (count entries, may be NULL) receive each
 * build's statistics (for a group built together, ms, ms_kernel and
 * launches are those of the group's build; the per-column arrays are filled
 * where given) and return code.  Returns the first error, else the first
 * warning, else SPAI_OK; handles that were built must be freed even when an
 * error is returned. */
int spai_build_batch(spai_ctx ctx, int count, const spai_csr* A, const spai_opts* opts,
                     spai_precond* P_out, spai_stats* st, int* status);

/* The tile tuner of the SPAI build (fixed patterns).  Columns with shadows of
 * 65..512 rows run in a warp kernel whose tile in shared memory has 32 R rows
 * and 16 or 32 columns; any tile that holds a column gives the same result
 * bit for bit (padding rows are zero and stay zero), so the shape is a cost
 * choice.  The columns are binned by |I_k| and |J_k| (bins 2..13: up to 16
 * columns and R = 3, 4, 5, 6, 7, 8, 10, 12, 16 for bins 2..10; 17..31 columns
 * and R = 4, 8, 16 for bins 11..13).  The first build in which a bin has at
 * least 8192 columns times the bin's candidate tiles (its own, the next two
 * larger row counts, a 32-column tile) on 4096 of them and keeps the fastest
 * for the device, u_f (SPAI_HALF / SPAI_SINGLE / SPAI_DOUBLE) and bin.
 * spai_tune_get returns the bin's choice (a candidate index 0..3, -1 while
 * untuned); spai_tune_set forces it (-1: tune again).  Both return
 * SPAI_ERR_INVALID_ARG for a bad bin, u_f or index. */
int spai_tune_get(int device, int uf, int bin);
int spai_tune_set(int device, int uf, int bin, int variant);

/* Size of P: *n and *nnz (either may be NULL).  SPAI_ERR_INVALID_ARG for a
 * NULL P. */
int spai_precond_info(spai_precond P, int64_t* n, int64_t* nnz);

/* Copy P to host buffers the caller owns: rowptr[n+1], col[nnz], val[nnz]
 * (float64, the unrounded values mbar_k * d(J_k)); any pointer may be NULL.
 * Waits for P's stream; SPAI_ERR_INVALID_ARG for a NULL P, SPAI_ERR_CUDA if a
 * copy fails. */
int spai_precond_export(spai_precond P, int64_t* rowptr, int32_t* col, double* val);

/* Release P's device memory (after the work queued on its stream); P must not
 * be used afterwards.  NULL is ignored. */
void spai_precond_free(spai_precond P);

/* Algorithm 3 (SPAI-GMRES-IR).  P: a preconditioner from spai_build; if NULL
 * and sopts != NULL one is built first (and freed); if both are NULL the
 * solve is unpreconditioned GMRES-IR (P = I).  b[n] and x[n] (float64) are
 * device pointers when A->on_device, host pointers otherwise; x is output
 * only.  st may be NULL. */
int gmres_ir_solve(spai_ctx ctx, const spai_csr* A, spai_precond P, const spai_opts* sopts,
                   const double* b, double* x, const ir_opts* opts, ir_stats* st);

/* Algorithm 3 for `count` independent systems with the same options (a batch
 * of the paper's solve; the batching is this library's).  The systems share
 * one persistent cooperative launch of the refinement kernel whose grid is
 * split into teams of blocks; each team solves one system after another,
 * larger systems first.  A system's team size depends on its order and the
 * options alone (about 8192 rows per block, more blocks where a block's rows
 * would not fit its shared memory, at most 16), so its result is the same
 * in any batch.  Systems of more than 65536 rows run afterwards, each on a
 * grid of its own as in gmres_ir_solve.  Every system's buffers are
 * allocated before the launch.  A[i] is a
 * host or device CSR and b[i], x[i] follow A[i].on_device.  P may be NULL or
 * hold NULL entries (that system is unpreconditioned); preconditioners come
 * from spai_build with the same u_f as opts->uf.  st (count entries, may be
 * NULL) receives each system's steps, iterations and backward errors, while
 * ms_ir, ms_kernel and launches describe the whole batch.  status (count
 * entries, may be NULL) receives each system's return code.  Returns the
 * first error, else the first warning, else SPAI_OK. */
int gmres_ir_solve_batch(spai_ctx ctx, int count, const spai_csr* A, const spai_precond* P,
                         const double* const* b, double* const* x, const ir_opts* opts,
                         ir_stats* st, int* status);

/* Serving queue with continuous batching.  solver_submit copies A and b
 * (host or device, as A->on_device says) into host memory the context owns
 * and returns a ticket; the caller's buffers may be reused once it returns.
 * Device inputs are copied with synchronous device-to-host copies (so that a
 * waiting request holds no device memory outside the admission budget) and
 * checked on the host.  An admission thread admits every waiting request whose
 * estimated device footprint fits what the context's HBM budget has left (a
 * request passed over for more than 200 ms is admitted before any later
 * one), uploads the admitted requests and builds their preconditioners
 * (requests with the same fixed-pattern options: one build over the
 * block-diagonal union, as spai_build_batch); a refinement thread solves the
 * prepared requests with the same options together, as gmres_ir_solve_batch
 * does.  Requests that arrive while others are being solved are admitted
 * and prepared meanwhile and join the next launch.  A request's result does
 * not depend on the other requests: alone or in a mix it is the same, bit
 * for bit.  Each request's A, P, b and x stay on the device until it is
 * solved.  Returns SPAI_ERR_ADMISSION if the request alone exceeds the
 * budget. */
int solver_submit(spai_ctx ctx, const spai_csr* A, const double* b, const spai_opts* sopts,
                  const ir_opts* opts, uint64_t* ticket);

/* SPAI_PENDING while the request runs; otherwise copies the solution into the
 * host buffer x[n] (may be NULL), fills st (may be NULL), releases the ticket
 * and returns the request's own status. */
int solver_poll(spai_ctx ctx, uint64_t ticket, double* x, ir_stats* st);

/* A static description of a status code; for SPAI_ERR_CUDA it names the last CUDA
 * error the library saw on the calling thread (a thread-local string, valid until
 * the thread's next call). */
const char* spai_strerror(int code);

/* Self-test of the bounded device-side waits (no counterpart in the paper).
 * Every wait of the refinement kernels (the exchange rounds among blocks and
 * the counter barrier) gives up after a clock budget, records
 * SPAI_ERR_TIMEOUT and leaves the kernel, so a block that never arrives
 * cannot hang the GPU.  This call launches a few blocks on `device` (made
 * current) whose exchange round (mode 0) or counter barrier (mode 1) waits
 * for one block more than the launch has, with a budget of limit_ms
 * milliseconds (0 < limit_ms <= 10000).  Returns SPAI_ERR_TIMEOUT when the
 * waits gave up as designed; the device stays usable afterwards.
 * SPAI_ERR_INVALID_ARG for a bad mode or limit. */
int spai_selftest_wait_timeout(int device, int mode, double limit_ms);

/* ---- allocation-free refinement solve --------------------------------
 * No counterpart in the paper: an engineering entry point for callers that
 * must not call the CUDA allocator -- real-time loops, where cudaMalloc and
 * cudaFree have no bounded latency and cudaFree synchronises the device;
 * hosts that hand all device memory to their own pool at start-up, so that
 * a later allocation would fail or break their accounting; and runtimes that
 * forbid allocation once running.  It runs the same refinement kernels as
 * gmres_ir_solve with a given preconditioner, but every scratch buffer lives
 * in one fixed device array of SPAI_NOALLOC_SCRATCH_BYTES (32 MiB) that each
 * GPU loading this library holds until the process exits.  It calls no
 * cudaMalloc, cudaFree or other allocating routine.  It runs on the calling
 * thread's current device, where A, P, b and x must reside.
 *   A, P : device CSR (on_device = 1); P holds the float64 entries of the
 *          left preconditioner (for instance spai_precond_export's output),
 *          or of the right one when opts->side = 1; P == NULL solves
 *          unpreconditioned.  Both are checked on the device first
 *          (SPAI_ERR_INVALID_ARG, SPAI_ERR_ZERO_ROW for an empty row of A).
 *   b, x : device float64 arrays of length n; x is output only.
 *   opts : as gmres_ir_solve (orth 0, 1 and 2, both sides, every stop rule),
 *          except that u_g and u_p are single or double: half Krylov storage
 *          returns SPAI_ERR_UNSUPPORTED here.
 *   cuda_stream: the cudaStream_t to run on (NULL: the legacy default stream).
 * The call reads sizes back to the host between its kernels, so it
 * synchronises the stream, and returns once x is complete.
 * Returns SPAI_ERR_UNSUPPORTED when the problem (n, nonzeros, gmres_max_it,
 * precisions) needs more than SPAI_NOALLOC_SCRATCH_BYTES, and the other
 * codes as gmres_ir_solve.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress); make that first call before any
 * stream capture.  All calls share the one array and the array keeps the
 * last call's contents (the call clears what must start at zero): calls
 * whose work overlaps on the GPU (other threads or streams) race and must be
 * serialised by the caller.  ir_stats' timing fields are left 0. */
#define SPAI_NOALLOC_SCRATCH_BYTES (32u << 20)
int gmres_ir_solve_noalloc(const spai_csr* A, const spai_csr* P, const double* b, double* x,
                           const ir_opts* opts, void* cuda_stream, ir_stats* st);

#ifdef __cplusplus
}
#endif

#endif /* SPAI_IR_H */
