"""ctypes binding of the C ABI in include/spai_ir.h (argument marshalling only).

Every numerical step runs in the CUDA library; this module only converts
numpy arrays / torch tensors to pointers.  Loading fails loudly when the
library has not been built -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libspai_ir.so")

HALF, SINGLE, DOUBLE, QUAD = 0, 1, 2, 3
PREC = {"half": HALF, "single": SINGLE, "double": DOUBLE, "quad": QUAD}
PAT_IDENTITY, PAT_A, PAT_A2 = 0, 1, 2
IR_STOP_BACKWARD, IR_STOP_FIXED, IR_STOP_CORRECTION = 0, 1, 2
IR_CONVERGED, IR_MAXSTEPS, IR_BREAKDOWN, IR_NONFINITE, IR_STAGNATED = 1, 2, 4, 8, 16
SPAI_IR_MAX_STEPS = 64

OK, WARN_NOT_CONVERGED, WARN_FILLCAP, PENDING = 0, 1, 2, 3
ERR_INVALID_ARG, ERR_ZERO_ROW, ERR_NONFINITE, ERR_NO_MEMORY = -1, -2, -3, -4
ERR_ADMISSION, ERR_TIMEOUT, ERR_CUDA, ERR_UNSUPPORTED, ERR_NOT_FOUND, ERR_INTERNAL = -5, -6, -7, -8, -9, -10

EXPORTED = ("spai_ctx_create", "spai_ctx_destroy", "spai_build", "spai_precond_info", "spai_precond_export",
            "spai_precond_free", "gmres_ir_solve", "solver_submit", "solver_poll", "spai_strerror",
            "gmres_ir_solve_noalloc", "gmres_ir_solve_batch", "spai_build_batch", "spai_selftest_wait_timeout",
            "spai_tune_get", "spai_tune_set")


class spai_csr(C.Structure):
    """CSR matrix of include/spai_ir.h: int64 rowptr[n+1], int32 col[nnz], float64 val[nnz];
    on_device = 1 for device pointers."""
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("on_device", C.c_int)]


SIDE_LEFT, SIDE_RIGHT = 0, 1


class spai_opts(C.Structure):
    """Options of Algorithm 1 (pattern, adaptive Grote-Huckle, eps, alpha, beta, fill cap, u_f,
    scaling, rho reading, side); built by make_spai_opts."""
    _fields_ = [("init", C.c_int), ("adaptive", C.c_int), ("eps", C.c_double), ("alpha", C.c_int),
                ("beta", C.c_int), ("max_fill", C.c_int), ("uf", C.c_int), ("scale", C.c_int),
                ("rho_restricted", C.c_int), ("side", C.c_int)]


class ir_opts(C.Structure):
    """Options of Algorithm 3 (the five precisions, tau, iteration limits, stop rule, Arnoldi form,
    side); built by make_ir_opts."""
    _fields_ = [("uf", C.c_int), ("u", C.c_int), ("ug", C.c_int), ("up", C.c_int), ("ur", C.c_int),
                ("tau", C.c_double), ("gmres_max_it", C.c_int), ("ir_max_steps", C.c_int), ("stop", C.c_int),
                ("stop_tol", C.c_double), ("orth", C.c_int), ("side", C.c_int)]


class spai_stats(C.Structure):
    """Statistics of one SPAI build, with optional per-column host arrays."""
    _fields_ = [("n", C.c_int64), ("nnz_P", C.c_int64), ("cols_converged", C.c_int64),
                ("cols_fillcap", C.c_int64), ("cols_nonfinite", C.c_int64), ("max_I", C.c_int),
                ("max_J", C.c_int), ("ms", C.c_double), ("ms_kernel", C.c_double), ("launches", C.c_int),
                ("colres", C.c_void_p), ("nJ", C.c_void_p), ("nI", C.c_void_p), ("flags", C.c_void_p)]


class ir_stats(C.Structure):
    """Statistics of one refinement solve: steps, GMRES iterations per step, backward errors."""
    _fields_ = [("steps", C.c_int), ("total_its", C.c_int), ("its", C.c_int * SPAI_IR_MAX_STEPS),
                ("nbe", C.c_double * (SPAI_IR_MAX_STEPS + 1)), ("final_nbe", C.c_double), ("flags", C.c_int),
                ("nnz_P", C.c_int64), ("ms_spai", C.c_double), ("ms_ir", C.c_double),
                ("ms_kernel", C.c_double), ("launches", C.c_int), ("grid", C.c_int)]


_lib = None
_lock = threading.Lock()


def lib():
    """Load the CUDA library; raise if it is missing (no fallback path)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libspai_ir.so is not built (run __graft_entry__.build()); "
                                   "the solver has no CPU fallback")
            L = C.CDLL(LIB_PATH)
            vp, i64p = C.c_void_p, C.POINTER(C.c_int64)
            L.spai_ctx_create.argtypes = [C.POINTER(vp), C.c_int, vp, C.c_size_t]
            L.spai_ctx_destroy.argtypes = [vp]
            L.spai_ctx_destroy.restype = None
            L.spai_build.argtypes = [vp, C.POINTER(spai_csr), C.POINTER(spai_opts), C.POINTER(vp),
                                     C.POINTER(spai_stats)]
            L.spai_precond_info.argtypes = [vp, i64p, i64p]
            L.spai_precond_export.argtypes = [vp, vp, vp, vp]
            L.spai_precond_free.argtypes = [vp]
            L.spai_precond_free.restype = None
            L.gmres_ir_solve.argtypes = [vp, C.POINTER(spai_csr), vp, C.POINTER(spai_opts), vp, vp,
                                         C.POINTER(ir_opts), C.POINTER(ir_stats)]
            L.solver_submit.argtypes = [vp, C.POINTER(spai_csr), vp, C.POINTER(spai_opts), C.POINTER(ir_opts),
                                        C.POINTER(C.c_uint64)]
            L.solver_poll.argtypes = [vp, C.c_uint64, vp, C.POINTER(ir_stats)]
            L.gmres_ir_solve_noalloc.argtypes = [C.POINTER(spai_csr), C.POINTER(spai_csr), vp, vp,
                                                 C.POINTER(ir_opts), vp, C.POINTER(ir_stats)]
            L.gmres_ir_solve_batch.argtypes = [vp, C.c_int, C.POINTER(spai_csr), C.POINTER(vp), C.POINTER(vp),
                                               C.POINTER(vp), C.POINTER(ir_opts), C.POINTER(ir_stats),
                                               C.POINTER(C.c_int)]
            L.spai_build_batch.argtypes = [vp, C.c_int, C.POINTER(spai_csr), C.POINTER(spai_opts), C.POINTER(vp),
                                           C.POINTER(spai_stats), C.POINTER(C.c_int)]
            L.spai_selftest_wait_timeout.argtypes = [C.c_int, C.c_int, C.c_double]
            L.spai_strerror.argtypes = [C.c_int]
            L.spai_strerror.restype = C.c_char_p
            _lib = L
        return _lib


def strerror(code: int) -> str:
    """The library's description of a status code (spai_strerror)."""
    return lib().spai_strerror(int(code)).decode()


class SpaiError(RuntimeError):
    """A negative status from the library; .code holds it."""

    def __init__(self, code, where):
        super().__init__("%s: %s (%d)" % (where, strerror(code), code))
        self.code = code


def _check(rc, where):
    if rc < 0:
        raise SpaiError(rc, where)
    return rc


def _prec(p):
    return PREC[p] if isinstance(p, str) else int(p)


def _ptr(a):
    """Pointer of a numpy array or a torch tensor (contiguous)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr()
    assert isinstance(a, np.ndarray) and a.flags.c_contiguous
    return a.ctypes.data


def make_csr(A, on_device=None):
    """A = (rowptr int64, col int32, val float64) as numpy arrays or CUDA tensors."""
    rp, ci, va = A
    dev = hasattr(rp, "is_cuda") and rp.is_cuda if on_device is None else on_device
    n = (rp.shape[0] if hasattr(rp, "shape") else len(rp)) - 1
    nnz = ci.shape[0]
    return spai_csr(n, nnz, _ptr(rp), _ptr(ci), _ptr(va), int(bool(dev)))


def make_spai_opts(init=PAT_A, adaptive=False, eps=0.5, alpha=-1, beta=8, max_fill=30, uf="single", scale=True,
                   rho_restricted=False, side=SIDE_LEFT):
    """side: SIDE_LEFT (P A ~ I, the paper's) or SIDE_RIGHT (A P ~ I)."""
    return spai_opts(int(init), int(bool(adaptive)), float(eps), int(alpha), int(beta), int(max_fill), _prec(uf),
                     int(bool(scale)), int(bool(rho_restricted)), int(side))


def make_ir_opts(uf="single", u="double", ug="double", up="double", ur="quad", tau=1e-8, gmres_max_it=0,
                 ir_max_steps=10, stop=IR_STOP_BACKWARD, stop_tol=0.0, orth=0, side=SIDE_LEFT):
    """orth: 0 modified Gram-Schmidt (default, the paper's), 1 classical Gram-Schmidt twice, 2 MGS with one
    reduction per iteration (inverse compact WY form, lagged normalisation).
    side: SIDE_LEFT (Algorithm 3) or SIDE_RIGHT (GMRES on A P u = r, d = P u).
    stop: IR_STOP_BACKWARD, IR_STOP_FIXED or IR_STOP_CORRECTION (stop_tol <= 0: the default threshold)."""
    return ir_opts(_prec(uf), _prec(u), _prec(ug), _prec(up), _prec(ur), float(tau), int(gmres_max_it),
                   int(ir_max_steps), int(stop), float(stop_tol), int(orth), int(side))


class Context:
    """A library context on one device and one CUDA stream."""

    def __init__(self, device=0, stream=None, hbm_budget=0):
        self.h = C.c_void_p()
        s = None
        if stream is not None:
            s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        _check(lib().spai_ctx_create(C.byref(self.h), int(device), s, C.c_size_t(int(hbm_budget))),
               "spai_ctx_create")

    def close(self):
        if self.h:
            lib().spai_ctx_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Precond:
    """A preconditioner P = M^T D on the device (spai_build); free() releases it."""

    def __init__(self, h, ctx=None):
        self.h = h
        self.ctx = ctx  # keeps the building context alive while the handle lives

    def info(self):
        n = C.c_int64()
        nnz = C.c_int64()
        _check(lib().spai_precond_info(self.h, C.byref(n), C.byref(nnz)), "spai_precond_info")
        return n.value, nnz.value

    def export(self):
        n, nnz = self.info()
        rp = np.zeros(n + 1, dtype=np.int64)
        ci = np.zeros(max(nnz, 1), dtype=np.int32)
        va = np.zeros(max(nnz, 1), dtype=np.float64)
        _check(lib().spai_precond_export(self.h, _ptr(rp), _ptr(ci), _ptr(va)), "spai_precond_export")
        return rp, ci[:nnz], va[:nnz]

    def free(self):
        if self.h:
            lib().spai_precond_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def spai_build(ctx: Context, A, opts: spai_opts, per_column=False):
    """Algorithm 1 on A^T D; returns (Precond, stats dict), the call's return code under "rc"
    (0, or SPAI_WARN_FILLCAP when some columns stopped at the fill cap)."""
    csr = make_csr(A)
    st = spai_stats()
    n = csr.n
    cols = {}
    if per_column:
        cols = dict(colres=np.zeros(n), nJ=np.zeros(n, dtype=np.int32), nI=np.zeros(n, dtype=np.int32),
                    flags=np.zeros(n, dtype=np.int32))
        st.colres, st.nJ, st.nI, st.flags = (_ptr(cols["colres"]), _ptr(cols["nJ"]), _ptr(cols["nI"]),
                                             _ptr(cols["flags"]))
    h = C.c_void_p()
    rc = _check(lib().spai_build(ctx.h, C.byref(csr), C.byref(opts), C.byref(h), C.byref(st)), "spai_build")
    out = dict(n=st.n, nnz_P=st.nnz_P, cols_converged=st.cols_converged, cols_fillcap=st.cols_fillcap,
               cols_nonfinite=st.cols_nonfinite, max_I=st.max_I, max_J=st.max_J, ms=st.ms,
               ms_kernel=st.ms_kernel, launches=st.launches, rc=rc)
    out.update(cols)
    return Precond(h, ctx), out


def _ir_dict(st, rc):
    s = st.steps
    return dict(steps=s, total_its=st.total_its, its=list(st.its[:s]), nbe=list(st.nbe[:s + 1]),
                final_nbe=st.final_nbe, flags=st.flags, nnz_P=st.nnz_P, ms_spai=st.ms_spai, ms_ir=st.ms_ir,
                ms_kernel=st.ms_kernel, launches=st.launches, grid=st.grid, rc=rc)


def gmres_ir_solve(ctx: Context, A, b, x, P: Precond | None = None, sopts: spai_opts | None = None,
                   opts: ir_opts | None = None):
    """Algorithm 3.  b, x: float64 numpy arrays (host) or CUDA tensors (device)."""
    csr = make_csr(A)
    st = ir_stats()
    rc = lib().gmres_ir_solve(ctx.h, C.byref(csr), P.h if P is not None else None,
                              C.byref(sopts) if sopts is not None else None, _ptr(b), _ptr(x), C.byref(opts),
                              C.byref(st))
    _check(rc, "gmres_ir_solve")
    return _ir_dict(st, rc)


def spai_build_batch(ctx: Context, As, opts: spai_opts, per_column=False):
    """spai_build for many matrices with the same options: fixed patterns in
    one build over the block-diagonal union of the matrices, adaptive ones as
    concurrent builds.  Returns (list of Precond, list of stats dicts); raises
    on the first error after freeing the handles that were built."""
    k = len(As)
    csrs = (spai_csr * max(k, 1))(*[make_csr(A) for A in As])
    hs = (C.c_void_p * max(k, 1))()
    sts = (spai_stats * max(k, 1))()
    status = (C.c_int * max(k, 1))()
    cols = [{} for _ in range(k)]
    if per_column:
        for i in range(k):
            n = csrs[i].n
            cols[i] = dict(colres=np.zeros(n), nJ=np.zeros(n, dtype=np.int32), nI=np.zeros(n, dtype=np.int32),
                           flags=np.zeros(n, dtype=np.int32))
            sts[i].colres, sts[i].nJ, sts[i].nI, sts[i].flags = (_ptr(cols[i]["colres"]), _ptr(cols[i]["nJ"]),
                                                                 _ptr(cols[i]["nI"]), _ptr(cols[i]["flags"]))
    rc = lib().spai_build_batch(ctx.h, k, csrs, C.byref(opts), hs, sts, status)
    Ps = [Precond(C.c_void_p(hs[i]), ctx) if hs[i] else None for i in range(k)]
    if rc < 0:
        for P in Ps:
            if P is not None:
                P.free()
        _check(rc, "spai_build_batch")
    out = [dict(n=sts[i].n, nnz_P=sts[i].nnz_P, cols_converged=sts[i].cols_converged,
                cols_fillcap=sts[i].cols_fillcap, cols_nonfinite=sts[i].cols_nonfinite, max_I=sts[i].max_I,
                max_J=sts[i].max_J, ms=sts[i].ms, ms_kernel=sts[i].ms_kernel, launches=sts[i].launches,
                rc=status[i], **cols[i]) for i in range(k)]
    return Ps, out


def gmres_ir_solve_batch(ctx: Context, As, bs, xs, Ps=None, opts: ir_opts | None = None):
    """Algorithm 3 for many systems with the same options in shared launches.

    As: list of CSR triples (numpy or CUDA tensors); bs, xs: matching float64
    vectors; Ps: None or a list of Precond / None.  Returns (stats list,
    status list); raises on the first error."""
    k = len(As)
    csrs = (spai_csr * max(k, 1))(*[make_csr(A) for A in As])
    vp = C.c_void_p
    bp = (vp * max(k, 1))(*[_ptr(b) for b in bs])
    xp = (vp * max(k, 1))(*[_ptr(x) for x in xs])
    pp = None
    if Ps is not None:
        pp = (vp * max(k, 1))(*[(P.h if P is not None else None) for P in Ps])
    sts = (ir_stats * max(k, 1))()
    status = (C.c_int * max(k, 1))()
    rc = lib().gmres_ir_solve_batch(ctx.h, k, csrs, pp, bp, xp, C.byref(opts), sts, status)
    _check(rc, "gmres_ir_solve_batch")
    return [_ir_dict(sts[i], status[i]) for i in range(k)], [status[i] for i in range(k)]


def solver_submit(ctx: Context, A, b, sopts: spai_opts | None, opts: ir_opts) -> int:
    """Queue one solve on the serving queue (continuous batching); returns its ticket."""
    csr = make_csr(A)
    t = C.c_uint64()
    _check(lib().solver_submit(ctx.h, C.byref(csr), _ptr(b), C.byref(sopts) if sopts is not None else None,
                               C.byref(opts), C.byref(t)), "solver_submit")
    return t.value


def solver_poll(ctx: Context, ticket: int, x=None):
    """Returns None while pending, else the stats dict (x filled when given)."""
    st = ir_stats()
    rc = lib().solver_poll(ctx.h, C.c_uint64(ticket), _ptr(x), C.byref(st))
    if rc == PENDING:
        return None
    _check(rc, "solver_poll")
    return _ir_dict(st, rc)


def tune_get(device: int, uf, bin_: int) -> int:
    """The SPAI tile tuner's choice for a bin (-1 while untuned); see spai_tune_get."""
    rc = lib().spai_tune_get(int(device), _prec(uf), int(bin_))
    if rc < -1:
        _check(rc, "spai_tune_get")
    return rc


def tune_set(device: int, uf, bin_: int, variant: int) -> None:
    """Force the SPAI tile tuner's choice for a bin (-1: tune again)."""
    _check(lib().spai_tune_set(int(device), _prec(uf), int(bin_), int(variant)), "spai_tune_set")


def selftest_wait_timeout(device=0, mode=0, limit_ms=50.0) -> int:
    """Runs the bounded-wait self-test; returns its code (ERR_TIMEOUT when the waits gave up)."""
    return lib().spai_selftest_wait_timeout(int(device), int(mode), float(limit_ms))


def gmres_ir_solve_noalloc(A, b, x, P=None, opts: ir_opts | None = None, stream=None):
    """Allocation-free refinement solve; A, P (CSR triples), b and x are CUDA tensors."""
    csr = make_csr(A, on_device=True)
    pcsr = make_csr(P, on_device=True) if P is not None else None
    st = ir_stats()
    s = None
    if stream is not None:
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    rc = lib().gmres_ir_solve_noalloc(C.byref(csr), C.byref(pcsr) if pcsr is not None else None, _ptr(b),
                                      _ptr(x), C.byref(opts), s, C.byref(st))
    _check(rc, "gmres_ir_solve_noalloc")
    return _ir_dict(st, rc)
