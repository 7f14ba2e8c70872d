"""Plain CPU oracle for SPAI-GMRES-IR (arXiv 2202.10204).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path (the
CUDA library and its binding) never imports this package.

The arithmetic lives in ``spai_ir_oracle.c`` (plain C, fp64, _Float128 for
quad, a hand-written half chop); this module only compiles it with gcc and
marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np
import scipy.sparse as sp

HALF, SINGLE, DOUBLE, QUAD = 0, 1, 2, 3
PREC_NAMES = {"half": HALF, "single": SINGLE, "double": DOUBLE, "quad": QUAD}
UNIT_ROUNDOFF = {HALF: 2.0 ** -11, SINGLE: 2.0 ** -24, DOUBLE: 2.0 ** -53, QUAD: 2.0 ** -113}
MODE_PEROP, MODE_ACC32 = 0, 1
PAT_IDENTITY, PAT_A, PAT_A2 = 0, 1, 2

CF_CONVERGED, CF_FILLCAP, CF_ALPHA, CF_NOCAND, CF_SINGULAR, CF_NONFINITE = 1, 2, 4, 8, 16, 32
IR_CONVERGED, IR_MAXSTEPS, IR_BREAKDOWN, IR_NONFINITE, IR_STAGNATED = 1, 2, 4, 8, 16
STOP_BACKWARD, STOP_FIXED, STOP_CORRECTION = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spai_ir_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class SpaiOpts(C.Structure):
    _fields_ = [("init", C.c_int), ("adaptive", C.c_int), ("eps", C.c_double),
                ("alpha", C.c_int), ("beta", C.c_int), ("max_fill", C.c_int),
                ("uf", C.c_int), ("mode", C.c_int), ("rho_restricted", C.c_int),
                ("scale", C.c_int)]


class GmresOpts(C.Structure):
    _fields_ = [("ug", C.c_int), ("up", C.c_int), ("tau", C.c_double), ("maxit", C.c_int), ("orth", C.c_int),
                ("side", C.c_int), ("kmode", C.c_int)]


class IrOpts(C.Structure):
    _fields_ = [("uf", C.c_int), ("u", C.c_int), ("ug", C.c_int), ("up", C.c_int),
                ("ur", C.c_int), ("mode", C.c_int), ("tau", C.c_double),
                ("gmres_maxit", C.c_int), ("imax", C.c_int), ("stop_tol", C.c_double), ("orth", C.c_int),
                ("side", C.c_int), ("stop_rule", C.c_int), ("kmode", C.c_int)]


def lib():
    """The compiled oracle (built on first use)."""
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _lib.orc_chop_half.restype = C.c_double
            _lib.orc_chop_half.argtypes = [C.c_double]
            _lib.orc_round.restype = C.c_double
            _lib.orc_round.argtypes = [C.c_double, C.c_int]
            _lib.orc_dot.restype = C.c_double
        return _lib


def set_threads(n: int = 0) -> int:
    """Threads of the SPAI column loop (0: keep); returns the number in use."""
    return int(lib().orc_set_threads(C.c_int(int(n))))


def _p(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _csr(A):
    rp = np.ascontiguousarray(A[0], dtype=np.int64)
    ci = np.ascontiguousarray(A[1], dtype=np.int32)
    va = np.ascontiguousarray(A[2], dtype=np.float64)
    return rp, ci, va


def prec(p) -> int:
    """Precision code of a name ("half", "single", "double", "quad") or of a code."""
    return PREC_NAMES[p] if isinstance(p, str) else int(p)


def chop_half(x):
    """Round to IEEE binary16, round-to-nearest-even with subnormals and overflow to
    infinity: the chop model of half precision the paper's experiments use (Section 4)."""
    L = lib()
    x = np.asarray(x, dtype=np.float64)
    return np.vectorize(L.orc_chop_half, otypes=[np.float64])(x) if x.ndim else L.orc_chop_half(float(x))


def round_to(x, p):
    """Round every entry to precision p (Table 1's formats; half by chop_half)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(x)
    lib().orc_round_array(C.c_int64(x.size), _p(x, C.c_double), C.c_int(prec(p)), _p(out, C.c_double))
    return out


def half_ops(a, b, op: int):
    """One half-precision operation per entry pair (op 0 +, 1 -, 2 *, 3 /, other sqrt|a|):
    operands rounded to binary16, the result computed in double (exact for + - *, and the
    second rounding of / and sqrt is innocuous since 53 >= 2 * 11 + 2) and rounded to binary16,
    the per-operation model of Section 4."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    out = np.empty_like(a)
    lib().orc_half_ops(C.c_int(a.size), _p(a, C.c_double), _p(b, C.c_double), C.c_int(op), _p(out, C.c_double))
    return out


def dot(x, y, p="double", mode=MODE_PEROP):
    """Inner product in precision p as every step of the oracle forms it."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    return lib().orc_dot(C.c_int(len(x)), _p(x, C.c_double), _p(y, C.c_double), C.c_int(prec(p)), C.c_int(mode))


def dense_ls(Abar, ebar, uf="double", mode=MODE_ACC32):
    """Householder least squares of Algorithm 1 on a dense (m x nc) block."""
    Abar = np.asfortranarray(Abar, dtype=np.float64)
    m, nc = Abar.shape
    ebar = np.ascontiguousarray(ebar, dtype=np.float64)
    mbar = np.zeros(nc)
    sbar = np.zeros(m)
    sn = C.c_double(0.0)
    fl = lib().orc_dense_ls(C.c_int(m), C.c_int(nc), _p(Abar, C.c_double), _p(ebar, C.c_double),
                            C.c_int(prec(uf)), C.c_int(mode), _p(mbar, C.c_double),
                            _p(sbar, C.c_double), C.byref(sn))
    return mbar, sbar, sn.value, fl


def rho(A, d, I, s, cand, uf="double", rho_restricted=False):
    """Candidate scores rho_j of the Grote-Huckle augmentation (Algorithm 1; reading R3):
    the norm of the residual s after its one-dimensional minimisation along column j of
    B = A^T D, rho_j^2 = ||s||^2 - (s^T b_j)^2 / ||b_j||^2."""
    rp, ci, va = _csr(A)
    n = len(rp) - 1
    I = np.ascontiguousarray(I, dtype=np.int32)
    s = np.ascontiguousarray(s, dtype=np.float64)
    cand = np.ascontiguousarray(cand, dtype=np.int32)
    d = np.ascontiguousarray(d, dtype=np.float64)
    out = np.zeros(len(cand))
    lib().orc_rho(C.c_int(n), _p(rp, C.c_int64), _p(ci, C.c_int32), _p(va, C.c_double), _p(d, C.c_double),
                  C.c_int(len(I)), _p(I, C.c_int32), _p(s, C.c_double), C.c_int(len(cand)),
                  _p(cand, C.c_int32), C.c_int(prec(uf)), C.c_int(int(rho_restricted)), _p(out, C.c_double))
    return out


def select(cand, rho_vals, nmax, uf="double"):
    """Indices Algorithm 1 adds (reading R4): of the candidates with rho at most the
    mean, the nmax smallest rho, ties to the smaller index."""
    cand = np.ascontiguousarray(cand, dtype=np.int32)
    rv = np.ascontiguousarray(rho_vals, dtype=np.float64)
    sel = np.zeros(max(nmax, 1), dtype=np.int32)
    k = lib().orc_select(C.c_int(len(cand)), _p(cand, C.c_int32), _p(rv, C.c_double), C.c_int(prec(uf)),
                         C.c_int(nmax), _p(sel, C.c_int32))
    return sel[:k].copy()


def spai(A, init=PAT_IDENTITY, adaptive=False, eps=0.5, alpha=-1, beta=8, max_fill=30, uf="double",
         mode=MODE_ACC32, rho_restricted=False, scale=True, cols=None):
    """SPAI of Algorithm 1 run on A^T D; returns a dict with P = M^T D pieces.

    ``P_rows[k]`` / ``P_vals[k]`` hold row k of P (= column k of M scaled by
    d(J_k)); ``mbar`` holds the u_f solution values.  With ``cols`` only
    those columns are computed (the other entries are left zero).
    """
    rp, ci, va = _csr(A)
    n = len(rp) - 1
    F = int(max_fill)
    o = SpaiOpts(int(init), int(bool(adaptive)), float(eps), int(alpha), int(beta), F, prec(uf), int(mode),
                 int(bool(rho_restricted)), int(bool(scale)))
    d = np.zeros(n)
    Jcnt = np.zeros(n, dtype=np.int32)
    Jidx = np.full(n * F, -1, dtype=np.int32)
    mval = np.zeros(n * F)
    colres = np.zeros(n)
    colres64 = np.zeros(n)
    flags = np.zeros(n, dtype=np.int32)
    nsolve = np.zeros(n, dtype=np.int32)
    Icnt = np.zeros(n, dtype=np.int32)
    if cols is None:
        ncols, cptr = 0, None
    else:
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        ncols, cptr = len(cols), _p(cols, C.c_int32)
    lib().orc_spai(C.c_int(n), _p(rp, C.c_int64), _p(ci, C.c_int32), _p(va, C.c_double), C.byref(o),
                   C.c_int(ncols), cptr, _p(d, C.c_double), _p(Jcnt, C.c_int32), _p(Jidx, C.c_int32),
                   _p(mval, C.c_double), _p(colres, C.c_double), _p(colres64, C.c_double),
                   _p(flags, C.c_int32), _p(nsolve, C.c_int32), _p(Icnt, C.c_int32))
    return dict(n=n, max_fill=F, d=d, Jcnt=Jcnt, Jidx=Jidx.reshape(n, F), mbar=mval.reshape(n, F),
                colres=colres, colres64=colres64, flags=flags, nsolve=nsolve, Icnt=Icnt)


def assemble_P(S, up="double", uf=None):
    """Row k of P = mbar_k * d(J_k) (P = M^T D), values rounded to u_p (and u_f).

    Returns (rowptr, col, val_up, val_uf) with val_* as float64 arrays.
    """
    n, F = S["n"], S["max_fill"]
    cnt = S["Jcnt"].astype(np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(cnt)
    mask = np.arange(F)[None, :] < cnt[:, None]
    col = S["Jidx"][mask].astype(np.int32)
    raw = (S["mbar"] * S["d"][np.clip(S["Jidx"], 0, None)])[mask]
    val_up = round_to(raw, up) if prec(up) != DOUBLE else raw.copy()
    val_uf = None if uf is None else (round_to(raw, uf) if prec(uf) != DOUBLE else raw.copy())
    return rowptr, col, val_up, val_uf


def transpose_csr(A):
    """CSR of A^T (sorted column indices); a library transpose, no arithmetic."""
    rp, ci, va = _csr(A)
    n = len(rp) - 1
    M = sp.csr_matrix((va, ci, rp), shape=(n, n)).T.tocsr()
    M.sort_indices()
    return M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float64)


def spai_right(A, up="double", uf=None, **kw):
    """Right SPAI (A P ~ I, reading R14): the transpose of the left SPAI of A^T.

    Algorithm 1 run on (A^T)^T D = A D with D scaling the columns of A gives
    M ~ (A D)^{-1}; the left assembly of that run is M^T D, whose transpose
    D M satisfies A (D M) ~ I.  Returns (S, P) with S the run's dict (per
    column of M, i.e. per row of P^T) and P = (rowptr, col, val_up, val_uf).
    """
    S = spai(transpose_csr(A), **kw)
    rp, ci, vup, vuf = assemble_P(S, up, uf)
    n = S["n"]
    perm = sp.csr_matrix((np.arange(len(ci), dtype=np.float64) + 1.0, ci, rp), shape=(n, n)).T.tocsr()
    perm.sort_indices()
    idx = perm.data.astype(np.int64) - 1
    P = (perm.indptr.astype(np.int64), perm.indices.astype(np.int32), vup[idx],
         None if vuf is None else vuf[idx])
    return S, P


def spmv(A, x, p="double", mode=MODE_PEROP):
    """y = A x in precision p (the products of Algorithm 3 in u_p; mode selects
    per-operation rounding or binary32 accumulation for half)."""
    rp, ci, va = _csr(A)
    n = len(rp) - 1
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(n)
    lib().orc_spmv(C.c_int(n), _p(rp, C.c_int64), _p(ci, C.c_int32), _p(va, C.c_double),
                   _p(x, C.c_double), C.c_int(prec(p)), C.c_int(mode), _p(y, C.c_double))
    return y


def residual(A, b, x, ur="double", u="double"):
    """r = b - A x computed in u_r and stored in u (Algorithm 3, residual line)."""
    rp, ci, va = _csr(A)
    n = len(rp) - 1
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    r = np.zeros(n)
    lib().orc_residual(C.c_int(n), _p(rp, C.c_int64), _p(ci, C.c_int32), _p(va, C.c_double),
                       _p(b, C.c_double), _p(x, C.c_double), C.c_int(prec(ur)), C.c_int(prec(u)),
                       _p(r, C.c_double))
    return r


ORTH_MGS, ORTH_CGS2, ORTH_MGS_ICWY = 0, 1, 2
SIDE_LEFT, SIDE_RIGHT = 0, 1


def gmres(A, r, P=None, ug="double", up="double", tau=1e-8, maxit=None, orth=ORTH_MGS, side=SIDE_LEFT,
          kmode=MODE_PEROP):
    """One GMRES solve from d = 0 (MGS, CGS2 or the one-reduction MGS): left, (P A) d = P r; right,
    (A P) u = r and d = P u.  kmode: at u_g or u_p = half, MODE_PEROP rounds every operation to half
    (the paper's chop model), MODE_ACC32 (orth 2 only) stores vectors in half and computes in binary32."""
    rp, ci, va = _csr(A)
    n = len(rp) - 1
    r = np.ascontiguousarray(r, dtype=np.float64)
    d = np.zeros(n)
    bd = C.c_int(0)
    rr = C.c_double(0.0)
    o = GmresOpts(prec(ug), prec(up), float(tau), int(maxit if maxit is not None else min(n, 500)), int(orth),
                  int(side), int(kmode))
    if P is None:
        pp = (None, None, None)
    else:
        prp, pci, pva = _csr(P)
        pp = (_p(prp, C.c_int64), _p(pci, C.c_int32), _p(pva, C.c_double))
    k = lib().orc_gmres(C.c_int(n), _p(rp, C.c_int64), _p(ci, C.c_int32), _p(va, C.c_double), pp[0], pp[1],
                        pp[2], _p(r, C.c_double), C.byref(o), _p(d, C.c_double), C.byref(bd), C.byref(rr))
    if k < 0:
        raise ValueError("kmode MODE_ACC32 at u_g or u_p = half is defined for the one-reduction MGS only")
    return d, k, bool(bd.value), rr.value


def default_stop_tol(A, u) -> float:
    """Reading R8: q * u with q the largest number of nonzeros in a row."""
    rp = np.asarray(A[0])
    q = int(np.max(np.diff(rp))) if len(rp) > 1 else 1
    return q * UNIT_ROUNDOFF[prec(u)]


def gmres_ir(A, b, P=None, uf="single", u="double", ug="double", up="double", ur="quad",
             tau=1e-8, gmres_maxit=None, imax=10, stop_tol=None, mode=MODE_ACC32, orth=ORTH_MGS, side=SIDE_LEFT,
             stop_rule=STOP_BACKWARD, kmode=MODE_PEROP):
    """SPAI-GMRES-IR (Algorithm 3) given P = (rowptr, col, val_up, val_uf) or None; side selects left
    (Algorithm 3) or right preconditioning of the GMRES solves (reading R14); stop_rule and stop_tol
    the stopping rule of reading R8 (default threshold: q u for the backward rule, u for the correction
    rule); kmode the arithmetic of the Krylov part at u_g or u_p = half (see gmres)."""
    if kmode == MODE_ACC32 and orth != ORTH_MGS_ICWY and (prec(ug) == HALF or prec(up) == HALF):
        raise ValueError("kmode MODE_ACC32 at u_g or u_p = half is defined for the one-reduction MGS only")
    rp, ci, va = _csr(A)
    n = len(rp) - 1
    b = np.ascontiguousarray(b, dtype=np.float64)
    if stop_tol is None:
        stop_tol = UNIT_ROUNDOFF[prec(u)] if stop_rule == STOP_CORRECTION else default_stop_tol(A, u)
    o = IrOpts(prec(uf), prec(u), prec(ug), prec(up), prec(ur), int(mode), float(tau),
               int(gmres_maxit if gmres_maxit is not None else min(n, 500)), int(imax), float(stop_tol), int(orth),
               int(side), int(stop_rule), int(kmode))
    x = np.zeros(n)
    its = np.zeros(imax + 1, dtype=np.int32)
    nbe = np.full(imax + 1, np.nan)
    steps = C.c_int(0)
    if P is None:
        pp = (None, None, None, None)
    else:
        prp = np.ascontiguousarray(P[0], dtype=np.int64)
        pci = np.ascontiguousarray(P[1], dtype=np.int32)
        pup = np.ascontiguousarray(P[2], dtype=np.float64)
        puf = np.ascontiguousarray(P[3] if P[3] is not None else P[2], dtype=np.float64)
        keep = (prp, pci, pup, puf)
        pp = (_p(prp, C.c_int64), _p(pci, C.c_int32), _p(pup, C.c_double), _p(puf, C.c_double))
    status = lib().orc_gmres_ir(C.c_int(n), _p(rp, C.c_int64), _p(ci, C.c_int32), _p(va, C.c_double),
                                pp[0], pp[1], pp[2], pp[3], _p(b, C.c_double), C.byref(o), _p(x, C.c_double),
                                _p(its, C.c_int32), _p(nbe, C.c_double), C.byref(steps))
    s = steps.value
    return dict(x=x, steps=s, its=its[:s].copy(), nbe=nbe[:s + 1].copy(), status=status,
                total_its=int(its[:s].sum()))


def arnoldi(A, r, P=None, k=10, ug="double", up="double", orth=ORTH_MGS):
    """k Arnoldi steps on (P A); returns (V n x (m), H (k+1) x k) with m columns produced."""
    rp, ci, va = _csr(A)
    n = len(rp) - 1
    r = np.ascontiguousarray(r, dtype=np.float64)
    V = np.zeros((k + 1, n))
    H = np.zeros((k, k + 1))
    if P is None:
        pp = (None, None, None)
    else:
        prp, pci, pva = _csr(P)
        pp = (_p(prp, C.c_int64), _p(pci, C.c_int32), _p(pva, C.c_double))
    m = lib().orc_arnoldi(C.c_int(n), _p(rp, C.c_int64), _p(ci, C.c_int32), _p(va, C.c_double), pp[0], pp[1],
                          pp[2], _p(r, C.c_double), C.c_int(prec(ug)), C.c_int(prec(up)), C.c_int(int(orth)),
                          C.c_int(k), _p(V, C.c_double), _p(H, C.c_double))
    return V[:m].T.copy(), H.T.copy()
