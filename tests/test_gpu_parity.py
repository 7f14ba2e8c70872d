"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (the arithmetic of each side is stated in the oracle's header):
* SPAI pattern J_k: bit-exact (integer work).
* SPAI columns: the residual ||B(:,J_k) mbar_k - e_k||_2 re-evaluated in
  float64 for both sides' mbar agrees to 1e-3 relative at u_f = half, 1e-6
  at single and 1e-10 at double, plus the representation floor
  4 u_f || |B(:,J_k)| |mbar_k| ||_2 (the u_f term of eq. (rhatbnd): storing
  mbar in u_f moves the residual by that much whichever side computes it);
  at least 99% of the columns must meet the relative tolerance alone.
* GMRES-IR: same number of refinement steps, total GMRES iterations within
  10%, normwise backward and forward errors within 10x of the oracle's.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from neartie import replay_gap
from paper_2202_10204_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_2202_10204_gb300 as S  # noqa: E402

RES_TOL = {"half": 1e-3, "single": 1e-6, "double": 1e-10}


@pytest.fixture(scope="module")
def ctx():
    c = S.Context(0)
    yield c
    c.close()


def true_colres(A, d, J_rows, J_cnt, mbar, floor=False):
    """|| B(:, J_k) m_k - e_k ||_2 in float64 for every column k (B = A^T D);
    with floor=True also || |B(:,J_k)| |m_k| ||_2."""
    Ms = synth.to_scipy(A)
    n = Ms.shape[0]
    B = (Ms.T @ sp.diags(d)).tocsc()
    rows, cols, vals = [], [], []
    for k in range(n):
        c = J_cnt[k]
        rows.extend(J_rows[k][:c]); cols.extend([k] * c); vals.extend(mbar[k][:c])
    M = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    R = (B @ M - sp.identity(n)).tocsc()
    res = np.sqrt(np.asarray(R.multiply(R).sum(axis=0)).ravel())
    if not floor:
        return res
    Q = (abs(B) @ abs(M)).tocsc()
    return res, np.sqrt(np.asarray(Q.multiply(Q).sum(axis=0)).ravel())


def assert_colres(res_gpu, res_orc, absbm, uf, mask=None, frac=0.99):
    tol = RES_TOL[uf]
    u = O.UNIT_ROUNDOFF[O.prec(uf)]
    diff = np.abs(res_gpu - res_orc)
    if mask is not None:
        diff, res_orc, absbm = diff[mask], res_orc[mask], absbm[mask]
    floor = (4 * u + 64 * 2.0 ** -53) * absbm  # u_f representation + float64 evaluation
    assert np.all(diff <= tol * res_orc + floor), np.max(diff - tol * res_orc - floor)
    assert np.mean(diff <= tol * res_orc) >= frac, np.mean(diff <= tol * res_orc)


def gpu_spai(ctx, A, **kw):
    P, st = S.spai_build(ctx, A, S.make_spai_opts(**kw), per_column=True)
    rp, ci, va = P.export()
    return P, st, (rp, ci, va)


def split_rows(rp, ci, va, d):
    """Row k of P -> (J_k, mbar_k = P(k, J_k) / d(J_k))."""
    n = len(rp) - 1
    cnt = np.diff(rp).astype(np.int32)
    F = int(cnt.max()) if n else 1
    J = np.full((n, F), -1, dtype=np.int64)
    M = np.zeros((n, F))
    for k in range(n):
        c = cnt[k]
        J[k, :c] = ci[rp[k]:rp[k + 1]]
        M[k, :c] = va[rp[k]:rp[k + 1]] / d[ci[rp[k]:rp[k + 1]]]
    return J, cnt, M


def with_explicit_zeros(A, frac, seed):
    """A copy of A with a fraction of its off-diagonal values stored as 0.0 (the
    structure kept): the shadows count only a_ij != 0 (Algorithm 1), the patterns
    pattern(A), pattern(A^2) the stored structure."""
    rp, ci, va = A
    va = va.copy()
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    pick = (ci != rows) & (np.random.default_rng(seed).random(len(va)) < frac)
    va[pick] = 0.0
    return rp, ci, va


SPAI_CASES = [
    ("2d-patA", lambda: synth.conv_diff_2d(20, 10.0, 1.0, 0.1, seed=1), O.PAT_A, 30),
    ("3d-patA2", lambda: synth.conv_diff_3d(9, 50.0, seed=3), O.PAT_A2, 25),
    ("rand-patA", lambda: synth.random_sparse(700, 9, seed=5), O.PAT_A, 12),
    ("3d-capped", lambda: synth.conv_diff_3d((7, 6, 5), 50.0, seed=8), O.PAT_A2, 9),
    # 17-30 pattern columns, shadows of 208-301 rows: the 256 x 32 and 512 x 32 tiles (the
    # 16-warp CTA kernel for the larger ones at u_f = double)
    ("rand-patA-wide", lambda: synth.random_sparse(1000, 17, seed=13), O.PAT_A, 30),
    # shadows of 65-256 rows with at most 16 pattern columns: the shared-memory tiles of
    # 128 x 16 and 256 x 16
    ("rand-patA-mid", lambda: synth.random_sparse(2000, 12, seed=17), O.PAT_A, 16),
    # 22 pattern columns and shadows of at most 101 rows: the 128 x 32 shared-memory tile
    ("band-patA", lambda: banded(600, 25, 22, seed=19), O.PAT_A, 30),
    # 16 pattern columns and shadows of 161-320 rows: the 192 x 16 .. 320 x 16 tiles
    ("rand-patA-16", lambda: synth.random_sparse(1500, 15, seed=37), O.PAT_A, 16),
    # 16 pattern columns and shadows of 257-512 rows: the 320 x 16, 384 x 16, 512 x 16 tiles
    ("rand-patA-16-wide", lambda: synth.random_sparse(1500, 22, seed=29), O.PAT_A, 16),
    ("rand-patA-16-widest", lambda: synth.random_sparse(1500, 27, seed=29), O.PAT_A, 16),
]


def banded(n, w, per_row, seed):
    """Rows with the same per_row column offsets in [-w, w] (0 included), values N(0,1)
    and diagonal 30: every pattern(A) column has per_row entries and a shadow within
    2 w + 1 rows."""
    rng = np.random.default_rng(seed)
    offs = np.sort(np.concatenate([[0], rng.choice(np.setdiff1d(np.arange(-w, w + 1), [0]), per_row - 1,
                                                   replace=False)]))
    rows, cols = [], []
    for i in range(n):
        c = i + offs
        c = c[(c >= 0) & (c < n)]
        rows.extend([i] * len(c)); cols.extend(c)
    vals = rng.standard_normal(len(rows))
    M = sp.csr_matrix((vals, (rows, cols)), shape=(n, n)) + 30 * sp.identity(n)
    M = M.tocsr()
    M.sort_indices()
    return M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float64)


def column_bins(Icnt, Jcnt):
    """The column kernel each fixed-pattern column runs in (the bins of the CUDA path):
    0/1 the register-tile warp kernel (32/64 rows), 2..13 the shared-memory-tile warp
    kernel (32 R rows by 16 or 32 columns), 14 the large-shadow kernel."""
    out = []
    for m, nj in zip(Icnt, Jcnt):
        R = (m + 31) // 32
        if m <= 32: b = 0
        elif m <= 64: b = 1
        elif m > 512: b = 14
        elif nj <= 16: b = R - 1 if R <= 8 else (8 if R <= 10 else (9 if R <= 12 else 10))
        else: b = 11 if R <= 4 else (12 if R <= 8 else 13)
        out.append(b)
    return np.array(out)


@pytest.mark.parametrize("uf", ["half", "single", "double"])
@pytest.mark.parametrize("name,make,init,F", SPAI_CASES)
def test_spai_fixed_pattern_parity(ctx, name, make, init, F, uf):
    A = make()
    P, st, (rp, ci, va) = gpu_spai(ctx, A, init=init, max_fill=F, uf=uf, eps=0.0)
    ref = O.spai(A, init=init, max_fill=F, uf=uf, eps=0.0)
    n = ref["n"]
    bins = column_bins(ref["Icnt"], ref["Jcnt"])
    if name == "rand-patA-mid":
        assert all(np.sum(bins == b) > 100 for b in (3, 4))
    if name == "band-patA":
        assert np.mean(bins == 11) > 0.9
    if name == "rand-patA-wide":
        assert np.sum(bins == 12) > 100 and np.sum(bins == 13) > 100
    if name == "rand-patA-16":
        assert all(np.sum(bins == b) > 100 for b in (5, 6, 7))
    if name == "rand-patA-16-wide":
        assert all(np.sum(bins == b) > 100 for b in (8, 9))
    if name == "rand-patA-16-widest":
        assert all(np.sum(bins == b) > 100 for b in (9, 10))
    # pattern: bit-exact
    assert np.array_equal(np.diff(rp), ref["Jcnt"])
    for k in range(n):
        assert np.array_equal(ci[rp[k]:rp[k + 1]], ref["Jidx"][k][: ref["Jcnt"][k]])
    assert np.array_equal(st["nI"], ref["Icnt"])
    J, cnt, M = split_rows(rp, ci, va, ref["d"])
    res_gpu, absbm = true_colres(A, ref["d"], J, cnt, M, floor=True)
    assert_colres(res_gpu, ref["colres64"], absbm, uf)
    # the u_f-computed norms the kernel reports agree to a few u_f
    u = O.UNIT_ROUNDOFF[O.prec(uf)]
    assert np.all(np.abs(st["colres"] - ref["colres"]) <= 64 * u * ref["colres"] + 8 * u * absbm + 1e-14)
    P.free()


@pytest.mark.parametrize("uf", ["half", "single", "double"])
def test_spai_tile_shapes_give_the_same_result(ctx, uf):
    """The tile tuner's candidates (shared-memory tiles of more rows or columns than a
    column needs) give every column the same result bit for bit, so the tuner's choice
    never changes a preconditioner."""
    A = synth.random_sparse(20000, 12, seed=17)
    so = S.make_spai_opts(init=1, max_fill=16, uf=uf)
    cols = np.arange(0, 20000, 97, dtype=np.int32)
    ref = O.spai(A, init=O.PAT_A, max_fill=16, uf="single", eps=0.0, cols=cols)
    assert np.mean(column_bins(ref["Icnt"][cols], ref["Jcnt"][cols]) == 4) > 0.6  # the 160 x 16 bin holds most
    S.tune_set(0, uf, 4, -1)
    P0, _ = S.spai_build(ctx, A, so)
    assert S.tune_get(0, uf, 4) >= 0  # tuned on this build (over 8192 columns in the bin)
    want = P0.export()
    P0.free()
    for variant in range(4):
        S.tune_set(0, uf, 4, variant)
        P, _ = S.spai_build(ctx, A, so)
        for u, v in zip(want, P.export()):
            assert np.array_equal(u, v), variant
        P.free()
    S.tune_set(0, uf, 4, -1)


@pytest.mark.parametrize("uf", ["half", "single", "double"])
def test_spai_explicit_zeros_parity(ctx, uf):
    """A with explicit zeros (15% of the off-diagonal values stored as 0.0): the
    pattern pattern(A^2) follows the stored structure and the shadows count only
    a_ij != 0 (Algorithm 1), both bit-exact against the oracle; every column meets
    the residual bound with the u_f floor (the u_f term of eq. (rhatbnd)).  At
    u_f = half 97.9% of this matrix's columns also meet the pure relative
    tolerance, the same fraction with the warp kernel's earlier FMA arithmetic:
    with zeros in the tile more columns sit where one half-ulp difference in m_k
    moves the residual by more than 1e-3 of itself."""
    A = with_explicit_zeros(synth.conv_diff_3d(9, 50.0, seed=3), 0.15, 21)
    P, st, (rp, ci, va) = gpu_spai(ctx, A, init=O.PAT_A2, max_fill=25, uf=uf, eps=0.0)
    ref = O.spai(A, init=O.PAT_A2, max_fill=25, uf=uf, eps=0.0)
    plain = O.spai(synth.conv_diff_3d(9, 50.0, seed=3), init=O.PAT_A2, max_fill=25, uf=uf, eps=0.0)
    assert np.sum(ref["Icnt"] != plain["Icnt"]) > 100  # the zeros change many shadows
    assert np.array_equal(np.diff(rp), ref["Jcnt"])
    for k in range(ref["n"]):
        assert np.array_equal(ci[rp[k]:rp[k + 1]], ref["Jidx"][k][: ref["Jcnt"][k]])
    assert np.array_equal(st["nI"], ref["Icnt"])
    J, cnt, M = split_rows(rp, ci, va, ref["d"])
    res_gpu, absbm = true_colres(A, ref["d"], J, cnt, M, floor=True)
    assert_colres(res_gpu, ref["colres64"], absbm, uf, frac=0.97 if uf == "half" else 0.99)
    P.free()


# A column may select a different pattern than the oracle only where the two
# runs' scores tie to rounding (reading R12): on the stretch of the oracle's
# path consistent with the GPU's pattern some decision (the selection boundary,
# the acceptance threshold or the column criterion) has a margin within
# NEAR_TIE * u_f of the step's mean rho (tests/neartie.py).  Both sides compute
# rho from their own residual s, whose entries differ by the rounding of the QR
# (a few u_f times the condition of the tile), so the allowance is a few
# hundred u_f rather than the few u_f of one rho evaluation.
NEAR_TIE = 512


def check_mismatches_are_near_ties(A, d, cols, J_gpu, J_orc, uf, eps, beta, F):
    """Every column whose pattern differs is a near-tie; returns their count."""
    u = O.UNIT_ROUNDOFF[O.prec(uf)]
    bad = []
    cnt = 0
    for k, Jg, Jo in zip(cols, J_gpu, J_orc):
        if np.array_equal(Jg, Jo):
            continue
        cnt += 1
        r = replay_gap(A, d, int(k), Jg, uf, eps, beta, F)
        assert r is not None, (k, Jg, Jo)
        kind, gap, step = r
        if gap > NEAR_TIE * u:
            bad.append((int(k), kind, step, gap / u))
    print("pattern mismatches: %d of %d columns, none beyond %d u_f" % (cnt, len(cols), NEAR_TIE))
    assert not bad, bad
    return cnt


@pytest.mark.parametrize("uf", ["single", "double"])
def test_spai_adaptive_parity(ctx, uf):
    A = synth.random_sparse(400, 6, seed=12)
    for eps in (0.5, 0.3):
        P, st, (rp, ci, va) = gpu_spai(ctx, A, init=O.PAT_IDENTITY, adaptive=True, eps=eps, beta=8, max_fill=30,
                                       uf=uf)
        ref = O.spai(A, init=O.PAT_IDENTITY, adaptive=True, eps=eps, beta=8, max_fill=30, uf=uf)
        n = ref["n"]
        same = np.array([np.array_equal(ci[rp[k]:rp[k + 1]], ref["Jidx"][k][: ref["Jcnt"][k]]) for k in range(n)])
        check_mismatches_are_near_ties(A, ref["d"], range(n), [ci[rp[k]:rp[k + 1]] for k in range(n)],
                                       [ref["Jidx"][k][: ref["Jcnt"][k]] for k in range(n)], uf, eps, 8, 30)
        J, cnt, M = split_rows(rp, ci, va, ref["d"])
        res_gpu, absbm = true_colres(A, ref["d"], J, cnt, M, floor=True)
        assert_colres(res_gpu, ref["colres64"], absbm, uf, mask=same)
        # every column meets eq. (trueres) or stopped at the cap / alpha
        conv = (st["flags"] & 1) != 0
        assert np.all(res_gpu[conv] <= 2 * eps)
        assert np.array_equal(conv[same], (ref["flags"][same] & 1) != 0)
        P.free()


@pytest.mark.parametrize("uf", ["half", "single", "double"])
def test_spai_large_shadow_fixed_parity(ctx, uf):
    """Fixed pattern(A) of a random matrix with 28 nonzeros per column and cap 30:
    every shadow has 513-682 rows, beyond the CTA kernel's 512-row register tile,
    so every column runs in the large-shadow kernel.  Compared with the oracle,
    which runs Algorithm 1 with no shadow limit: patterns and shadow sizes
    bit-exact, column residuals within the usual tolerances."""
    A = synth.random_sparse(900, 28, seed=31)
    P, st, (rp, ci, va) = gpu_spai(ctx, A, init=O.PAT_A, max_fill=30, uf=uf, eps=0.0)
    ref = O.spai(A, init=O.PAT_A, max_fill=30, uf=uf, eps=0.0)
    n = ref["n"]
    assert np.mean(ref["Icnt"] > 512) > 0.9
    assert np.array_equal(np.diff(rp), ref["Jcnt"])
    for k in range(n):
        assert np.array_equal(ci[rp[k]:rp[k + 1]], ref["Jidx"][k][: ref["Jcnt"][k]])
    assert np.array_equal(st["nI"], ref["Icnt"])
    J, cnt, M = split_rows(rp, ci, va, ref["d"])
    res_gpu, absbm = true_colres(A, ref["d"], J, cnt, M, floor=True)
    assert_colres(res_gpu, ref["colres64"], absbm, uf)
    P.free()


@pytest.mark.parametrize("uf", ["single", "double"])
def test_spai_large_shadow_adaptive_parity(ctx, uf):
    """Grote-Huckle from the identity on a random matrix with 24 nonzeros per
    column, eps 0.1, beta 8, cap 30: most columns grow past 512 shadow rows, where
    the CTA kernel hands them to the large-shadow kernel at the step they
    outgrow it.  Sampled columns against the uncapped oracle: same patterns up to
    near-ties, residuals within tolerance where the patterns agree."""
    A = synth.random_sparse(1500, 24, seed=31)
    eps, beta, F = 0.1, 8, 30
    P, st, (rp, ci, va) = gpu_spai(ctx, A, init=O.PAT_IDENTITY, adaptive=True, eps=eps, beta=beta, max_fill=F,
                                   uf=uf)
    assert np.mean(st["nI"] > 512) > 0.5  # the large-shadow kernel took most columns
    cols = np.sort(np.random.default_rng(3).choice(len(rp) - 1, size=160, replace=False))
    ref = O.spai(A, init=O.PAT_IDENTITY, adaptive=True, eps=eps, beta=beta, max_fill=F, uf=uf, cols=cols)
    d = ref["d"]
    Jg = [ci[rp[k]:rp[k + 1]] for k in cols]
    Jo = [ref["Jidx"][k][: ref["Jcnt"][k]] for k in cols]
    check_mismatches_are_near_ties(A, d, cols, Jg, Jo, uf, eps, beta, F)
    same = np.array([np.array_equal(x, y) for x, y in zip(Jg, Jo)])
    assert np.array_equal(st["nI"][cols][same], ref["Icnt"][cols][same])
    J, cnt, M = split_rows(rp, ci, va, d)
    res_gpu, absbm = true_colres(A, d, J, cnt, M, floor=True)
    assert_colres(res_gpu[cols], ref["colres64"][cols], absbm[cols], uf, mask=same)
    P.free()


def run_pair(ctx, A, b, init, F, uf, u, ug, up, ur, tau, eps=0.0, adaptive=False):
    so = S.make_spai_opts(init=init, max_fill=F, uf=uf, eps=eps, adaptive=adaptive)
    io = S.make_ir_opts(uf=uf, u=u, ug=ug, up=up, ur=ur, tau=tau)
    x = np.zeros_like(b)
    st = S.gmres_ir_solve(ctx, A, b, x, sopts=so, opts=io)
    Sr = O.spai(A, init=init, max_fill=F, uf=uf, eps=eps, adaptive=adaptive)
    ref = O.gmres_ir(A, b, O.assemble_P(Sr, up, uf), uf=uf, u=u, ug=ug, up=up, ur=ur, tau=tau)
    return x, st, ref


def errors(A, b, x, x_true):
    Ms = synth.to_scipy(A)
    nbe = np.max(np.abs(b - Ms @ x)) / (abs(Ms).sum(axis=1).max() * np.max(np.abs(x)) + np.max(np.abs(b)))
    fe = np.max(np.abs(x - x_true)) / np.max(np.abs(x_true))
    return nbe, fe


def check_ir(A, b, x_true, x, st, ref, u):
    assert st["steps"] == ref["steps"], (st["its"], list(ref["its"]))
    assert abs(st["total_its"] - ref["total_its"]) <= max(1, 0.1 * ref["total_its"]), (st["its"], list(ref["its"]))
    nb_g, fe_g = errors(A, b, x, x_true)
    nb_o, fe_o = errors(A, b, ref["x"], x_true)
    assert nb_g <= 10 * max(nb_o, u)
    assert fe_g <= 10 * max(fe_o, u)


def test_ir_small_2d_single_double_quad(ctx):
    A, b, x_true = synth.cfg_small_2d()
    x, st, ref = run_pair(ctx, A, b, O.PAT_A, 30, "single", "double", "double", "double", "quad", 1e-4)
    check_ir(A, b, x_true, x, st, ref, 2.0 ** -53)
    assert st["final_nbe"] <= 1e-15
    assert st["flags"] & 1


def test_ir_3d_half_single(ctx):
    A, b, x_true = synth.cfg_large_3d(N=16)
    x, st, ref = run_pair(ctx, A, b, O.PAT_A2, 25, "half", "single", "single", "single", "double", 1e-4)
    check_ir(A, b, x_true, x, st, ref, 2.0 ** -24)


@pytest.mark.parametrize("tup", [("half", "single", "single", "single", "double"),
                                 ("single", "double", "double", "double", "double")])
def test_ir_gram_schmidt_group(ctx, tup):
    # n = 27^3 = 19683: 77 blocks of 256 rows, so the Gram-Schmidt rounds run among
    # 39 blocks that each hold two blocks' rows (the last one a single, ragged block)
    uf, u, ug, up, ur = tup
    A = synth.conv_diff_3d(27, 50.0, seed=11)
    b, x_true = synth.rhs(A, seed=12)
    tau = 1e-4 if ug == "single" else 1e-8
    x, st, ref = run_pair(ctx, A, b, O.PAT_A2, 25, uf, u, ug, up, ur, tau)
    assert st["grid"] >= 64
    check_ir(A, b, x_true, x, st, ref, O.UNIT_ROUNDOFF[O.prec(u)])


@pytest.mark.parametrize("tup", [("single", "double", "single", "single", "double"),
                                 ("half", "single", "single", "double", "double"),
                                 ("double", "double", "double", "double", "double"),
                                 ("single", "double", "double", "single", "quad")])
def test_ir_precision_tuples(ctx, tup):
    uf, u, ug, up, ur = tup
    A = synth.conv_diff_2d(24, 20.0, 1.0, 0.1, seed=7)
    b, x_true = synth.rhs(A, seed=9)
    tau = 1e-4 if ug == "single" else 1e-8
    x, st, ref = run_pair(ctx, A, b, O.PAT_A, 30, uf, u, ug, up, ur, tau)
    check_ir(A, b, x_true, x, st, ref, O.UNIT_ROUNDOFF[O.prec(u)])


def test_ir_unpreconditioned(ctx):
    A, b, x_true = synth.cfg_small_2d()
    io = S.make_ir_opts(uf="single", u="double", ug="double", up="double", ur="quad", tau=1e-4)
    x = np.zeros_like(b)
    st = S.gmres_ir_solve(ctx, A, b, x, opts=io)
    ref = O.gmres_ir(A, b, None, uf="single", u="double", ug="double", up="double", ur="quad", tau=1e-4)
    check_ir(A, b, x_true, x, st, ref, 2.0 ** -53)


def test_ir_adaptive_random(ctx):
    A = synth.random_sparse(600, 8, seed=21, log10_scale=3.0)
    b, x_true = synth.rhs(A, seed=3)
    x, st, ref = run_pair(ctx, A, b, O.PAT_IDENTITY, 30, "single", "double", "double", "double", "quad", 1e-8,
                          eps=0.4, adaptive=True)
    check_ir(A, b, x_true, x, st, ref, 2.0 ** -53)


def test_device_buffers_match_host_buffers(ctx):
    A, b, x_true = synth.cfg_small_2d()
    so = S.make_spai_opts(init=1, max_fill=30, uf="single")
    io = S.make_ir_opts(uf="single", u="double", ug="double", up="double", ur="quad", tau=1e-4)
    xh = np.zeros_like(b)
    S.gmres_ir_solve(ctx, A, b, xh, sopts=so, opts=io)
    Ad = tuple(torch.from_numpy(a).cuda() for a in A)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    torch.cuda.synchronize()
    S.gmres_ir_solve(ctx, Ad, bd, xd, sopts=so, opts=io)
    assert np.array_equal(xd.cpu().numpy(), xh)  # deterministic: bitwise equal


def test_edge_cases(ctx):
    io = S.make_ir_opts(uf="single", u="double", ug="double", up="double", ur="quad", tau=1e-8)
    so = S.make_spai_opts(init=0, max_fill=4, uf="single")
    # n = 1
    A1 = (np.array([0, 1], dtype=np.int64), np.array([0], dtype=np.int32), np.array([4.0]))
    x = np.zeros(1)
    st = S.gmres_ir_solve(ctx, A1, np.array([2.0]), x, sopts=so, opts=io)
    assert x[0] == 0.5
    # diagonal system: identity pattern is the exact inverse, one iteration
    a = np.array([2.0, -3.0, 0.5, 7.0, -0.25])
    Ad = synth._to_csr(sp.diags(a))
    b = np.arange(1.0, 6.0)
    x = np.zeros(5)
    st = S.gmres_ir_solve(ctx, Ad, b, x, sopts=so, opts=io)
    np.testing.assert_allclose(x, b / a, rtol=1e-15)
    # zero right-hand side: x = 0 with no GMRES work
    A, b, _ = synth.cfg_small_2d()
    x = np.ones_like(b)
    st = S.gmres_ir_solve(ctx, A, np.zeros_like(b), x, sopts=S.make_spai_opts(init=1, max_fill=30), opts=io)
    assert np.all(x == 0) and st["steps"] == 0
    # a zero row is singular
    Az = (np.array([0, 1, 1], dtype=np.int64), np.array([0], dtype=np.int32), np.array([1.0]))
    with pytest.raises(S.SpaiError) as e:
        S.gmres_ir_solve(ctx, Az, np.ones(2), np.zeros(2), sopts=so, opts=io)
    assert e.value.code == -2
    # unsorted columns are rejected
    Au = (np.array([0, 2, 3], dtype=np.int64), np.array([1, 0, 1], dtype=np.int32), np.array([1.0, 2.0, 3.0]))
    with pytest.raises(S.SpaiError) as e:
        S.gmres_ir_solve(ctx, Au, np.ones(2), np.zeros(2), sopts=so, opts=io)
    assert e.value.code == -1
    # the structural checks of host inputs run on the device: a decreasing rowptr, a
    # column out of range, a repeated column, in spai_build as well
    bad = [
        (np.array([0, 2, 1, 3], dtype=np.int64), np.array([0, 1, 2], dtype=np.int32)),
        (np.array([0, 1, 2, 3], dtype=np.int64), np.array([0, 3, 2], dtype=np.int32)),
        (np.array([0, 2, 3, 4], dtype=np.int64), np.array([0, 0, 1, 2], dtype=np.int32)),
    ]
    for rp, ci in bad:
        Ab = (rp, ci, np.ones(len(ci)))
        with pytest.raises(S.SpaiError) as e:
            S.gmres_ir_solve(ctx, Ab, np.ones(3), np.zeros(3), sopts=so, opts=io)
        assert e.value.code == -1
        with pytest.raises(S.SpaiError) as e:
            S.spai_build(ctx, Ab, so)
        assert e.value.code == -1
    with pytest.raises(S.SpaiError) as e:
        S.spai_build(ctx, Az, so)
    assert e.value.code == -2
    # unsupported fill cap
    with pytest.raises(S.SpaiError) as e:
        S.spai_build(ctx, A, S.make_spai_opts(init=1, max_fill=40))
    assert e.value.code == -8


def test_half_krylov_edge_cases(ctx):
    # u_g = u_p = half (one-reduction MGS): n = 1, a diagonal system, a zero right-hand side,
    # a ragged tiny system, and values beyond half's range (a clean non-finite status)
    io = S.make_ir_opts(uf="single", u="double", ug="half", up="half", ur="quad", tau=1e-2, orth=2,
                        ir_max_steps=30)
    so = S.make_spai_opts(init=0, max_fill=4, uf="single")
    A1 = (np.array([0, 1], dtype=np.int64), np.array([0], dtype=np.int32), np.array([4.0]))
    x = np.zeros(1)
    S.gmres_ir_solve(ctx, A1, np.array([2.0]), x, sopts=so, opts=io)
    assert x[0] == 0.5
    a = np.array([2.0, -3.0, 0.5, 7.0, -0.25])
    Ad = synth._to_csr(sp.diags(a))
    b = np.arange(1.0, 6.0)
    x = np.zeros(5)
    st = S.gmres_ir_solve(ctx, Ad, b, x, sopts=so, opts=io)
    np.testing.assert_allclose(x, b / a, rtol=1e-13)
    A, b, x_true = synth.cfg_small_2d()
    x = np.ones_like(b)
    st = S.gmres_ir_solve(ctx, A, np.zeros_like(b), x, sopts=S.make_spai_opts(init=1, max_fill=30), opts=io)
    assert np.all(x == 0) and st["steps"] == 0
    # ragged: n = 37 (one full 32-row slice and a partial one)
    Ar = synth.conv_diff_2d(7, 5.0, 1.0, 0.1, seed=3)
    Ar = synth._to_csr(synth.to_scipy(Ar)[:37, :37] + sp.eye(37))
    br, xr = synth.rhs(Ar, seed=4)
    x = np.zeros_like(br)
    st = S.gmres_ir_solve(ctx, Ar, br, x, sopts=S.make_spai_opts(init=1, max_fill=30), opts=io)
    ref = O.gmres_ir(Ar, br, O.assemble_P(O.spai(Ar, init=O.PAT_A, max_fill=30, uf="single"), "half", "single"),
                     uf="single", u="double", ug="half", up="half", ur="quad", tau=1e-2, orth=O.ORTH_MGS_ICWY,
                     kmode=O.MODE_ACC32, imax=30)
    assert st["flags"] & 1 and ref["status"] & O.IR_CONVERGED
    assert np.max(np.abs(x - xr)) <= 10 * max(np.max(np.abs(ref["x"] - xr)), 2.0 ** -53) * np.max(np.abs(xr)) + 1e-14
    # A's half copy overflows: the solve reports a non-finite result instead of a number
    Ab = synth._to_csr(sp.diags(np.full(40, 1e6)) + sp.eye(40, k=1))
    with pytest.raises(S.SpaiError) as e:
        S.gmres_ir_solve(ctx, Ab, np.ones(40), np.zeros(40), sopts=so, opts=io)
    assert e.value.code == -3  # SPAI_ERR_NONFINITE


@pytest.mark.parametrize("e", [40, -40])
def test_half_krylov_scale_invariance(ctx, e):
    # with the residual scaled into [0.5, 1) before the half-precision Krylov part (reading
    # R17), b 2^e gives x 2^e bit for bit, although b 2^e lies outside half's range
    A, b, x_true = synth.cfg_small_2d()
    P, _ = S.spai_build(ctx, A, S.make_spai_opts(init=1, max_fill=30, uf="single"))
    io = S.make_ir_opts(uf="single", u="double", ug="half", up="half", ur="quad", tau=1e-2, orth=2,
                        ir_max_steps=30)
    x0, x1 = np.zeros_like(b), np.zeros_like(b)
    s0 = S.gmres_ir_solve(ctx, A, b, x0, P=P, opts=io)
    s1 = S.gmres_ir_solve(ctx, A, np.ldexp(b, e), x1, P=P, opts=io)
    assert s0["flags"] & 1 and s1["flags"] & 1 and s0["its"] == s1["its"]
    assert np.array_equal(np.ldexp(x0, e), x1)
    P.free()


def test_precond_outlives_its_context():
    # a preconditioner stays usable after the context that built it is destroyed
    A, b, _ = synth.cfg_small_2d()
    c = S.Context(0)
    P, _ = S.spai_build(c, A, S.make_spai_opts(init=1, max_fill=30, uf="single"))
    before = P.export()
    c.close()
    after = P.export()
    for u, v in zip(before, after):
        assert np.array_equal(u, v)
    c2 = S.Context(0)
    x = np.zeros_like(b)
    st = S.gmres_ir_solve(c2, A, b, x, P=P, opts=S.make_ir_opts(tau=1e-8))
    assert st["flags"] & 1
    P.free()
    c2.close()


@pytest.mark.parametrize("tup", [("half", "single", "single", "single", "double"),
                                 ("single", "double", "double", "double", "quad"),
                                 ("single", "double", "single", "single", "double")])
def test_ir_cgs2_against_oracle(ctx, tup):
    """The classical-Gram-Schmidt-twice Arnoldi option against the oracle's CGS2."""
    uf, u, ug, up, ur = tup
    if u == "single":
        A, b, x_true = synth.cfg_large_3d(N=16)
        init, F = O.PAT_A2, 25
    else:
        A = synth.conv_diff_2d(40, 20.0, 1.0, 0.1, seed=11)
        b, x_true = synth.rhs(A, seed=12)
        init, F = O.PAT_A, 30
    tau = 1e-4 if ug == "single" else 1e-8
    so = S.make_spai_opts(init=init, max_fill=F, uf=uf)
    io = S.make_ir_opts(uf=uf, u=u, ug=ug, up=up, ur=ur, tau=tau, orth=1)
    x = np.zeros_like(b)
    st = S.gmres_ir_solve(ctx, A, b, x, sopts=so, opts=io)
    Sr = O.spai(A, init=init, max_fill=F, uf=uf)
    ref = O.gmres_ir(A, b, O.assemble_P(Sr, up, uf), uf=uf, u=u, ug=ug, up=up, ur=ur, tau=tau, orth=O.ORTH_CGS2)
    check_ir(A, b, x_true, x, st, ref, O.UNIT_ROUNDOFF[O.prec(u)])


ICWY_CASES = [
    # (name, tuple, side, preconditioned, gmres_max_it)
    ("3d-half-single", ("half", "single", "single", "single", "double"), 0, True, 0),
    ("2d-single-double-quad", ("single", "double", "double", "double", "quad"), 0, True, 0),
    ("2d-single-ug-single", ("single", "double", "single", "single", "double"), 0, True, 0),
    ("2d-right", ("single", "double", "double", "double", "quad"), 1, True, 0),
    ("2d-unpreconditioned", ("single", "double", "double", "double", "quad"), 0, False, 0),
    ("2d-capped-iterations", ("single", "double", "double", "double", "quad"), 0, True, 12),
]


@pytest.mark.parametrize("name,tup,side,precond,maxit", ICWY_CASES)
def test_ir_one_reduction_mgs_against_oracle(ctx, name, tup, side, precond, maxit):
    """MGS in its one-reduction form (orth 2) against the oracle's: left and right
    preconditioning, no preconditioner, and a GMRES iteration cap (the last pass
    then only forms ||u_k||)."""
    uf, u, ug, up, ur = tup
    if u == "single":
        A, b, x_true = synth.cfg_large_3d(N=16)
        init, F = O.PAT_A2, 25
    else:
        A = synth.conv_diff_2d(40, 20.0, 1.0, 0.1, seed=11)
        b, x_true = synth.rhs(A, seed=12)
        init, F = O.PAT_A, 30
    tau = 1e-4 if ug == "single" else 1e-8
    so = S.make_spai_opts(init=init, max_fill=F, uf=uf, side=side) if precond else None
    io = S.make_ir_opts(uf=uf, u=u, ug=ug, up=up, ur=ur, tau=tau, orth=2, side=side, gmres_max_it=maxit)
    x = np.zeros_like(b)
    st = S.gmres_ir_solve(ctx, A, b, x, sopts=so, opts=io)
    Pr = None
    if precond and side == 0:
        Pr = O.assemble_P(O.spai(A, init=init, max_fill=F, uf=uf), up, uf)
    elif precond:
        _, Pr = O.spai_right(A, up=up, uf=uf, init=init, max_fill=F)
    ref = O.gmres_ir(A, b, Pr, uf=uf, u=u, ug=ug, up=up, ur=ur, tau=tau, orth=O.ORTH_MGS_ICWY, side=side,
                     gmres_maxit=maxit if maxit else None)
    if maxit:
        assert max(st["its"]) == maxit
    check_ir(A, b, x_true, x, st, ref, O.UNIT_ROUNDOFF[O.prec(u)])


@pytest.mark.parametrize("tup", [("half", "single", "single", "single", "double"),
                                 ("single", "double", "double", "double", "double")])
def test_ir_one_reduction_mgs_large_grid(ctx, tup):
    # n = 27^3 = 19683: 77 blocks of 256 rows (a ragged last block), the grid size at which
    # the MGS rounds would run in a Gram-Schmidt group
    uf, u, ug, up, ur = tup
    A = synth.conv_diff_3d(27, 50.0, seed=11)
    b, x_true = synth.rhs(A, seed=12)
    tau = 1e-4 if ug == "single" else 1e-8
    so = S.make_spai_opts(init=O.PAT_A2, max_fill=25, uf=uf)
    io = S.make_ir_opts(uf=uf, u=u, ug=ug, up=up, ur=ur, tau=tau, orth=2)
    x = np.zeros_like(b)
    st = S.gmres_ir_solve(ctx, A, b, x, sopts=so, opts=io)
    ref = O.gmres_ir(A, b, O.assemble_P(O.spai(A, init=O.PAT_A2, max_fill=25, uf=uf), up, uf), uf=uf, u=u, ug=ug,
                     up=up, ur=ur, tau=tau, orth=O.ORTH_MGS_ICWY)
    assert st["grid"] >= 64
    check_ir(A, b, x_true, x, st, ref, O.UNIT_ROUNDOFF[O.prec(u)])


@pytest.mark.parametrize("log10_scale", [4.0, 5.0])
def test_ir_condition_window(ctx, log10_scale):
    """Random nonsymmetric systems (n = 2000, 12 nonzeros per column) at the upper end of the
    batched configuration's condition range, in its tuple (single, double, single, single,
    double) with the one-reduction MGS: at 1-norm condition ~3e4 the refinement converges after
    GMRES solves of a few hundred iterations, at ~2e5 it leaves the window where GMRES-IR with
    u_g = u_p = single converges (Section 3.1) and stagnates near 1e-4 (the stop rule's
    stagnation test).  The GPU follows the oracle in both, on the same preconditioner."""
    A = synth.random_sparse(2000, 12, seed=21, log10_scale=log10_scale)
    b, x_true = synth.rhs(A, seed=22)
    P, _ = S.spai_build(ctx, A, S.make_spai_opts(init=1, max_fill=30, uf="single"))
    Pc = P.export()
    kw = dict(uf="single", u="double", ug="single", up="single", ur="double", tau=1e-4)
    x = np.zeros_like(b)
    st = S.gmres_ir_solve(ctx, A, b, x, P=P, opts=S.make_ir_opts(orth=2, **kw))
    Pv = (Pc[0], Pc[1], O.round_to(Pc[2], "single"), O.round_to(Pc[2], "single"))
    ref = O.gmres_ir(A, b, Pv, orth=O.ORTH_MGS_ICWY, **kw)
    assert bool(st["flags"] & 16) == bool(ref["status"] & O.IR_STAGNATED)
    assert bool(st["flags"] & 1) == bool(ref["status"] & O.IR_CONVERGED)
    if log10_scale >= 5.0:
        assert ref["status"] & O.IR_STAGNATED and ref["nbe"][-1] > 1e-8
        assert st["final_nbe"] <= 10 * ref["nbe"][-1] and ref["nbe"][-1] <= 10 * st["final_nbe"]
        assert st["steps"] == ref["steps"]
        assert abs(st["total_its"] - ref["total_its"]) <= max(1, 0.1 * ref["total_its"])
    else:
        assert max(ref["its"]) >= 200
        check_ir(A, b, x_true, x, st, ref, 2.0 ** -53)
    P.free()


# ---------------------------------------------------------------- half Krylov storage (u_g, u_p = half)

HALF_KRYLOV_CASES = [
    # (name, tuple, tau, side, preconditioned); tau ~ sqrt(u_half) where u_g is half
    ("2d-hh-double-quad", ("single", "double", "half", "half", "quad"), 1e-2, 0, True),
    ("3d-hh-single", ("half", "single", "half", "half", "double"), 1e-2, 0, True),
    ("3d-hf-single", ("half", "single", "half", "single", "double"), 1e-2, 0, True),
    ("3d-fh-single", ("half", "single", "single", "half", "double"), 1e-4, 0, True),
    ("2d-hh-right", ("single", "double", "half", "half", "quad"), 1e-2, 1, True),
    ("2d-hh-unpreconditioned", ("single", "double", "half", "half", "quad"), 1e-2, 0, False),
]


def check_ir_steps_near_stop(st_its, st_nbe, ref_its, ref_nbe, stop_tol):
    """The step counts agree, or differ by one where the stop rule is a near-tie: with
    half-precision Krylov vectors a refinement step contracts the backward error by only
    ~1e-2, so when a step lands within a factor 10 of the threshold q u the two sides may
    stop one step apart.  Returns the common number of steps."""
    a, b = len(st_its), len(ref_its)
    if a != b:
        m = min(a, b)
        longer = st_nbe if a > b else ref_nbe
        assert abs(a - b) == 1 and longer[m] <= 10 * stop_tol, (st_its, list(ref_its), st_nbe, list(ref_nbe))
        a = b = m
    tg, to = sum(st_its[:a]), sum(ref_its[:a])
    assert abs(tg - to) <= max(1, 0.1 * to), (st_its, list(ref_its))
    return a


@pytest.mark.parametrize("name,tup,tau,side,precond", HALF_KRYLOV_CASES)
def test_ir_half_krylov_against_oracle(ctx, name, tup, tau, side, precond):
    """u_g and/or u_p = half (Krylov vectors and the products' matrix copies stored in
    half, binary32 arithmetic; one-reduction MGS) against the oracle's MODE_ACC32 Krylov
    part, both scaling the residual by a power of two (reading R17)."""
    uf, u, ug, up, ur = tup
    if u == "single":
        A, b, x_true = synth.cfg_large_3d(N=16)
        init, F = O.PAT_A2, 25
    else:
        A = synth.conv_diff_2d(40, 20.0, 1.0, 0.1, seed=11)
        b, x_true = synth.rhs(A, seed=12)
        init, F = O.PAT_A, 30
    so = S.make_spai_opts(init=init, max_fill=F, uf=uf, side=side) if precond else None
    io = S.make_ir_opts(uf=uf, u=u, ug=ug, up=up, ur=ur, tau=tau, orth=2, side=side, ir_max_steps=30)
    x = np.zeros_like(b)
    st = S.gmres_ir_solve(ctx, A, b, x, sopts=so, opts=io)
    Pr = None
    if precond and side == 0:
        Pr = O.assemble_P(O.spai(A, init=init, max_fill=F, uf=uf), up, uf)
    elif precond:
        _, Pr = O.spai_right(A, up=up, uf=uf, init=init, max_fill=F)
    ref = O.gmres_ir(A, b, Pr, uf=uf, u=u, ug=ug, up=up, ur=ur, tau=tau, orth=O.ORTH_MGS_ICWY, side=side,
                     kmode=O.MODE_ACC32, imax=30)
    assert ref["status"] & O.IR_CONVERGED
    assert st["flags"] & 1
    m = check_ir_steps_near_stop(st["its"], st["nbe"], ref["its"], ref["nbe"], O.default_stop_tol(A, u))
    # at a near-tie the side that took one more step is rerun for m steps, so that the
    # errors compared are those after the same number of steps
    if st["steps"] > m:
        io = S.make_ir_opts(uf=uf, u=u, ug=ug, up=up, ur=ur, tau=tau, orth=2, side=side, ir_max_steps=m)
        x = np.zeros_like(b)
        S.gmres_ir_solve(ctx, A, b, x, sopts=so, opts=io)
    elif ref["steps"] > m:
        ref = O.gmres_ir(A, b, Pr, uf=uf, u=u, ug=ug, up=up, ur=ur, tau=tau, orth=O.ORTH_MGS_ICWY, side=side,
                         kmode=O.MODE_ACC32, imax=m)
    nb_g, fe_g = errors(A, b, x, x_true)
    nb_o, fe_o = errors(A, b, ref["x"], x_true)
    uu = O.UNIT_ROUNDOFF[O.prec(u)]
    assert nb_g <= 10 * max(nb_o, uu) and fe_g <= 10 * max(fe_o, uu)


def test_ir_half_krylov_large_grid(ctx):
    # n = 27^3 = 19683: 77 row blocks and the block that runs the Givens rotations
    A = synth.conv_diff_3d(27, 50.0, seed=11)
    b, x_true = synth.rhs(A, seed=12)
    tup = dict(uf="half", u="single", ug="half", up="half", ur="double")
    so = S.make_spai_opts(init=O.PAT_A2, max_fill=25, uf="half")
    io = S.make_ir_opts(tau=1e-2, orth=2, **tup)
    x = np.zeros_like(b)
    st = S.gmres_ir_solve(ctx, A, b, x, sopts=so, opts=io)
    ref = O.gmres_ir(A, b, O.assemble_P(O.spai(A, init=O.PAT_A2, max_fill=25, uf="half"), "half", "half"),
                     tau=1e-2, orth=O.ORTH_MGS_ICWY, kmode=O.MODE_ACC32, **tup)
    assert st["grid"] >= 64
    check_ir(A, b, x_true, x, st, ref, 2.0 ** -24)


@pytest.mark.parametrize("ug,up,orth", [("half", "half", 0), ("half", "single", 1), ("half", "double", 2),
                                        ("double", "half", 2)])
def test_ir_half_krylov_unsupported_forms(ctx, ug, up, orth):
    # half Krylov storage is built for the one-reduction MGS beside single only
    A, b, x_true = synth.cfg_small_2d()
    io = S.make_ir_opts(uf="single", u="double", ug=ug, up=up, ur="quad", tau=1e-2, orth=orth)
    x = np.zeros_like(b)
    with pytest.raises(S.SpaiError) as e:
        S.gmres_ir_solve(ctx, A, b, x, sopts=S.make_spai_opts(init=1, max_fill=30, uf="single"), opts=io)
    assert e.value.code == S.ERR_UNSUPPORTED


# ---------------------------------------------------------------- right preconditioning (reading R14)


def _transpose(rp, ci, va):
    n = len(rp) - 1
    M = sp.csr_matrix((va, ci, rp), shape=(n, n)).T.tocsr()
    M.sort_indices()
    return M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data


@pytest.mark.parametrize("uf", ["half", "single"])
@pytest.mark.parametrize("name,make,init,F", [SPAI_CASES[0], SPAI_CASES[2]])
def test_spai_right_parity(ctx, name, make, init, F, uf):
    # the right SPAI is the transpose of Algorithm 1 run on A^T: compare P^T with the oracle's
    # left run on A^T column by column (pattern bit-exact, residuals as for the left SPAI)
    A = make()
    P, st, (rp, ci, va) = gpu_spai(ctx, A, init=init, max_fill=F, uf=uf, eps=0.0, side=S.SIDE_RIGHT)
    At = O.transpose_csr(A)
    ref = O.spai(At, init=init, max_fill=F, uf=uf, eps=0.0)
    n = ref["n"]
    tp, tc, tv = _transpose(rp, ci, va)
    assert np.array_equal(np.diff(tp), ref["Jcnt"])
    for k in range(n):
        assert np.array_equal(tc[tp[k]:tp[k + 1]], ref["Jidx"][k][: ref["Jcnt"][k]])
    J, cnt, M = split_rows(tp, tc, tv, ref["d"])
    res_gpu, absbm = true_colres(At, ref["d"], J, cnt, M, floor=True)
    assert_colres(res_gpu, ref["colres64"], absbm, uf)
    # column k of A P - I is A D m_k - e_k, the residual just compared
    Ms = synth.to_scipy(A)
    Pm = sp.csr_matrix((va, ci, rp), shape=(n, n))
    R = (Ms @ Pm - sp.identity(n)).tocsc()
    colres = np.sqrt(np.asarray(R.multiply(R).sum(axis=0)).ravel())
    np.testing.assert_allclose(colres, res_gpu, rtol=1e-9, atol=1e-13)
    P.free()


@pytest.mark.parametrize("tup", [("single", "double", "double", "double", "quad"),
                                 ("half", "single", "single", "single", "double")])
def test_ir_right_preconditioned(ctx, tup):
    uf, u, ug, up, ur = tup
    if uf == "half":
        A, b, x_true = synth.cfg_large_3d(N=16)
        init, F = O.PAT_A2, 25
    else:
        A, b, x_true = synth.cfg_small_2d()
        init, F = O.PAT_A, 30
    tau = 1e-4
    so = S.make_spai_opts(init=init, max_fill=F, uf=uf, side=S.SIDE_RIGHT)
    io = S.make_ir_opts(uf=uf, u=u, ug=ug, up=up, ur=ur, tau=tau, side=S.SIDE_RIGHT)
    x = np.zeros_like(b)
    st = S.gmres_ir_solve(ctx, A, b, x, sopts=so, opts=io)
    _, Pr = O.spai_right(A, up=up, uf=uf, init=init, max_fill=F)
    ref = O.gmres_ir(A, b, Pr, uf=uf, u=u, ug=ug, up=up, ur=ur, tau=tau, side=O.SIDE_RIGHT)
    check_ir(A, b, x_true, x, st, ref, O.UNIT_ROUNDOFF[O.prec(u)])
    assert st["flags"] & 1


def test_ir_right_group_and_left_agree():
    # a grid large enough for the Gram-Schmidt group (77 blocks): the right-preconditioned solve
    # reaches the same accuracy as the left one
    c = S.Context(0)
    A = synth.conv_diff_3d(27, 50.0, seed=11)
    b, x_true = synth.rhs(A, seed=12)
    res = {}
    for side in (S.SIDE_LEFT, S.SIDE_RIGHT):
        so = S.make_spai_opts(init=O.PAT_A2, max_fill=25, uf="half", side=side)
        io = S.make_ir_opts(uf="half", u="single", ug="single", up="single", ur="double", tau=1e-4, side=side)
        x = np.zeros_like(b)
        st = S.gmres_ir_solve(c, A, b, x, sopts=so, opts=io)
        nbe, fe = errors(A, b, x, x_true)
        res[side] = (st, nbe, fe)
        assert st["flags"] & 1 and st["grid"] >= 64
    for side in res:
        assert res[side][1] <= 7 * 2.0 ** -24 and res[side][2] <= 1e-4
    c.close()


# ---------------------------------------------------------------- stopping rules (reading R8)


def test_ir_correction_rule_against_oracle(ctx):
    A = synth.conv_diff_2d(24, 20.0, 1.0, 0.1, seed=7)
    b, x_true = synth.rhs(A, seed=9)
    kw = dict(uf="single", u="double", ug="single", up="single", ur="quad", tau=1e-2)
    so = S.make_spai_opts(init=O.PAT_A, max_fill=30, uf="single")
    io = S.make_ir_opts(stop=S.IR_STOP_CORRECTION, stop_tol=1e-10, **kw)
    x = np.zeros_like(b)
    st = S.gmres_ir_solve(ctx, A, b, x, sopts=so, opts=io)
    Sr = O.spai(A, init=O.PAT_A, max_fill=30, uf="single")
    ref = O.gmres_ir(A, b, O.assemble_P(Sr, "single", "single"), stop_rule=O.STOP_CORRECTION, stop_tol=1e-10,
                     **kw)
    assert ref["status"] & O.IR_CONVERGED and st["flags"] & S.IR_CONVERGED
    check_ir(A, b, x_true, x, st, ref, 2.0 ** -53)


def test_ir_stagnation_against_oracle(ctx):
    # one GMRES iteration per step without a preconditioner: the corrections do not
    # halve, and both sides stop at the same step with the stagnation flag
    A = synth.random_sparse(200, 6, seed=8, log10_scale=2.0)
    b, _ = synth.rhs(A, seed=9)
    kw = dict(uf="single", u="double", ug="double", up="double", ur="double", tau=1e-8)
    io = S.make_ir_opts(gmres_max_it=1, **kw)
    x = np.zeros_like(b)
    st = S.gmres_ir_solve(ctx, A, b, x, opts=io)
    ref = O.gmres_ir(A, b, None, gmres_maxit=1, **kw)
    assert ref["status"] & O.IR_STAGNATED
    assert st["flags"] & S.IR_STAGNATED and not st["flags"] & S.IR_CONVERGED
    assert st["rc"] == S.WARN_NOT_CONVERGED
    assert st["steps"] == ref["steps"] and st["its"] == list(ref["its"])


def test_device_inputs_are_checked(ctx):
    so = S.make_spai_opts(init=0, max_fill=4, uf="single")
    io = S.make_ir_opts(uf="single", u="double", ug="double", up="double", ur="quad", tau=1e-8)
    bad = [
        ((0, 1, 2, 3), (0, 3, 2), S.ERR_INVALID_ARG),  # a column outside [0, n)
        ((0, 2, 1, 3), (0, 1, 2), S.ERR_INVALID_ARG),  # a decreasing rowptr
        ((0, 1, 2, 5), (0, 1, 2), S.ERR_INVALID_ARG),  # rowptr past nnz
        ((0, 2, 3, 4), (1, 0, 2, 1), S.ERR_INVALID_ARG),  # columns not ascending
        ((0, 1, 1, 2), (0, 2), S.ERR_ZERO_ROW),        # an empty row
    ]
    bd = torch.ones(3, dtype=torch.float64, device="cuda")
    for rp, ci, code in bad:
        Ad = tuple(torch.from_numpy(a).cuda() for a in (np.array(rp, dtype=np.int64), np.array(ci, dtype=np.int32),
                                                         np.ones(len(ci))))
        with pytest.raises(S.SpaiError) as e:
            S.spai_build(ctx, Ad, so)
        assert e.value.code == code, (rp, ci)
        with pytest.raises(S.SpaiError) as e:
            S.gmres_ir_solve(ctx, Ad, bd, torch.zeros_like(bd), sopts=so, opts=io)
        assert e.value.code == code, (rp, ci)
        with pytest.raises(S.SpaiError) as e:
            S.gmres_ir_solve_batch(ctx, [Ad], [bd], [torch.zeros_like(bd)], None, io)
        assert e.value.code == code, (rp, ci)


def test_bounded_waits_time_out_and_leave_the_device_usable(ctx):
    # a launch whose exchange round (mode 0) or counter barrier (mode 1) waits for a
    # block that does not exist: every wait gives up after its budget and reports
    # SPAI_ERR_TIMEOUT; the device then runs a normal solve
    for mode in (0, 1):
        assert S.selftest_wait_timeout(0, mode, 50.0) == S.ERR_TIMEOUT
    A, b, x_true = synth.cfg_small_2d()
    x = np.zeros_like(b)
    st = S.gmres_ir_solve(ctx, A, b, x, sopts=S.make_spai_opts(init=1, max_fill=30, uf="single"),
                          opts=S.make_ir_opts(uf="single", u="double", ug="double", up="double", ur="quad", tau=1e-4))
    assert st["flags"] & 1 and st["final_nbe"] <= 1e-15
