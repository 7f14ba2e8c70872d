"""Pins for the CPU oracle: checks against facts the paper and mathematics fix.

Each test compares the oracle with something other than itself: a library
routine (numpy float16, numpy/scipy least squares), exact rational
arithmetic, a closed form from the paper (eq. trueres, the 2 sqrt(n) eps and
2 n eps bounds of Section 3, GMRES finite termination), or a hand-computed
example.
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import minimize_scalar

import oracle as O
from paper_2202_10204_gb300 import synth


def dense_to_csr(M):
    return synth._to_csr(sp.csr_matrix(np.asarray(M, dtype=np.float64)))


# ---------------------------------------------------------------- Table 1: chop


def test_chop_half_matches_numpy_float16_conversion():
    rng = np.random.default_rng(0)
    # spread over normal, subnormal and overflow ranges
    x = rng.normal(size=200000) * 2.0 ** rng.integers(-30, 18, size=200000)
    # exact ties at half precision (odd multiples of half a quantum)
    ties = (rng.integers(0, 2 ** 11, size=5000) * 2 + 1) * 2.0 ** -12
    x = np.concatenate([x, ties, -ties, [65504.0, 65519.99, 65520.0, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26, 0.0]])
    with np.errstate(over="ignore"):  # the overflow range is part of the comparison
        ref = x.astype(np.float16).astype(np.float64)
    got = O.chop_half(x)
    assert np.array_equal(np.isinf(got), np.isinf(ref))
    fin = np.isfinite(ref)
    assert np.array_equal(got[fin], ref[fin])


@pytest.mark.parametrize("op", [0, 1, 2, 3, 4])
def test_half_arithmetic_matches_numpy_float16(op):
    rng = np.random.default_rng(op + 1)
    a = (rng.normal(size=100000) * 2.0 ** rng.integers(-16, 9, size=100000)).astype(np.float16)
    b = (rng.normal(size=100000) * 2.0 ** rng.integers(-16, 9, size=100000)).astype(np.float16)
    b[b == 0] = np.float16(1.0)
    with np.errstate(all="ignore"):
        ref = {0: a + b, 1: a - b, 2: a * b, 3: a / b, 4: np.sqrt(np.abs(a))}[op].astype(np.float64)
    got = O.half_ops(a.astype(np.float64), b.astype(np.float64), op)
    same = (got == ref) | (np.isnan(got) & np.isnan(ref))
    assert same.all()


def test_unit_roundoffs_table1():
    # Table 1: half 2^-11, single 2^-24, double 2^-53 -- the spacing just above 1 is 2u
    for p, u in ((O.HALF, 2.0 ** -11), (O.SINGLE, 2.0 ** -24)):
        assert O.round_to(1.0 + u, p) == 1.0          # tie to even
        assert O.round_to(1.0 + 1.5 * u, p) == 1.0 + 2 * u
    assert O.UNIT_ROUNDOFF[O.DOUBLE] == np.finfo(np.float64).eps / 2


# ---------------------------------------------------------------- least squares


def exact_lstsq(A, e):
    """Normal equations in exact rational arithmetic (brute force)."""
    m, nc = A.shape
    Af = [[Fraction(float(A[i, j])) for j in range(nc)] for i in range(m)]
    ef = [Fraction(float(v)) for v in e]
    G = [[sum(Af[i][a] * Af[i][b] for i in range(m)) for b in range(nc)] for a in range(nc)]
    r = [sum(Af[i][a] * ef[i] for i in range(m)) for a in range(nc)]
    for c in range(nc):  # Gaussian elimination (G is SPD: no pivoting needed)
        for rr in range(c + 1, nc):
            f = G[rr][c] / G[c][c]
            for q in range(c, nc):
                G[rr][q] -= f * G[c][q]
            r[rr] -= f * r[c]
    x = [Fraction(0)] * nc
    for c in range(nc - 1, -1, -1):
        x[c] = (r[c] - sum(G[c][q] * x[q] for q in range(c + 1, nc))) / G[c][c]
    return np.array([float(v) for v in x])


@pytest.mark.parametrize("shape", [(3, 1), (5, 3), (8, 5), (7, 7)])
def test_dense_ls_double_matches_exact(shape):
    rng = np.random.default_rng(sum(shape))
    m, nc = shape
    for trial in range(5):
        A = rng.normal(size=(m, nc))
        e = np.zeros(m); e[rng.integers(m)] = 1.0
        x_ex = exact_lstsq(A, e)
        mb, sb, sn, fl = O.dense_ls(A, e, "double")
        kappa = np.linalg.cond(A)
        assert fl == 0
        assert np.max(np.abs(mb - x_ex)) <= 50 * 2.0 ** -53 * kappa ** 2 * max(1, np.max(np.abs(x_ex)))
        # explicit residual and its norm
        s_ref = A @ x_ex - e
        assert abs(sn - np.linalg.norm(s_ref)) <= 1e-12 * max(1.0, np.linalg.norm(e))
        np.testing.assert_allclose(sb, A @ mb - e, atol=1e-14)


@pytest.mark.parametrize("uf,u", [("single", 2.0 ** -24), ("half", 2.0 ** -11)])
@pytest.mark.parametrize("mode", [O.MODE_PEROP, O.MODE_ACC32])
def test_dense_ls_low_precision_error_bound(uf, u, mode):
    rng = np.random.default_rng(7)
    for trial in range(20):
        m, nc = 9, 4
        A = O.round_to(rng.uniform(-1, 1, size=(m, nc)), uf)
        e = np.zeros(m); e[trial % m] = 1.0
        x_ex = np.linalg.lstsq(A, e, rcond=None)[0]
        mb, sb, sn, fl = O.dense_ls(A, e, uf, mode)
        kappa = np.linalg.cond(A)
        # Householder LS (Higham, ASNA Thm 20.3): error O(m nc u kappa^2) relative
        rel = np.linalg.norm(mb - x_ex) / np.linalg.norm(x_ex)
        assert rel <= 4 * m * nc * u * kappa ** 2
        # values are representable in u_f
        assert np.array_equal(mb, O.round_to(mb, uf))
        # the reported ||sbar|| is the u_f norm of the explicit residual
        r_true = np.linalg.norm(A @ mb - e)
        assert abs(sn - r_true) <= 4 * m * nc * u * max(r_true, 1.0)


def test_dense_ls_square_is_solve():
    rng = np.random.default_rng(3)
    A = rng.normal(size=(6, 6)) + 6 * np.eye(6)
    e = np.eye(6)[2]
    mb, sb, sn, fl = O.dense_ls(A, e, "double")
    np.testing.assert_allclose(mb, np.linalg.solve(A, e), rtol=1e-13, atol=1e-14)
    assert sn <= 1e-14


# ---------------------------------------------------------------- SPAI special cases


def test_spai_diagonal_identity_pattern_is_exact_inverse():
    a = np.array([2.0, -3.0, 0.5, 7.0, -0.25])
    A = dense_to_csr(np.diag(a))
    for uf in ("double", "single", "half"):
        S = O.spai(A, init=O.PAT_IDENTITY, uf=uf, max_fill=4)
        rp, col, val, _ = O.assemble_P(S, up="double")
        assert np.array_equal(col, np.arange(5))
        np.testing.assert_allclose(val, 1.0 / a, rtol=4 * O.UNIT_ROUNDOFF[O.prec(uf)])
        assert np.all(S["flags"] & O.CF_CONVERGED)


def test_spai_full_pattern_gives_inverse():
    rng = np.random.default_rng(11)
    n = 10
    Ad = rng.normal(size=(n, n)) + 4 * np.eye(n)
    A = dense_to_csr(Ad)
    S = O.spai(A, init=O.PAT_A, uf="double", max_fill=n, eps=1e-12)
    rp, col, val, _ = O.assemble_P(S, up="double")
    P = sp.csr_matrix((val, col, rp), shape=(n, n)).toarray()
    np.testing.assert_allclose(P @ Ad, np.eye(n), atol=1e-12 * np.linalg.cond(Ad))
    # and GMRES on P A converges in one iteration (P A = I)
    b = rng.normal(size=n)
    d, k, bd, rr = O.gmres(A, b, (rp, col, val), tau=1e-10)
    assert k == 1
    np.testing.assert_allclose(Ad @ d, b, atol=1e-10)


def test_spai_block_diagonal_exact_block_inverse():
    rng = np.random.default_rng(5)
    blocks = [rng.normal(size=(s, s)) + 3 * np.eye(s) for s in (3, 4, 2, 5)]
    Ad = sp.block_diag([sp.coo_matrix(bk) for bk in blocks]).toarray()
    n = Ad.shape[0]
    A = dense_to_csr(Ad)
    S = O.spai(A, init=O.PAT_A, uf="double", max_fill=8, eps=1e-10)
    rp, col, val, _ = O.assemble_P(S, up="double")
    P = sp.csr_matrix((val, col, rp), shape=(n, n)).toarray()
    np.testing.assert_allclose(P, np.linalg.inv(Ad), atol=1e-12)
    assert np.max(S["colres64"]) < 1e-13


def test_spai_column_matches_library_lstsq():
    A, b, x = synth.cfg_small_2d()
    Ms = synth.to_scipy(A)
    n = Ms.shape[0]
    S = O.spai(A, init=O.PAT_A, uf="double", max_fill=30, cols=[0, 17, 500, 1023])
    rowmax = np.abs(Ms).max(axis=1).toarray().ravel()
    B = (Ms.T @ sp.diags(1.0 / rowmax)).tocsc()  # B = A^T D
    for k in (0, 17, 500, 1023):
        J = S["Jidx"][k][: S["Jcnt"][k]]
        assert np.array_equal(J, np.sort(Ms[:, [k]].nonzero()[0]))  # pattern(A), column k
        BJ = B[:, J].toarray()
        I = np.union1d(np.nonzero(np.any(BJ != 0, axis=1))[0], [k])
        e = (I == k).astype(float)
        m_ref = np.linalg.lstsq(BJ[I], e, rcond=None)[0]
        np.testing.assert_allclose(S["mbar"][k][: len(J)], m_ref, rtol=1e-12, atol=1e-13)
        assert abs(S["colres64"][k] - np.linalg.norm(BJ @ m_ref - np.eye(n)[k])) < 1e-12


def _lstsq_column(Ms, d, J, k):
    """numpy lstsq of min ||B(I, J) m - e_k(I)|| with B = A^T D and I the nonzero
    rows of B(:, J) plus k; returns (m, I)."""
    n = Ms.shape[0]
    B = (Ms.T @ sp.diags(d)).tocsc()
    BJ = B[:, J].toarray()
    I = np.union1d(np.nonzero(np.any(BJ != 0, axis=1))[0], [k])
    e = (I == k).astype(float)
    return np.linalg.lstsq(BJ[I], e, rcond=None)[0], I


def test_spai_large_shadows_match_library_lstsq():
    # Algorithm 1 has no bound on the shadow |I_k|: fixed pattern(A) columns of a
    # matrix with 28 nonzeros per column (shadows of 500-700 rows) and adaptive
    # columns grown to 30 entries are the least-squares solutions on their full
    # shadows, and the adaptive ones keep augmenting past 512 rows
    A = synth.random_sparse(1500, 28, seed=31)
    Ms = synth.to_scipy(A)
    cols = [0, 101, 333, 1499]
    S = O.spai(A, init=O.PAT_A, uf="double", max_fill=30, cols=cols)
    for k in cols:
        J = S["Jidx"][k][: S["Jcnt"][k]]
        m_ref, I = _lstsq_column(Ms, S["d"], J, k)
        assert len(I) == S["Icnt"][k]
        np.testing.assert_allclose(S["mbar"][k][: len(J)], m_ref, rtol=1e-10, atol=1e-12)
    assert min(S["Icnt"][k] for k in cols) > 512
    A = synth.random_sparse(1500, 24, seed=5)
    Ms = synth.to_scipy(A)
    cols = list(range(0, 1500, 75))
    S = O.spai(A, init=O.PAT_IDENTITY, adaptive=True, eps=0.1, beta=8, max_fill=30, uf="double", cols=cols)
    big = [k for k in cols if S["Icnt"][k] > 512]
    assert len(big) >= len(cols) // 2
    for k in big:
        J = S["Jidx"][k][: S["Jcnt"][k]]
        assert len(J) == 30 or (S["flags"][k] & O.CF_CONVERGED)
        m_ref, I = _lstsq_column(Ms, S["d"], J, k)
        assert len(I) == S["Icnt"][k]
        np.testing.assert_allclose(S["mbar"][k][: len(J)], m_ref, rtol=1e-9, atol=1e-11)


def test_pattern_A2_matches_scipy():
    A = synth.conv_diff_3d(6, 50.0, seed=3)
    Ms = synth.to_scipy(A)
    A2 = (abs(Ms) @ abs(Ms)).tocsc()
    S = O.spai(A, init=O.PAT_A2, uf="single", max_fill=25, cols=list(range(0, 216, 7)))
    for k in range(0, 216, 7):
        J = S["Jidx"][k][: S["Jcnt"][k]]
        ref = np.sort(A2[:, k].nonzero()[0])
        assert len(ref) <= 25
        assert np.array_equal(J, ref)
    # interior column of the 7-point stencil: |pattern(A^2)| = 25
    k = 2 * 36 + 2 * 6 + 2
    assert S["Jcnt"][k] == 25 or k not in range(0, 216, 7)


def test_explicit_zeros_pattern_structural_shadow_by_value():
    """Explicit zeros of A: pattern(A^2) follows the stored structure (a boolean
    product of the structure, scipy), the shadow I_k counts only rows with a
    nonzero value in B(:, J_k) (Algorithm 1), and m_k is the library
    least-squares solution on that shadow."""
    A = synth.conv_diff_3d(5, 50.0, seed=4)
    rp, ci, va = A
    va = va.copy()
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    va[(ci != rows) & (np.random.default_rng(7).random(len(va)) < 0.3)] = 0.0
    Az = (rp, ci, va)
    n = len(rp) - 1
    cols = list(range(0, n, 9))
    S = O.spai(Az, init=O.PAT_A2, uf="double", max_fill=25, cols=cols)
    Ms = sp.csr_matrix((va, ci, rp), shape=(n, n))  # explicit zeros kept
    St = sp.csr_matrix((np.ones(len(ci)), ci, rp), shape=(n, n))
    A2 = (St @ St).tocsc()
    rowmax = np.array([np.abs(va[rp[i]:rp[i + 1]]).max() for i in range(n)])
    B = (Ms.T @ sp.diags(1.0 / rowmax)).tocsc()
    fewer = 0
    for k in cols:
        J = S["Jidx"][k][: S["Jcnt"][k]]
        assert np.array_equal(J, np.sort(A2[:, k].nonzero()[0]))
        BJ = B[:, J].toarray()
        I = np.union1d(np.nonzero(np.any(BJ != 0, axis=1))[0], [k])
        assert S["Icnt"][k] == len(I)
        Ist = np.union1d(np.nonzero(np.asarray((St.T[:, J]).sum(axis=1)).ravel())[0], [k])
        fewer += len(I) < len(Ist)
        e = (I == k).astype(float)
        m_ref = np.linalg.lstsq(BJ[I], e, rcond=None)[0]
        np.testing.assert_allclose(S["mbar"][k][: len(J)], m_ref, rtol=1e-10, atol=1e-12)
    assert fewer > 0  # the zeros shrink some shadows below the structural ones


def test_fill_cap_keeps_k_and_nearest():
    A = synth.conv_diff_3d(6, 50.0, seed=3)
    k = 2 * 36 + 3 * 6 + 2
    S = O.spai(A, init=O.PAT_A2, uf="double", max_fill=7, cols=[k])
    J = S["Jidx"][k][: S["Jcnt"][k]]
    assert S["Jcnt"][k] == 7 and k in J
    Ms = synth.to_scipy(A)
    full = np.sort((abs(Ms) @ abs(Ms))[:, k].nonzero()[0])
    order = sorted(full, key=lambda j: (j != k, abs(j - k), j))
    assert np.array_equal(J, np.sort(order[:7]))


# ---------------------------------------------------------------- Grote-Huckle


def test_rho_is_univariate_residual_minimum():
    A = synth.random_sparse(60, 6, seed=2)
    Ms = synth.to_scipy(A)
    rowmax = np.abs(Ms).max(axis=1).toarray().ravel()
    d = 1.0 / rowmax
    B = (Ms.T @ sp.diags(d)).toarray()
    rng = np.random.default_rng(1)
    I = np.sort(rng.choice(60, size=20, replace=False))
    s = np.zeros(60); s[I] = rng.normal(size=20)
    cand = np.array([3, 10, 25, 41, 59], dtype=np.int32)
    rho = O.rho(A, d, I, s[I], cand, "double")
    for c, j in enumerate(cand):
        f = lambda mu: np.linalg.norm(s + mu * B[:, j])
        best = minimize_scalar(f, bounds=(-100, 100), method="bounded", options={"xatol": 1e-12}).fun
        assert abs(rho[c] - best) <= 1e-7 * max(1.0, best)
    # literal (restricted) reading uses ||b_j(I)|| instead of ||b_j||
    rho_r = O.rho(A, d, I, s[I], cand, "double", rho_restricted=True)
    for c, j in enumerate(cand):
        bI = B[I, j]
        if np.linalg.norm(bI) > 0:
            ref = np.sqrt(max(0.0, s @ s - (s[I] @ bI) ** 2 / (bI @ bI)))
            assert abs(rho_r[c] - ref) <= 1e-12


def test_selection_hand_example():
    # candidates and scores; mean = (0.5+0.2+0.9+0.2+0.4+0.8)/6 = 0.5
    cand = [3, 7, 1, 9, 4, 6]
    rho = [0.5, 0.2, 0.9, 0.2, 0.4, 0.8]
    # acceptable (rho <= 0.5): 3, 7, 9, 4; order by rho then index: 7, 9, 4, 3
    assert list(O.select(cand, rho, 3)) == [7, 9, 4]
    assert list(O.select(cand, rho, 8)) == [7, 9, 4, 3]
    assert list(O.select(cand, rho, 0)) == []
    assert list(O.select([5], [0.3], 2)) == [5]


@pytest.mark.parametrize("uf", ["double", "single"])
def test_adaptive_meets_column_criterion(uf):
    # eq. (trueres): every column of an uncapped adaptive run satisfies
    # ||e_k - A^T D m_k|| <= eps up to the rounding term (<= 2 eps, Section 3)
    A = synth.conv_diff_2d(8, 10.0, 1.0, 0.1, seed=4)
    n = 64
    for eps in (0.5, 0.3, 0.1):
        S = O.spai(A, init=O.PAT_IDENTITY, adaptive=True, eps=eps, beta=8, alpha=n, max_fill=n, uf=uf)
        assert np.all(S["flags"] & O.CF_CONVERGED)
        assert np.all(S["colres"] <= eps)
        assert np.all(S["colres64"] <= 2 * eps)


def test_adaptive_global_bounds():
    # ||I - A^T D M||_F <= 2 sqrt(n) eps and ||I - P A||_inf <= 2 n eps (eq. AM1)
    A = synth.random_sparse(80, 5, seed=9)
    n = 80
    Ad = synth.to_scipy(A).toarray()
    for eps in (0.4, 0.2):
        S = O.spai(A, init=O.PAT_IDENTITY, adaptive=True, eps=eps, alpha=n, max_fill=n, uf="single")
        assert np.all(S["flags"] & O.CF_CONVERGED)
        rp, col, val, _ = O.assemble_P(S, up="double")
        P = sp.csr_matrix((val, col, rp), shape=(n, n)).toarray()
        d = S["d"]
        M = (P / d[None, :]).T  # P = M^T D
        B = Ad.T @ np.diag(d)
        assert np.linalg.norm(np.eye(n) - B @ M, "fro") <= 2 * np.sqrt(n) * eps
        assert np.linalg.norm(np.eye(n) - P @ Ad, np.inf) <= 2 * n * eps


def test_larger_eps_gives_sparser_preconditioner():
    # qualitative trend of Section 4 (Tables 4-6): larger eps -> fewer nonzeros
    A = synth.random_sparse(200, 6, seed=12)
    nnz = []
    for eps in (0.2, 0.35, 0.5):
        S = O.spai(A, init=O.PAT_IDENTITY, adaptive=True, eps=eps, max_fill=60, uf="single")
        nnz.append(int(S["Jcnt"].sum()))
    assert nnz[0] > nnz[1] > nnz[2]


def test_half_modes_agree_to_half_precision():
    A, b, x = synth.cfg_small_2d()
    S1 = O.spai(A, init=O.PAT_A, uf="half", mode=O.MODE_PEROP, max_fill=30)
    S2 = O.spai(A, init=O.PAT_A, uf="half", mode=O.MODE_ACC32, max_fill=30)
    rel = np.abs(S1["colres64"] - S2["colres64"]) / S2["colres64"]
    assert np.max(rel) < 1e-2
    # both are near the double-precision optimum (the LS residual is stationary)
    S3 = O.spai(A, init=O.PAT_A, uf="double", max_fill=30)
    assert np.max(np.abs(S2["colres64"] - S3["colres64"]) / S3["colres64"]) < 1e-3


# ---------------------------------------------------------------- GMRES


def test_gmres_terminates_in_at_most_n_iterations():
    rng = np.random.default_rng(21)
    for n in (5, 17, 40, 64):
        Ad = rng.normal(size=(n, n)) + np.sqrt(n) * np.eye(n)
        A = dense_to_csr(Ad)
        r = rng.normal(size=n)
        d, k, bd, rr = O.gmres(A, r, None, tau=1e-14, maxit=n)
        assert k <= n
        assert np.linalg.norm(Ad @ d - r) <= 1e-10 * np.linalg.norm(r)


def test_gmres_distinct_eigenvalues_bound():
    rng = np.random.default_rng(4)
    n = 30
    S = rng.normal(size=(n, n)) + 5 * np.eye(n)
    lam = np.array([1.0, 2.0, 5.0])[rng.integers(0, 3, size=n)]
    Ad = S @ np.diag(lam) @ np.linalg.inv(S)
    A = dense_to_csr(Ad)
    r = rng.normal(size=n)
    d, k, bd, rr = O.gmres(A, r, None, tau=1e-12, maxit=n)
    assert k <= 3
    np.testing.assert_allclose(Ad @ d, r, atol=1e-8 * np.linalg.norm(r))


def test_gmres_zero_rhs():
    A = dense_to_csr(np.eye(4) * 2)
    d, k, bd, rr = O.gmres(A, np.zeros(4), None)
    assert k == 0 and np.all(d == 0)


def test_gmres_preconditioned_equals_unpreconditioned_on_PA():
    # left preconditioning: GMRES on (P, A) behaves like GMRES on the product P A
    rng = np.random.default_rng(8)
    n = 20
    Ad = rng.normal(size=(n, n)) + 5 * np.eye(n)
    Pd = np.diag(1.0 / np.diag(Ad))
    r = rng.normal(size=n)
    d1, k1, _, _ = O.gmres(dense_to_csr(Ad), r, dense_to_csr(Pd), tau=1e-10)
    d2, k2, _, _ = O.gmres(dense_to_csr(Pd @ Ad), Pd @ r, None, tau=1e-10)
    assert k1 == k2
    np.testing.assert_allclose(d1, d2, rtol=1e-8, atol=1e-10)


# ---------------------------------------------------------------- residual and IR


def test_quad_residual_is_exactly_rounded():
    rng = np.random.default_rng(2)
    n = 12
    Ad = rng.normal(size=(n, n))
    A = dense_to_csr(Ad)
    x = rng.normal(size=n)
    b = Ad @ x + rng.normal(size=n) * 1e-14
    r = O.residual(A, b, x, "quad", "double")
    for i in range(n):
        ex = Fraction(b[i]) - sum(Fraction(Ad[i, j]) * Fraction(x[j]) for j in range(n))
        assert r[i] == float(ex)  # Fraction -> float rounds to nearest


def exact_solve(Ad, b):
    n = len(b)
    M = [[Fraction(float(v)) for v in row] + [Fraction(float(b[i]))] for i, row in enumerate(Ad)]
    for c in range(n):
        p = max(range(c, n), key=lambda r: abs(M[r][c]))
        M[c], M[p] = M[p], M[c]
        for r in range(c + 1, n):
            f = M[r][c] / M[c][c]
            if f:
                for q in range(c, n + 1):
                    M[r][q] -= f * M[c][q]
    x = [Fraction(0)] * n
    for c in range(n - 1, -1, -1):
        x[c] = (M[c][n] - sum(M[c][q] * x[q] for q in range(c + 1, n))) / M[c][c]
    return np.array([float(v) for v in x])


def test_ir_reaches_working_accuracy_quad_residual():
    # Theorems 1-2: with u_r = quad, forward error ~ u and backward error <= q u
    A = synth.conv_diff_2d(5, 10.0, 1.0, 0.1, seed=3)
    Ad = synth.to_scipy(A).toarray()
    b = np.random.default_rng(1).normal(size=25)
    x_ex = exact_solve(Ad, b)
    S = O.spai(A, init=O.PAT_A, uf="single", max_fill=30)
    P = O.assemble_P(S, up="double", uf="single")
    R = O.gmres_ir(A, b, P, uf="single", u="double", ug="double", up="double", ur="quad", tau=1e-4)
    assert R["status"] & O.IR_CONVERGED
    u = 2.0 ** -53
    assert np.max(np.abs(R["x"] - x_ex)) / np.max(np.abs(x_ex)) <= 2 * u
    assert R["nbe"][-1] <= 5 * u


def test_ir_single_working_precision():
    A, b, x = synth.cfg_small_2d()
    S = O.spai(A, init=O.PAT_A, uf="half", max_fill=30)
    P = O.assemble_P(S, up="single", uf="half")
    R = O.gmres_ir(A, b, P, uf="half", u="single", ug="single", up="single", ur="double", tau=1e-4)
    assert R["status"] & O.IR_CONVERGED
    assert R["nbe"][-1] <= 5 * 2.0 ** -24
    assert np.array_equal(R["x"], O.round_to(R["x"], "single"))
    ferr = np.max(np.abs(R["x"] - x)) / np.max(np.abs(x))
    assert ferr < 1e-5


def test_ir_without_preconditioner_is_plain_gmres_ir():
    A, b, x = synth.cfg_small_2d()
    R = O.gmres_ir(A, b, None, uf="single", u="double", ug="double", up="double", ur="quad", tau=1e-4)
    assert R["status"] & O.IR_CONVERGED
    S = O.spai(A, init=O.PAT_A, uf="single", max_fill=30)
    R2 = O.gmres_ir(A, b, O.assemble_P(S, "double", "single"), uf="single", u="double", ug="double",
                    up="double", ur="quad", tau=1e-4)
    # the preconditioner lowers the iteration count (Tables 4-6 trend)
    assert R2["total_its"] < R["total_its"]


# ---------------------------------------------------------------- products in u_p / u_f


@pytest.mark.parametrize("p,u", [("double", 2.0 ** -53), ("single", 2.0 ** -24), ("half", 2.0 ** -11)])
@pytest.mark.parametrize("mode", [O.MODE_PEROP, O.MODE_ACC32])
def test_spmv_error_bound(p, u, mode):
    # |fl(M x) - M x| <= gamma_q |M||x| with the operands first rounded to p
    A = synth.conv_diff_3d(5, 50.0, seed=2)
    Ms = synth.to_scipy(A)
    x = np.random.default_rng(0).normal(size=Ms.shape[0])
    Mp = Ms.copy(); Mp.data = O.round_to(Mp.data, p)
    xp = O.round_to(x, p)
    y = O.spmv(A, x, p, mode)
    exact = Mp @ xp
    bound = abs(Mp) @ abs(xp)
    q = 7
    assert np.all(np.abs(y - exact) <= (q + 1) * u * bound + 1e-300)
    assert np.array_equal(y, O.round_to(y, p))
    if p == "double":
        np.testing.assert_allclose(y, Ms @ x, rtol=1e-13, atol=1e-13)


def test_gmres_single_precision_converges_to_tau():
    A, b, x = synth.cfg_small_2d()
    Ad = synth.to_scipy(A)
    r = np.random.default_rng(3).normal(size=1024)
    d, k, bd, rr = O.gmres(A, r, None, ug="single", up="single", tau=1e-4)
    assert rr <= 1e-4
    assert np.linalg.norm(Ad @ d - r) / np.linalg.norm(r) <= 1e-3
    assert np.array_equal(d, O.round_to(d, "single"))


# ---------------------------------------------------------------- Gram-Schmidt variants


@pytest.mark.parametrize("orth", [O.ORTH_MGS, O.ORTH_CGS2, O.ORTH_MGS_ICWY])
def test_arnoldi_matches_krylov_qr(orth):
    # Arnoldi builds an orthonormal basis of the Krylov space K_k(A, r) with
    # A V_k = V_{k+1} H; compare with numpy's QR of the explicit Krylov matrix
    rng = np.random.default_rng(5)
    n, k = 12, 6
    Ad = rng.normal(size=(n, n)) + 3 * np.eye(n)
    r = rng.normal(size=n)
    V, H = O.arnoldi(dense_to_csr(Ad), r, None, k=k, orth=orth)
    K = np.column_stack([np.linalg.matrix_power(Ad, i) @ r for i in range(k + 1)])
    Q, _ = np.linalg.qr(K)
    # same subspace column by column (up to signs)
    for c in range(k + 1):
        assert abs(abs(Q[:, c] @ V[:, c]) - 1.0) < 1e-9
    np.testing.assert_allclose(Ad @ V[:, :k], V @ H, atol=1e-12)
    np.testing.assert_allclose(V.T @ V, np.eye(k + 1), atol=1e-13)


def test_cgs2_keeps_orthogonality_in_single():
    # twice is enough: CGS2's basis is orthogonal to O(u) even where MGS
    # drifts (loss of orthogonality ~ u * cond); single precision, 60 steps
    A, b, x = synth.cfg_small_2d()
    r = np.random.default_rng(2).normal(size=1024)
    V2, _ = O.arnoldi(A, r, None, k=60, ug="single", up="single", orth=O.ORTH_CGS2)
    Vm, _ = O.arnoldi(A, r, None, k=60, ug="single", up="single", orth=O.ORTH_MGS)
    e2 = np.linalg.norm(V2.T @ V2 - np.eye(V2.shape[1]))
    em = np.linalg.norm(Vm.T @ Vm - np.eye(Vm.shape[1]))
    assert e2 <= 100 * 2.0 ** -24 * np.sqrt(V2.shape[1])
    assert e2 <= em


def test_icwy_mgs_equals_mgs_in_double():
    # the one-reduction form of MGS (inverse compact WY, lagged normalisation) is
    # MGS in exact arithmetic: on well-conditioned Krylov bases in double the two
    # agree to rounding, column by column and coefficient by coefficient
    rng = np.random.default_rng(5)
    Ad = rng.normal(size=(40, 40)) + 8 * np.eye(40)
    r = rng.normal(size=40)
    Vm, Hm = O.arnoldi(dense_to_csr(Ad), r, None, k=20, orth=O.ORTH_MGS)
    Vi, Hi = O.arnoldi(dense_to_csr(Ad), r, None, k=20, orth=O.ORTH_MGS_ICWY)
    assert Vi.shape == Vm.shape
    np.testing.assert_allclose(Vi, Vm, atol=1e-13)
    np.testing.assert_allclose(Hi, Hm, atol=1e-12)
    # with the SPAI preconditioner on the 2D system (P A well conditioned)
    A, b, x = synth.cfg_small_2d()
    P = O.assemble_P(O.spai(A, init=O.PAT_A, uf="double", max_fill=30), "double", "double")
    Pc = (P[0], P[1], P[2])
    Vm, Hm = O.arnoldi(A, b, Pc, k=20, orth=O.ORTH_MGS)
    Vi, Hi = O.arnoldi(A, b, Pc, k=20, orth=O.ORTH_MGS_ICWY)
    np.testing.assert_allclose(Vi, Vm, atol=1e-12)
    np.testing.assert_allclose(Hi, Hm, atol=1e-12 * np.max(np.abs(Hm)))


def test_icwy_mgs_loses_orthogonality_like_mgs_in_single():
    # MGS-like stability: in single precision the basis of the one-reduction form
    # loses orthogonality as MGS's does (~ u cond), not more; CGS2 keeps O(u)
    A = synth.random_sparse(800, 8, seed=3, log10_scale=4.0)
    r = np.random.default_rng(3).normal(size=800)
    e = {}
    for orth in (O.ORTH_MGS, O.ORTH_CGS2, O.ORTH_MGS_ICWY):
        V, _ = O.arnoldi(A, r, None, k=120, ug="single", up="single", orth=orth)
        assert V.shape[1] == 121
        e[orth] = np.linalg.norm(V.T @ V - np.eye(121))
    assert e[O.ORTH_MGS_ICWY] <= 4 * e[O.ORTH_MGS]
    assert e[O.ORTH_CGS2] < e[O.ORTH_MGS]


def test_gmres_ir_icwy_matches_mgs_solution():
    A, b, x_true = synth.cfg_small_2d()
    S = O.spai(A, init=O.PAT_A, uf="single", max_fill=30)
    P = O.assemble_P(S, "double", "single")
    Rm = O.gmres_ir(A, b, P, tau=1e-4, orth=O.ORTH_MGS)
    Ri = O.gmres_ir(A, b, P, tau=1e-4, orth=O.ORTH_MGS_ICWY)
    assert Ri["status"] & O.IR_CONVERGED
    assert Ri["steps"] == Rm["steps"] and abs(Ri["total_its"] - Rm["total_its"]) <= 1
    assert np.max(np.abs(Ri["x"] - Rm["x"])) <= 4 * 2.0 ** -53 * np.max(np.abs(Rm["x"]))
    # right preconditioning and single-precision Krylov vectors as well
    _, Pr = O.spai_right(A, up="single", uf="single", init=O.PAT_A, max_fill=30)
    kw = dict(uf="single", u="double", ug="single", up="single", ur="quad", tau=1e-4, side=O.SIDE_RIGHT)
    Rm = O.gmres_ir(A, b, Pr, orth=O.ORTH_MGS, **kw)
    Ri = O.gmres_ir(A, b, Pr, orth=O.ORTH_MGS_ICWY, **kw)
    assert Ri["status"] & O.IR_CONVERGED and Ri["steps"] == Rm["steps"]
    assert abs(Ri["total_its"] - Rm["total_its"]) <= max(1, 0.1 * Rm["total_its"])


def test_gmres_ir_cgs2_matches_mgs_solution():
    A, b, x_true = synth.cfg_small_2d()
    S = O.spai(A, init=O.PAT_A, uf="single", max_fill=30)
    P = O.assemble_P(S, "double", "single")
    Rm = O.gmres_ir(A, b, P, tau=1e-4, orth=O.ORTH_MGS)
    Rc = O.gmres_ir(A, b, P, tau=1e-4, orth=O.ORTH_CGS2)
    assert Rc["status"] & O.IR_CONVERGED
    assert Rc["steps"] == Rm["steps"]
    assert abs(Rc["total_its"] - Rm["total_its"]) <= 1
    assert np.max(np.abs(Rc["x"] - Rm["x"])) <= 4 * 2.0 ** -53 * np.max(np.abs(Rm["x"]))


# ---------------------------------------------------------------- right preconditioning (reading R14)


def test_right_gmres_equals_unpreconditioned_on_AP():
    # right preconditioning: GMRES on (A, P) from the right is GMRES on the product A P, and
    # its correction is d = P u
    rng = np.random.default_rng(18)
    n = 20
    Ad = rng.normal(size=(n, n)) + 5 * np.eye(n)
    Pd = np.diag(1.0 / np.diag(Ad)) + 0.01 * rng.normal(size=(n, n))
    r = rng.normal(size=n)
    d1, k1, _, _ = O.gmres(dense_to_csr(Ad), r, dense_to_csr(Pd), tau=1e-10, side=O.SIDE_RIGHT)
    u2, k2, _, _ = O.gmres(dense_to_csr(Ad @ Pd), r, None, tau=1e-10)
    assert k1 == k2
    np.testing.assert_allclose(d1, Pd @ u2, rtol=1e-8, atol=1e-10)


def test_right_gmres_estimate_is_the_true_residual():
    # the Givens estimate of right-preconditioned GMRES is ||r - A d|| / ||r|| (exact arithmetic);
    # the left one is the preconditioned residual ||P (r - A d)|| / ||P r||
    rng = np.random.default_rng(19)
    n = 40
    Ad = rng.normal(size=(n, n)) + 8 * np.eye(n)
    Pd = np.linalg.inv(Ad + 0.5 * rng.normal(size=(n, n)))
    r = rng.normal(size=n)
    for side in (O.SIDE_LEFT, O.SIDE_RIGHT):
        d, k, _, rr = O.gmres(dense_to_csr(Ad), r, dense_to_csr(Pd), tau=1e-6, side=side)
        if side == O.SIDE_RIGHT:
            true = np.linalg.norm(r - Ad @ d) / np.linalg.norm(r)
        else:
            true = np.linalg.norm(Pd @ (r - Ad @ d)) / np.linalg.norm(Pd @ r)
        assert rr <= 1e-6 and abs(true - rr) <= 1e-9, (side, k, rr, true)


def test_right_gmres_without_preconditioner_is_left():
    A = synth.conv_diff_2d(10, 20.0, 1.0, 0.1, seed=3)
    r = np.random.default_rng(2).normal(size=100)
    d1, k1, _, _ = O.gmres(A, r, None, ug="single", up="single", tau=1e-4)
    d2, k2, _, _ = O.gmres(A, r, None, ug="single", up="single", tau=1e-4, side=O.SIDE_RIGHT)
    assert k1 == k2 and np.array_equal(d1, d2)


def test_spai_right_full_pattern_gives_inverse_from_the_right():
    rng = np.random.default_rng(21)
    n = 10
    Ad = rng.normal(size=(n, n)) + 4 * np.eye(n)
    A = dense_to_csr(Ad)
    S, (rp, col, val, _) = O.spai_right(A, up="double", init=O.PAT_A, uf="double", max_fill=n, eps=1e-12)
    P = sp.csr_matrix((val, col, rp), shape=(n, n)).toarray()
    np.testing.assert_allclose(Ad @ P, np.eye(n), atol=1e-12 * np.linalg.cond(Ad))
    # and right-preconditioned GMRES on A P = I converges in one iteration
    b = rng.normal(size=n)
    d, k, bd, rr = O.gmres(A, b, (rp, col, val), tau=1e-10, side=O.SIDE_RIGHT)
    assert k == 1
    np.testing.assert_allclose(Ad @ d, b, atol=1e-10)


def test_spai_right_columns_minimise_the_right_residual():
    # the right SPAI's column k minimises ||A D m - e_k|| over its pattern (Algorithm 1 on A D):
    # check against numpy lstsq on the columns of A D for a random sparse matrix
    A = synth.random_sparse(60, 4, seed=9)
    Ms = synth.to_scipy(A).toarray()
    S, (rp, col, val, _) = O.spai_right(A, up="double", init=O.PAT_A, uf="double", max_fill=10, eps=0.0)
    dcol = 1.0 / np.max(np.abs(Ms), axis=0)
    B = Ms * dcol[None, :]
    P = sp.csr_matrix((val, col, rp), shape=(60, 60)).toarray()
    for k in (0, 7, 33, 59):
        J = S["Jidx"][k][: S["Jcnt"][k]]
        e = np.zeros(60); e[k] = 1.0
        m, *_ = np.linalg.lstsq(B[:, J], e, rcond=None)
        # column k of P = D m (rows J)
        np.testing.assert_allclose(P[J, k], dcol[J] * m, rtol=1e-10, atol=1e-14)
        assert np.count_nonzero(P[:, k]) == len(J)


def test_ir_right_reaches_working_accuracy():
    A, b, x_true = synth.cfg_small_2d()
    S, P = O.spai_right(A, up="double", uf="single", init=O.PAT_A, max_fill=30)
    r = O.gmres_ir(A, b, P, uf="single", u="double", ug="double", up="double", ur="quad", tau=1e-4,
                   side=O.SIDE_RIGHT)
    Ms = synth.to_scipy(A)
    x = r["x"]
    nbe = np.max(np.abs(b - Ms @ x)) / (abs(Ms).sum(axis=1).max() * np.max(np.abs(x)) + np.max(np.abs(b)))
    assert r["steps"] >= 1 and nbe <= 5 * 2.0 ** -53
    assert np.max(np.abs(x - x_true)) / np.max(np.abs(x_true)) < 1e-12


def _iterates(A, b, P, steps, **kw):
    """x_0 .. x_steps from runs with the fixed-step rule (reading R8)."""
    return [O.gmres_ir(A, b, P, imax=s, stop_rule=O.STOP_FIXED, **kw)["x"] for s in range(steps + 1)]


def test_ir_correction_rule_stops_at_small_correction():
    # reading R8, correction rule: stop before step i once ||d_{i-1}|| / ||x_i|| <= stop_tol;
    # the expected step is read off the iterates of fixed-step runs
    A = synth.conv_diff_2d(12, 10.0, 1.0, 0.1, seed=3)
    b, _ = synth.rhs(A, seed=4)
    P = O.assemble_P(O.spai(A, init=O.PAT_A, max_fill=30, uf="single"), "single", "single")
    kw = dict(uf="single", u="double", ug="single", up="single", ur="quad", tau=1e-2)
    X = _iterates(A, b, P, 8, **kw)
    q = [None] + [np.max(np.abs(X[s] - X[s - 1])) / np.max(np.abs(X[s])) for s in range(1, 9)]
    want = next(s for s in range(1, 9) if q[s] <= 1e-10)
    assert all(q[s] < 0.5 * q[s - 1] for s in range(2, want + 1))  # no stagnation on the way
    R = O.gmres_ir(A, b, P, stop_rule=O.STOP_CORRECTION, stop_tol=1e-10, **kw)
    assert R["steps"] == want and R["status"] & O.IR_CONVERGED
    np.testing.assert_array_equal(R["x"], X[want])
    # the backward rule converges too, without the stagnation flag
    Rb = O.gmres_ir(A, b, P, **kw)
    assert Rb["status"] & O.IR_CONVERGED and not Rb["status"] & O.IR_STAGNATED


def test_ir_stagnation_stops_without_convergence():
    # reading R8, stagnation: stop before step i >= 2 once q_i >= q_{i-1} / 2.  One GMRES
    # iteration per refinement step on an unpreconditioned nonsymmetric system barely
    # shrinks the corrections
    A = synth.random_sparse(200, 6, seed=8, log10_scale=2.0)
    b, _ = synth.rhs(A, seed=9)
    kw = dict(uf="single", u="double", ug="double", up="double", ur="double", tau=1e-8, gmres_maxit=1)
    X = _iterates(A, b, None, 6, **kw)
    q = [None] + [np.max(np.abs(X[s] - X[s - 1])) / np.max(np.abs(X[s])) for s in range(1, 7)]
    want = next(s for s in range(2, 7) if q[s] >= 0.5 * q[s - 1])
    R = O.gmres_ir(A, b, None, **kw)
    assert R["steps"] == want
    assert R["status"] & O.IR_STAGNATED and not R["status"] & O.IR_CONVERGED
    np.testing.assert_array_equal(R["x"], X[want])



def _pairwise_f32(t):
    # the pairwise order written out with numpy float32 arithmetic (each add rounded)
    if len(t) == 1:
        return t[0]
    m = len(t) // 2
    return np.float32(_pairwise_f32(t[:m]) + _pairwise_f32(t[m:]))


def test_inner_products_single_are_pairwise():
    # single-precision inner products: rounded products summed pairwise, bit for bit
    rng = np.random.default_rng(17)
    for n in (1, 2, 3, 7, 64, 1000, 4097):
        x = rng.normal(size=n).astype(np.float32).astype(np.float64)
        y = rng.normal(size=n).astype(np.float32).astype(np.float64)
        t = (x.astype(np.float32) * y.astype(np.float32)).astype(np.float32)
        assert O.dot(x, y, "single") == float(_pairwise_f32(list(t))), n
    # a case where the order matters: 1 + 4 * 2^-25 is 1 left to right, 1 + 2^-23 pairwise
    x = np.array([1.0, 2.0 ** -25, 2.0 ** -25, 2.0 ** -25, 2.0 ** -25])
    assert O.dot(x, np.ones(5), "single") == 1.0 + 2.0 ** -23


def test_inner_product_error_bounds():
    # pairwise: |error| <= gamma_{ceil(log2 n)+1} sum |x_i y_i| (Higham, Accuracy and Stability,
    # eq. (4.6) with the product's rounding); double is checked against the exact (fsum) value
    import math
    rng = np.random.default_rng(3)
    for n, p in ((262144, "single"), (100000, "double"), (5000, "single")):
        u = O.UNIT_ROUNDOFF[O.prec(p)]
        x = rng.normal(size=n)
        y = rng.normal(size=n)
        if p == "single":
            x = x.astype(np.float32).astype(np.float64)
            y = y.astype(np.float32).astype(np.float64)
        exact = math.fsum(x * y)  # products of single values are exact in double
        k = math.ceil(math.log2(n)) + 1
        gamma = k * u / (1 - k * u)
        bound = gamma * np.sum(np.abs(x * y))
        if p == "double":
            bound += 2.0 ** -53 * np.sum(np.abs(x * y))  # x*y themselves rounded in double
        assert abs(O.dot(x, y, p) - exact) <= bound, (n, p)


def test_spai_threads_do_not_change_results():
    # the SPAI columns are independent: any number of threads gives the same bits, for
    # adaptive patterns and for fixed patterns cut by the fill cap
    cases = [(synth.random_sparse(600, 8, seed=4, log10_scale=2.0),
              dict(init=O.PAT_IDENTITY, adaptive=True, eps=0.3, max_fill=20, uf="single")),
             (synth.conv_diff_3d((7, 6, 5), 50.0, seed=8), dict(init=O.PAT_A2, max_fill=9, uf="half", eps=0.0))]
    for A, kw in cases:
        out = []
        for th in (1, 4):
            O.set_threads(th)
            out.append(O.spai(A, **kw))
        O.set_threads(0)
        for key in ("Jcnt", "Jidx", "mbar", "colres", "colres64", "flags", "nsolve", "Icnt"):
            assert np.array_equal(out[0][key], out[1][key]), key


def test_round_to_matches_scalar_rounding():
    x = np.random.default_rng(1).normal(size=1000) * 10.0 ** np.random.default_rng(2).uniform(-8, 6, size=1000)
    for p in ("half", "single", "double"):
        r = O.round_to(x, p)
        assert all(r[i] == O.lib().orc_round(float(x[i]), O.prec(p)) for i in range(0, 1000, 7))
    np.testing.assert_array_equal(O.round_to(x, "single"), x.astype(np.float32).astype(np.float64))


# ---------------------------------------------------------------- half-storage Krylov part (kmode)


def test_half_krylov_acc32_is_perop_at_single_and_double():
    # the Krylov arithmetic mode only concerns half: with u_g, u_p single or
    # double the two modes give the same bits
    A, b, x = synth.cfg_small_2d()
    P = O.assemble_P(O.spai(A, init=O.PAT_A, uf="single", max_fill=30), "single", "single")
    r = np.random.default_rng(7).normal(size=1024)
    for ug, up in (("single", "single"), ("double", "single"), ("single", "double")):
        d0 = O.gmres(A, r, (P[0], P[1], P[2]), ug=ug, up=up, tau=1e-4, orth=O.ORTH_MGS_ICWY)
        d1 = O.gmres(A, r, (P[0], P[1], P[2]), ug=ug, up=up, tau=1e-4, orth=O.ORTH_MGS_ICWY,
                     kmode=O.MODE_ACC32)
        assert d0[1] == d1[1] and np.array_equal(d0[0], d1[0])


def test_half_krylov_finite_termination():
    # textbook: GMRES on a diagonalisable matrix with two distinct eigenvalues
    # terminates after two iterations; with the vectors stored in half (values
    # 1 and 2, and a right-hand side of ones, are exact in half) the third
    # Arnoldi vector is at the level of half's rounding, and d = A^{-1} r to
    # that level
    n = 64
    Ad = np.diag(np.where(np.arange(n) < 40, 1.0, 2.0))
    r = np.ones(n)
    d, k, bd, rr = O.gmres(dense_to_csr(Ad), r, None, ug="half", up="half", tau=1e-2,
                           orth=O.ORTH_MGS_ICWY, kmode=O.MODE_ACC32)
    assert k <= 2
    np.testing.assert_allclose(d, r / np.diag(Ad), rtol=8 * 2.0 ** -11)


def test_half_krylov_acc32_refinement_reaches_working_accuracy():
    # Algorithm 3 with u_g = u_p = half (FP16 storage, FP32 operations) on a
    # well-conditioned SPAI-preconditioned system, tau ~ sqrt(u_half): each GMRES
    # solve is only accurate to ~u_half, but the refinement (u = double, u_r =
    # quad) still converges to a backward error of q u (Theorem 2's limit); the
    # vectors stored in half cost refinement steps, not accuracy.  Without the
    # power-of-two scaling of the residual (reading R17) the residuals of later
    # steps fall below half's range and the refinement stagnates near 1e-8.
    A, b, x_true = synth.cfg_small_2d()
    P = O.assemble_P(O.spai(A, init=O.PAT_A, uf="single", max_fill=30), "half", "single")
    R = O.gmres_ir(A, b, P, uf="single", u="double", ug="half", up="half", ur="quad", tau=1e-2,
                   orth=O.ORTH_MGS_ICWY, kmode=O.MODE_ACC32, imax=30)
    assert R["status"] & O.IR_CONVERGED
    assert R["nbe"][-1] <= O.default_stop_tol(A, "double")
    ferr = np.max(np.abs(R["x"] - x_true)) / np.max(np.abs(x_true))
    assert ferr <= 1e-12
    # the half-precision Krylov part needs more refinement steps than single's
    Ps = O.assemble_P(O.spai(A, init=O.PAT_A, uf="single", max_fill=30), "single", "single")
    S = O.gmres_ir(A, b, Ps, uf="single", u="double", ug="single", up="single", ur="quad", tau=1e-2,
                   orth=O.ORTH_MGS_ICWY)
    assert R["steps"] > S["steps"]


def test_half_krylov_acc32_beats_per_operation_half():
    # binary32 operations on half-stored vectors give a more accurate GMRES
    # solution than rounding every operation to half (the chop model), measured
    # by the true preconditioned residual of a long solve
    A, b, x = synth.cfg_small_2d()
    Ad = synth.to_scipy(A)
    S = O.spai(A, init=O.PAT_A, uf="single", max_fill=30)
    P = O.assemble_P(S, "half", "single")
    Pd = sp.csr_matrix((P[2], P[1], P[0]), shape=(1024, 1024))
    r = np.random.default_rng(11).normal(size=1024)
    z = Pd @ r
    res = {}
    for km in (O.MODE_PEROP, O.MODE_ACC32):
        d, k, bd, rr = O.gmres(A, r, (P[0], P[1], P[2]), ug="half", up="half", tau=1e-6, maxit=80,
                               orth=O.ORTH_MGS_ICWY, kmode=km)
        res[km] = np.linalg.norm(z - Pd @ (Ad @ d)) / np.linalg.norm(z)
    assert res[O.MODE_ACC32] < res[O.MODE_PEROP]
    assert res[O.MODE_ACC32] <= 50 * 2.0 ** -11


# ---------------------------------------------------------------- Table 1 (golden fixture)


def _table1():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_ieee_precisions.txt")
    rows = {}
    for line in open(path):
        line = line.split("#")[0].split()
        if line:
            rows[line[0]] = (int(line[1]), int(line[2]), int(line[3]))
    return rows


def test_table1_golden_unit_roundoffs_and_ranges():
    # the oracle's precisions against the values printed in Table 1: unit
    # roundoff exactly, storage size, and the order of magnitude of the
    # largest normalised number of the formats it rounds to
    rows = _table1()
    assert set(rows) == {"half", "single", "double", "quad"}
    for name, (bits, rng, ulog2) in rows.items():
        assert O.UNIT_ROUNDOFF[O.prec(name)] == 2.0 ** ulog2, name
    for name, dt in (("half", np.float16), ("single", np.float32), ("double", np.float64)):
        bits, rng, ulog2 = rows[name]
        fi = np.finfo(dt)
        assert fi.bits == bits
        big, tiny = float(fi.max), float(fi.tiny)
        assert abs(np.log10(big) - rng) <= 1 and abs(np.log10(tiny) + rng) <= 1
        if name != "double":
            # the oracle's rounding keeps the largest finite value and overflows past it
            assert O.round_to(np.array([big]), name)[0] == big
            assert np.isinf(O.round_to(np.array([big * (1 + 2.0 ** ulog2)]), name)[0])
            # and the spacing at 1 is 2u
            assert O.round_to(np.array([1.0 + 2.0 * 2.0 ** ulog2]), name)[0] == 1.0 + 2.0 * 2.0 ** ulog2


def test_ir_non_finite_iterate_is_reported():
    # A's half copy overflows (1e6 > 65504): the products are non-finite, so is the
    # correction, and the refinement must stop with the non-finite status instead of
    # taking a NaN residual for a zero one
    Ab = synth._to_csr(sp.diags(np.full(40, 1e6)) + sp.eye(40, k=1))
    P = O.assemble_P(O.spai(Ab, init=O.PAT_IDENTITY, max_fill=4, uf="single"), "half", "single")
    R = O.gmres_ir(Ab, np.ones(40), P, uf="single", u="double", ug="half", up="half", ur="quad", tau=1e-2,
                   orth=O.ORTH_MGS_ICWY, kmode=O.MODE_ACC32, imax=30)
    assert R["status"] & O.IR_NONFINITE and not R["status"] & O.IR_CONVERGED


@pytest.mark.parametrize("e", [40, -40])
def test_half_krylov_refinement_is_scale_invariant(e):
    # binary floating point is invariant under power-of-two scaling while nothing over- or
    # underflows; with the residual scaled into [0.5, 1) before the half-precision Krylov
    # part (reading R17), b 2^e gives x 2^e bit for bit even where b 2^e alone would fall
    # outside half's range
    A, b, x_true = synth.cfg_small_2d()
    P = O.assemble_P(O.spai(A, init=O.PAT_A, uf="single", max_fill=30), "half", "single")
    kw = dict(uf="single", u="double", ug="half", up="half", ur="quad", tau=1e-2, orth=O.ORTH_MGS_ICWY,
              kmode=O.MODE_ACC32, imax=30)
    R0 = O.gmres_ir(A, b, P, **kw)
    R1 = O.gmres_ir(A, np.ldexp(b, e), P, **kw)
    assert R0["status"] & O.IR_CONVERGED and R1["status"] & O.IR_CONVERGED
    assert list(R0["its"]) == list(R1["its"])
    assert np.array_equal(np.ldexp(R0["x"], e), R1["x"])


@pytest.mark.parametrize("uf,u,tf,tu", [("half", "double", np.float16, np.float64),
                                        ("single", "double", np.float32, np.float64),
                                        ("double", "single", np.float64, np.float32),
                                        ("half", "single", np.float16, np.float32)])
def test_x0_is_b_rounded_to_u_f_then_u_without_preconditioner(uf, u, tf, tu):
    # Algorithm 3, line 2 with P = I: x0 = P b computed in u_f and stored in u, which for
    # A = I is b rounded to u_f and then to u (numpy's IEEE conversions); imax = 0 returns x0
    n = 64
    b = np.random.default_rng(3).normal(size=n)
    eye = synth._to_csr(sp.eye(n, format="csr"))
    R = O.gmres_ir(eye, b, None, uf=uf, u=u, ug="double", up="double", ur="quad", imax=0)
    assert R["steps"] == 0
    assert np.array_equal(R["x"], b.astype(tf).astype(tu).astype(np.float64))


def test_x0_uses_the_u_f_copy_of_P():
    # reading R9: x0 = P b takes P's values in u_f, GMRES its values in u_p.  The two copies
    # are given different values (powers of two and small integers, so every product is
    # exact in half), and x0 shows which copy was used
    rng = np.random.default_rng(4)
    n = 32
    a = 2.0 ** rng.integers(-3, 4, size=n)
    b = rng.integers(-8, 9, size=n).astype(np.float64)
    A = synth._to_csr(sp.diags(a, format="csr"))
    rp, ci = np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32)
    P = (rp, ci, 1.0 / a, 2.0 / a)  # (structure, values in u_p, values in u_f)
    R = O.gmres_ir(A, b, P, uf="half", u="double", ug="double", up="double", ur="quad", imax=0)
    assert np.array_equal(R["x"], 2.0 * b / a)


@pytest.mark.parametrize("orth", [O.ORTH_MGS, O.ORTH_CGS2])
def test_half_storage_mode_is_refused_outside_the_one_reduction_form(orth):
    # the binary32-arithmetic model of half Krylov storage (R17) is defined for the
    # one-reduction MGS only: the other forms must refuse it, not run another model silently
    A, b, _ = synth.cfg_small_2d()
    with pytest.raises(ValueError):
        O.gmres_ir(A, b, None, uf="single", u="double", ug="half", up="single", ur="double", tau=1e-2,
                   orth=orth, kmode=O.MODE_ACC32)
    with pytest.raises(ValueError):
        O.gmres(A, b, None, ug="single", up="half", tau=1e-2, orth=orth, kmode=O.MODE_ACC32)
