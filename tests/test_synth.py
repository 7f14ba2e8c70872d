"""The seeded input generators against the structure their recipe states:
stencil sizes, the signs and row sums of the discretised operators, the
convection term as the only nonsymmetric part, exact nonzeros per column of
the random matrices and their scalings, and determinism under a seed."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2202_10204_gb300 import synth


def check_csr(A, n):
    rp, ci, va = A
    assert rp.dtype == np.int64 and ci.dtype == np.int32 and va.dtype == np.float64
    assert len(rp) == n + 1 and rp[0] == 0 and rp[-1] == len(ci) == len(va)
    for i in range(n):
        row = ci[rp[i]:rp[i + 1]]
        assert np.all(np.diff(row) > 0), i  # sorted, no duplicates
    assert ci.min() >= 0 and ci.max() < n


@pytest.mark.parametrize("N", [1, 2, 7])
def test_conv_diff_2d_stencil_and_row_sums(N):
    A = synth.conv_diff_2d(N, peclet=10.0, diag_shift=0.1, seed=1)
    n = N * N
    check_csr(A, n)
    assert len(A[1]) == 5 * n - 4 * N  # five points, minus the missing neighbours on the boundary
    M = synth.to_scipy(A)
    d = M.diagonal()
    off = M - sp.diags(d)
    assert np.all(d > 0) and np.all(off.data <= 0)
    # upwind convection and diffusion cancel in the row sums of interior rows, leaving the
    # U(0, 0.1) diagonal term; boundary rows keep the missing neighbours' weight
    s = np.asarray(M.sum(axis=1)).ravel()
    iy, ix = np.divmod(np.arange(n), N)
    interior = (iy > 0) & (iy < N - 1) & (ix > 0) & (ix < N - 1)
    assert np.all(s > -1e-12)
    assert np.all(s[interior] < 0.1 + 1e-12)
    if N > 2:
        assert np.all(s[~interior] > 0.9)  # at least one missing neighbour of weight >= nu = 1


@pytest.mark.parametrize("N", [1, 3, (4, 3, 2)])
def test_conv_diff_3d_stencil_signs_and_symmetric_part(N):
    A = synth.conv_diff_3d(N, peclet=50.0, seed=3)
    Nx, Ny, Nz = (N, N, N) if np.isscalar(N) else N
    n = Nx * Ny * Nz
    check_csr(A, n)
    assert len(A[1]) == 7 * n - 2 * (Ny * Nz + Nx * Nz + Nx * Ny)
    M = synth.to_scipy(A)
    d = M.diagonal()
    off = (M - sp.diags(d)).tocsr()
    off.eliminate_zeros()
    assert np.all(d > 0) and np.all(off.data < 0)
    # the diffusion part is symmetric (harmonic-mean faces); the nonsymmetric part is the
    # upwind convection, h w on one side of every neighbour pair
    h = 1.0 / (max(Nx, Ny, Nz) + 1)
    hw = h * 50.0 / np.sqrt(3.0)
    K = (M - M.T).tocoo()
    K.eliminate_zeros()
    assert np.allclose(np.abs(K.data), hw, rtol=1e-12)
    assert K.nnz == 2 * (off.nnz // 2)
    # rows of interior cells sum to zero; cells on the boundary keep their boundary faces
    s = np.asarray(M.sum(axis=1)).ravel()
    iz, rem = np.divmod(np.arange(n), Nx * Ny)
    iy, ix = np.divmod(rem, Nx)
    interior = (iz > 0) & (iz < Nz - 1) & (iy > 0) & (iy < Ny - 1) & (ix > 0) & (ix < Nx - 1)
    scale = np.abs(M).sum(axis=1).A.ravel()
    assert np.all(np.abs(s[interior]) <= 1e-13 * scale[interior])
    assert np.all(s[~interior] > 0)


def test_conv_diff_3d_bench_size():
    A = synth.conv_diff_3d(64, peclet=50.0, seed=3)
    assert len(A[0]) - 1 == 262144 and len(A[1]) == 1810432


@pytest.mark.parametrize("k", [1, 8, 16])
def test_random_sparse_nonzeros_per_column(k):
    n = 300
    A = synth.random_sparse(n, nnz_per_col=k, seed=6)
    check_csr(A, n)
    M = synth.to_scipy(A).tocsc()
    assert np.all(np.diff(M.indptr) == k)  # distinct rows: no duplicates were summed away
    d = M.diagonal()
    shift = 2.0 * np.sqrt(max(k - 1, 1))
    assert np.all(np.abs(d) >= shift)


def test_random_sparse_scaling_is_two_sided_diagonal():
    # with log10_scale s the matrix is D_r R D_c, D_r and D_c on [1, 10^(s/2)], R the unscaled
    # matrix of the same seed: every entry ratio is dr_i dc_j, a rank-one pattern in logs
    n, s = 200, 6.0
    R = synth.to_scipy(synth.random_sparse(n, 8, seed=6)).tocoo()
    S = synth.to_scipy(synth.random_sparse(n, 8, seed=6, log10_scale=s)).tocsr()
    ratio = np.asarray(S[R.row, R.col]).ravel() / R.data
    assert np.all(ratio >= 1.0 - 1e-12) and np.all(ratio <= 10.0 ** s * (1 + 1e-12))
    # log ratio = a_i + b_j: fit by least squares over the pattern, residual at rounding level
    rows = np.concatenate([np.arange(len(R.data)), np.arange(len(R.data))])
    cols = np.concatenate([R.row, n + R.col])
    X = sp.csr_matrix((np.ones(2 * len(R.data)), (rows, cols)), shape=(len(R.data), 2 * n))
    y = np.log10(ratio)
    sol = sp.linalg.lsqr(X, y, atol=1e-14, btol=1e-14, iter_lim=20000)[0]
    assert np.max(np.abs(X @ sol - y)) < 1e-9


def test_generators_are_deterministic_under_their_seeds():
    for make in (lambda sd: synth.conv_diff_2d(6, seed=sd), lambda sd: synth.conv_diff_3d(4, seed=sd),
                 lambda sd: synth.random_sparse(100, 8, seed=sd, log10_scale=2.0)):
        a, b, c = make(1), make(1), make(2)
        assert all(np.array_equal(x, y) for x, y in zip(a, b))
        assert not np.array_equal(a[2], c[2])
    A = synth.conv_diff_2d(6)
    b1, x1 = synth.rhs(A, seed=2)
    b2, x2 = synth.rhs(A, seed=2)
    assert np.array_equal(b1, b2) and np.array_equal(x1, x2)
    assert np.allclose(synth.to_scipy(A) @ x1, b1, rtol=0, atol=1e-13 * np.abs(b1).max())
