"""GPU: the batched refinement entry point (gmres_ir_solve_batch).

Systems solved together in one persistent launch run on teams of fewer
blocks than alone (about 2048 rows per block), so their reductions round
differently; the bar is the GMRES-IR one of the other tests: the same number
of refinement steps as the same system solved alone (or by the oracle),
GMRES iterations within 10%, backward and forward errors within 10x.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_2202_10204_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_2202_10204_gb300 as S  # noqa: E402

TUPLE = dict(uf="single", u="double", ug="single", up="single", ur="double")


@pytest.fixture(scope="module")
def ctx():
    c = S.Context(0)
    yield c
    c.close()


def errors(A, b, x, x_true):
    Ms = synth.to_scipy(A)
    nbe = np.max(np.abs(b - Ms @ x)) / (abs(Ms).sum(axis=1).max() * np.max(np.abs(x)) + np.max(np.abs(b)))
    return nbe, np.max(np.abs(x - x_true)) / np.max(np.abs(x_true))


def mixed_systems():
    out = []
    for i, N in enumerate((20, 45, 64, 100, 130)):
        A = synth.conv_diff_2d(N, 10.0 + 8 * i, 1.0, 0.1, seed=40 + i)
        out.append(A)
    for i, n in enumerate((3000, 9000, 20000)):
        out.append(synth.random_sparse(n, 8 + 2 * i, seed=50 + i, log10_scale=2.0))
    out.append(synth.conv_diff_3d(18, 50.0, seed=60))
    return out


def test_batch_matches_single_solves(ctx):
    As = mixed_systems()
    io = S.make_ir_opts(tau=1e-4, **TUPLE)
    so = S.make_spai_opts(init=1, max_fill=30, uf="single")
    Ps = [S.spai_build(ctx, A, so)[0] for A in As]
    Ps[3] = None  # one system without a preconditioner
    bs, xts = zip(*[synth.rhs(A, seed=70 + i) for i, A in enumerate(As)])
    xs = [np.zeros_like(b) for b in bs]
    sts, status = S.gmres_ir_solve_batch(ctx, As, list(bs), xs, Ps, io)
    assert all(s_ >= 0 for s_ in status)
    for i, A in enumerate(As):
        x1 = np.zeros_like(bs[i])
        st1 = S.gmres_ir_solve(ctx, A, bs[i], x1, P=Ps[i], opts=io)
        assert sts[i]["steps"] == st1["steps"], (i, sts[i]["its"], st1["its"])
        assert abs(sts[i]["total_its"] - st1["total_its"]) <= max(1, 0.1 * st1["total_its"]), (i, sts[i]["its"],
                                                                                          st1["its"])
        nb_b, fe_b = errors(A, bs[i], xs[i], xts[i])
        nb_s, fe_s = errors(A, bs[i], x1, xts[i])
        u = 2.0 ** -53
        assert nb_b <= 10 * max(nb_s, u) and fe_b <= 10 * max(fe_s, u), (i, nb_b, nb_s, fe_b, fe_s)
        assert sts[i]["flags"] & 1
    for P in Ps:
        if P is not None:
            P.free()


def test_batch_against_oracle(ctx):
    As = [synth.conv_diff_2d(24, 20.0, 1.0, 0.1, seed=7), synth.random_sparse(1500, 8, seed=3, log10_scale=2.0)]
    io = S.make_ir_opts(tau=1e-4, **TUPLE)
    Ps, refs, bs, xts = [], [], [], []
    for i, A in enumerate(As):
        b, xt = synth.rhs(A, seed=90 + i)
        bs.append(b); xts.append(xt)
        P, _ = S.spai_build(ctx, A, S.make_spai_opts(init=1, max_fill=30, uf="single"))
        Ps.append(P)
        Sr = O.spai(A, init=O.PAT_A, max_fill=30, uf="single")
        refs.append(O.gmres_ir(A, b, O.assemble_P(Sr, "single", "single"), tau=1e-4, **TUPLE))
    xs = [np.zeros_like(b) for b in bs]
    sts, _ = S.gmres_ir_solve_batch(ctx, As, bs, xs, Ps, io)
    for i, A in enumerate(As):
        ref = refs[i]
        assert sts[i]["steps"] == ref["steps"], (sts[i]["its"], list(ref["its"]))
        assert abs(sts[i]["total_its"] - ref["total_its"]) <= max(1, 0.1 * ref["total_its"])
        nb_g, fe_g = errors(A, bs[i], xs[i], xts[i])
        nb_o, fe_o = errors(A, bs[i], ref["x"], xts[i])
        assert nb_g <= 10 * max(nb_o, 2.0 ** -53) and fe_g <= 10 * max(fe_o, 2.0 ** -53)
        Ps[i].free()


def test_batch_more_systems_than_teams_device_inputs(ctx):
    # 24 systems of n = 65536 on teams of 8 blocks (19 teams on 152 SMs): some teams
    # solve two systems one after another; inputs and outputs on the device
    dev = torch.device("cuda", 0)
    io = S.make_ir_opts(tau=1e-4, **TUPLE)
    As, bs, xts, Ps = [], [], [], []
    for i in range(24):
        A = synth.conv_diff_2d(256, 5.0 + i, 1.0, 0.1, seed=100 + i)
        b, xt = synth.rhs(A, seed=200 + i)
        Ad = tuple(torch.from_numpy(a).to(dev) for a in A)
        As.append(Ad); bs.append(torch.from_numpy(b).to(dev)); xts.append((A, b, xt))
        Ps.append(S.spai_build(ctx, Ad, S.make_spai_opts(init=1, max_fill=30, uf="single"))[0])
    xs = [torch.zeros_like(b) for b in bs]
    sts, status = S.gmres_ir_solve_batch(ctx, As, bs, xs, Ps, io)
    assert all(s_ == 0 for s_ in status)
    assert sts[0]["launches"] >= 1 + 24  # one batched launch + per-system kernels
    for i in range(24):
        A, b, xt = xts[i]
        nbe, fe = errors(A, b, xs[i].cpu().numpy(), xt)
        assert nbe <= 20 * 2.0 ** -53 and fe <= 1e-10, (i, nbe, fe)
        assert sts[i]["grid"] == 8  # about 8192 rows per block
        Ps[i].free()


def test_batch_edge_cases(ctx):
    io = S.make_ir_opts(tau=1e-4, **TUPLE)
    assert S.gmres_ir_solve_batch(ctx, [], [], [], None, io) == ([], [])
    A = synth.conv_diff_2d(16, 10.0, 1.0, 0.1, seed=1)
    b, _ = synth.rhs(A, seed=2)
    P, _ = S.spai_build(ctx, A, S.make_spai_opts(init=1, uf="half"))
    with pytest.raises(S.SpaiError) as e:  # P built with another u_f
        S.gmres_ir_solve_batch(ctx, [A], [b], [np.zeros_like(b)], [P], io)
    assert e.value.code == -1
    P.free()
    # a zero right-hand side among others: x = 0 with no GMRES work
    A2 = synth.conv_diff_2d(30, 10.0, 1.0, 0.1, seed=3)
    b2, _ = synth.rhs(A2, seed=4)
    xs = [np.ones(256), np.zeros_like(b2)]
    sts, status = S.gmres_ir_solve_batch(ctx, [A, A2], [np.zeros(256), b2], xs, None, io)
    assert np.all(xs[0] == 0) and sts[0]["steps"] == 0 and sts[1]["flags"] & 1


BUILD_CASES = {
    # fixed patterns: one build over the block-diagonal union of the batch
    "pattern(A)-half": dict(init=1, max_fill=30, uf="half"),
    "pattern(A^2)-single-right": dict(init=2, max_fill=25, uf="single", side=1),
    "pattern(A)-double": dict(init=1, max_fill=30, uf="double"),
    # adaptive: concurrent builds, one per matrix
    "adaptive-single": dict(init=0, adaptive=True, eps=0.4, beta=8, max_fill=20, uf="single"),
}


@pytest.mark.parametrize("case", list(BUILD_CASES))
def test_spai_build_batch_matches_single_builds(ctx, case):
    # the batched build gives every matrix the preconditioner and statistics of its own build, bit for bit
    As = mixed_systems()
    big = BUILD_CASES[case]["init"] == 1
    if big:
        # columns of every kernel: shadows above 512 rows (large-shadow kernel) beside small ones
        As.insert(2, synth.random_sparse(900, 28, seed=31))
    so = S.make_spai_opts(**BUILD_CASES[case])
    Ps, sts = S.spai_build_batch(ctx, As, so, per_column=True)
    assert len(Ps) == len(As) and all(P is not None for P in Ps)
    for i, A in enumerate(As):
        P1, st1 = S.spai_build(ctx, A, so, per_column=True)
        for u, v in zip(P1.export(), Ps[i].export()):
            assert np.array_equal(u, v), i
        for key in ("n", "nnz_P", "cols_converged", "cols_fillcap", "cols_nonfinite", "max_I", "max_J", "rc"):
            assert sts[i][key] == st1[key], (i, key, sts[i][key], st1[key])
        for key in ("colres", "nJ", "nI", "flags"):
            assert np.array_equal(sts[i][key], st1[key]), (i, key)
        P1.free()
        Ps[i].free()
    if big:
        assert max(st["max_I"] for st in sts) > 512
    if not BUILD_CASES[case].get("adaptive"):
        assert len(set(st["launches"] for st in sts)) == 1  # one build for the whole batch


def test_spai_build_batch_device_inputs_and_failures(ctx):
    # device inputs; a matrix with a non-finite value makes its group's build fail, and the
    # matrices are then built one by one: that matrix alone reports the error
    dev = torch.device("cuda", 0)
    As = mixed_systems()[:5]
    rp, ci, va = As[3]
    va = va.copy()
    va[7] = np.inf
    As[3] = (rp, ci, va)
    Ad = [tuple(torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in A) for A in As]
    so = S.make_spai_opts(init=1, max_fill=30, uf="single")
    csrs = (S._lib.spai_csr * len(Ad))(*[S._lib.make_csr(A) for A in Ad])
    hs = (C.c_void_p * len(Ad))()
    status = (C.c_int * len(Ad))()
    rc = S._lib.lib().spai_build_batch(ctx.h, len(Ad), csrs, C.byref(so), hs, None, status)
    assert rc == S._lib.ERR_NONFINITE
    assert status[3] == S._lib.ERR_NONFINITE
    assert not hs[3] and all(hs[i] for i in (0, 1, 2, 4))
    for i in (0, 1, 2, 4):
        P = S._lib.Precond(C.c_void_p(hs[i]), ctx)
        P1, _ = S.spai_build(ctx, As[i], so)
        for u, v in zip(P1.export(), P.export()):
            assert np.array_equal(u, v), i
        assert status[i] >= 0
        P.free()
        P1.free()
    # a device CSR whose last entry names a column beyond its own matrix, inside the
    # rows of the batch (still sorted: a check of the union alone would pass it)
    bad = (Ad[0][0], Ad[0][1].clone(), Ad[0][2])
    bad[1][-1] = int(Ad[0][0].numel() - 1) + 5
    csrs = (S._lib.spai_csr * 2)(S._lib.make_csr(bad), S._lib.make_csr(Ad[1]))
    hs = (C.c_void_p * 2)()
    status = (C.c_int * 2)()
    rc = S._lib.lib().spai_build_batch(ctx.h, 2, csrs, C.byref(so), hs, None, status)
    assert rc == S._lib.ERR_INVALID_ARG and status[0] == S._lib.ERR_INVALID_ARG and status[1] >= 0
    assert not hs[0] and hs[1]
    S._lib.Precond(C.c_void_p(hs[1]), ctx).free()


@pytest.mark.parametrize("orth,side", [(1, 0), (0, 1), (2, 0), (2, 1)])
def test_batch_cgs2_and_right_preconditioning(ctx, orth, side):
    As = mixed_systems()[:6]
    io = S.make_ir_opts(tau=1e-4, orth=orth, side=side, **TUPLE)
    so = S.make_spai_opts(init=1, max_fill=30, uf="single", side=side)
    Ps, _ = S.spai_build_batch(ctx, As, so)
    bs, xts = zip(*[synth.rhs(A, seed=300 + i) for i, A in enumerate(As)])
    xs = [np.zeros_like(b) for b in bs]
    sts, status = S.gmres_ir_solve_batch(ctx, As, list(bs), xs, Ps, io)
    for i, A in enumerate(As):
        x1 = np.zeros_like(bs[i])
        st1 = S.gmres_ir_solve(ctx, A, bs[i], x1, P=Ps[i], opts=io)
        assert sts[i]["steps"] == st1["steps"], (i, sts[i]["its"], st1["its"])
        assert abs(sts[i]["total_its"] - st1["total_its"]) <= max(1, 0.1 * st1["total_its"])
        nb_b, fe_b = errors(A, bs[i], xs[i], xts[i])
        nb_s, fe_s = errors(A, bs[i], x1, xts[i])
        assert nb_b <= 10 * max(nb_s, 2.0 ** -53) and fe_b <= 10 * max(fe_s, 2.0 ** -53)
        Ps[i].free()


def test_batch_half_krylov_matches_single_solves(ctx):
    # u_g = u_p = half (one-reduction MGS) in the batched launch: each system as solved alone
    As = mixed_systems()[:6]
    tup = dict(uf="single", u="double", ug="half", up="half", ur="double")
    io = S.make_ir_opts(tau=1e-2, orth=2, ir_max_steps=30, **tup)
    so = S.make_spai_opts(init=1, max_fill=30, uf="single")
    Ps, _ = S.spai_build_batch(ctx, As, so)
    bs, xts = zip(*[synth.rhs(A, seed=500 + i) for i, A in enumerate(As)])
    xs = [np.zeros_like(b) for b in bs]
    sts, status = S.gmres_ir_solve_batch(ctx, As, list(bs), xs, Ps, io)
    assert all(s_ >= 0 for s_ in status)
    for i, A in enumerate(As):
        x1 = np.zeros_like(bs[i])
        st1 = S.gmres_ir_solve(ctx, A, bs[i], x1, P=Ps[i], opts=io)
        assert sts[i]["flags"] & 1 and st1["flags"] & 1
        # the step counts agree, or differ by one at a near-tie of the stop rule (a
        # half-precision Krylov step contracts the backward error by only ~1e-2)
        a, b = sts[i]["steps"], st1["steps"]
        if a != b:
            m = min(a, b)
            longer = sts[i]["nbe"] if a > b else st1["nbe"]
            assert abs(a - b) == 1 and longer[m] <= 10 * O.default_stop_tol(A, "double"), (i, sts[i], st1)
        m = min(a, b)
        assert abs(sum(sts[i]["its"][:m]) - sum(st1["its"][:m])) <= max(1, 0.1 * sum(st1["its"][:m]))
        xb = xs[i]
        if a > m:  # errors after the same number of steps
            xb = np.zeros_like(bs[i])
            S.gmres_ir_solve_batch(ctx, [A], [bs[i]], [xb], [Ps[i]], S.make_ir_opts(
                tau=1e-2, orth=2, ir_max_steps=m, **tup))
        elif b > m:
            x1 = np.zeros_like(bs[i])
            S.gmres_ir_solve(ctx, A, bs[i], x1, P=Ps[i], opts=S.make_ir_opts(tau=1e-2, orth=2, ir_max_steps=m, **tup))
        nb_b, fe_b = errors(A, bs[i], xb, xts[i])
        nb_s, fe_s = errors(A, bs[i], x1, xts[i])
        assert nb_b <= 10 * max(nb_s, 2.0 ** -53) and fe_b <= 10 * max(fe_s, 2.0 ** -53)
        Ps[i].free()


def test_batch_large_system_runs_alone_and_matches_single_solve(ctx):
    # a system of more than 65536 rows runs on a grid of its own inside the batch, exactly as
    # gmres_ir_solve runs it: the same bits; the small ones beside it run in the shared launch
    io = S.make_ir_opts(tau=1e-4, orth=2, **TUPLE)
    so = S.make_spai_opts(init=1, max_fill=30, uf="single")
    As = [synth.conv_diff_2d(300, 20.0, 1.0, 0.1, seed=11), synth.conv_diff_2d(40, 10.0, 1.0, 0.1, seed=12)]
    Ps, _ = S.spai_build_batch(ctx, As, so)
    bs = [synth.rhs(A, seed=20 + i)[0] for i, A in enumerate(As)]
    xs = [np.zeros_like(b) for b in bs]
    sts, status = S.gmres_ir_solve_batch(ctx, As, bs, xs, Ps, io)
    assert all(s_ >= 0 for s_ in status)
    x1 = np.zeros_like(bs[0])
    st1 = S.gmres_ir_solve(ctx, As[0], bs[0], x1, P=Ps[0], opts=io)
    assert sts[0]["grid"] == st1["grid"] and sts[0]["its"] == st1["its"]
    assert np.array_equal(xs[0], x1)
    assert sts[1]["grid"] == 1  # 1600 rows: a team of one block
    for P in Ps:
        P.free()
