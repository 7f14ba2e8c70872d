"""GPU parity at full workload sizes (sampled against the oracle) and the
serving queue.

* The 64^3 bench workload, in the launch configuration bench.py times:
  the pattern of every column is checked against pattern(A^2) with the cap
  (from scipy), a seeded sample of columns against the oracle's own column
  computation, and the refinement against properties that hold at any size
  (backward error at the stop tolerance, bounded steps).
* An adaptive (Grote-Huckle) build on a 100,000-column random nonsymmetric
  matrix, 16 nonzeros per column, condition raised by row/column scaling:
  sampled columns against the oracle.
* Serving: requests of different sizes and precisions submitted together
  give bitwise the same solution as the same request solved alone.
"""
import time

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
    c = S.Context(0, stream=torch.cuda.current_stream())
    yield c
    c.close()


def col_residuals(A, d, cols, J_list, m_list):
    """float64 ||B(:,J_k) m_k - e_k|| and || |B(:,J_k)| |m_k| || for the sampled columns."""
    Ms = synth.to_scipy(A)
    n = Ms.shape[0]
    B = (Ms.T @ sp.diags(d)).tocsc()
    res, absbm = [], []
    for k, J, m in zip(cols, J_list, m_list):
        BJ = B[:, J]
        r = BJ @ m
        r[k] -= 1.0
        res.append(np.linalg.norm(r))
        absbm.append(np.linalg.norm(abs(BJ) @ np.abs(m)))
    return np.array(res), np.array(absbm)


# pattern mismatches must be near-ties of rho (see test_gpu_parity.NEAR_TIE)
NEAR_TIE = 512


def check_sampled_columns(A, P_csr, ref, cols, uf, adaptive=None):
    """adaptive = (eps, beta, max_fill) for Grote-Huckle runs: a column whose
    pattern differs from the oracle's must be a near-tie (replayed)."""
    rp, ci, va = P_csr
    d = ref["d"]
    same, Jg, mg, Jo, mo = [], [], [], [], []
    for k in cols:
        J = ci[rp[k]:rp[k + 1]]
        Jr = ref["Jidx"][k][: ref["Jcnt"][k]]
        same.append(np.array_equal(J, Jr))
        Jg.append(J); mg.append(va[rp[k]:rp[k + 1]] / d[J])
        Jo.append(Jr); mo.append(ref["mbar"][k][: ref["Jcnt"][k]])
    same = np.array(same)
    if adaptive is None:
        assert same.all()
    else:
        eps, beta, F = adaptive
        u = O.UNIT_ROUNDOFF[O.prec(uf)]
        bad = []
        for k, g, o, sm in zip(cols, Jg, Jo, same):
            if sm:
                continue
            r = replay_gap(A, d, int(k), g, uf, eps, beta, F)
            assert r is not None, (k, g, o)
            if r[1] > NEAR_TIE * u:
                bad.append((int(k), r[0], r[2], r[1] / u))
        print("pattern mismatches: %d of %d sampled columns" % (int((~same).sum()), len(cols)))
        assert not bad, bad
    cols = np.asarray(cols)
    rg, ag = col_residuals(A, d, cols, Jg, mg)
    ro, _ = col_residuals(A, d, cols, Jo, mo)
    u = O.UNIT_ROUNDOFF[O.prec(uf)]
    diff = np.abs(rg - ro)[same]
    bound = RES_TOL[uf] * ro[same] + (4 * u + 64 * 2.0 ** -53) * ag[same]
    assert np.all(diff <= bound), np.max(diff - bound)
    assert np.mean(diff <= RES_TOL[uf] * ro[same]) >= 0.99


def test_bench_workload_full_size(ctx):
    A, b, x_true = synth.cfg_large_3d(N=64)
    n = len(A[0]) - 1
    Ad = tuple(torch.from_numpy(a).cuda() for a in A)
    so = S.make_spai_opts(init=2, max_fill=25, uf="half", eps=0.3)
    P, st = S.spai_build(ctx, Ad, so, per_column=True)
    Pc = P.export()
    # every column's pattern: column k of pattern(A^2), at most 25 (interior columns have exactly 25)
    Ms = synth.to_scipy(A)
    A2 = (abs(Ms) @ abs(Ms)).tocsc()
    A2.sort_indices()
    assert np.array_equal(np.diff(Pc[0]), np.diff(A2.indptr))
    assert np.array_equal(Pc[1], A2.indices)
    assert st["max_I"] == 63 and st["max_J"] == 25
    # sampled columns against the oracle
    cols = np.sort(np.random.default_rng(7).choice(n, size=384, replace=False))
    cols = np.unique(np.concatenate([cols, [0, 1, n // 2, n - 1]]))
    ref = O.spai(A, init=O.PAT_A2, max_fill=25, uf="half", eps=0.3, cols=cols)
    check_sampled_columns(A, Pc, ref, cols, "half")
    assert np.array_equal(st["nI"][cols], ref["Icnt"][cols])
    # the refinement: stops at the backward-error tolerance within i_max
    io = S.make_ir_opts(uf="half", u="single", ug="single", up="single", ur="double", tau=1e-4)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    r = S.gmres_ir_solve(ctx, Ad, bd, xd, P=P, opts=io)
    x = xd.cpu().numpy()
    assert r["flags"] & 1 and 1 <= r["steps"] <= 10
    q = 7
    nbe = np.max(np.abs(b - Ms @ x)) / (abs(Ms).sum(axis=1).max() * np.max(np.abs(x)) + np.max(np.abs(b)))
    assert nbe <= q * 2.0 ** -24
    assert abs(r["final_nbe"] - nbe) <= 0.5 * nbe  # the kernel's own estimate (single-precision iterate)
    assert np.max(np.abs(x - x_true)) / np.max(np.abs(x_true)) < 1e-4
    P.free()


def check_ir_against_oracle(A, b, x_true, x, st, ref, u):
    """Same number of refinement steps, total GMRES iterations within 10%,
    normwise backward and forward errors within 10x of the oracle's."""
    Ms = synth.to_scipy(A)
    assert st["steps"] == ref["steps"], (st["its"], list(ref["its"]))
    assert abs(st["total_its"] - ref["total_its"]) <= max(1, 0.1 * ref["total_its"]), (st["its"], list(ref["its"]))
    def errs(xx):
        nbe = np.max(np.abs(b - Ms @ xx)) / (abs(Ms).sum(axis=1).max() * np.max(np.abs(xx)) + np.max(np.abs(b)))
        return nbe, np.max(np.abs(xx - x_true)) / np.max(np.abs(x_true))
    nb_g, fe_g = errs(x)
    nb_o, fe_o = errs(ref["x"])
    assert nb_g <= 10 * max(nb_o, u) and fe_g <= 10 * max(fe_o, u), (nb_g, nb_o, fe_g, fe_o)


@pytest.mark.parametrize("orth", [2, 0])
def test_bench_workload_refinement_full_size(ctx, orth):
    """The 64^3 bench workload solved in the launch configuration bench.py times,
    against a full oracle solve of the same system (every SPAI column, then the
    refinement): every column's residual within the half-precision tolerance,
    and the refinement's steps, iterations and errors (one-reduction MGS, the
    headline's, and the MGS exchange rounds)."""
    A, b, x_true = synth.cfg_large_3d(N=64)
    Ad = tuple(torch.from_numpy(a).cuda() for a in A)
    so = S.make_spai_opts(init=2, max_fill=25, uf="half", eps=0.3)
    P, st = S.spai_build(ctx, Ad, so, per_column=True)
    Pc = P.export()
    O.set_threads(0)
    ref_s = O.spai(A, init=O.PAT_A2, max_fill=25, uf="half", eps=0.3)
    assert np.array_equal(np.diff(Pc[0]), ref_s["Jcnt"])
    assert np.array_equal(st["nI"], ref_s["Icnt"])
    # every column: float64 residuals of both sides' m_k within 1e-3 relative plus the
    # u_f representation floor, 99% within the pure relative tolerance
    Ms = synth.to_scipy(A)
    d = ref_s["d"]
    n = len(b)
    B = (Ms.T @ sp.diags(d)).tocsc()
    rows = np.repeat(np.arange(n), np.diff(Pc[0]))
    Mg = sp.csr_matrix((Pc[2] / d[Pc[1]], (Pc[1], rows)), shape=(n, n))
    mask = np.arange(25)[None, :] < ref_s["Jcnt"][:, None]
    Mo = sp.csr_matrix((ref_s["mbar"][mask], (ref_s["Jidx"][mask], np.repeat(np.arange(n), ref_s["Jcnt"]))),
                       shape=(n, n))
    def colnorm(M):
        return np.sqrt(np.asarray(M.multiply(M).sum(axis=0)).ravel())
    rg = colnorm((B @ Mg - sp.identity(n)).tocsc())
    ro = colnorm((B @ Mo - sp.identity(n)).tocsc())
    ag = colnorm((abs(B) @ abs(Mg)).tocsc())
    floor = (4 * 2.0 ** -11 + 64 * 2.0 ** -53) * ag
    diff = np.abs(rg - ro)
    assert np.all(diff <= RES_TOL["half"] * ro + floor), np.max(diff - RES_TOL["half"] * ro - floor)
    assert np.mean(diff <= RES_TOL["half"] * ro) >= 0.99
    # the refinement
    kw = dict(uf="half", u="single", ug="single", up="single", ur="double", tau=1e-4)
    io = S.make_ir_opts(orth=orth, **kw)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    r = S.gmres_ir_solve(ctx, Ad, bd, xd, P=P, opts=io)
    ref = O.gmres_ir(A, b, O.assemble_P(ref_s, "single", "half"), orth=orth, **kw)
    check_ir_against_oracle(A, b, x_true, xd.cpu().numpy(), r, ref, 2.0 ** -24)
    P.free()


def test_adaptive_ill_conditioned_refinement():
    """A random nonsymmetric system in the style of the ill-conditioned stress
    configuration: n = 10,000, 16 nonzeros per column, row and column scalings of
    up to 10^3 each; Grote-Huckle SPAI from the identity (eps 0.5, beta 8, cap 30,
    u_f single) and the refinement with (single, double, double, double, quad),
    whose GMRES solves run to their 500-iteration cap.  Against the oracle: the
    patterns up to near-ties of rho, and the refinement's steps, iterations and
    errors (modified Gram-Schmidt, the paper's method, and its one-reduction form)."""
    c = S.Context(0)
    A = synth.random_sparse(10000, 16, seed=6, log10_scale=6.0)
    b, x_true = synth.rhs(A, seed=7)
    so = S.make_spai_opts(init=0, adaptive=True, eps=0.5, beta=8, max_fill=30, uf="single")
    P, st = S.spai_build(c, A, so, per_column=True)
    O.set_threads(0)
    ref_s = O.spai(A, init=O.PAT_IDENTITY, adaptive=True, eps=0.5, beta=8, max_fill=30, uf="single")
    Pc = P.export()
    cols = np.arange(0, 10000, 7)
    check_sampled_columns(A, Pc, ref_s, cols, "single", adaptive=(0.5, 8, 30))
    kw = dict(uf="single", u="double", ug="double", up="double", ur="quad", tau=1e-8)
    x = np.zeros_like(b)
    r = S.gmres_ir_solve(c, A, b, x, P=P, opts=S.make_ir_opts(**kw))
    # the refinement is compared on the same preconditioner (the GPU's, whose near-tie
    # columns may differ from the oracle's): its values rounded to u_p and u_f
    Pv = (Pc[0], Pc[1], O.round_to(Pc[2], "double"), O.round_to(Pc[2], "single"))
    ref = O.gmres_ir(A, b, Pv, **kw)
    assert max(ref["its"]) >= 300
    check_ir_against_oracle(A, b, x_true, x, r, ref, 2.0 ** -53)
    # the one-reduction MGS on the same system: its GMRES solves run long enough that the
    # sums over blocks are split among the blocks (2 (j + 1) partials x blocks >= 32768)
    x2 = np.zeros_like(b)
    r2 = S.gmres_ir_solve(c, A, b, x2, P=P, opts=S.make_ir_opts(orth=2, **kw))
    assert 2 * (max(r2["its"]) + 1) * r2["grid"] >= 32768, (r2["its"], r2["grid"])
    ref2 = O.gmres_ir(A, b, Pv, orth=O.ORTH_MGS_ICWY, **kw)
    check_ir_against_oracle(A, b, x_true, x2, r2, ref2, 2.0 ** -53)
    P.free()
    c.close()


def test_adaptive_100k_sampled(ctx):
    A = synth.random_sparse(100_000, 16, seed=6, log10_scale=6.0)
    n = len(A[0]) - 1
    so = S.make_spai_opts(init=0, adaptive=True, eps=0.5, beta=8, max_fill=30, uf="single")
    t0 = time.time()
    P, st = S.spai_build(ctx, A, so, per_column=True)
    assert time.time() - t0 < 120
    Pc = P.export()
    cols = np.sort(np.random.default_rng(11).choice(n, size=48, replace=False))
    ref = O.spai(A, init=O.PAT_IDENTITY, adaptive=True, eps=0.5, beta=8, max_fill=30, uf="single", cols=cols)
    # a column may select differently from the oracle only on a near-tie of rho
    check_sampled_columns(A, Pc, ref, cols, "single", adaptive=(0.5, 8, 30))
    conv = (st["flags"][cols] & 1) != 0
    assert np.mean(conv == ((ref["flags"][cols] & 1) != 0)) >= 0.95
    P.free()


def _requests():
    reqs = []
    A, b, _ = synth.cfg_small_2d()
    reqs.append((A, b, S.make_spai_opts(init=1, max_fill=30, uf="single"),
                 S.make_ir_opts(uf="single", u="double", ug="double", up="double", ur="quad", tau=1e-4)))
    for N, seed in ((12, 3), (16, 5), (20, 9)):
        A3 = synth.conv_diff_3d(N, 50.0, seed=seed)
        b3, _ = synth.rhs(A3, seed=seed + 1)
        reqs.append((A3, b3, S.make_spai_opts(init=2, max_fill=25, uf="half"),
                     S.make_ir_opts(uf="half", u="single", ug="single", up="single", ur="double", tau=1e-4)))
    Ar = synth.random_sparse(3000, 8, seed=4, log10_scale=2.0)
    br, _ = synth.rhs(Ar, seed=1)
    reqs.append((Ar, br, S.make_spai_opts(init=0, adaptive=True, eps=0.4, max_fill=20, uf="single"),
                 S.make_ir_opts(uf="single", u="double", ug="single", up="single", ur="double", tau=1e-4)))
    A2, b2, _ = synth.cfg_small_2d(seed_mat=5, seed_rhs=6)
    reqs.append((A2, b2, None, S.make_ir_opts(uf="single", u="double", ug="double", up="double", ur="double",
                                              tau=1e-8)))
    # half-precision Krylov storage (u_g = u_p = half, one-reduction MGS)
    A4 = synth.conv_diff_3d(14, 50.0, seed=11)
    b4, _ = synth.rhs(A4, seed=12)
    reqs.append((A4, b4, S.make_spai_opts(init=2, max_fill=25, uf="half"),
                 S.make_ir_opts(uf="half", u="single", ug="half", up="half", ur="double", tau=1e-2, orth=2,
                                ir_max_steps=30)))
    return reqs


def _serve(ctx, reqs, stagger=0.0):
    """Submit reqs (the second half `stagger` seconds after the first) and poll
    until every request is done; returns [(x, stats)] in submission order."""
    half = (len(reqs) + 1) // 2 if stagger > 0 else len(reqs)
    tickets = [S.solver_submit(ctx, A, b, so, io) for (A, b, so, io) in reqs[:half]]
    if stagger > 0:
        time.sleep(stagger)
        tickets += [S.solver_submit(ctx, A, b, so, io) for (A, b, so, io) in reqs[half:]]
    results = {}
    t0 = time.time()
    while len(results) < len(tickets):
        assert time.time() - t0 < 300
        for i, t in enumerate(tickets):
            if i in results:
                continue
            x = np.zeros_like(reqs[i][1])
            st = S.solver_poll(ctx, t, x)
            if st is not None:
                results[i] = (x, st)
        time.sleep(0.002)
    return [results[i] for i in range(len(reqs))]


def test_serving_mix_matches_standalone():
    # continuous batching: each request gives the same bits alone in the queue, all at once,
    # and when half of them arrive while the first half is on the GPU
    reqs = _requests()
    alone = []
    for req in reqs:
        c1 = S.Context(0, hbm_budget=8 << 30)
        alone.append(_serve(c1, [req])[0])
        c1.close()
    for stagger in (0.0, 0.005):
        c2 = S.Context(0, hbm_budget=8 << 30)
        mix = _serve(c2, reqs, stagger)
        c2.close()
        for i in range(len(reqs)):
            xa, sa = alone[i]
            xm, sm = mix[i]
            assert sm["steps"] == sa["steps"] and sm["its"] == sa["its"], (stagger, i)
            assert np.array_equal(xm, xa), (stagger, i)  # deterministic kernels: the same bits alone and in the mix
            if len(reqs[i][1]) <= 65536:
                assert sm["grid"] <= 16, sm["grid"]  # solved by a team of the batched launch
    # and within the refinement tolerance of the single-system entry point
    c3 = S.Context(0)
    for i, (A, b, so, io) in enumerate(reqs):
        if io.ug == 0:
            continue  # half Krylov storage: compared with the oracle in test_gpu_parity.py
        x = np.zeros_like(b)
        st = S.gmres_ir_solve(c3, A, b, x, sopts=so, opts=io)
        xa, sa = alone[i]
        assert sa["steps"] == st["steps"], (i, sa["its"], st["its"])
        assert abs(sa["total_its"] - st["total_its"]) <= max(1, 0.1 * st["total_its"]), (i, sa["its"], st["its"])
        Ms = synth.to_scipy(A)
        nb = lambda y: np.max(np.abs(b - Ms @ y)) / (abs(Ms).sum(axis=1).max() * np.max(np.abs(y)) + np.max(np.abs(b)))
        assert nb(xa) <= 10 * max(nb(x), 2.0 ** -53), (i, nb(xa), nb(x))
    c3.close()


def test_serving_failed_request_does_not_affect_others():
    # a request with a non-finite value fails on its own; the requests admitted with it are
    # solved as they would be alone
    reqs = _requests()[1:4]
    A, b, so, io = reqs[1]
    rp, ci, va = A
    va = va.copy()
    va[3] = np.nan
    bad = ((rp, ci, va), b, so, io)
    c1 = S.Context(0, hbm_budget=8 << 30)
    alone = [_serve(c1, [r])[0] for r in (reqs[0], reqs[2])]
    c1.close()
    c2 = S.Context(0, hbm_budget=8 << 30)
    tickets = [S.solver_submit(c2, A_, b_, so_, io_) for (A_, b_, so_, io_) in (reqs[0], bad, reqs[2])]
    got = {}
    t0 = time.time()
    while len(got) < 3:
        assert time.time() - t0 < 120
        for i, t in enumerate(tickets):
            if i in got:
                continue
            x = np.zeros(len(b) if i == 1 else len((reqs[0], bad, reqs[2])[i][1]))
            try:
                st = S.solver_poll(c2, t, x)
            except S.SpaiError as e:
                got[i] = e.code
                continue
            if st is not None:
                got[i] = (x, st)
        time.sleep(0.002)
    c2.close()
    assert got[1] == S._lib.ERR_NONFINITE
    for i, j in ((0, 0), (2, 1)):
        assert np.array_equal(got[i][0], alone[j][0]) and got[i][1]["its"] == alone[j][1]["its"]


def test_serving_admission_budget():
    A, b, _ = synth.cfg_small_2d()
    c = S.Context(0, hbm_budget=1 << 20)
    with pytest.raises(S.SpaiError) as e:
        S.solver_submit(c, A, b, S.make_spai_opts(init=1), S.make_ir_opts())
    assert e.value.code == -5
    with pytest.raises(S.SpaiError) as e:
        S.solver_poll(c, 12345)
    assert e.value.code == -9
    c.close()
