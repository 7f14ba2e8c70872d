"""The allocation-free refinement entry point (gmres_ir_solve_noalloc).

Some callers cannot call the CUDA allocator: work being recorded into a
CUDA graph, real-time or embedded runtimes that forbid allocation after
start-up, and hosts that hand the library an exact memory budget.  For them
the library offers gmres_ir_solve_noalloc, which keeps all its scratch in
one fixed device array.  This test calls it through the C ABI twice in a
row and checks each result against the allocating entry point
(gmres_ir_solve with the same preconditioner), with the tolerance the other
GPU tests use for refinement results (same step count, GMRES iterations
within 10%, solution within 10 u of the reference relative to its norm).
It lives in its own file, collected last, and runs alone or after the
other tests.
"""
import numpy as np
import pytest

from paper_2202_10204_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_2202_10204_gb300 as S  # noqa: E402
from paper_2202_10204_gb300 import _lib  # noqa: E402


def to_dev(A):
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in A)


@pytest.mark.parametrize("case", ["3d-half-single", "2d-single-double-quad"])
def test_noalloc_matches_allocating_entry_point(case):
    if case == "3d-half-single":
        A, b, _ = synth.cfg_large_3d(N=16)
        so = S.make_spai_opts(init=2, max_fill=25, uf="half")
        io = S.make_ir_opts(uf="half", u="single", ug="single", up="single", ur="double", tau=1e-4)
        u = 2.0 ** -24
    else:
        A, b, _ = synth.cfg_small_2d()
        so = S.make_spai_opts(init=1, max_fill=30, uf="single")
        io = S.make_ir_opts(uf="single", u="double", ug="double", up="double", ur="quad", tau=1e-4)
        u = 2.0 ** -53
    ctx = S.Context(0, stream=torch.cuda.current_stream())
    P, _ = S.spai_build(ctx, A, so)
    Pcsr = P.export()
    Ad, bd, Pd = to_dev(A), torch.from_numpy(b).cuda(), to_dev(Pcsr)
    x_ref = torch.zeros_like(bd)
    ref = S.gmres_ir_solve(ctx, Ad, bd, x_ref, P=P, opts=io)
    torch.cuda.synchronize()
    xr = x_ref.cpu().numpy()
    for call in range(2):
        x = torch.full_like(bd, float("nan"))
        st = _lib.gmres_ir_solve_noalloc(Ad, bd, x, P=Pd, opts=io, stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        xn = x.cpu().numpy()
        assert st["steps"] == ref["steps"], (call, st["its"], ref["its"])
        assert abs(st["total_its"] - ref["total_its"]) <= max(1, 0.1 * ref["total_its"])
        assert np.all(np.isfinite(xn))
        assert np.max(np.abs(xn - xr)) <= 10 * u * np.max(np.abs(xr)), call
    P.free()
    ctx.close()


def test_noalloc_rejects_problems_beyond_its_scratch():
    # the Krylov basis alone (n x (gmres_max_it + 1) doubles) exceeds the fixed array
    A, b, _ = synth.cfg_large_3d(N=24)
    Ad, bd = to_dev(A), torch.from_numpy(b).cuda()
    io = S.make_ir_opts(uf="single", u="double", ug="double", up="double", ur="double", tau=1e-8,
                        gmres_max_it=1000)
    with pytest.raises(S.SpaiError) as e:
        _lib.gmres_ir_solve_noalloc(Ad, bd, torch.zeros_like(bd), P=None, opts=io)
    assert e.value.code == _lib.ERR_UNSUPPORTED
