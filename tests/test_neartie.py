"""The near-tie replay (tests/neartie.py) that the adaptive parity tests use to
accept a column whose pattern differs from the oracle's: it returns nothing
for the oracle's own patterns, a zero margin for an exact tie of the
selection rule, and, for patterns with a planted wrong index, margins far
above the NEAR_TIE allowance in nearly every column, so that a selection bug
on the GPU could not pass as rounding."""
import numpy as np
import scipy.sparse as sp

import oracle as O
from neartie import _col_lists, replay_gap
from paper_2202_10204_gb300 import synth

NEAR_TIE = 512  # the allowance of the parity tests, in units of u_f


def test_oracle_patterns_replay_to_none():
    A = synth.random_sparse(400, 6, seed=12)
    ref = O.spai(A, init=O.PAT_IDENTITY, adaptive=True, eps=0.3, beta=8, max_fill=30, uf="single")
    cols = _col_lists(A)
    for k in range(ref["n"]):
        J = ref["Jidx"][k][: ref["Jcnt"][k]]
        assert replay_gap(A, ref["d"], k, J, "single", 0.3, 8, 30, colsA=cols) is None, k


def test_exact_tie_is_a_zero_selection_margin():
    # column 0: J = {0}, I = {0, 1}, residual s on rows 0 and 1; rows 2 and 3 of A agree on
    # columns 0 and 1 and have equal norms, so the candidates 2 and 3 have the same rho
    # bit for bit; beta = 1 takes one, the smaller index (reading R4)
    Ad = np.array([[2, 1, 0, 0], [0, 0, 3, 1], [1, 1, 1, 0], [1, 1, 0, 1]], float)
    A = synth._to_csr(sp.csr_matrix(Ad))
    ref = O.spai(A, init=O.PAT_IDENTITY, adaptive=True, eps=1e-3, beta=1, max_fill=2, uf="double")
    assert list(ref["Jidx"][0][: ref["Jcnt"][0]]) == [0, 2]
    assert replay_gap(A, ref["d"], 0, [0, 2], "double", 1e-3, 1, 2) is None
    assert replay_gap(A, ref["d"], 0, [0, 3], "double", 1e-3, 1, 2) == ("selection", 0.0, 0)


def test_planted_wrong_index_is_not_a_near_tie():
    A = synth.random_sparse(400, 6, seed=12)
    ref = O.spai(A, init=O.PAT_IDENTITY, adaptive=True, eps=0.3, beta=8, max_fill=30, uf="single")
    cols = _col_lists(A)
    u = O.UNIT_ROUNDOFF[O.SINGLE]
    rng = np.random.default_rng(0)
    gaps = []
    for k in range(ref["n"]):
        J = [int(j) for j in ref["Jidx"][k][: ref["Jcnt"][k]]]
        if len(J) < 2:
            continue
        r = int(rng.integers(0, ref["n"]))
        while r in J:
            r = int(rng.integers(0, ref["n"]))
        planted = sorted(J[:-1] + [r])  # the last index the oracle added, swapped for another
        g = replay_gap(A, ref["d"], k, planted, "single", 0.3, 8, 30, colsA=cols)
        assert g is not None, k
        gaps.append(g[1] / u)
    gaps = np.array(gaps)
    assert len(gaps) >= 200
    # the replay explains a mismatch by the smallest margin on the consistent stretch of the
    # oracle's path, so a planted index passes only where that stretch holds a genuinely
    # close decision: a few columns, not the many a selection bug would touch
    assert np.mean(gaps > NEAR_TIE) > 0.9
