"""Near-tie analysis of adaptive SPAI columns whose patterns differ between
the CUDA path and the oracle (reading R12 of the selection rule).

Both sides score the candidates of a Grote-Huckle step by rho_j computed
from their own least-squares residual, so the two scores of one candidate
differ by rounding; where two decisions are that close the sides may take
different ones, and their patterns differ from then on.  For a column k
whose GPU pattern J_g differs from the oracle's, the oracle's path is
replayed step by step with the oracle's own exported steps (the dense least
squares, rho and the selection of Algorithm 1).  The GPU's intermediate
patterns are not known, so the replay covers the stretch of the oracle's
path that is consistent with J_g: from the first step up to and including
the first step whose additions leave J_g (or the oracle's last step).  On
that stretch every decision's margin is measured, relative to the step's
mean rho: the selection boundary (the largest rho taken against the
smallest acceptable rho left out), the acceptance threshold (the mean
against the nearest rho on either side) and the column criterion
(||s|| against eps, relative to eps).  The smallest margin is returned: a
pattern mismatch is explained by rounding only if it is small.
"""
import numpy as np

import oracle as O


def _col_lists(A):
    rp, ci, va = A
    n = len(rp) - 1
    cols = [[] for _ in range(n)]
    for i in range(n):
        for q in range(rp[i], rp[i + 1]):
            cols[ci[q]].append(i)
    return cols


def replay_gap(A, d, k, J_gpu, uf, eps, beta, max_fill, alpha=None, colsA=None):
    """Smallest decision margin on the oracle's path consistent with J_gpu:
    (kind, margin, step), kind in {"selection", "threshold", "criterion"};
    None when the oracle's own pattern equals J_gpu."""
    rp, ci, va = A
    n = len(rp) - 1
    if alpha is None:
        alpha = (n + beta - 1) // beta
    if colsA is None:
        colsA = _col_lists(A)
    Jg = set(int(j) for j in J_gpu)
    J = [int(k)]
    best = None

    def note(kind, margin, step):
        nonlocal best
        if best is None or margin < best[1]:
            best = (kind, float(margin), step)

    for step in range(alpha + 1):
        I = set([int(k)])
        for j in J:
            for q in range(rp[j], rp[j + 1]):
                if va[q] != 0.0:
                    I.add(int(ci[q]))
        I = np.array(sorted(I), dtype=np.int64)
        pos = {int(v): t for t, v in enumerate(I)}
        Ab = np.zeros((len(I), len(J)))
        for c, j in enumerate(J):
            for q in range(rp[j], rp[j + 1]):
                if va[q] != 0.0:
                    Ab[pos[int(ci[q])], c] = va[q] * d[j]
        Ab = O.round_to(Ab, uf) if O.prec(uf) != O.DOUBLE else Ab
        e = (I == k).astype(float)
        _, s, sn, _ = O.dense_ls(Ab, e, uf)
        note("criterion", abs(sn - eps) / eps, step)
        if sn <= eps or step == alpha or len(J) >= max_fill:
            break
        cand = set()
        for t, l in enumerate(I):
            if s[t] != 0.0:
                cand.update(colsA[l])
        cand = np.array(sorted(cand - set(J)), dtype=np.int32)
        if len(cand) == 0:
            break
        rho = O.rho(A, d, I, s, cand, uf)
        mean = float(np.mean(rho))
        scale = mean if mean > 0 else 1.0
        nmax = min(beta, max_fill - len(J))
        sel = [int(x) for x in O.select(cand, rho, nmax, uf)]
        r = dict(zip((int(c) for c in cand), rho))
        taken = [r[j] for j in sel]
        left = sorted(r[int(c)] for c in cand if int(c) not in sel and r[int(c)] <= mean)
        if taken and left and len(sel) == nmax:
            note("selection", abs(left[0] - max(taken)) / scale, step)
        below = [v for v in rho if v <= mean]
        above = [v for v in rho if v > mean]
        if below:
            note("threshold", abs(mean - max(below)) / scale, step)
        if above:
            note("threshold", abs(min(above) - mean) / scale, step)
        if not sel or not set(sel) <= Jg:
            break  # the oracle stops here, or its path leaves J_g
        J = sorted(set(J) | set(sel))
    if set(J) == Jg:
        return None
    return best
