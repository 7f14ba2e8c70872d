"""Near-tie analysis of adaptive SPAI columns whose patterns differ between
the CUDA path and the oracle (reading R12 of the selection rule).

For a column k whose GPU pattern J_g differs from the oracle's, the oracle's
Grote-Huckle path is replayed step by step with the oracle's own exported
steps (the dense least squares, rho and the selection of Algorithm 1) until
the first step whose additions leave J_g.  There the two runs took a
different decision on nearly equal scores: the returned gap is the smallest
distance, relative to the mean rho of that step, between the rho of an index
the oracle added but the GPU did not and either the rho of an index the GPU
added instead or the acceptance threshold (the mean); where the oracle found
no candidate at or below the mean but the GPU went on, the distance of the
GPU's additions to the mean.  A path that never leaves J_g but stops earlier
(the column criterion ||s|| <= eps) returns the relative distance of ||s||
to eps.
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
    rp, ci, va = A
    n = len(rp) - 1
    if alpha is None:
        alpha = (n + beta - 1) // beta
    if colsA is None:
        colsA = _col_lists(A)
    Jg = set(int(j) for j in J_gpu)
    J = [int(k)]
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
        if sn <= eps:
            return ("converged", abs(sn - eps) / eps) if set(J) != Jg else None
        if step == alpha or len(J) >= max_fill:
            return None
        cand = set()
        for t, l in enumerate(I):
            if s[t] != 0.0:
                cand.update(colsA[l])
        cand = np.array(sorted(cand - set(J)), dtype=np.int32)
        if len(cand) == 0:
            return None
        rho = O.rho(A, d, I, s, cand, uf)
        sel = O.select(cand, rho, min(beta, max_fill - len(J)), uf)
        if len(sel) == 0:
            # no candidate at or below the mean: the oracle stops here; if the GPU went
            # on, it accepted an index whose rho ties with the mean
            if set(J) == Jg:
                return None
            mean = float(np.mean(rho))
            r = dict(zip((int(c) for c in cand), rho))
            ext = [r[j] for j in Jg if j in r]
            gap = min((abs(v - mean) for v in ext), default=np.inf)
            return ("threshold", gap / mean if mean > 0 else np.inf)
        if not set(int(x) for x in sel) <= Jg:
            mean = float(np.mean(rho))
            r = dict(zip((int(c) for c in cand), rho))
            X = [int(x) for x in sel if int(x) not in Jg]
            Y = [j for j in Jg if j in r and j not in J and j not in set(int(x) for x in sel)]
            gap = np.inf
            for x in X:
                gap = min(gap, abs(r[x] - mean))
                for y in Y:
                    gap = min(gap, abs(r[x] - r[y]))
            return ("selection", gap / mean if mean > 0 else np.inf)
        J = sorted(set(J) | set(int(x) for x in sel))
    return None
