"""FP64 oracle of partial selection for nonadjacent groups (Section 5.1.1, Section 5.2
"Partial selection", Appendix C.3) -- TEST INFRASTRUCTURE ONLY.

A group's targets P = {i_1 < ... < i_m} need not be consecutive in the elimination order, and
a candidate j conditions only the targets before it (i < j).  Target i's column holds
s_i = {i} + {targets after i} + {picks after i}, and the objective is
    sum_{i in P} log Theta_{ii | s_i \\ i}                    (eq. partial_kl)
-- the log-determinant of the partially conditioned target covariance -- minimised greedily.

The algorithm (Appendix C.3) keeps the Cholesky factor L of the joint covariance restricted
to the selected points and the targets, its columns sorted from the latest position to the
earliest (so that a column's pivot is conditioned on exactly the later points), with a row
for every candidate and target:
  * score of candidate j: walk the columns in order carrying v = Theta_{jj | columns so far};
    at column c of element e with pivot d = L_ec^2 and covariance L_jc L_ec, a target e that
    j conditions (e < j) would get the variance d - (L_jc L_ec)^2 / v (eq. obj_partial); then
    v -= L_jc^2 (eq. partial_induct).  The score is the sum over those targets of
    log d - log(new variance): the decrease of the objective.
  * inserting the pick k at its place p (the number of selected points and targets after
    it): columns before p are unchanged; the new column is u = Theta_{:,k | first p} /
    sqrt(Theta_{kk | first p}) by left-looking over the first p columns; the columns from p
    on become the factor of the joint covariance conditioned on k, i.e. a rank-one downdate
    by u, done in place column by column (eq. chol_partial_update).

Readings (the same on the GPU): ties go to the earliest candidate in the list; a candidate is
exhausted when its variance conditioned on every selected point and target (v after the
last column) is below the floor, as in the multiple-target selection (with every candidate
after the group the two selections coincide); candidates must lie after the first target.

Pinned in tests/test_oracle_partial.py by a brute-force greedy on the objective
(dense conditional variances), by the multiple-target selection when every candidate follows
the group, and by the dense Cholesky of the final joint covariance.
"""
from __future__ import annotations

import math

import numpy as np

from . import exhaustion_floor, theta_matrix


def select_partial(kp, pts, P, cand, k: int, floor=None, forced=None):
    """Greedy partial selection for the targets P (positions, any order) from the candidate
    positions `cand`.  forced[t] >= 0 replays a pick given as an index into cand.  Returns
    dict(sel, decrease, best, chosen, L, order): the picks, each pick's decrease of the
    objective (= chosen), the largest decrease at each step (best), and the final factor
    (rows: candidates then targets; columns in the order `order`, latest position first)."""
    P = sorted(int(x) for x in P)
    cand = [int(x) for x in cand]
    floor = exhaustion_floor(kp) if floor is None else floor
    C, m = len(cand), len(P)
    rows = cand + P                       # row r <-> point rows[r]
    is_target = [False] * C + [True] * m
    T = theta_matrix(kp, pts, rows)       # Theta over every row
    order: list[int] = []                 # rows of the selected points and targets, latest first
    L = np.zeros((C + m, 0))
    taken = [False] * C

    def insert(r):
        """Insert row r's point into the factor (left-looking column + in-place downdate)."""
        nonlocal L
        pos = rows[r]
        p = sum(1 for e in order if rows[e] > pos)     # its place: the points after it come first
        d = T[r, r] - L[r, :p] @ L[r, :p]             # Theta_{rr | first p}
        u = (T[:, r] - L[:, :p] @ L[r, :p]) / math.sqrt(d)
        u[order[:p]] = 0.0                              # rows of the points before it in the order
        new = L.copy()
        x = u.copy()
        x[r] = 0.0
        # columns from p on: the factor of the covariance conditioned on r as well, i.e. a
        # rank-one downdate by u, column by column; the rows still below a column's pivot
        # (later pivots and the candidates) are updated, the pivot row takes the new diagonal
        for c in range(p, len(order)):
            e = order[c]
            lee = new[e, c]
            rr = math.sqrt(lee * lee - x[e] * x[e])
            cth, sth = rr / lee, x[e] / lee
            above = set(order[:c + 1])
            below = [y for y in range(C + m) if y not in above and y != r]
            col = (new[below, c] - sth * x[below]) / cth
            x[below] = cth * x[below] - sth * col
            new[below, c] = col
            new[e, c] = rr
        new[r, p:] = 0.0
        L = np.concatenate([new[:, :p], u.reshape(-1, 1), new[:, p:]], axis=1)
        order.insert(p, r)

    for r in range(C, C + m):             # the targets first
        insert(r)
    sel, dec, bests = [], [], []
    for t in range(k):
        best, best_r = None, -1
        scores = {}
        for j in range(C):
            if taken[j]:
                continue
            v = T[j, j]
            score = 0.0
            for c, e in enumerate(order):
                d = L[e, c] ** 2
                cov = L[j, c] * L[e, c]
                if is_target[e] and rows[e] < rows[j]:
                    score += math.log(d) - math.log(d - cov * cov / v)
                v -= L[j, c] ** 2
            if v < floor:
                continue
            scores[j] = score
            if best is None or score > best:
                best, best_r = score, j
        if best_r < 0:
            break
        q = best_r
        if forced is not None and t < len(forced) and forced[t] >= 0:
            q = int(forced[t])
        taken[q] = True
        insert(q)
        sel.append(rows[q])
        dec.append(scores.get(q, -math.inf))
        bests.append(best)
    return dict(sel=np.array(sel, np.int32), decrease=np.array(dec), best=np.array(bests), chosen=np.array(dec),
                L=L, order=[rows[e] for e in order])


def objective(kp, pts, P, S) -> float:
    """sum_{i in P} log Theta_{ii | s_i \\ i}, s_i = targets after i and picks after i, by
    dense conditional variances (eq. partial_kl)."""
    P = sorted(int(x) for x in P)
    S = [int(x) for x in S]
    tot = 0.0
    for i in P:
        cond = [x for x in P + S if x > i]
        K = theta_matrix(kp, pts, cond + [i])
        c = len(cond)
        v = K[c, c] - (K[:c, c] @ np.linalg.solve(K[:c, :c], K[:c, c]) if c else 0.0)
        tot += math.log(v)
    return tot
