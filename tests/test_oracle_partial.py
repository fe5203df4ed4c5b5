"""Pins of the partial-selection oracle (oracle/partial.py; Section 5.2, Appendix C.3).

  * brute force: a greedy that, at every step, evaluates the objective
    sum_i log Theta_{ii | s_i \\ i} (eq. partial_kl) for every candidate by dense conditional
    variances and keeps the least -- no factor, no insertion, no downdate;
  * the factor after the last insertion equals the dense Cholesky factor of the joint
    covariance of the targets and picks, latest position first (eq. chol_partial);
  * each pick's reported decrease equals the change of the dense objective;
  * with every candidate after a consecutive group, partial selection is the
    multiple-target selection (eq. greedy_mult).
"""
import math

import numpy as np
import pytest

import synthetic


def _ordered(oracle, n, seed):
    pts = synthetic.points(n, 2, seed)
    order, _ = oracle.maximin(pts)
    return pts[order]


def _brute(oracle, kp, pts, P, cand, k):
    from oracle import partial
    floor = oracle.exhaustion_floor(kp)
    S = []
    for _ in range(k):
        best, bj = None, None
        for j in cand:
            j = int(j)
            if j in S:
                continue
            cond = sorted(int(x) for x in P) + S
            K = oracle.theta_matrix(kp, pts, cond + [j])
            c = len(cond)
            if K[c, c] - K[:c, c] @ np.linalg.solve(K[:c, :c], K[:c, c]) < floor:
                continue
            v = partial.objective(kp, pts, P, S + [j])
            if best is None or v < best:
                best, bj = v, j
        if bj is None:
            break
        S.append(bj)
    return S


def _problem(oracle, seed, n=70, m=5, C=18):
    """Targets spread over the ordering; candidates the nearest later points of any target
    (so some fall between targets)."""
    pts = _ordered(oracle, n, seed)
    rng = np.random.default_rng(seed)
    P = sorted(rng.choice(np.arange(3, n // 2), size=m, replace=False).tolist())
    d = ((pts[:, None, :] - pts[None, P, :]) ** 2).sum(-1).min(1)
    pool = [j for j in np.argsort(d, kind="stable") if j > P[0] and j not in P]
    return pts, P, [int(j) for j in pool[:C]]


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_partial_matches_brute_force(oracle_lib, seed):
    oracle = oracle_lib
    from oracle import partial
    pts, P, cand = _problem(oracle, seed)
    kp = oracle.kernel(2, 3, 0.3, 1.0, 1e-6)
    r = partial.select_partial(kp, pts, P, cand, 6)
    assert list(r["sel"]) == _brute(oracle, kp, pts, P, cand, 6)
    assert any(P[0] < j < P[-1] for j in cand)  # candidates between targets: the case the method exists for


@pytest.mark.parametrize("seed", [5, 6])
def test_partial_factor_and_decreases(oracle_lib, seed):
    oracle = oracle_lib
    from oracle import partial
    pts, P, cand = _problem(oracle, seed, n=90, m=6, C=25)
    kp = oracle.kernel(2, 5, 0.25, 1.3, 1e-5)
    r = partial.select_partial(kp, pts, P, cand, 10)
    order = r["order"]
    assert order == sorted(order, reverse=True)
    G = np.linalg.cholesky(oracle.theta_matrix(kp, pts, order))
    rows = cand + sorted(P)
    ri = [rows.index(x) for x in order]
    assert np.abs(r["L"][ri, :] - G).max() <= 1e-12
    S, base = [], partial.objective(kp, pts, P, [])
    for q, dec in zip(r["sel"], r["decrease"]):
        S.append(int(q))
        new = partial.objective(kp, pts, P, S)
        assert dec == pytest.approx(base - new, rel=1e-10, abs=1e-12)
        base = new


def test_partial_is_multi_target_for_a_consecutive_group(oracle_lib):
    oracle = oracle_lib
    from oracle import partial
    pts = _ordered(oracle, 300, 8)
    kp = oracle.kernel(2, 3, 0.2, 1.0, 1e-6)
    gp = np.array([0, 6, 13], np.int64)
    gptr, gidx = oracle.group_candidates(pts, gp, 40)
    for g in range(2):
        g0, m = int(gp[g]), int(gp[g + 1] - gp[g])
        cand = gidx[gptr[g]:gptr[g + 1]]
        a = partial.select_partial(kp, pts, range(g0, g0 + m), cand, 12)
        b = oracle.select_multi(kp, pts, g0, m, cand, 12)
        assert list(a["sel"]) == list(b["sel"])
        np.testing.assert_allclose(a["decrease"], np.log(b["chosen"]), rtol=1e-9)
