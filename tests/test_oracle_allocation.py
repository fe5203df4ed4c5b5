"""Pins of the global greedy allocation oracle (Section 5.4, oracle/allocation.py).

The queue is pinned against (1) a brute-force global greedy that, after every pick,
re-scores every candidate of every unit by dense log-determinants (no trajectories, no
queue), (2) an independent formulation of the queue's pop order (running minimum of each
unit's decreases, sorted), (3) hand-worked budgets, and (4) a closed form for the first
picks of an Ornstein-Uhlenbeck process on a line.
"""
import math

import numpy as np
import pytest

import synthetic


def _ordered(oracle, n, dim, seed, clustered=False):
    pts = synthetic.clustered_points(n, dim, seed) if clustered else synthetic.points(n, dim, seed)
    order, _ = oracle.maximin(pts)
    return pts[order]


def _cond_var(oracle, kp, pts, j, cond):
    K = oracle.theta_matrix(kp, pts, list(cond) + [j])
    if not cond:
        return K[-1, -1]
    return K[-1, -1] - K[:-1, -1] @ np.linalg.solve(K[:-1, :-1], K[:-1, -1])


def _brute_force(oracle, kp, pts, units, cand_lists, k, budget, single):
    """Global greedy by exhaustive re-scoring: every step evaluates, for every unit below k
    picks and every candidate not yet picked and not exhausted, the exact decrease of
    logdet Theta_{P,P|S} per nonzero, and takes the largest one if its nonzeros still fit."""
    floor = oracle.exhaustion_floor(kp)
    S = [[] for _ in units]
    done = [False] * len(units)
    left = budget
    while True:
        best = None
        for u, P in enumerate(units):
            if done[u] or len(S[u]) >= k:
                continue
            base = oracle.logdet_cond(kp, pts, P, S[u])
            ub = None
            for j in cand_lists[u]:
                j = int(j)
                if j in S[u]:
                    continue
                if _cond_var(oracle, kp, pts, j, S[u] if single else list(P) + S[u]) < floor:
                    continue
                gain = (base - oracle.logdet_cond(kp, pts, P, S[u] + [j])) / len(P)
                if ub is None or gain > ub[0]:
                    ub = (gain, j)
            if ub is None or (single and not ub[0] > 0):
                done[u] = True  # the unit's greedy has ended
                continue
            if best is None or ub[0] > best[0]:
                best = (ub[0], u, ub[1])
        if best is None:
            break
        _, u, j = best
        if len(units[u]) > left:
            break
        S[u].append(j)
        left -= len(units[u])
    return S


def _pop_order_counts(gains, costs, budget):
    """The queue's result from the order (running minimum of a unit's decreases descending,
    unit ascending, pick ascending), accepted while the nonzeros fit."""
    items = []
    for u, g in enumerate(gains):
        run = math.inf
        for t, x in enumerate(g):
            run = min(run, float(x))
            items.append((-run, u, t))
    items.sort()
    counts = np.zeros(len(gains), np.int32)
    left = budget
    for _, u, _t in items:
        if costs[u] > left:
            break
        left -= costs[u]
        counts[u] += 1
    return counts


@pytest.mark.parametrize("budget", [0, 7, 25, 40, 10_000])
def test_columns_global_matches_brute_force(oracle_lib, budget):
    oracle = oracle_lib
    from oracle import allocation
    pts = _ordered(oracle, 28, 2, 11)
    kp = oracle.kernel(2, 3, 0.3, 1.0, 1e-6)
    ptr, idx = oracle.column_candidates(pts, 6)
    cl = [idx[ptr[i]:ptr[i + 1]] for i in range(len(pts))]
    sel, counts = allocation.select_columns_global(kp, pts, None, cl, 3, budget)
    ref = _brute_force(oracle, kp, pts, [[i] for i in range(len(pts))], cl, 3, budget, True)
    assert [list(s) for s in sel] == ref
    assert counts.sum() == sum(len(r) for r in ref) <= budget


@pytest.mark.parametrize("budget", [0, 9, 30, 61, 10_000])
def test_groups_global_matches_brute_force(oracle_lib, budget):
    """Supernodes of 1 to 4 members: nonzeros and the per-nonzero key both count members."""
    oracle = oracle_lib
    from oracle import allocation
    pts = _ordered(oracle, 30, 2, 12)
    kp = oracle.kernel(2, 3, 0.3, 1.0, 1e-6)
    sizes = [1, 3, 2, 4, 1, 2, 3, 1, 2, 4, 3, 2, 1, 1]
    assert sum(sizes) == len(pts)
    grp_ptr = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    gptr, gidx = oracle.group_candidates(pts, grp_ptr, 6)
    cl = [gidx[gptr[g]:gptr[g + 1]] for g in range(len(sizes))]
    sel, counts = allocation.select_groups_global(kp, pts, grp_ptr, cl, 3, budget)
    units = [list(range(int(grp_ptr[g]), int(grp_ptr[g + 1]))) for g in range(len(sizes))]
    ref = _brute_force(oracle, kp, pts, units, cl, 3, budget, False)
    assert [list(s) for s in sel] == ref
    assert int((counts * np.array(sizes)).sum()) <= budget


def test_queue_matches_running_minimum_order():
    """Random decrease sequences with many exact ties (small integers), costs 1..4."""
    from oracle import allocation
    rng = np.random.default_rng(5)
    for _ in range(3000):
        n = int(rng.integers(1, 7))
        gains = [rng.integers(-1, 5, size=int(rng.integers(0, 6))).astype(float) for _ in range(n)]
        costs = [int(c) for c in rng.integers(1, 5, size=n)]
        total = sum(c * len(g) for c, g in zip(costs, gains))
        budget = int(rng.integers(0, total + 2))
        got = allocation.queue_allocate(gains, costs, budget)
        assert np.array_equal(got, _pop_order_counts(gains, costs, budget))


def test_queue_hand_worked():
    from oracle import allocation
    qa = allocation.queue_allocate
    # everything fits; nothing fits
    assert list(qa([[3.0, 1.0], [2.0]], [1, 1], 10)) == [2, 1]
    assert list(qa([[3.0, 1.0], [2.0]], [1, 1], 0)) == [0, 0]
    # order 3 (u0), 2 (u1), 1 (u0)
    assert list(qa([[3.0, 1.0], [2.0]], [1, 1], 2)) == [1, 1]
    # a later, larger decrease of a unit waits for its smaller predecessor
    assert list(qa([[1.0, 9.0], [2.0]], [1, 1], 1)) == [0, 1]
    assert list(qa([[1.0, 9.0], [2.0]], [1, 1], 3)) == [2, 1]
    # equal keys: lower unit first
    assert list(qa([[2.0], [2.0], [2.0]], [1, 1, 1], 2)) == [1, 1, 0]
    # the queue stops at the first pick that does not fit, even if a cheaper one would
    assert list(qa([[5.0], [4.0]], [8, 1], 7)) == [0, 0]
    assert list(qa([[5.0], [4.0]], [8, 1], 9)) == [1, 1]
    # empty units never enter
    assert list(qa([[], [1.0]], [1, 1], 5)) == [0, 1]


def test_first_picks_of_ou_line_closed_form(oracle_lib):
    """Exponential kernel (nu = 1/2, the Ornstein-Uhlenbeck process) on a line, one pick per
    column: the decrease of picking the nearest later point at distance d is
    -log(1 - exp(-2 d / ell)), so a budget of B picks goes to the B columns whose nearest
    later point is closest."""
    oracle = oracle_lib
    from oracle import allocation
    pts = _ordered(oracle, 40, 1, 3)
    ell = 0.2
    kp = oracle.kernel(1, 1, ell, 1.0, 0.0)
    ptr, idx = oracle.column_candidates(pts, 4)
    cl = [idx[ptr[i]:ptr[i + 1]] for i in range(len(pts))]
    sels, gains = allocation.column_gains(kp, pts, None, cl, 1)
    for i in range(len(pts) - 1):
        d = np.abs(pts[i + 1:, 0] - pts[i, 0]).min()
        assert gains[i][0] == pytest.approx(-math.log1p(-math.exp(-2 * d / ell)), rel=1e-9)
    dmin = [np.abs(pts[i + 1:, 0] - pts[i, 0]).min() for i in range(len(pts) - 1)]
    B = 15
    _, counts = allocation.select_columns_global(kp, pts, None, cl, 1, B)
    assert sorted(np.nonzero(counts)[0].tolist()) == sorted(np.argsort(dmin, kind="stable")[:B].tolist())


@pytest.mark.parametrize("clustered", [False, True])
def test_global_allocation_lowers_kl_at_equal_nonzeros(oracle_lib, clustered):
    """The point of Section 5.4: at the nonzero count of k entries per column, letting the
    columns compete lowers sum log v (= 2 KL + logdet Theta) below the even allocation,
    the more so in an inhomogeneous cloud."""
    oracle = oracle_lib
    from oracle import allocation
    pts = _ordered(oracle, 1500, 2, 3, clustered)
    kp = oracle.kernel(2, 3, 0.1, 1.0, 1e-8)
    ptr, idx = oracle.column_candidates(pts, 32)
    cl = [idx[ptr[i]:ptr[i + 1]] for i in range(len(pts))]
    sels, gains = allocation.column_gains(kp, pts, None, cl, 16)
    even = [min(6, len(g)) for g in gains]
    _, counts = allocation.select_columns_global(kp, pts, None, cl, 16, sum(even))
    s_even = -sum(g[:c].sum() for g, c in zip(gains, even))
    s_glob = -sum(g[:c].sum() for g, c in zip(gains, counts))
    # the selection's own decreases agree with the fill's log v_i
    col_ptr, row_idx, val, logv = oracle.factor_columns(kp, pts, [s[:c] for s, c in zip(sels, counts)], threads=4)
    assert logv.sum() == pytest.approx(len(pts) * math.log(1 + 1e-8) + s_glob, abs=1e-6 * len(pts))
    assert s_glob < s_even - 10.0
