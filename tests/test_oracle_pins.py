"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test pins an oracle routine to something other than itself: closed forms from
textbooks, identities derived in the paper's appendices, brute force on tiny inputs,
special cases with a known exact answer, and a hand-worked example.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.special

import synthetic

HERE = os.path.dirname(os.path.abspath(__file__))


def _ordered(oracle, n, dim, seed):
    pts = synthetic.points(n, dim, seed)
    order, ell2 = oracle.maximin(pts)
    return pts[order], ell2


# ----------------------------------------------------------------- kernel --

@pytest.mark.parametrize("nu_x2", [1, 3, 5])
def test_matern_matches_bessel_form(oracle_lib, nu_x2):
    """Half-integer closed forms vs the general Matern definition with the modified
    Bessel function K_nu (Rasmussen & Williams eq. 4.14), cited by the paper for its kernels."""
    oracle = oracle_lib
    nu = nu_x2 / 2.0
    ell, s2 = 0.37, 1.7
    kp = oracle.kernel(2, nu_x2, ell, s2, 0.0)
    for r in [1e-3, 0.05, 0.2, 0.9, 2.5]:
        z = math.sqrt(2 * nu) * r / ell
        ref = s2 * 2 ** (1 - nu) / math.gamma(nu) * z ** nu * scipy.special.kv(nu, z)
        assert abs(oracle.matern(kp, r) - ref) <= 1e-12 * max(1.0, abs(ref))
    assert oracle.matern(kp, 0.0) == pytest.approx(s2, rel=0, abs=0)


def test_theta_nugget_on_diagonal_only(oracle_lib):
    oracle = oracle_lib
    kp = oracle.kernel(2, 3, 0.2, 1.0, 1e-3)
    pts = np.array([[0.1, 0.1], [0.1, 0.1], [0.5, 0.2]])
    T = oracle.theta_matrix(kp, pts, [0, 1, 2])
    assert T[0, 0] == 1.0 + 1e-3 and T[0, 1] == 1.0
    assert np.allclose(T, T.T)


# ------------------------------------------------------------------- prep --

@pytest.mark.parametrize("dim", [1, 2, 3])
def test_maximin_property(oracle_lib, dim):
    """eq. maximin: ell_k is the distance to the later set, and no earlier point is farther
    from the later set than the point placed at k."""
    oracle = oracle_lib
    pts = synthetic.points(300, dim, 5)
    order, ell2 = oracle.maximin(pts)
    assert sorted(order.tolist()) == list(range(300)) and order[-1] == 0
    P = pts[order]
    D = ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)
    for k in range(299):
        later = D[:k + 1, k + 1:].min(axis=1)   # distance of each of positions 0..k to the set after k
        assert later[k] == ell2[k]
        assert np.all(later[:k] <= ell2[k])
    assert np.all(np.diff(ell2[:-1]) >= 0)     # length scales grow along the ordering


def test_knn_later_property(oracle_lib):
    oracle = oracle_lib
    P, _ = _ordered(oracle, 500, 2, 3)
    for tgt, first, C in [([10], 11, 40), ([100, 101, 102], 103, 64), ([480], 481, 64), ([499], 500, 8)]:
        got = oracle.knn_later(P, tgt, first, C)
        cand = np.arange(first, 500)
        key = np.min(((P[cand][:, None, :] - P[tgt][None, :, :]) ** 2).sum(-1), axis=1)
        ref = cand[np.lexsort((cand, key))][:C]
        assert got.tolist() == ref.tolist()


def test_groups_partition_and_rule(oracle_lib):
    """Groups partition the positions, respect the size cap, and every member of a group's
    first pass lies in the opening point's neighbour list with ell_j <= 1.5 ell_i."""
    oracle = oracle_lib
    P, ell2 = _ordered(oracle, 2048, 2, 1)
    members, gp = oracle.group(P, ell2, 64, 1.5, 8, 64)
    assert sorted(members.tolist()) == list(range(2048))
    sz = np.diff(gp)
    assert sz.max() <= 64 and sz.min() >= 1
    for g in range(len(sz)):
        grp = members[gp[g]:gp[g + 1]]
        assert np.all(np.diff(grp) > 0)
    # first group: opened by position 0; its first pass takes, in distance order, the
    # neighbours with ell_j <= 1.5 ell_0 (a later small group may have been merged in)
    nb = oracle.knn_later(P, [0], 1, 64).tolist()
    first_pass = [0] + [j for j in nb if ell2[j] <= 2.25 * ell2[0]][:63]
    g0 = members[gp[0]:gp[1]]
    assert set(first_pass) <= set(g0.tolist())


# -------------------------------------------------------------- selection --

@pytest.mark.parametrize("seed,nu_x2,C,k", [(0, 1, 24, 6), (1, 3, 32, 8), (2, 5, 20, 8), (3, 3, 12, 12)])
def test_T1_naive_equals_cholesky_form(oracle_lib, seed, nu_x2, C, k):
    """eq. obj_gp <=> eq. cond_cov: the O(C k^2) Cholesky form picks what re-factorising
    picks, and its running target variance equals the re-factorised one."""
    oracle = oracle_lib
    kp = oracle.kernel(2, nu_x2, 0.3, 1.0, 1e-6)
    P, _ = _ordered(oracle, 200, 2, seed)
    tgt = 7
    cand = oracle.knn_later(P, [tgt], tgt + 1, C)
    r = oracle.select_single(kp, P, tgt, cand, k)
    S, v = oracle.select_single_naive(kp, P, tgt, cand, k)
    assert r["sel"].tolist() == S.tolist()
    assert np.allclose(r["vtar"][1:], v, rtol=1e-8, atol=0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_T2_brute_force_subsets(oracle_lib, seed):
    """Greedy is never better than the exhaustive optimum, and is optimal for k = 1 and k = C."""
    oracle = oracle_lib
    kp = oracle.kernel(2, 3, 0.4, 1.0, 1e-6)
    P, _ = _ordered(oracle, 100, 2, seed)
    tgt = 3
    cand = oracle.knn_later(P, [tgt], tgt + 1, 10)
    for k in [1, 2, 3, 10]:
        r = oracle.select_single(kp, P, tgt, cand, k)
        _, vstar = oracle.brute_force_subset(kp, P, tgt, cand, k)
        vg = r["vtar"][-1]
        assert vstar <= vg * (1 + 1e-10)
        if k in (1, 10):
            assert vg == pytest.approx(vstar, rel=1e-8)


def test_T3_target_variance_is_inverse_entry(oracle_lib):
    """eq. inverse_cond: after the picks S, Theta_{tt|S} = 1 / (Theta_{s,s}^{-1})_{11}, s = (t, S)."""
    oracle = oracle_lib
    kp = oracle.kernel(2, 3, 0.1, 1.0, 1e-8)
    P, _ = _ordered(oracle, 1024, 2, 0)
    for tgt in [0, 17, 500, 1000]:
        cand = oracle.knn_later(P, [tgt], tgt + 1, 64)
        r = oracle.select_single(kp, P, tgt, cand, 16)
        T = oracle.theta_matrix(kp, P, [tgt] + r["sel"].tolist())
        inv11 = np.linalg.inv(T)[0, 0]
        kappa = np.linalg.cond(T)
        assert abs(r["vtar"][-1] * inv11 - 1.0) <= 1e-15 * kappa * 10 + 1e-12


def test_T4_fill_normalisation_and_T13_solve(oracle_lib):
    """KL-optimal columns satisfy L_{s,i}^T Theta_{s,s} L_{s,i} = 1 (Appendix A.1), and equal
    a library solve of Theta_{s,s} x = e_1 scaled by 1/sqrt(x_1) (eq. L_col)."""
    oracle = oracle_lib
    kp = oracle.kernel(3, 5, 0.2, 1.0, 1e-6)
    P, _ = _ordered(oracle, 600, 3, 4)
    for i in [0, 50, 400]:
        cand = oracle.knn_later(P, [i], i + 1, 48)
        r = oracle.select_single(kp, P, i, cand, 12)
        rows, L, lv = oracle.fill_column(kp, P, i, r["sel"])
        T = oracle.theta_matrix(kp, P, rows)
        assert L @ T @ L == pytest.approx(1.0, rel=1e-9)
        x = np.linalg.solve(T, np.eye(len(rows))[0])
        assert np.allclose(L, x / np.sqrt(x[0]), rtol=1e-8, atol=1e-8 * np.abs(L).max())
        assert lv == pytest.approx(-np.log(x[0]), rel=1e-10)
        assert rows[0] == i and np.all(np.diff(rows[1:]) > 0)


def test_T5_nested_and_monotone(oracle_lib):
    """Greedy picks for k are a prefix of those for k+1; sum of log v is non-increasing in k;
    KL >= 0 against the dense log-determinant."""
    oracle = oracle_lib
    kp = oracle.kernel(2, 3, 0.15, 1.0, 1e-6)
    P, _ = _ordered(oracle, 256, 2, 9)
    ptr, idx = oracle.column_candidates(P, 32)
    logdet = oracle.logdet_theta(kp, P)
    prev_sel, prev_sum = None, None
    for k in [0, 1, 2, 4, 8, 16]:
        sels = [oracle.select_single(kp, P, i, idx[ptr[i]:ptr[i + 1]], k)["sel"] for i in range(256)]
        if prev_sel is not None:
            for a, b in zip(prev_sel, sels):
                assert b[:len(a)].tolist() == a.tolist()
        _, _, _, logv = oracle.factor_columns(kp, P, sels)
        s = logv.sum()
        if prev_sum is not None:
            assert s <= prev_sum + 1e-9 * abs(prev_sum)
        assert oracle.kl_from_logv(s, logdet) >= -1e-8
        prev_sel, prev_sum = sels, s


def test_T6_complete_pattern_is_exact(oracle_lib):
    """With every later point as candidate and k = all of them, the factor is the exact inverse
    Cholesky factor U^{-T} (U the reverse Cholesky factor, Appendix A.4) and KL = 0."""
    oracle = oracle_lib
    n = 24
    kp = oracle.kernel(2, 3, 0.5, 1.0, 1e-4)
    P, _ = _ordered(oracle, n, 2, 2)
    sels = []
    for i in range(n):
        cand = np.arange(i + 1, n, dtype=np.int32)
        sels.append(oracle.select_single(kp, P, i, cand, n)["sel"])
        assert len(sels[-1]) == n - 1 - i
    cp, ri, val, logv = oracle.factor_columns(kp, P, sels)
    L = np.zeros((n, n))
    for c in range(n):
        L[ri[cp[c]:cp[c + 1]], c] = val[cp[c]:cp[c + 1]]
    T = oracle.theta_matrix(kp, P, np.arange(n))
    U = np.linalg.cholesky(T[::-1, ::-1])[::-1, ::-1]
    ref = np.linalg.inv(U).T
    assert np.allclose(L, ref, rtol=1e-8, atol=1e-8 * np.abs(ref).max())
    assert abs(oracle.kl_from_logv(logv.sum(), oracle.logdet_theta(kp, P))) < 1e-8


def test_T7_k0_diagonal(oracle_lib):
    """k = 0: L_ii = 1/sqrt(Theta_ii) and 2 KL = sum log Theta_ii - logdet Theta."""
    oracle = oracle_lib
    n = 64
    kp = oracle.kernel(2, 1, 0.2, 2.0, 1e-3)
    P, _ = _ordered(oracle, n, 2, 6)
    cp, ri, val, logv = oracle.factor_columns(kp, P, [np.zeros(0, np.int32)] * n)
    assert np.allclose(val, 1 / np.sqrt(2.0 + 1e-3), rtol=1e-14)
    ld = oracle.logdet_theta(kp, P)
    assert 2 * oracle.kl_from_logv(logv.sum(), ld) == pytest.approx(n * np.log(2.001) - ld, rel=1e-12)


def test_kl_closed_form_orientation(oracle_lib):
    """eq. kl with Theta_1 = Theta, Theta_2 = (L L^T)^{-1} equals the eq. obj_chol sum."""
    oracle = oracle_lib
    n = 80
    kp = oracle.kernel(2, 3, 0.2, 1.0, 1e-5)
    P, _ = _ordered(oracle, n, 2, 8)
    ptr, idx = oracle.column_candidates(P, 16)
    sels = [oracle.select_single(kp, P, i, idx[ptr[i]:ptr[i + 1]], 4)["sel"] for i in range(n)]
    cp, ri, val, logv = oracle.factor_columns(kp, P, sels)
    L = np.zeros((n, n))
    for c in range(n):
        L[ri[cp[c]:cp[c + 1]], c] = val[cp[c]:cp[c + 1]]
    T = oracle.theta_matrix(kp, P, np.arange(n))
    Q = L @ L.T
    two_kl = np.trace(Q @ T) - np.linalg.slogdet(Q)[1] - np.linalg.slogdet(T)[1] - n
    assert 2 * oracle.kl_from_logv(logv.sum(), oracle.logdet_theta(kp, P)) == pytest.approx(two_kl, rel=1e-7, abs=1e-9)


def test_T8_markov_1d_golden(oracle_lib):
    """Hand-worked 1-D exponential-kernel example: k = 2 picks the nearest later point on
    each side, and the resulting v_i is the full conditional variance Theta_{ii | i+1:}."""
    oracle = oracle_lib
    g = json.load(open(os.path.join(HERE, "golden", "ou_markov_1d.json")))
    x = np.array(g["x"])[:, None]
    n = len(x)
    kp = oracle.kernel(1, g["nu_x2"], g["length_scale"], g["variance"], g["nugget"])
    T = oracle.theta_matrix(kp, x, np.arange(n))
    for i in range(n - 1):
        cand = np.arange(i + 1, n, dtype=np.int32)
        r = oracle.select_single(kp, x, i, cand, 2)
        assert r["sel"].tolist() == g["expected_picks"][str(i)]
        rest = np.arange(i + 1, n)
        full = T[i, i] - T[i, rest] @ np.linalg.solve(T[np.ix_(rest, rest)], T[rest, i])
        assert r["vtar"][-1] == pytest.approx(full, rel=1e-9)


def test_T9_planted_factor_recovery(oracle_lib):
    """Section 6.5: recover a planted sparse factor L from Theta = (L L^T)^{-1}.  Columns whose
    selected set covers the planted pattern reproduce L exactly (KL-optimality)."""
    oracle = oracle_lib
    n, s = 256, 32
    Lp = synthetic.planted_factor(n, s, seed=0)
    Q = Lp @ Lp.T
    Theta = np.linalg.inv(Q)
    Theta = 0.5 * (Theta + Theta.T)
    kp, dummy = oracle.dense_kernel(Theta)
    inter = union = 0
    exact_cols = 0
    for i in range(n):
        true = set(np.nonzero(Lp[i + 1:, i])[0] + i + 1)
        cand = np.arange(i + 1, n, dtype=np.int32)
        r = oracle.select_single(kp, dummy, i, cand, len(true))
        got = set(r["sel"].tolist())
        inter += len(got & true)
        union += len(got | true)
        if got >= true:
            rows, L, _ = oracle.fill_column(kp, dummy, i, r["sel"])
            ref = Lp[rows, i]
            assert np.allclose(L, ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())
            exact_cols += 1
    iou = inter / union
    print(f"planted recovery IOU = {iou:.4f}, exact columns = {exact_cols}/{n}")
    assert iou > 0.9 and exact_cols > n // 2


def test_T10_multi_with_one_target_is_single(oracle_lib):
    oracle = oracle_lib
    kp = oracle.kernel(2, 3, 0.1, 1.0, 1e-8)
    P, _ = _ordered(oracle, 2048, 2, 0)
    for i in [0, 100, 1500]:
        cand = oracle.knn_later(P, [i], i + 1, 128)
        a = oracle.select_single(kp, P, i, cand, 16)["sel"]
        b = oracle.select_multi(kp, P, i, 1, cand, 16)["sel"]
        assert a.tolist() == b.tolist()


@pytest.mark.parametrize("m", [2, 5])
def test_T11_multi_score_is_logdet_change(oracle_lib, m):
    """eq. greedy_mult (matrix determinant lemma): the two-factor ratio var1/var2 of the pick
    equals exp(-(logdet Theta_{PP|S+q} - logdet Theta_{PP|S})) from dense factorisations,
    and the two-factor greedy picks what the naive re-factorising greedy picks."""
    oracle = oracle_lib
    kp = oracle.kernel(2, 3, 0.3, 1.0, 1e-6)
    P, _ = _ordered(oracle, 300, 2, 1)
    g0 = 20
    cand = oracle.knn_later(P, np.arange(g0, g0 + m), g0 + m, 24)
    r = oracle.select_multi(kp, P, g0, m, cand, 6)
    S, _ = oracle.select_multi_naive(kp, P, g0, m, cand, 6)
    assert r["sel"].tolist() == S.tolist()
    tg = list(range(g0, g0 + m))
    for t in range(len(r["sel"])):
        before = oracle.logdet_cond(kp, P, tg, r["sel"][:t])
        after = oracle.logdet_cond(kp, P, tg, r["sel"][:t + 1])
        assert np.log(r["chosen"][t]) == pytest.approx(before - after, rel=1e-7, abs=1e-10)


def test_T12_aggregated_kl_and_reverse_cholesky(oracle_lib):
    """eq. obj_mult: sum over members of log v_i = logdet Theta_{PP | S~}; the reverse-Cholesky
    fill (Appendix A.4) equals the per-member dense fill."""
    oracle = oracle_lib
    kp = oracle.kernel(2, 3, 0.1, 1.0, 1e-6)
    P, ell2 = _ordered(oracle, 1024, 2, 2)
    members, gp = oracle.group(P, ell2, 32, 1.5, 4, 16)
    P = P[members]
    for g in [0, 3, len(gp) // 2]:
        g0, g1 = int(gp[g]), int(gp[g + 1])
        m = g1 - g0
        cand = oracle.knn_later(P, np.arange(g0, g1), g1, 64)
        sel = oracle.select_multi(kp, P, g0, m, cand, 12)["sel"]
        rows_r, Lr, logv_r = oracle.fill_group_reverse_chol(kp, P, g0, m, sel)
        lsum = 0.0
        for a in range(m):
            rows, L, lv = oracle.fill_member(kp, P, g0, m, a, sel)
            assert rows.tolist() == rows_r[a:].tolist()
            ref = Lr[a:, a]
            assert np.allclose(L, ref, rtol=1e-8, atol=1e-8 * np.abs(ref).max())
            assert lv == pytest.approx(logv_r[a], rel=1e-9, abs=1e-12)
            lsum += lv
        assert lsum == pytest.approx(oracle.logdet_cond(kp, P, range(g0, g1), sel), rel=1e-9, abs=1e-9)


@pytest.mark.parametrize("op", [0, 1, 2])
def test_apply_factor_dense(oracle_lib, op):
    oracle = oracle_lib
    n = 120
    kp = oracle.kernel(2, 3, 0.2, 1.0, 1e-5)
    P, _ = _ordered(oracle, n, 2, 3)
    ptr, idx = oracle.column_candidates(P, 12)
    sels = [oracle.select_single(kp, P, i, idx[ptr[i]:ptr[i + 1]], 5)["sel"] for i in range(n)]
    cp, ri, val, _ = oracle.factor_columns(kp, P, sels)
    L = np.zeros((n, n))
    for c in range(n):
        L[ri[cp[c]:cp[c + 1]], c] = val[cp[c]:cp[c + 1]]
    x = synthetic.normal(1, n * 3).reshape(n, 3)
    ref = [L @ x, L.T @ x, L @ (L.T @ x)][op]
    assert np.allclose(oracle.apply_factor(n, cp, ri, val, op, x), ref, rtol=1e-12, atol=1e-12)


def test_pcg_oracle_textbook_properties():
    """CG terminates in as many iterations as the matrix has distinct eigenvalues, and the
    preconditioned solve agrees with a direct solve."""
    from oracle.pcg import pcg
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    eig = np.repeat([1.0, 4.0, 9.0], 10)
    A = Q @ np.diag(eig) @ Q.T
    b = rng.standard_normal(30)
    x, it, rel = pcg(A, b, tol=1e-12)
    assert it == 3 and np.allclose(A @ x, b, atol=1e-10)
    B = rng.standard_normal((40, 40))
    A2 = B @ B.T + 40 * np.eye(40)
    M = np.diag(1 / np.diag(A2))
    x2, it2, _ = pcg(A2, b[:20].repeat(2), Minv=M, tol=1e-12)
    assert np.allclose(x2, np.linalg.solve(A2, b[:20].repeat(2)), rtol=1e-9)
    assert it2 <= 40


# ------------------------------------------------- FP64 side state (pivots) --

def test_pivot_variances_match_cholesky_greedy(oracle_lib):
    """The dense Schur complements agree with the Cholesky-form greedy's own quantities:
    var1 / var2 of each pick is the multiple-target score of that pick (eq. greedy_mult),
    and for one target the decrease log(var1 / var2) is log(v_t / v_t+1) of the target's
    variance (the two sides of the determinant lemma)."""
    oracle = oracle_lib
    pts, _ = _ordered(oracle, 400, 2, 21)
    kp = oracle.kernel(2, 3, 0.2, 1.0, 1e-6)
    gptr, gidx = oracle.group_candidates(pts, np.array([0, 5, 9], np.int64), 40)
    for g, (g0, m) in enumerate([(0, 5), (5, 4)]):
        cand = gidx[gptr[g]:gptr[g + 1]]
        r = oracle.select_multi(kp, pts, g0, m, cand, 12)
        v1, v2 = oracle.pivot_variances(kp, pts, range(g0, g0 + m), r["sel"])
        np.testing.assert_allclose(v1 / v2, r["chosen"], rtol=1e-9)
    cptr, cidx = oracle.column_candidates(pts, 40)
    for i in [0, 17, 150]:
        cand = cidx[cptr[i]:cptr[i + 1]]
        r = oracle.select_single(kp, pts, i, cand, 12)
        v1, v2 = oracle.pivot_variances(kp, pts, [i], r["sel"])
        np.testing.assert_allclose(np.log(v1 / v2), np.log(r["vtar"][:-1] / r["vtar"][1:]), rtol=1e-8)


def test_pivot_variances_ou_closed_form(oracle_lib):
    """Exponential kernel on a line (Ornstein-Uhlenbeck, Markov): a pick's variance given
    earlier picks depends only on its nearest earlier picks on each side --
    sigma^2 (1 - e^{-2d/ell}) beyond the outermost pick at distance d, and the bridge
    variance sigma^2 (1 - e^{-2a/ell})(1 - e^{-2b/ell}) / (1 - e^{-2(a+b)/ell}) between
    picks at distances a and b; the first pick has the full variance."""
    oracle = oracle_lib
    ell = 0.3
    kp = oracle.kernel(1, 1, ell, 2.0, 0.0)
    pts = np.array([[0.0], [0.55], [0.1], [0.9], [0.3]])
    picks = [1, 2, 3, 4]
    v1, v2 = oracle.pivot_variances(kp, pts, [0], picks)
    e = lambda d: 1.0 - math.exp(-2.0 * d / ell)
    bridge = lambda a, b: 2.0 * e(a) * e(b) / e(a + b)
    assert v1[0] == pytest.approx(2.0, rel=1e-12)
    assert v1[1] == pytest.approx(2.0 * e(0.45), rel=1e-10)      # 0.1 beyond 0.55
    assert v1[2] == pytest.approx(2.0 * e(0.35), rel=1e-10)      # 0.9 beyond 0.55
    assert v1[3] == pytest.approx(bridge(0.2, 0.25), rel=1e-10)  # 0.3 between 0.1 and 0.55
    # with the target at 0 as well
    assert v2[0] == pytest.approx(2.0 * e(0.55), rel=1e-10)
    assert v2[1] == pytest.approx(bridge(0.1, 0.45), rel=1e-10)  # 0.1 between 0 and 0.55
    assert v2[3] == pytest.approx(bridge(0.2, 0.25), rel=1e-10)
