"""Pins of the directed GP regression oracle (oracle/gp.py), Section 3."""
import math

import numpy as np
import pytest

import synthetic
from oracle import gp as OG


def test_ou_bridge_closed_form(oracle_lib):
    """Matern 1/2 in 1-D without nugget is the Ornstein-Uhlenbeck process: greedy
    selection picks the two neighbours of the target (screening), and the posterior is
    the OU bridge -- with r1 = exp(-d1), r2 = exp(-d2), d1, d2 the scaled distances to
    the left and right neighbour:
        mean = [r1 (1 - r2^2) y_a + r2 (1 - r1^2) y_b] / (1 - r1^2 r2^2)
        var  = (1 - r1^2)(1 - r2^2) / (1 - r1^2 r2^2)."""
    oracle = oracle_lib
    ell = 0.3
    kp = oracle.kernel(1, 1, ell, 1.0, 0.0)
    xs = np.sort(synthetic.uniform(91, 0, 40))
    t = 0.5 * (xs[17] + xs[18]) + 0.1 * (xs[18] - xs[17])
    pts = np.concatenate([[t], xs]).reshape(-1, 1)  # the target first, then the training points
    y = np.concatenate([[0.0], synthetic.normal(92, 40)])
    cand = np.arange(1, 41)
    sel = oracle.select_single(kp, pts, 0, cand, 2)["sel"]
    assert sorted(sel.tolist()) == [18, 19]  # positions of xs[17], xs[18]
    mean, var = OG.predict(kp, pts, 0, sel, y)
    r1, r2 = math.exp(-(t - xs[17]) / ell), math.exp(-(xs[18] - t) / ell)
    m_ref = (r1 * (1 - r2 * r2) * y[18] + r2 * (1 - r1 * r1) * y[19]) / (1 - r1 * r1 * r2 * r2)
    v_ref = (1 - r1 * r1) * (1 - r2 * r2) / (1 - r1 * r1 * r2 * r2)
    assert mean == pytest.approx(m_ref, rel=1e-12, abs=1e-14)
    assert var == pytest.approx(v_ref, rel=1e-12)
    # more picks cannot change an OU posterior that the neighbours screen
    m4, v4 = OG.predict(kp, pts, 0, oracle.select_single(kp, pts, 0, cand, 4)["sel"], y)
    assert m4 == pytest.approx(m_ref, rel=1e-9, abs=1e-12) and v4 == pytest.approx(v_ref, rel=1e-9)


def test_interpolates_a_training_point(oracle_lib):
    """Without nugget the posterior at a training location is the observation, with
    zero variance."""
    oracle = oracle_lib
    kp = oracle.kernel(2, 3, 0.2, 1.3, 0.0)
    P = synthetic.points(60, 2, 93)
    pts = np.vstack([P[7:8], P])  # target = a copy of training point 7 (position 8)
    y = np.concatenate([[0.0], synthetic.normal(94, 60)])
    sel = [8, 3, 20, 41]
    mean, var = OG.predict(kp, pts, 0, sel, y)
    assert mean == pytest.approx(y[8], abs=1e-10)
    assert abs(var) <= 1e-10


def test_full_conditioning_matches_joint_cholesky(oracle_lib):
    """With every training point picked, the posterior equals the conditional read off
    the Cholesky factor of the joint covariance of (training, target): for
    L L^T = [[K, k], [k^T, s2]], var = L_tt^2 and mean = L_tI L_II^{-1} y."""
    oracle = oracle_lib
    kp = oracle.kernel(2, 5, 0.25, 0.8, 1e-3)
    P = synthetic.points(41, 2, 95)
    y = synthetic.normal(96, 41)
    sel = np.arange(1, 41)
    mean, var = OG.predict(kp, P, 0, sel, y)
    J = oracle.theta_matrix(kp, P, list(sel) + [0])
    J[-1, -1] = kp.variance  # the latent value at the target: no nugget
    L = np.linalg.cholesky(J)
    m_ref = L[-1, :-1] @ np.linalg.solve(np.tril(L[:-1, :-1]), y[1:])
    assert var == pytest.approx(L[-1, -1] ** 2, rel=1e-10)
    assert mean == pytest.approx(m_ref, rel=1e-10, abs=1e-12)
