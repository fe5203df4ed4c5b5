"""Pins of the learned-proposal oracle: analytic gradients against central finite
differences, GELU against its defining integral, AdamW against a hand-unrolled step,
and the features against their geometric definitions on a hand-made group."""
import math

import numpy as np
import pytest
from scipy import integrate

import synthetic
from oracle import learned as OL


def _params(seed, scale=0.3):
    u = synthetic.uniform(seed, 40, OL.N_PARAMS)
    return (u * 2 - 1) * scale


def test_gelu_is_x_times_normal_cdf():
    for z in [-3.0, -0.7, 0.0, 0.4, 2.5]:
        cdf, _ = integrate.quad(lambda t: math.exp(-t * t / 2) / math.sqrt(2 * math.pi), -np.inf, z)
        assert OL.gelu(np.array(z)) == pytest.approx(z * cdf, abs=1e-12)
        h = 1e-6
        fd = (OL.gelu(np.array(z + h)) - OL.gelu(np.array(z - h))) / (2 * h)
        assert OL.dgelu(np.array(z)) == pytest.approx(fd, rel=1e-7, abs=1e-9)


def test_T14_gradients_match_finite_differences():
    """Central differences with h = 1e-6 on FP64 agree with the analytic backward to 1e-6."""
    p = _params(1)
    X = synthetic.normal(2, 24 * 8).reshape(24, 8)
    y = (synthetic.uniform(3, 5, 24) < 0.3).astype(np.float64)
    g = OL.grads(p, X, y, pos_weight=4.0)
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.choice(OL.OFF_B1, 12, replace=False), rng.integers(OL.OFF_B1, OL.N_PARAMS, 40),
                          [OL.OFF_B3]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (OL.loss(p + e, X, y, 4.0) - OL.loss(p - e, X, y, 4.0)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-9), i


def test_adamw_first_steps():
    p = np.array([1.0, -2.0])
    m = np.zeros(2)
    v = np.zeros(2)
    g = np.array([0.5, -0.25])
    p1, m1, v1 = OL.adamw_step(p, m, v, g, 1, lr=0.1, wd=0.01)
    # step 1: m_hat = g, v_hat = g^2, so the update is lr * (sign(g) + wd * p) up to eps
    assert np.allclose(p1, p - 0.1 * (np.sign(g) * np.abs(g) / (np.abs(g) + 1e-8) + 0.01 * p), rtol=1e-12)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)


def test_features_on_a_hand_made_group():
    from oracle import kernel
    kp = kernel(2, 3, 0.5, 2.0, 0.0)
    pts = np.array([[0.0, 0.0], [0.2, 0.0], [0.3, 0.4], [1.0, 1.0], [0.0, 0.1]])
    f = OL.features(kp, pts, 0, 2, [2, 3, 4])
    ell = 0.1  # the last candidate (0, 0.1) is at distance 0.1 from its nearest member
    # candidate 2 (0.3, 0.4): nearest member is point 1 (0.2, 0): offset (0.1, 0.4)
    assert f[0, 0] == pytest.approx(0.1 / ell) and f[0, 1] == pytest.approx(0.4 / ell)
    assert f[0, 2] == pytest.approx(math.hypot(0.1, 0.4) / ell)
    assert f[0, 3] == pytest.approx(math.hypot(0.2, 0.4) / ell)
    assert f[:, 4].tolist() == [0.0, 1 / 3, 2 / 3]
    assert np.all(f[:, 6] == 2 / 64)
    # candidate 4 (0, 0.1): nearest member is point 0 at distance 0.1
    t = math.sqrt(3) * 0.1 / 0.5
    assert f[2, 5] == pytest.approx((1 + t) * math.exp(-t))
    assert f[2, 7] <= f[2, 5] + 1e-15
    assert f[2, 2] == pytest.approx(1.0)
