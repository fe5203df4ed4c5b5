"""FP64 oracle of the learned candidate proposal -- TEST INFRASTRUCTURE ONLY.

The paper has no learned component; this follows the proposal's definition as stated
in this repository: 8 features per (group, candidate), an MLP 8 -> 128 -> 128 -> 1 with
exact (erf) GELU, a weighted binary cross-entropy against plain-greedy labels and AdamW.
Plain numpy, unblocked; pinned by central finite differences in the tests.

Features of candidate j (list rank r of C) for the group P = positions g0..g0+m-1,
with R the distance from the last candidate of the list to its nearest member (1 if
zero), a* the nearest member (lowest index on ties), K the kernel without nugget and
sigma^2 its variance:
  f0, f1  (x_j - x_a*)[0], [1] / R            (0 for a missing coordinate)
  f2      |x_j - x_a*| / R
  f3      |x_j - mean_a x_a| / R
  f4      r / C
  f5      K(|x_j - x_a*|) / sigma^2
  f6      m / 64
  f7      mean_a K(|x_j - x_a|) / sigma^2
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

N_FEAT, HIDDEN = 8, 128
# flat parameter layout (FP32 on the device, FP64 here)
OFF_W1, OFF_B1 = 0, 8 * 128
OFF_W2 = OFF_B1 + 128
OFF_B2 = OFF_W2 + 128 * 128
OFF_W3 = OFF_B2 + 128
OFF_B3 = OFF_W3 + 128
N_PARAMS = OFF_B3 + 1


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return dict(W1=p[OFF_W1:OFF_B1].reshape(8, 128), b1=p[OFF_B1:OFF_W2], W2=p[OFF_W2:OFF_B2].reshape(128, 128),
                b2=p[OFF_B2:OFF_W3], w3=p[OFF_W3:OFF_B3], b3=p[OFF_B3])


def pack(d):
    return np.concatenate([d["W1"].ravel(), d["b1"], d["W2"].ravel(), d["b2"], d["w3"], np.atleast_1d(d["b3"])])


def matern_np(nu_x2, ell, s2, r):
    c = {1: 1.0, 3: math.sqrt(3.0), 5: math.sqrt(5.0)}[nu_x2]
    t = c * r / ell
    if nu_x2 == 1:
        return s2 * np.exp(-t)
    if nu_x2 == 3:
        return s2 * (1 + t) * np.exp(-t)
    return s2 * (1 + t + t * t / 3) * np.exp(-t)


def features(kp, pts, g0, m, cand):
    """8 features of every candidate of one group (definitions in the module docstring)."""
    P = pts[g0:g0 + m]
    X = pts[np.asarray(cand, dtype=np.int64)]
    C = len(cand)
    D = np.sqrt(((X[:, None, :] - P[None, :, :]) ** 2).sum(-1))  # C x m
    a = np.argmin(D, axis=1)
    dmin = D[np.arange(C), a]
    ell = dmin[-1] if C and dmin[-1] > 0 else 1.0
    diff = X - P[a]
    f = np.zeros((C, N_FEAT))
    f[:, 0] = diff[:, 0] / ell
    if pts.shape[1] > 1:
        f[:, 1] = diff[:, 1] / ell
    f[:, 2] = dmin / ell
    f[:, 3] = np.sqrt(((X - P.mean(0)) ** 2).sum(-1)) / ell
    f[:, 4] = np.arange(C) / C
    f[:, 5] = matern_np(kp.nu_x2, kp.length_scale, kp.variance, dmin) / kp.variance
    f[:, 6] = m / 64.0
    f[:, 7] = matern_np(kp.nu_x2, kp.length_scale, kp.variance, D).mean(1) / kp.variance
    return f


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def dgelu(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(p, X):
    """Returns the scores and the intermediates (Z1, H1, Z2, H2)."""
    d = unpack(p)
    Z1 = X @ d["W1"] + d["b1"]
    H1 = gelu(Z1)
    Z2 = H1 @ d["W2"] + d["b2"]
    H2 = gelu(Z2)
    s = H2 @ d["w3"] + d["b3"]
    return s, (Z1, H1, Z2, H2)


def softplus(x):
    return np.logaddexp(0.0, x)


def loss(p, X, y, pos_weight):
    """Mean weighted BCE with logits: pos_weight * y * softplus(-s) + (1 - y) * softplus(s)."""
    s, _ = forward(p, X)
    return float(np.mean(pos_weight * y * softplus(-s) + (1 - y) * softplus(s)))


def grads(p, X, y, pos_weight):
    """Analytic gradient of `loss` (backpropagation through the three layers)."""
    d = unpack(p)
    s, (Z1, H1, Z2, H2) = forward(p, X)
    B = X.shape[0]
    sig = 1.0 / (1.0 + np.exp(-s))
    dS = (pos_weight * y * (sig - 1.0) + (1 - y) * sig) / B
    g = {}
    g["w3"] = H2.T @ dS
    g["b3"] = np.array(dS.sum())
    dZ2 = np.outer(dS, d["w3"]) * dgelu(Z2)
    g["W2"] = H1.T @ dZ2
    g["b2"] = dZ2.sum(0)
    dZ1 = (dZ2 @ d["W2"].T) * dgelu(Z1)
    g["W1"] = X.T @ dZ1
    g["b1"] = dZ1.sum(0)
    return pack(g)


def adamw_step(p, m, v, g, step, lr, b1=0.9, b2=0.999, eps=1e-8, wd=0.0):
    """One AdamW step (decoupled weight decay), bias-corrected; returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    p = p - lr * (mh / (np.sqrt(vh) + eps) + wd * p)
    return p, m, v
