"""FP64 oracle of directed GP regression (Section 3) -- TEST INFRASTRUCTURE ONLY.

For a target point t with selected training points I (e.g. by `select_single` on its
candidate set), the posterior of the latent process at t given the noisy observations
y_I (the nugget is the observation-noise variance, on the diagonal of Theta_II only):
    mean_t = Theta_{t,I} Theta_{I,I}^{-1} y_I
    var_t  = K(t,t) - Theta_{t,I} Theta_{I,I}^{-1} Theta_{I,t}
K(t,t) = variance (no nugget: the latent value, not a new observation).  Plain dense
numpy solves; pinned in tests/test_oracle_gp.py by the Ornstein-Uhlenbeck bridge in
closed form, interpolation at a training point, and the full-conditioning posterior
from the Cholesky factor of the joint covariance.
"""
from __future__ import annotations

import numpy as np

from . import matern, theta_matrix


def predict(kp, pts, target: int, sel, y):
    """(mean, var) at position `target` of `pts` from the picks `sel` (positions of
    pts) with observations y[sel]."""
    sel = np.asarray(sel, dtype=np.int64)
    if sel.size == 0:
        return 0.0, float(kp.variance)
    K = theta_matrix(kp, pts, sel)
    P = np.asarray(pts, dtype=np.float64)
    r = np.sqrt(((P[sel] - P[target]) ** 2).sum(-1))
    k = np.array([matern(kp, float(v)) for v in r])
    w = np.linalg.solve(K, k)
    return float(w @ np.asarray(y, dtype=np.float64)[sel]), float(kp.variance - w @ k)
