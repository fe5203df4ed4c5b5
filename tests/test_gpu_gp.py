"""GPU directed GP regression (Section 3) against the oracle and on GP draws.

Tolerances: the picks follow the selection tolerances of the parity tests (FP64 exact
up to the 1e-10 tie band); given the picks, the FP64 posterior mean agrees with the
oracle's dense solve to 1e-9 relative (plus 1e-12 absolute) and the variance to 1e-9 of
the prior variance -- FP64 rounding through a Cholesky of at most k = 32 picks with the
nugget as the smallest eigenvalue bound.
"""
import numpy as np
import pytest

import synthetic
from oracle import gp as OG
from parity import ReplayStats, replay_single

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_11648_gb300 import build
    build.build()
    from paper_2307_11648_gb300 import gp, sic
    return torch, sic, gp, sic.Handle(0)


@pytest.mark.parametrize("prec_name", ["fp64", "fp32"])
def test_gp_predict_matches_oracle(env, oracle_lib, prec_name):
    torch, sic, gp, h = env
    oracle = oracle_lib
    kp = sic.kernel(2, 3, 0.1, 1.5, 1e-4)
    okp = oracle.kernel(2, 3, 0.1, 1.5, 1e-4)
    xtr = synthetic.points(2000, 2, 31)
    ytr = synthetic.normal(32, 2000)
    xte = synthetic.points(300, 2, 33)
    prec = sic.SIC_FP64 if prec_name == "fp64" else sic.SIC_FP32_MIXED
    model = gp.DirectedGP(h, kp, xtr, ytr, n_cand=128, k=24, prec=prec)
    mean, var = model.predict(xte)
    h.sync()
    mean, var = mean.cpu().numpy(), var.cpu().numpy()
    d = model.last
    pts = d["pts"].cpu().numpy()
    ptr, idx = d["ptr"].cpu().numpy(), d["idx"].cpu().numpy()
    sel = d["sel_idx"].view(-1, 24).cpu().numpy()
    cnt = d["sel_count"].cpu().numpy()
    y = np.concatenate([np.zeros(300), ytr])
    stats = ReplayStats()
    for t in range(0, 300, 5):
        cand = idx[ptr[t]:ptr[t + 1]]
        assert np.all(cand >= 300)
        picks = sel[t, :cnt[t]]
        if prec_name == "fp64":
            replay_single(oracle, okp, pts, t, cand, 24, picks, stats)
        m_ref, v_ref = OG.predict(okp, pts, t, picks, y)
        assert mean[t] == pytest.approx(m_ref, rel=1e-9, abs=1e-12), t
        assert abs(var[t] - v_ref) <= 1e-9 * kp.variance, t
    print(prec_name, stats, "mean var", var.mean())


def test_gp_calibrated_on_draws(env):
    """Draw one GP realisation on training + test points (dense Cholesky of the joint
    covariance, test infrastructure), observe the training values with noise of the
    nugget's variance, predict the latent test values: the standardised errors have
    mean square ~1 and the predictions explain most of the prior variance."""
    torch, sic, gp, h = env
    ntr, nte = 2500, 800
    kp = sic.kernel(2, 3, 0.15, 1.0, 1e-3)
    X = np.vstack([synthetic.points(nte, 2, 41), synthetic.points(ntr, 2, 42)])
    D = np.sqrt(((X[:, None, :] - X[None, :, :]) ** 2).sum(-1))
    t = np.sqrt(3.0) * D / 0.15
    K = (1 + t) * np.exp(-t)
    f = np.linalg.cholesky(K + 1e-10 * np.eye(len(X))) @ synthetic.normal(43, len(X))
    y = f[nte:] + np.sqrt(1e-3) * synthetic.normal(44, ntr)
    model = gp.DirectedGP(h, kp, X[nte:], y, n_cand=128, k=32)
    mean, var = model.predict(X[:nte])
    h.sync()
    mean, var = mean.cpu().numpy(), var.cpu().numpy()
    assert np.all(var > 0)
    z2 = (f[:nte] - mean) ** 2 / var
    rmse = np.sqrt(np.mean((f[:nte] - mean) ** 2))
    print("mean z^2", z2.mean(), "rmse", rmse, "prior sd 1")
    assert 0.75 < z2.mean() < 1.33
    assert rmse < 0.2
