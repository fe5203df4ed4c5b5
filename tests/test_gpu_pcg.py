"""GPU tests of the on-the-fly kernel matvec and of preconditioned CG with the factor.

Tolerances: FP64 matvec vs the dense oracle product to 1e-12 relative; FP32 matvec to
1e-5 relative (FP32 kernel entries, ~6e-8 relative each; products summed with double-FP32
compensation).  PCG in FP64 mode against the oracle's textbook PCG with the oracle's own
factor: iteration counts within 1, and the device solution's true residual |b - A x| / |b|
(A formed densely by the oracle) below 1e-7 (the solvers stop at recursive residual 1e-8;
the solutions themselves may differ by up to cond(A) * 1e-8).
"""
import math

import numpy as np
import pytest

import synthetic
from oracle.pcg import pcg as oracle_pcg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_11648_gb300 import build
    build.build()
    from paper_2307_11648_gb300 import pipeline, sic
    return torch, sic, pipeline, sic.Handle(0)


@pytest.mark.parametrize("nrhs", [1, 2, 3, 8])
def test_matvec_matches_dense(env, oracle_lib, nrhs):
    torch, sic, pipeline, h = env
    n = 3000
    kp = sic.kernel(2, 3, 0.08, 1.0, 1e-6)
    P = synthetic.points(n, 2, 4)
    x = synthetic.normal(5, n * nrhs).reshape(n, nrhs)
    T = oracle_lib.theta_matrix(oracle_lib.kernel(2, 3, 0.08, 1.0, 1e-6), P, np.arange(n)) + 1e-4 * np.eye(n)
    ref = T @ x
    for prec, tol in [(sic.SIC_FP64, 1e-12), (sic.SIC_FP32_MIXED, 1e-5)]:
        y = torch.empty((n, nrhs), dtype=torch.float64, device="cuda")
        sic.matern_matvec(h, torch.from_numpy(P).cuda(), kp, 1e-4, prec, torch.from_numpy(x).cuda(), y)
        h.sync()
        err = np.abs(y.cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err <= tol, (prec, err)


def _factor_for(env, hp, prec):
    torch, sic, pipeline, h = env
    dp = pipeline.DeviceProblem(hp)
    fb = pipeline.FactorBuilder(h, hp, prec)
    fb.run(dp)
    nnz = int(fb.col_ptr[-1].item())
    return dp, fb, (fb.col_ptr, fb.row_idx[:nnz].contiguous(), fb.val[:nnz].contiguous())


def test_pcg_matches_oracle(env, oracle_lib):
    """FP64 PCG on the device against the oracle's textbook PCG with the oracle's own factor:
    N = 4096, Matern 3/2 with the config-3 spacing ratio, system Theta(nugget 1e-6) + 1e-4 I,
    preconditioner = supernodal factor (C = 1024, k = 64) of that same matrix, 4 right-hand
    sides."""
    torch, sic, pipeline, h = env
    oracle = oracle_lib
    n, nrhs = 4096, 4
    ell = 0.02 * math.sqrt((1 << 20) / n)
    kp = sic.kernel(2, 3, ell, 1.0, 1e-6 + 1e-4)       # the solved matrix, shift folded into the nugget
    okp = oracle.kernel(2, 3, ell, 1.0, 1e-6 + 1e-4)
    hp = pipeline.prepare_groups(synthetic.points(n, 2, 0), kp, 1024, 64, 8, 64)
    P = hp.pts
    sels = []
    for g in range(len(hp.grp_ptr) - 1):
        g0, g1 = int(hp.grp_ptr[g]), int(hp.grp_ptr[g + 1])
        cand = oracle.knn_later(P, np.arange(g0, g1), g1, 1024)
        sels.append(oracle.select_multi(okp, P, g0, g1 - g0, cand, 64)["sel"])
    cp, ri, val, _ = oracle.factor_groups(okp, P, hp.grp_ptr, sels)
    L = np.zeros((n, n))
    for c in range(n):
        L[ri[cp[c]:cp[c + 1]], c] = val[cp[c]:cp[c + 1]]
    A = oracle.theta_matrix(okp, P, np.arange(n))
    B = synthetic.normal(3, n * nrhs).reshape(n, nrhs)
    dp, fb, factor = _factor_for(env, hp, sic.SIC_FP64)
    Xd = torch.empty((n, nrhs), dtype=torch.float64, device="cuda")
    ws = sic._ws(sic.pcg_workspace(n, nrhs), "cuda")
    its, rel = sic.pcg_solve(h, dp.pts, kp, 0.0, sic.SIC_FP64, factor, torch.from_numpy(B).cuda(), Xd, 1e-8, 500, ws)
    X = Xd.cpu().numpy()
    its0, _ = sic.pcg_solve(h, dp.pts, kp, 0.0, sic.SIC_FP64, None, torch.from_numpy(B).cuda(), Xd, 1e-8, 400, ws)
    M = L @ L.T
    for r in range(nrhs):
        xo, it, rl = oracle_pcg(A, B[:, r], Minv=M, tol=1e-8, max_iter=500)
        assert rl < 1e-8 and rel[r] < 1e-8
        assert abs(int(its[r]) - it) <= 1, (r, its[r], it)
        true_res = np.linalg.norm(B[:, r] - A @ X[:, r]) / np.linalg.norm(B[:, r])
        assert true_res <= 1e-7, (r, true_res)
    print("PCG iterations: factor", its.tolist(), "none (cap 400)", its0.tolist())
    assert np.all(its < its0)


def test_pcg_preconditioner_quality(env):
    """Config-5 comparison at N = 2^16 (config-3 spacing ratio, C = 1024, k = 64, 8 right-hand
    sides, FP32-entry matvec with compensated sums): iterations to 1e-8 with the greedy
    (conditional) factor and with the k-nearest-neighbour factor (first k candidates), both
    built for the solved matrix Theta + 1e-4 I, and without preconditioner.  Conditional
    selection needs no more iterations than k-nearest neighbours (Section 6.4 reports about
    half)."""
    torch, sic, pipeline, h = env
    n, nrhs, k = 1 << 16, 8, 64
    kp = sic.kernel(2, 3, 0.02 * math.sqrt((1 << 20) / n), 1.0, 1e-6 + 1e-4)
    hp = pipeline.prepare_groups(synthetic.points(n, 2, 0), kp, 1024, k, 8, 64)
    B = torch.from_numpy(synthetic.normal(7, n * nrhs).reshape(n, nrhs)).cuda()
    ws = sic._ws(sic.pcg_workspace(n, nrhs), "cuda")
    res = {}
    dp, fb, factor = _factor_for(env, hp, sic.SIC_FP32_MIXED)
    res["conditional"], rel = sic.pcg_solve(h, dp.pts, kp, 0.0, sic.SIC_FP32_MIXED, factor, B, torch.empty_like(B),
                                            1e-8, 1000, ws)
    assert np.all(rel < 1e-8)
    U = hp.n_units
    sel = np.full((U, k), -1, np.int32)
    cnt = np.zeros(U, np.int32)
    for g in range(U):
        c = hp.cand_idx[hp.cand_ptr[g]:hp.cand_ptr[g + 1]][:k]
        sel[g, :len(c)] = c
        cnt[g] = len(c)
    fb.sel_idx.copy_(torch.from_numpy(sel.ravel()))
    fb.sel_count.copy_(torch.from_numpy(cnt))
    fb.fill(dp)
    nnz = int(fb.col_ptr[-1].item())
    factor = (fb.col_ptr, fb.row_idx[:nnz].contiguous(), fb.val[:nnz].contiguous())
    res["knn"], _ = sic.pcg_solve(h, dp.pts, kp, 0.0, sic.SIC_FP32_MIXED, factor, B, torch.empty_like(B), 1e-8,
                                  1000, ws)
    res["none"], _ = sic.pcg_solve(h, dp.pts, kp, 0.0, sic.SIC_FP32_MIXED, None, B, torch.empty_like(B), 1e-8, 300,
                                   ws)
    print({k2: v.tolist() for k2, v in res.items()})
    assert np.all(res["conditional"] <= res["knn"])
    assert np.all(res["conditional"] < res["none"])
