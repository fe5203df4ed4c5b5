"""GPU FP64 side state of a selection (the picks' FP64 conditional variances) against the
oracle's dense Schur complements.

The picks given to the kernel come from the oracle (its FP64 greedy) or from a seeded
random draw of distinct candidates, never from the GPU.  Tolerance per variance v (FP64
rounding through at most m + k elimination steps of entries of size sigma^2):
|dv| <= 1e-9 v + 1e-13 sigma^2; for the decrease log(v1 / v2) / m the same bound carried
through the logarithm: |dg| <= (1e-9 + 1e-13 sigma^2 / v1 + 1e-9 + 1e-13 sigma^2 / v2) / m.
"""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu

REL, ABS = 1e-9, 1e-13


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_11648_gb300 import build
    build.build()
    from paper_2307_11648_gb300 import pipeline, sic
    return torch, sic, pipeline, sic.Handle(0)


def _okernel(oracle, kp):
    return oracle.kernel(kp.dim, kp.nu_x2, kp.length_scale, kp.variance, kp.nugget)


def _run_side(env, pts, kp, sel, cnt, k, grp_ptr=None, max_m=1):
    torch, sic, _, h = env
    U = len(cnt)
    si = np.full((U, k), -1, np.int32)
    for u in range(U):
        c = min(cnt[u], k, len(sel[u]))
        si[u, :c] = sel[u][:c]
    d = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).cuda()
    out = [torch.full((U * k,), -1.0, dtype=torch.float64, device="cuda") for _ in range(3)]
    sic.side_state_fp64(h, d(pts, np.float64), kp, d(si.reshape(-1), np.int32), d(np.asarray(cnt), np.int32), k,
                        grp_ptr=None if grp_ptr is None else d(grp_ptr, np.int64), max_m=max_m,
                        pvar=out[0], pvar_p=out[1], gain=out[2])
    h.sync()
    return [o.view(U, k).cpu().numpy() for o in out]


def _compare(oracle, okp, pts, units, sel, cnt, res, s2, sample):
    v1g, v2g, gg = res
    worst = 0.0
    for u in sample:
        P = units[u]
        v1, v2 = oracle.pivot_variances(okp, pts, P, sel[u][:cnt[u]])
        c = cnt[u]
        for a, b in ((v1g[u, :c], v1), (v2g[u, :c], v2)):
            err = np.abs(a - b)
            assert np.all(err <= REL * np.abs(b) + ABS * s2), (u, err.max())
            worst = max(worst, float((err / np.abs(b)).max()) if c else 0.0)
        g = np.log(v1 / v2) / len(P)
        tol = (2 * REL + ABS * s2 / v1 + ABS * s2 / v2) / len(P)
        assert np.all(np.abs(gg[u, :c] - g) <= tol), u
        assert np.all(v1g[u, c:] == -1.0) and np.all(gg[u, c:] == -1.0)  # untouched
    return worst


def test_side_state_columns_on_oracle_picks(env, oracle_lib):
    """N = 4096 single columns (2-D, Matern 3/2, ell = 0.1, nugget 1e-8), 64 candidates,
    up to 16 picks of the oracle's FP64 greedy."""
    torch, sic, pipeline, h = env
    oracle = oracle_lib
    kp = sic.kernel(2, 3, 0.1, 1.0, 1e-8)
    okp = _okernel(oracle, kp)
    hp = pipeline.prepare_columns(synthetic.points(4096, 2, 0), kp, 64, 16)
    P = hp.pts
    sel, cnt, vtar = [], [], []
    for i in range(hp.n):
        r = oracle.select_single(okp, P, i, hp.cand_idx[hp.cand_ptr[i]:hp.cand_ptr[i + 1]], 16)
        sel.append(r["sel"])
        cnt.append(len(r["sel"]))
        vtar.append(r["vtar"])
    res = _run_side(env, P, kp, sel, cnt, 16)
    # every column against the oracle's own Cholesky recursion; a sample against dense solves
    for i in range(hp.n):
        g = np.log(vtar[i][:-1] / vtar[i][1:])
        np.testing.assert_allclose(res[2][i, :cnt[i]], g, rtol=1e-8, atol=1e-12, err_msg=str(i))
    worst = _compare(oracle, okp, P, [[i] for i in range(hp.n)], sel, cnt, res, 1.0, range(0, hp.n, 37))
    print(f"columns: worst relative variance error {worst:.2e}")


def test_side_state_groups_on_oracle_picks(env, oracle_lib):
    """Supernodes of 8-64 members over N = 4096 points (Matern 3/2, ell = 0.05, nugget
    1e-6), 128 candidates, up to 32 picks of the oracle's FP64 multiple-target greedy."""
    torch, sic, pipeline, h = env
    oracle = oracle_lib
    kp = sic.kernel(2, 3, 0.05, 1.0, 1e-6)
    okp = _okernel(oracle, kp)
    hp = pipeline.prepare_groups(synthetic.points(4096, 2, 1), kp, 128, 32)
    P, gp = hp.pts, hp.grp_ptr
    G = len(gp) - 1
    sel, cnt, chosen = [], [], []
    for g in range(G):
        r = oracle.select_multi(okp, P, int(gp[g]), int(gp[g + 1] - gp[g]),
                                hp.cand_idx[hp.cand_ptr[g]:hp.cand_ptr[g + 1]], 32)
        sel.append(r["sel"])
        cnt.append(len(r["sel"]))
        chosen.append(r["chosen"])
    res = _run_side(env, P, kp, sel, cnt, 32, gp, hp.max_m)
    for g in range(G):
        m = int(gp[g + 1] - gp[g])
        np.testing.assert_allclose(res[2][g, :cnt[g]], np.log(chosen[g]) / m, rtol=1e-8, atol=1e-12, err_msg=str(g))
    units = [list(range(int(gp[g]), int(gp[g + 1]))) for g in range(G)]
    worst = _compare(oracle, okp, P, units, sel, cnt, res, 1.0, range(0, G, 5))
    print(f"groups {G}: worst relative variance error {worst:.2e}")


def test_side_state_random_picks_largest_layout(env, oracle_lib):
    """Picks drawn at random (distinct, seeded) among 256 candidates, k = 128 and groups of
    up to 64 members (the largest shared-memory layout), including units with no pick."""
    torch, sic, pipeline, h = env
    oracle = oracle_lib
    kp = sic.kernel(2, 5, 0.08, 1.3, 1e-5)
    okp = _okernel(oracle, kp)
    hp = pipeline.prepare_groups(synthetic.points(6000, 2, 7), kp, 256, 64)
    P, gp = hp.pts, hp.grp_ptr
    G = len(gp) - 1
    rng = np.random.default_rng(11)
    k = 128
    sel, cnt = [], []
    for g in range(G):
        cand = hp.cand_idx[hp.cand_ptr[g]:hp.cand_ptr[g + 1]]
        c = int(rng.integers(0, min(k, len(cand)) + 1)) if g % 7 else 0
        sel.append(rng.permutation(cand)[:c].astype(np.int32))
        cnt.append(c)
    res = _run_side(env, P, kp, sel, cnt, k, gp, hp.max_m)
    units = [list(range(int(gp[g]), int(gp[g + 1]))) for g in range(G)]
    sample = [g for g in range(G) if cnt[g] > 100][:6] + list(range(0, G, 23))
    worst = _compare(oracle, okp, P, units, sel, cnt, res, 1.3, sample)
    print(f"random picks, max m {hp.max_m}: worst relative variance error {worst:.2e}")


def test_side_state_errors_reported(env):
    torch, sic, pipeline, h = env
    kp = sic.kernel(2, 3, 0.1, 1.0, 1e-8)
    pts = synthetic.points(300, 2, 3)
    with pytest.raises(sic.SicError):  # a repeated pick without nugget: Theta_SS is singular
        _run_side(env, pts, sic.kernel(2, 3, 0.1, 1.0, 0.0), [np.array([5, 5], np.int32)], [2], 4)
    with pytest.raises(sic.SicError):  # a pick outside the points
        _run_side(env, pts, kp, [np.array([5, 300], np.int32)], [2], 4)
    with pytest.raises(sic.SicError):  # a count above k
        _run_side(env, pts, kp, [np.array([5, 6], np.int32)], [5], 4)
    v1, v2, g = _run_side(env, pts, kp, [np.array([5, 6], np.int32), np.array([], np.int32)], [2, 0], 4)
    assert v1[0, 0] == pytest.approx(1.0 + 1e-8) and np.isfinite(g[0, :2]).all() and v1[1, 0] == -1.0


def test_side_state_no_units(env):
    torch, sic, pipeline, h = env
    kp = sic.kernel(2, 3, 0.1, 1.0, 1e-8)
    pts = torch.from_numpy(synthetic.points(50, 2, 1)).cuda()
    z = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    sic.side_state_fp64(h, pts, kp, z, z[:0], 4, gain=out)  # nothing launched
    h.sync()
    with pytest.raises(sic.SicError):  # no output requested
        sic.side_state_fp64(h, pts, kp, z, z[:0], 4)


def test_side_state_full_size_sampled(env, oracle_lib):
    """The bench's configuration: N = 2^20 supernodes (Matern 3/2, ell = 0.02, nugget 1e-6,
    8-64 members, k = 64), candidate lists cut to their 256 nearest, FP32 selection with a
    global budget of 48 picks per column and the decreases from the FP64 side state.
    Sampled groups: the side state's variances against dense Schur complements of the same
    picks; the allocation is a valid one (within budget, prefixes, no dropped pick ranked
    above a kept one)."""
    torch, sic, pipeline, h = env
    oracle = oracle_lib
    cfg = synthetic.PRESETS["cfg3_aggregated"]
    kp = sic.kernel(cfg["dim"], cfg["nu_x2"], cfg["length_scale"], cfg["variance"], cfg["nugget"])
    pts = synthetic.points(cfg["n"], cfg["dim"], cfg["seed"])
    hp = pipeline.prepare_groups(pts, kp, 256, cfg["k"], cfg["m_min"], cfg["m_max"])
    sizes = np.diff(hp.grp_ptr)
    B = int(48 * sizes.sum())
    dp = pipeline.DeviceProblem(hp)
    fb = pipeline.FactorBuilder(h, hp, sic.SIC_FP32_MIXED, budget=B, side_fp64=True)
    fb.run(dp)
    h.sync()
    G, k = hp.n_units, hp.k
    v1 = torch.empty(G * k, dtype=torch.float64, device="cuda")
    v2 = torch.empty(G * k, dtype=torch.float64, device="cuda")
    sic.side_state_fp64(h, dp.pts, kp, fb.sel_idx, fb.local_count, k, grp_ptr=dp.grp_ptr, max_m=hp.max_m,
                        pvar=v1, pvar_p=v2)
    h.sync()
    v1, v2 = v1.view(G, k).cpu().numpy(), v2.view(G, k).cpu().numpy()
    gain = fb.gain.view(G, k).cpu().numpy()
    sel = fb.sel_idx.view(G, k).cpu().numpy()
    lcnt, cnt = fb.local_count.cpu().numpy(), fb.sel_count.cpu().numpy()
    okp = _okernel(oracle, kp)
    rng = np.random.default_rng(8)
    groups = sorted(set(rng.choice(G, 10, replace=False).tolist()) | {0, G - 1})
    for g in groups:
        P = list(range(int(hp.grp_ptr[g]), int(hp.grp_ptr[g + 1])))
        c = int(lcnt[g])
        o1, o2 = oracle.pivot_variances(okp, hp.pts, P, sel[g, :c])
        assert np.all(np.abs(v1[g, :c] - o1) <= REL * o1 + ABS * kp.variance), g
        assert np.all(np.abs(v2[g, :c] - o2) <= REL * o2 + ABS * kp.variance), g
        tol = (2 * REL + ABS * kp.variance / o1 + ABS * kp.variance / o2) / len(P)
        assert np.all(np.abs(gain[g, :c] - np.log(o1 / o2) / len(P)) <= tol), g
    assert np.all(cnt >= 0) and np.all(cnt <= lcnt) and int(np.dot(cnt, sizes)) <= B
    keys = [np.minimum.accumulate(gain[u, :lcnt[u]]) for u in range(G)]
    kept = min(keys[u][cnt[u] - 1] for u in range(G) if cnt[u] > 0)
    dropped = max((keys[u][cnt[u]] for u in range(G) if cnt[u] < lcnt[u]), default=-np.inf)
    assert kept >= dropped
    print(f"groups {G}: kept {int(np.dot(cnt, sizes))} of {B} nonzeros; sum log v {float(fb.sum_logv.cpu()[0]):.1f}")
