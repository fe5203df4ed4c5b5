"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle.

Tolerances (stated per result; FP64 rounding differences come from FMA contraction
and a different exp implementation, ~1e-16 relative per operation):
  * selections by oracle replay, compared on each pick's FP64 decrease of the unit's
    objective (nats of 2 KL; tests/parity.py derives the rule): FP64 picks identical
    except at near-ties of the scores within 1e-10 relative; FP32 picks within 1e-3
    relative of the best decrease plus what FP32 cannot resolve in that state.  Every
    test asserts the fraction of steps that differ and the worst decrease gap against
    the caps in CAPS (measured on GB300, with margin);
  * FP32 in aggregate (the survey's FP32 tolerance): sum log v of the FP32 selection
    <= sum log v of the FP64 selection + 1e-3 KL_plain, KL_plain exact (dense logdet)
    at N = 4096 and by the 2k-pick proxy at full size (a smaller KL, so a stricter bound);
  * fill: row indices identical; values max|dL| <= 1e-8 * max|L| per column (the benchmark spec's
    factor tolerance); log v_i to 1e-9 absolute (log v is O(10), so 1e-10 relative);
  * KL sum: 1e-9 relative.
"""
import numpy as np
import pytest

import synthetic
from parity import ReplayStats, column_errors, replay_multi, replay_single

pytestmark = pytest.mark.gpu

L_TOL = 1e-8
LOGV_TOL = 1e-9
KL_BOUND = 1e-3  # sum log v_FP32 <= sum log v_FP64 + KL_BOUND * KL_plain

# (fraction of replayed steps whose pick differs from the oracle's, worst decrease gap in
# nats) allowed per test and precision
CAPS = {
    "fp64": (1e-3, 1e-9),
    "columns_small_full_fp32": (3e-3, 5e-3),       # measured 7.3e-4, 1.5e-3
    "columns_batched_fp32": (1e-2, 1e-3),          # measured 0, 0
    "columns_shapes_fp32": (4e-2, 1e-4),           # measured <= 1.7e-2 (k = 64), 4.9e-6
    "aggregated_small_full_fp32": (5e-3, 1e-5),    # measured 1.0e-3, 1.2e-7
    "aggregated_shapes_fp32": (6e-2, 2e-2),        # k > 64: worst gaps 1.2e-3, 4.5e-3
    "aggregated_full_fp32": (8e-2, 1e-2),          # measured 3.8e-2, 3.0e-3
    "aggregated_top256_fp32": (0.15, 0.3),         # measured 8.75e-2, 0.108
    "directed_fp32": (0.5, 3e-2),                  # one target, 24 picks: measured 0.375, 8.5e-3
}


def _caps(name, prec_name):
    return CAPS["fp64"] if prec_name == "fp64" else CAPS[f"{name}_fp32"]


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_11648_gb300 import build
    build.build()
    from paper_2307_11648_gb300 import pipeline, sic
    h = sic.Handle(0)
    return torch, sic, pipeline, h


def _okernel(oracle, kp):
    return oracle.kernel(kp.dim, kp.nu_x2, kp.length_scale, kp.variance, kp.nugget)


def _run(env, hp, prec):
    torch, sic, pipeline, h = env
    dp = pipeline.DeviceProblem(hp)
    fb = pipeline.FactorBuilder(h, hp, prec)
    fb.run(dp)
    h.sync()
    return fb


def _check_fill_columns(oracle, okp, P, cols, sels, cp, ri, val, logv):
    worst = 0.0
    for i in cols:
        rows, L, lv = oracle.fill_column(okp, P, i, sels[i])
        a, b = cp[i], cp[i + 1]
        assert ri[a:b].tolist() == rows.tolist(), f"rows of column {i}"
        e = column_errors(val[a:b], L)
        worst = max(worst, e)
        assert e <= L_TOL, f"column {i}: rel err {e}"
        assert abs(logv[i] - lv) <= LOGV_TOL, f"column {i}: logv {logv[i]} vs {lv}"
    return worst


# ------------------------------------------------------- single columns --

@pytest.mark.parametrize("prec_name", ["fp64", "fp32"])
def test_columns_small_full(env, oracle_lib, prec_name):
    """Config-1 workload (N=4096, 2-D, Matern 3/2, ell=0.1, nugget 1e-8, C=256, k=16),
    every column compared."""
    torch, sic, pipeline, h = env
    oracle = oracle_lib
    cfg = synthetic.PRESETS["cfg1_single_fp64"]
    kp = sic.kernel(cfg["dim"], cfg["nu_x2"], cfg["length_scale"], cfg["variance"], cfg["nugget"])
    pts = synthetic.points(cfg["n"], cfg["dim"], cfg["seed"])
    hp = pipeline.prepare_columns(pts, kp, cfg["n_cand"], cfg["k"])
    prec = sic.SIC_FP64 if prec_name == "fp64" else sic.SIC_FP32_MIXED
    fb = _run(env, hp, prec)
    sels = fb.sel_lists()
    okp = _okernel(oracle, kp)
    P = hp.pts
    stats = ReplayStats()
    for i in range(hp.n):
        cand = hp.cand_idx[hp.cand_ptr[i]:hp.cand_ptr[i + 1]]
        replay_single(oracle, okp, P, i, cand, hp.k, sels[i], stats, fp32=prec_name == "fp32")
    print(prec_name, stats)
    stats.check(*_caps("columns_small_full", prec_name))
    cp, ri, val, logv = fb.csc()
    worst = _check_fill_columns(oracle, okp, P, range(hp.n), sels, cp, ri, val, logv)
    _, _, _, ologv = oracle.factor_columns(okp, P, sels)
    s = float(fb.sum_logv.cpu()[0])
    assert s == pytest.approx(float(np.sum(ologv)), rel=1e-9)
    ld = oracle.logdet_theta(okp, P)
    kl = oracle.kl_from_logv(s, ld)
    print(f"{prec_name}: worst fill err {worst:.2e}, KL = {kl:.6g}")
    assert kl >= 0


@pytest.mark.parametrize("prec_name", ["fp64", "fp32"])
def test_columns_batched_full_size_sampled(env, oracle_lib, prec_name):
    """Config-2 workload at full size (N=65536, 3-D, Matern 5/2, ell=0.05, nugget 1e-6,
    C=512, k=32) in the launch configuration the benchmark uses; sampled columns
    (random ones plus the ragged tail) are checked, with the oracle computing their
    candidate lists itself; the ordering is checked by the maximin property."""
    torch, sic, pipeline, h = env
    oracle = oracle_lib
    cfg = synthetic.PRESETS["cfg2_single_batched"]
    kp = sic.kernel(cfg["dim"], cfg["nu_x2"], cfg["length_scale"], cfg["variance"], cfg["nugget"])
    pts = synthetic.points(cfg["n"], cfg["dim"], cfg["seed"])
    hp = pipeline.prepare_columns(pts, kp, cfg["n_cand"], cfg["k"])
    prec = sic.SIC_FP64 if prec_name == "fp64" else sic.SIC_FP32_MIXED
    fb = _run(env, hp, prec)
    sels = fb.sel_lists()
    okp = _okernel(oracle, kp)
    P = hp.pts
    n = hp.n
    rng = np.random.default_rng(7)
    cols = sorted(set(rng.choice(n - 600, 40, replace=False).tolist()) |
                  {n - 513, n - 512, n - 300, n - 33, n - 32, n - 2, n - 1})
    _check_ordering_sampled(oracle, pts, hp, rng)
    stats = ReplayStats()
    for i in cols:
        cand = oracle.knn_later(P, [i], i + 1, cfg["n_cand"])
        assert cand.tolist() == hp.cand_idx[hp.cand_ptr[i]:hp.cand_ptr[i + 1]].tolist()
        replay_single(oracle, okp, P, i, cand, hp.k, sels[i], stats, fp32=prec_name == "fp32")
    print(prec_name, stats)
    stats.check(*_caps("columns_batched", prec_name))
    cp, ri, val, logv = fb.csc()
    _check_fill_columns(oracle, okp, P, cols, sels, cp, ri, val, logv)
    assert np.all(np.isfinite(logv))


# every launch shape of the single-target kernel: candidate rows per thread (1, 2, 4 for up to
# 256, 512, 1024 candidates) x factor entries kept per row (16, 32, 64 for k up to 16, 32, 64)
SHAPES = [("fp32", 200, 16), ("fp32", 400, 16), ("fp32", 1000, 16), ("fp32", 200, 32), ("fp32", 400, 32),
          ("fp32", 1000, 32), ("fp32", 200, 64), ("fp32", 400, 64),
          ("fp64", 200, 16), ("fp64", 400, 16), ("fp64", 1000, 16), ("fp64", 200, 32), ("fp64", 400, 32),
          ("fp64", 200, 64)]


@pytest.mark.parametrize("prec_name,n_cand,k", SHAPES)
def test_columns_launch_shapes(env, oracle_lib, prec_name, n_cand, k):
    """N = 1536 in 2-D (Matern 3/2, ell = 0.1, nugget 1e-6): the early columns have the full
    candidate count, the late ones ragged lists down to none; every 5th column and the last
    ones replayed by the oracle, their fill checked, the KL sum against the oracle's."""
    torch, sic, pipeline, h = env
    oracle = oracle_lib
    kp = sic.kernel(2, 3, 0.1, 1.0, 1e-6)
    hp = pipeline.prepare_columns(synthetic.points(1536, 2, 11), kp, n_cand, k)
    assert hp.max_cand == n_cand
    prec = sic.SIC_FP64 if prec_name == "fp64" else sic.SIC_FP32_MIXED
    fb = _run(env, hp, prec)
    sels = fb.sel_lists()
    okp = _okernel(oracle, kp)
    P = hp.pts
    cols = sorted(set(range(0, hp.n, 5)) | set(range(hp.n - 40, hp.n)))
    stats = ReplayStats()
    for i in cols:
        cand = hp.cand_idx[hp.cand_ptr[i]:hp.cand_ptr[i + 1]]
        replay_single(oracle, okp, P, i, cand, hp.k, sels[i], stats, fp32=prec_name == "fp32")
    print(prec_name, n_cand, k, stats)
    stats.check(*_caps("columns_shapes", prec_name))
    cp, ri, val, logv = fb.csc()
    _check_fill_columns(oracle, okp, P, cols, sels, cp, ri, val, logv)
    _, _, _, ologv = oracle.factor_columns(okp, P, sels)
    assert float(fb.sum_logv.cpu()[0]) == pytest.approx(float(np.sum(ologv)), rel=1e-9)


def _check_ordering_sampled(oracle, pts, hp, rng, n_pos=24, n_earlier=64):
    """Reverse-maximin at any size: ell2[p] is the squared distance to the later set and no
    sampled earlier point is farther from that set."""
    P = hp.pts if hp.grp_ptr is None else pts[hp.order]
    n = P.shape[0]
    assert sorted(hp.order.tolist()) == list(range(n)) if n <= 70000 else True
    assert hp.order[-1] == 0 or hp.grp_ptr is not None
    if hp.grp_ptr is not None:
        return
    for p in rng.choice(n - 1, n_pos, replace=False):
        later = P[p + 1:]
        d = np.min(np.sum((later - P[p]) ** 2, axis=1))
        assert d == hp.ell2[p]
        for j in rng.choice(p + 1, min(n_earlier, p + 1), replace=False):
            assert np.min(np.sum((later - P[j]) ** 2, axis=1)) <= hp.ell2[p]


# ----------------------------------------------------------- supernodes --

@pytest.mark.parametrize("prec_name", ["fp64", "fp32"])
def test_aggregated_small_full(env, oracle_lib, prec_name):
    """Supernodes on a small problem (N=4096, 2-D, Matern 3/2, ell=0.05, nugget 1e-6,
    C=192, k=24, m in [4, 32]); every group compared."""
    torch, sic, pipeline, h = env
    oracle = oracle_lib
    kp = sic.kernel(2, 3, 0.05, 1.0, 1e-6)
    pts = synthetic.points(4096, 2, 11)
    hp = pipeline.prepare_groups(pts, kp, 192, 24, mmin=4, mmax=32)
    prec = sic.SIC_FP64 if prec_name == "fp64" else sic.SIC_FP32_MIXED
    fb = _run(env, hp, prec)
    sels = fb.sel_lists()
    okp = _okernel(oracle, kp)
    P = hp.pts
    stats = ReplayStats()
    gp = hp.grp_ptr
    for g in range(len(gp) - 1):
        g0, g1 = int(gp[g]), int(gp[g + 1])
        cand = hp.cand_idx[hp.cand_ptr[g]:hp.cand_ptr[g + 1]]
        replay_multi(oracle, okp, P, g0, g1 - g0, cand, hp.k, sels[g], stats, fp32=prec_name == "fp32")
    print(prec_name, stats)
    stats.check(*_caps("aggregated_small_full", prec_name))
    cp, ri, val, logv = fb.csc()
    worst = 0.0
    for g in range(len(gp) - 1):
        g0, g1 = int(gp[g]), int(gp[g + 1])
        for a in range(g1 - g0):
            rows, L, lv = oracle.fill_member(okp, P, g0, g1 - g0, a, sels[g])
            c = g0 + a
            assert ri[cp[c]:cp[c + 1]].tolist() == rows.tolist()
            e = column_errors(val[cp[c]:cp[c + 1]], L)
            worst = max(worst, e)
            assert e <= L_TOL, f"member {a} of group {g}: {e}"
            assert abs(logv[c] - lv) <= LOGV_TOL
    ld = oracle.logdet_theta(okp, P)
    print(f"{prec_name}: worst fill err {worst:.2e}; KL {oracle.kl_from_logv(float(fb.sum_logv.cpu()[0]), ld):.6g}")


# launch shapes of the shared-memory / workspace supernodal kernel not met by the other tests:
# (precision, candidates, k, largest group) -> threads per CTA, state in shared memory or not
AGG_SHAPES = [("fp32", 200, 80, 16),    # 256 threads, shared memory (k > 64: not the register kernel)
              ("fp32", 200, 128, 64),   # 256 threads, workspace
              ("fp32", 400, 16, 16),    # 512 threads, shared memory
              ("fp64", 200, 64, 64),    # 256 threads, workspace
              ("fp64", 300, 16, 16)]    # 512 threads, shared memory


@pytest.mark.parametrize("prec_name,n_cand,k,mmax", AGG_SHAPES)
def test_aggregated_launch_shapes(env, oracle_lib, prec_name, n_cand, k, mmax):
    """N = 2048 in 2-D (Matern 3/2, ell = 0.1, nugget 1e-6), supernodes of 4..mmax members;
    every third group replayed by the oracle and its members' columns checked."""
    torch, sic, pipeline, h = env
    oracle = oracle_lib
    kp = sic.kernel(2, 3, 0.1, 1.0, 1e-6)
    hp = pipeline.prepare_groups(synthetic.points(2048, 2, 12), kp, n_cand, k, mmin=4, mmax=mmax)
    assert hp.max_cand == n_cand
    prec = sic.SIC_FP64 if prec_name == "fp64" else sic.SIC_FP32_MIXED
    fb = _run(env, hp, prec)
    sels = fb.sel_lists()
    okp = _okernel(oracle, kp)
    P = hp.pts
    stats = ReplayStats()
    gp = hp.grp_ptr
    G = len(gp) - 1
    groups = sorted(set(range(0, G, 3)) | {G - 2, G - 1})
    cp, ri, val, logv = fb.csc()
    for g in groups:
        g0, g1 = int(gp[g]), int(gp[g + 1])
        cand = hp.cand_idx[hp.cand_ptr[g]:hp.cand_ptr[g + 1]]
        replay_multi(oracle, okp, P, g0, g1 - g0, cand, hp.k, sels[g], stats, fp32=prec_name == "fp32")
        for a in range(g1 - g0):
            rows, L, lv = oracle.fill_member(okp, P, g0, g1 - g0, a, sels[g])
            c = g0 + a
            assert ri[cp[c]:cp[c + 1]].tolist() == rows.tolist()
            assert column_errors(val[cp[c]:cp[c + 1]], L) <= L_TOL, f"member {a} of group {g}"
            assert abs(logv[c] - lv) <= LOGV_TOL
    print(prec_name, n_cand, k, mmax, stats)
    stats.check(*_caps("aggregated_shapes", prec_name))
    assert np.all(np.isfinite(logv))


@pytest.mark.parametrize("prec_name", ["fp32", "fp64"])
def test_aggregated_full_size_sampled(env, oracle_lib, prec_name):
    """Config-3 workload at full size (N=2^20, 2-D, Matern 3/2, ell=0.02, nugget 1e-6,
    C=1024, k=64, supernodes m in [8, 64]) in the benchmark's launch configuration;
    sampled groups are checked against the oracle, which computes their candidate
    lists itself."""
    torch, sic, pipeline, h = env
    oracle = oracle_lib
    cfg = synthetic.PRESETS["cfg3_aggregated"]
    kp = sic.kernel(cfg["dim"], cfg["nu_x2"], cfg["length_scale"], cfg["variance"], cfg["nugget"])
    hp = _cfg3_problem(env)
    prec = sic.SIC_FP64 if prec_name == "fp64" else sic.SIC_FP32_MIXED
    fb = _run(env, hp, prec)
    sels = fb.sel_lists()
    okp = _okernel(oracle, kp)
    P = hp.pts
    gp = hp.grp_ptr
    G = len(gp) - 1
    rng = np.random.default_rng(3)
    groups = sorted(set(rng.choice(G - 50, 10, replace=False).tolist()) | {G - 40, G - 3, G - 1})
    stats = ReplayStats()
    cp, ri, val, logv = fb.csc()
    for g in groups:
        g0, g1 = int(gp[g]), int(gp[g + 1])
        cand = oracle.knn_later(P, np.arange(g0, g1), g1, cfg["n_cand"])
        assert cand.tolist() == hp.cand_idx[hp.cand_ptr[g]:hp.cand_ptr[g + 1]].tolist()
        replay_multi(oracle, okp, P, g0, g1 - g0, cand, hp.k, sels[g], stats, fp32=prec_name == "fp32")
        for a in range(g1 - g0):
            rows, L, lv = oracle.fill_member(okp, P, g0, g1 - g0, a, sels[g])
            c = g0 + a
            assert ri[cp[c]:cp[c + 1]].tolist() == rows.tolist()
            assert column_errors(val[cp[c]:cp[c + 1]], L) <= L_TOL
            assert abs(logv[c] - lv) <= LOGV_TOL
    print(prec_name, stats, "sum logv", float(fb.sum_logv.cpu()[0]))
    stats.check(*_caps("aggregated_full", prec_name))
    assert np.all(np.isfinite(logv))


@pytest.mark.parametrize("prec_name", ["fp32", "fp64"])
def test_aggregated_full_size_top256_sampled(env, oracle_lib, prec_name):
    """Config-3 workload at full size with every candidate list cut to its 256 nearest
    entries (the list length the learned proposal hands to the selection; it runs the
    two-threads-per-candidate shared-memory kernel).  Sampled groups against the oracle,
    which computes the 256 nearest later points itself."""
    torch, sic, pipeline, h = env
    oracle = oracle_lib
    cfg = synthetic.PRESETS["cfg3_aggregated"]
    kp = sic.kernel(cfg["dim"], cfg["nu_x2"], cfg["length_scale"], cfg["variance"], cfg["nugget"])
    hp = _cfg3_problem(env)
    top = 256
    cnt = np.minimum(np.diff(hp.cand_ptr), top)
    dptr = np.zeros(len(cnt) + 1, np.int64)
    dptr[1:] = np.cumsum(cnt)
    keep = np.repeat(hp.cand_ptr[:-1], cnt) + (np.arange(int(dptr[-1])) - np.repeat(dptr[:-1], cnt))
    didx = np.ascontiguousarray(hp.cand_idx[keep])
    dhp = pipeline.HostProblem(hp.pts, hp.kp, hp.k, dptr, didx, hp.grp_ptr, hp.order, hp.ell2)
    prec = sic.SIC_FP64 if prec_name == "fp64" else sic.SIC_FP32_MIXED
    fb = _run(env, dhp, prec)
    sels = fb.sel_lists()
    okp = _okernel(oracle, kp)
    P = hp.pts
    gp = hp.grp_ptr
    G = len(gp) - 1
    rng = np.random.default_rng(5)
    groups = sorted(set(rng.choice(G - 50, 12, replace=False).tolist()) | {0, G - 7, G - 2, G - 1})
    stats = ReplayStats()
    cp, ri, val, logv = fb.csc()
    for g in groups:
        g0, g1 = int(gp[g]), int(gp[g + 1])
        cand = oracle.knn_later(P, np.arange(g0, g1), g1, top)
        assert cand.tolist() == didx[dptr[g]:dptr[g + 1]].tolist()
        replay_multi(oracle, okp, P, g0, g1 - g0, cand, hp.k, sels[g], stats, fp32=prec_name == "fp32")
        for a in range(g1 - g0):
            rows, L, lv = oracle.fill_member(okp, P, g0, g1 - g0, a, sels[g])
            c = g0 + a
            assert ri[cp[c]:cp[c + 1]].tolist() == rows.tolist()
            assert column_errors(val[cp[c]:cp[c + 1]], L) <= L_TOL
            assert abs(logv[c] - lv) <= LOGV_TOL
    # T4 on the device's output: every sampled member column is Theta-normalised,
    # L_{s,i}^T Theta_{s,s} L_{s,i} = 1 (eq. L_col), with Theta from the oracle
    worst = 0.0
    for g in groups:
        for c in range(int(gp[g]), int(gp[g + 1])):
            rows = ri[cp[c]:cp[c + 1]]
            v = val[cp[c]:cp[c + 1]]
            worst = max(worst, abs(float(v @ oracle.theta_matrix(okp, P, rows) @ v) - 1.0))
    assert worst <= 1e-8, worst
    print(prec_name, "top-256", stats, "sum logv", float(fb.sum_logv.cpu()[0]), "T4 worst", worst)
    stats.check(*_caps("aggregated_top256", prec_name))
    assert np.all(np.isfinite(logv))


_CFG3 = {}


def _cfg3_problem(env):
    torch, sic, pipeline, h = env
    if "hp" not in _CFG3:
        cfg = synthetic.PRESETS["cfg3_aggregated"]
        kp = sic.kernel(cfg["dim"], cfg["nu_x2"], cfg["length_scale"], cfg["variance"], cfg["nugget"])
        pts = synthetic.points(cfg["n"], cfg["dim"], cfg["seed"])
        _CFG3["hp"] = pipeline.prepare_groups(pts, kp, cfg["n_cand"], cfg["k"], cfg["m_min"], cfg["m_max"])
    return _CFG3["hp"]


# -------------------------------------------------------- other entries --

@pytest.mark.parametrize("prec_name", ["fp64", "fp32"])
def test_select_single_directed(env, oracle_lib, prec_name):
    """Directed GP selection over 5000 training points for one target (Section 3)."""
    torch, sic, pipeline, h = env
    oracle = oracle_lib
    kp = sic.kernel(2, 5, 0.2, 1.0, 1e-6)
    xtr = synthetic.points(5000, 2, 21)
    xt = np.array([0.43, 0.61])
    prec = sic.SIC_FP64 if prec_name == "fp64" else sic.SIC_FP32_MIXED
    k = 24
    ws = sic._ws(sic.select_single_workspace(5000, k, prec), "cuda")
    oi = torch.empty(k, dtype=torch.int32, device="cuda")
    ov = torch.empty(k + 1, dtype=torch.float64, device="cuda")
    oc = torch.empty(1, dtype=torch.int32, device="cuda")
    sic.select_single(h, torch.from_numpy(xtr).cuda(), torch.from_numpy(xt).cuda(), kp, k, prec, oi, ov, oc, ws)
    h.sync()
    cnt = int(oc.cpu()[0])
    sel = oi.cpu().numpy()[:cnt]
    okp = _okernel(oracle, kp)
    P = np.vstack([xt[None, :], xtr])  # row 0 = target, rows 1.. = training points
    cand = np.arange(1, 5001, dtype=np.int32)
    stats = ReplayStats()
    replay_single(oracle, okp, P, 0, cand, k, sel + 1, stats, fp32=prec_name == "fp32")
    if prec_name == "fp64":
        r = oracle.select_single(okp, P, 0, cand, k, forced=(sel).tolist())
        assert np.allclose(ov.cpu().numpy()[:cnt + 1], r["vtar"], rtol=1e-8)
    print(prec_name, stats)
    stats.check(*_caps("directed", prec_name))


@pytest.mark.parametrize("nrhs", [1, 2, 3, 8])
def test_apply_factor(env, oracle_lib, nrhs):
    torch, sic, pipeline, h = env
    oracle = oracle_lib
    kp = sic.kernel(2, 3, 0.1, 1.0, 1e-6)
    pts = synthetic.points(3000, 2, 5)
    hp = pipeline.prepare_columns(pts, kp, 64, 12)
    fb = _run(env, hp, sic.SIC_FP64)
    cp, ri, val, _ = fb.csc()
    x = synthetic.normal(9, hp.n * nrhs).reshape(hp.n, nrhs)
    xd = torch.from_numpy(x).cuda()
    for op in [sic.SIC_OP_L, sic.SIC_OP_LT, sic.SIC_OP_LLT]:
        y = torch.empty_like(xd)
        ws = sic._ws(sic.apply_factor_workspace(hp.n, nrhs, op), "cuda")
        nnz = int(cp[-1])
        sic.apply_factor(h, fb.col_ptr, fb.row_idx[:nnz].contiguous(), fb.val[:nnz].contiguous(), op, xd, y, ws)
        h.sync()
        ref = oracle.apply_factor(hp.n, cp, ri, val, op, x)
        assert np.allclose(y.cpu().numpy(), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_edge_cases_and_determinism(env, oracle_lib):
    """Tiny problems (n = 1, 2, 3: empty and single candidate lists), k larger than the
    candidate count, and bit-identical repeated FP64 runs."""
    torch, sic, pipeline, h = env
    oracle = oracle_lib
    kp = sic.kernel(2, 3, 0.3, 1.0, 1e-6)
    okp = _okernel(oracle, kp)
    for n in [1, 2, 3, 40]:
        pts = synthetic.points(n, 2, 4)
        hp = pipeline.prepare_columns(pts, kp, 8, 16)
        fb = _run(env, hp, sic.SIC_FP64)
        sels = fb.sel_lists()
        for i in range(n):
            cand = hp.cand_idx[hp.cand_ptr[i]:hp.cand_ptr[i + 1]]
            r = oracle.select_single(okp, hp.pts, i, cand, 16)
            assert sels[i].tolist() == r["sel"].tolist()
        cp, ri, val, logv = fb.csc()
        _, _, oval, ologv = oracle.factor_columns(okp, hp.pts, sels)
        assert np.allclose(val, oval, rtol=1e-9, atol=1e-9 * np.abs(oval).max())
    pts = synthetic.points(2048, 2, 6)
    hp = pipeline.prepare_columns(pts, kp, 100, 20)
    a = _run(env, hp, sic.SIC_FP64)
    b = _run(env, hp, sic.SIC_FP64)
    nnz = int(a.col_ptr[-1].item())
    assert torch.equal(a.sel_idx, b.sel_idx) and torch.equal(a.col_ptr, b.col_ptr)
    assert torch.equal(a.val[:nnz], b.val[:nnz]) and torch.equal(a.row_idx[:nnz], b.row_idx[:nnz])
    assert float(a.sum_logv.cpu()[0]) == float(b.sum_logv.cpu()[0])


def test_errors_reported_by_sync(env):
    """Kernel-detected errors come back through sic_sync: a candidate list longer than the
    stated bound (invalid) and a singular pattern (duplicate points, no nugget)."""
    torch, sic, pipeline, h = env
    kp = sic.kernel(2, 3, 0.3, 1.0, 1e-6)
    pts = synthetic.points(300, 2, 8)
    hp = pipeline.prepare_columns(pts, kp, 32, 8)
    dp = pipeline.DeviceProblem(hp)
    fb = pipeline.FactorBuilder(h, hp, sic.SIC_FP64)
    sic.select_columns(h, dp.pts, kp, dp.cand_ptr, dp.cand_idx, 16, 8, sic.SIC_FP64, fb.sel_idx, fb.sel_count)
    with pytest.raises(sic.SicError) as e:
        h.sync()
    assert e.value.code == sic.SIC_ERR_INVALID and 0 <= e.value.unit < 300
    h.sync()  # cleared
    # duplicate points without a nugget: with k = 1 the pattern {i, duplicate} is
    # exactly singular (Theta_{ss} = [[1, 1], [1, 1]])
    kp0 = sic.kernel(2, 3, 0.3, 1.0, 0.0)
    p2 = synthetic.points(64, 2, 9)
    hp2 = pipeline.prepare_columns(p2, kp0, 16, 1)
    P = hp2.pts.copy()
    P[5] = P[hp2.cand_idx[hp2.cand_ptr[5]]]  # column 5's nearest candidate coincides with it
    hp2.pts = P
    dp2 = pipeline.DeviceProblem(hp2)
    fb2 = pipeline.FactorBuilder(h, hp2, sic.SIC_FP64)
    fb2.select(dp2)
    h.sync()
    sels = fb2.sel_lists()
    assert sels[5][0] == hp2.cand_idx[hp2.cand_ptr[5]]
    fb2.fill(dp2)
    with pytest.raises(sic.SicError) as e:
        h.sync()
    assert e.value.code == sic.SIC_ERR_NOT_PD and e.value.unit == 5


def test_supernodal_fp32_errors_reported_by_sync(env):
    """The FP32 supernodal path for short candidate lists (targets' factors in their own
    launch, register-resident selection) reports through sic_sync: a candidate inside its
    own group (invalid), a group larger than the stated max_m (invalid), and coincident
    targets without a nugget (the targets' factor is singular)."""
    torch, sic, pipeline, h = env
    kp = sic.kernel(2, 3, 0.05, 1.0, 1e-6)
    hp = pipeline.prepare_groups(synthetic.points(4096, 2, 12), kp, 128, 16, mmin=4, mmax=32)
    g = 10
    g0 = int(hp.grp_ptr[g])

    def run(hp_, max_m=None):
        dp = pipeline.DeviceProblem(hp_)
        fb = pipeline.FactorBuilder(h, hp_, sic.SIC_FP32_MIXED)
        mm = hp_.max_m if max_m is None else max_m
        ws = sic._ws(sic.select_aggregated_workspace(h, hp_.n_units, hp_.max_cand, mm, hp_.k, sic.SIC_FP32_MIXED),
                     "cuda")
        sic.select_aggregated(h, dp.pts, hp_.kp, dp.grp_ptr, dp.cand_ptr, dp.cand_idx, hp_.max_cand, mm, hp_.k,
                              sic.SIC_FP32_MIXED, fb.sel_idx, fb.sel_count, ws)

    run(hp)
    h.sync()  # the clean problem runs without error
    bad = pipeline.HostProblem(hp.pts, hp.kp, hp.k, hp.cand_ptr, hp.cand_idx.copy(), hp.grp_ptr, hp.order, hp.ell2)
    bad.cand_idx[hp.cand_ptr[g]] = g0  # a member of the group itself
    run(bad)
    with pytest.raises(sic.SicError) as e:
        h.sync()
    assert e.value.code == sic.SIC_ERR_INVALID and e.value.unit == g
    m_big = int(np.argmax(np.diff(hp.grp_ptr)))
    run(hp, max_m=int(np.diff(hp.grp_ptr)[m_big]) - 1)
    with pytest.raises(sic.SicError) as e:
        h.sync()
    assert e.value.code == sic.SIC_ERR_INVALID
    kp0 = sic.kernel(2, 3, 0.05, 1.0, 0.0)
    P = hp.pts.copy()
    P[g0 + 1] = P[g0]  # two coincident members: Theta_PP singular without a nugget
    sing = pipeline.HostProblem(P, kp0, hp.k, hp.cand_ptr, hp.cand_idx, hp.grp_ptr, hp.order, hp.ell2)
    run(sing)
    with pytest.raises(sic.SicError) as e:
        h.sync()
    assert e.value.code == sic.SIC_ERR_NOT_PD and e.value.unit == g


# ----------------------------------------------------- FP32 in aggregate --
# The survey's FP32 tolerance: sum log v_FP32 <= sum log v_FP64 + 1e-3 KL_plain, with KL_plain the
# KL divergence of the plain FP64 greedy factor (eq. obj_chol: KL = (sum log v - logdet Theta) / 2).

def _sum_logv(env, hp, prec):
    fb = _run(env, hp, prec)
    s = float(fb.sum_logv.cpu()[0])
    del fb
    return s


def test_fp32_kl_bound_columns_exact(env, oracle_lib):
    """Config-1 workload (single columns, nugget 1e-8), exact KL from the dense logdet."""
    torch, sic, pipeline, h = env
    oracle = oracle_lib
    cfg = synthetic.PRESETS["cfg1_single_fp64"]
    kp = sic.kernel(cfg["dim"], cfg["nu_x2"], cfg["length_scale"], cfg["variance"], cfg["nugget"])
    hp = pipeline.prepare_columns(synthetic.points(cfg["n"], cfg["dim"], cfg["seed"]), kp, cfg["n_cand"], cfg["k"])
    s64, s32 = _sum_logv(env, hp, sic.SIC_FP64), _sum_logv(env, hp, sic.SIC_FP32_MIXED)
    kl64 = oracle.kl_from_logv(s64, oracle.logdet_theta(_okernel(oracle, kp), hp.pts))
    print(f"cfg1: KL_plain {kl64:.6g}, sum log v FP32 - FP64 = {s32 - s64:.4g} "
          f"({(s32 - s64) / kl64:.3e} KL_plain)")
    assert kl64 > 0
    assert s32 <= s64 + KL_BOUND * kl64


def test_fp32_kl_bound_aggregated_exact(env, oracle_lib):
    """Supernodes at N = 4096 (Matern 3/2, ell = 0.05, nugget 1e-6, C = 192, k = 24, m in [4, 32]),
    exact KL from the dense logdet."""
    torch, sic, pipeline, h = env
    oracle = oracle_lib
    kp = sic.kernel(2, 3, 0.05, 1.0, 1e-6)
    hp = pipeline.prepare_groups(synthetic.points(4096, 2, 11), kp, 192, 24, mmin=4, mmax=32)
    s64, s32 = _sum_logv(env, hp, sic.SIC_FP64), _sum_logv(env, hp, sic.SIC_FP32_MIXED)
    kl64 = oracle.kl_from_logv(s64, oracle.logdet_theta(_okernel(oracle, kp), hp.pts))
    print(f"supernodes 4096: KL_plain {kl64:.6g}, sum log v FP32 - FP64 = {s32 - s64:.4g} "
          f"({(s32 - s64) / kl64:.3e} KL_plain)")
    assert kl64 > 0
    assert s32 <= s64 + KL_BOUND * kl64


def _truncate(pipeline, hp, top):
    cnt = np.minimum(np.diff(hp.cand_ptr), top)
    ptr = np.zeros(len(cnt) + 1, np.int64)
    ptr[1:] = np.cumsum(cnt)
    keep = np.repeat(hp.cand_ptr[:-1], cnt) + (np.arange(int(ptr[-1])) - np.repeat(ptr[:-1], cnt))
    return pipeline.HostProblem(hp.pts, hp.kp, hp.k, ptr, np.ascontiguousarray(hp.cand_idx[keep]), hp.grp_ptr,
                                hp.order, hp.ell2)


@pytest.mark.parametrize("top", [0, 256])
def test_fp32_kl_bound_full_size_proxy(env, top):
    """Config-3 workload at full size (N = 2^20), all 1024 candidates or the first 256 (the
    headline path's selection kernel): KL_plain by the 2k-pick proxy, (S_64 - S_ref) / 2 with
    S_ref from 128 picks per supernode over all candidates (S_ref >= logdet Theta, so the proxy
    is below KL_plain and the bound stricter)."""
    torch, sic, pipeline, h = env
    hp = _cfg3_problem(env)
    ref_hp = pipeline.HostProblem(hp.pts, hp.kp, 2 * hp.k, hp.cand_ptr, hp.cand_idx, hp.grp_ptr, hp.order, hp.ell2)
    s_ref = _sum_logv(env, ref_hp, sic.SIC_FP32_MIXED)
    php = _truncate(pipeline, hp, top) if top else hp
    s64, s32 = _sum_logv(env, php, sic.SIC_FP64), _sum_logv(env, php, sic.SIC_FP32_MIXED)
    kl_proxy = 0.5 * (s64 - s_ref)
    print(f"full size, top {top or 1024}: KL proxy {kl_proxy:.6g}, sum log v FP32 - FP64 = {s32 - s64:.4g} "
          f"({(s32 - s64) / kl_proxy:.3e} KL proxy)")
    assert kl_proxy > 0
    assert s32 <= s64 + KL_BOUND * kl_proxy


def test_fp32_kl_bound_columns_full_size_proxy(env):
    """Config-2 workload at full size (N = 65,536, 3-D, C = 512, k = 32): KL_plain by the proxy
    with 64 picks per column."""
    torch, sic, pipeline, h = env
    cfg = synthetic.PRESETS["cfg2_single_batched"]
    kp = sic.kernel(cfg["dim"], cfg["nu_x2"], cfg["length_scale"], cfg["variance"], cfg["nugget"])
    hp = pipeline.prepare_columns(synthetic.points(cfg["n"], cfg["dim"], cfg["seed"]), kp, cfg["n_cand"], cfg["k"])
    ref_hp = pipeline.HostProblem(hp.pts, hp.kp, 2 * hp.k, hp.cand_ptr, hp.cand_idx, None, hp.order, hp.ell2)
    s_ref = _sum_logv(env, ref_hp, sic.SIC_FP32_MIXED)
    s64, s32 = _sum_logv(env, hp, sic.SIC_FP64), _sum_logv(env, hp, sic.SIC_FP32_MIXED)
    kl_proxy = 0.5 * (s64 - s_ref)
    print(f"cfg2: KL proxy {kl_proxy:.6g}, sum log v FP32 - FP64 = {s32 - s64:.4g} "
          f"({(s32 - s64) / kl_proxy:.3e} KL proxy)")
    assert kl_proxy > 0
    assert s32 <= s64 + KL_BOUND * kl_proxy
