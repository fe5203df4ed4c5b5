"""GPU global greedy allocation of nonzeros (Section 5.4) against the oracle's priority queue.

Tolerances:
  * sic_allocate_global on decreases given to both sides: the per-unit counts are integer
    results and must be identical, ties, costs and the stop-at-the-first-misfit rule
    included;
  * FP64 selection with decreases: the picks follow the parity tests' selection rule
    (identical up to the 1e-10 tie band, by oracle replay); where the picks agree the
    decreases log(v_t / v_t+1) (columns) and log(var|I / var|I,P) / m (supernodes) agree
    with the oracle's to 1e-9 relative plus 1e-12 absolute (FP64 rounding through at most
    k downdates of variances no smaller than the nugget);
  * the allocation after an FP64 selection: counts equal the oracle queue's, except where
    the running-minimum keys of the picks in question lie within 1e-9 relative of the
    queue's cut key (a near-tie at the cut that FP64 rounding may decide either way);
  * FP32 selections: the allocation is valid (within budget, a prefix of every unit's
    picks, no dropped pick ranked above a kept one).  The factor's sum of log v is within
    1e-4 relative of the FP64 path's with the decreases from the FP64 side state, within
    1e-3 with the FP32 selection's own decreases: on the clustered cloud the FP32
    conditional variances near the nugget carry errors of several percent, which misrank
    picks at the cut (measured: the side state halves that gap; the rest comes from the FP32
    picks themselves).  On clustered single columns with nugget 1e-8 the FP32
    selection itself is unreliable (the target variance falls below FP32 resolution), so the
    KL claim there is asserted for the FP64 selection.
"""
import dataclasses
import math

import numpy as np
import pytest

import synthetic
from parity import ReplayStats, replay_multi, replay_single

pytestmark = pytest.mark.gpu

TIE_BAND = 1e-10
GAIN_REL, GAIN_ABS = 1e-9, 1e-12
CUT_REL = 1e-9


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


def _gpu_allocate(env, gain, cnt, k, budget, sizes=None):
    torch, sic, _, h = env
    U = len(cnt)
    g = torch.from_numpy(np.ascontiguousarray(gain.reshape(U * k))).cuda()
    c = torch.from_numpy(cnt.astype(np.int32)).cuda()
    gp = None
    if sizes is not None:
        gp = torch.from_numpy(np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)).cuda()
    out = torch.full((U,), -7, dtype=torch.int32, device="cuda")
    ws = sic._ws(sic.allocate_global_workspace(U, k), "cuda")
    sic.allocate_global(h, g, c, k, budget, out, ws, grp_ptr=gp)
    h.sync()
    return out.cpu().numpy()


def _running_min_keys(gains):
    return [np.minimum.accumulate(np.asarray(g, dtype=np.float64)) if len(g) else np.zeros(0) for g in gains]


def _cut_key(gains, costs, budget):
    """Running-minimum key of the first pick the queue rejects (None if all fit)."""
    items = []
    for u, e in enumerate(_running_min_keys(gains)):
        items += [(-float(x), u, t) for t, x in enumerate(e)]
    items.sort()
    left = budget
    for neg, u, _ in items:
        if costs[u] > left:
            return -neg
        left -= costs[u]
    return None


def _check_counts_near_cut(got, ref, gains, costs, budget):
    """Counts equal, or differing only over picks whose keys are near-ties of the cut."""
    bad = np.nonzero(got != ref)[0]
    if len(bad) == 0:
        return 0
    tau = _cut_key(gains, costs, budget)
    assert tau is not None, "counts differ although every pick fits"
    keys = _running_min_keys(gains)
    for u in bad:
        lo, hi = sorted((int(got[u]), int(ref[u])))
        for x in keys[u][lo:hi]:
            assert abs(x - tau) <= CUT_REL * abs(tau), f"unit {u}: counts {got[u]} vs {ref[u]}, key {x} cut {tau}"
    return len(bad)


# --------------------------------------------- the allocation on given decreases --

CASES = {  # name: (seed, units, k, integer decreases (many ties), group costs)
    "ties_groups": (1, 3000, 64, True, True),
    "real_columns": (2, 20000, 37, False, False),
    "k128": (3, 500, 128, False, True),
    "one_unit": (4, 1, 5, True, False),
    "many_units": (5, 300000, 8, False, False),
}


def _case(name):
    seed, n, k, ints, costs = CASES[name]
    rng = np.random.default_rng(seed)
    cnt = rng.integers(0, k + 1, size=n)
    cnt[: n // 10] = k
    if ints:
        gain = rng.integers(-2, 6, size=(n, k)).astype(np.float64)
    else:
        gain = rng.normal(size=(n, k)) * np.exp(rng.normal(size=(n, 1)))
    for u in range(n):
        gain[u, cnt[u]:] = np.nan  # never read
    sizes = rng.integers(1, 65, size=n) if costs else None
    return gain, cnt, k, sizes


@pytest.mark.parametrize("name", list(CASES))
def test_allocate_matches_queue(env, name):
    from oracle import allocation
    gain, cnt, k, sizes = _case(name)
    costs = [int(s) for s in sizes] if sizes is not None else [1] * len(cnt)
    gains = [gain[u, :cnt[u]] for u in range(len(cnt))]
    total = sum(c * int(n) for c, n in zip(costs, cnt))
    fracs = [0.0, 0.5, 1.0, 1.5] if name == "many_units" else [0.0, 0.01, 0.3, 0.5, 0.77, 0.999, 1.0, 1.5]
    for f in fracs:
        budget = int(f * total)
        got = _gpu_allocate(env, gain, cnt, k, budget, sizes)
        ref = allocation.queue_allocate(gains, costs, budget)
        assert np.array_equal(got, ref), f"{name} budget {budget}: {np.nonzero(got != ref)[0][:10]}"
        assert int(np.dot(got, costs)) <= budget


def test_allocate_edge_cases(env):
    torch, sic, _, h = env
    from oracle import allocation
    # every budget over a small case with equal keys across units of different cost
    gain = np.array([[3.0, 2.0, 2.0], [2.0, 2.0, 9.0], [2.0, 1.0, 0.0]])
    cnt = np.array([3, 3, 3])
    sizes = np.array([2, 3, 1])
    for budget in range(0, 20):
        got = _gpu_allocate(env, gain, cnt, 3, budget, sizes)
        ref = allocation.queue_allocate([gain[u] for u in range(3)], [2, 3, 1], budget)
        assert np.array_equal(got, ref), budget
    # no units: nothing launched, nothing read
    ws = sic._ws(sic.allocate_global_workspace(0, 4), "cuda")
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    z = torch.zeros(1, dtype=torch.int32, device="cuda")
    sic.allocate_global(h, e, z[:0], 4, 10, z[:0], ws)
    h.sync()


def test_allocate_errors_reported(env):
    torch, sic, _, h = env
    gain = np.ones((4, 3))
    with pytest.raises(sic.SicError):
        _gpu_allocate(env, gain, np.array([1, 4, 0, 2]), 3, 5)  # count above k
    g2 = gain.copy()
    g2[2, 0] = np.nan
    with pytest.raises(sic.SicError):
        _gpu_allocate(env, g2, np.array([1, 1, 1, 1]), 3, 5)  # NaN decrease
    with pytest.raises(sic.SicError):
        _gpu_allocate(env, gain, np.array([1, 1, 1, 1]), 3, -1)  # negative budget
    # the handle stays usable
    assert list(_gpu_allocate(env, gain, np.array([1, 2, 3, 0]), 3, 4)) == [1, 2, 1, 0]


# ------------------------------------------------ selection + allocation + fill --

def _columns_problem(env, n, seed, n_cand, k, clustered=False):
    torch, sic, pipeline, h = env
    kp = sic.kernel(2, 3, 0.1, 1.0, 1e-8)
    pts = synthetic.clustered_points(n, 2, seed) if clustered else synthetic.points(n, 2, seed)
    return kp, pipeline.prepare_columns(pts, kp, n_cand, k)


def test_columns_global_fp64_matches_oracle(env, oracle_lib):
    """N = 4096 (the small single-column workload), 64 candidates, at most 16 picks per
    column, a budget of 8 N nonzeros."""
    torch, sic, pipeline, h = env
    oracle = oracle_lib
    from oracle import allocation
    kp, hp = _columns_problem(env, 4096, 0, 64, 16)
    B = 8 * hp.n
    dp = pipeline.DeviceProblem(hp)
    fb = pipeline.FactorBuilder(h, hp, sic.SIC_FP64, budget=B)
    fb.run(dp)
    h.sync()
    okp = _okernel(oracle, kp)
    P, k = hp.pts, hp.k
    cl = [hp.cand_idx[hp.cand_ptr[i]:hp.cand_ptr[i + 1]] for i in range(hp.n)]
    osel, ogain = allocation.column_gains(okp, P, None, cl, k)
    sel = fb.sel_idx.view(-1, k).cpu().numpy()
    lcnt = fb.local_count.cpu().numpy()
    gain = fb.gain.view(-1, k).cpu().numpy()
    cnt = fb.sel_count.cpu().numpy()
    stats = ReplayStats()
    same = 0
    for i in range(hp.n):
        picks = sel[i, :lcnt[i]]
        replay_single(oracle, okp, P, i, cl[i], k, picks, stats)
        if np.array_equal(picks, osel[i]):
            same += 1
            np.testing.assert_allclose(gain[i, :lcnt[i]], ogain[i], rtol=GAIN_REL, atol=GAIN_ABS, err_msg=str(i))
    assert same >= hp.n - 5
    ref = allocation.queue_allocate(ogain, [1] * hp.n, B)
    nd = _check_counts_near_cut(cnt, ref, ogain, [1] * hp.n, B)
    assert int(cnt.sum()) == min(B, int(lcnt.sum()))
    # the fill of the allocated pattern against the oracle's fill of the same pattern
    sels = fb.sel_lists()
    _, _, _, ologv = oracle.factor_columns(okp, P, sels)
    s = float(fb.sum_logv.cpu()[0])
    assert s == pytest.approx(float(np.sum(ologv)), rel=1e-9)
    even = hp.n * math.log(1 + kp.nugget) - sum(float(g[:8].sum()) for g in ogain)
    print(f"replay {stats}; counts differing at the cut: {nd}; sum log v global {s:.4f} even(8) {even:.4f}")
    assert s < even


def _groups_problem(env, n, seed, n_cand, k, clustered=False):
    torch, sic, pipeline, h = env
    kp = sic.kernel(2, 3, 0.05, 1.0, 1e-6)
    pts = synthetic.clustered_points(n, 2, seed) if clustered else synthetic.points(n, 2, seed)
    return kp, pipeline.prepare_groups(pts, kp, n_cand, k)


def test_groups_global_fp64_matches_oracle(env, oracle_lib):
    """Supernodes of 8-64 members over N = 4096 points, 128 candidates, at most 32 picks, a
    budget of half the nonzeros of 32 picks everywhere; each pick costs its group's size."""
    torch, sic, pipeline, h = env
    oracle = oracle_lib
    from oracle import allocation
    kp, hp = _groups_problem(env, 4096, 1, 128, 32)
    sizes = np.diff(hp.grp_ptr).astype(int)
    B = int(16 * sizes.sum())
    dp = pipeline.DeviceProblem(hp)
    fb = pipeline.FactorBuilder(h, hp, sic.SIC_FP64, budget=B)
    fb.run(dp)
    h.sync()
    okp = _okernel(oracle, kp)
    P, k, G = hp.pts, hp.k, len(sizes)
    cl = [hp.cand_idx[hp.cand_ptr[g]:hp.cand_ptr[g + 1]] for g in range(G)]
    osel, ogain = allocation.group_gains(okp, P, hp.grp_ptr, cl, k)
    sel = fb.sel_idx.view(-1, k).cpu().numpy()
    lcnt = fb.local_count.cpu().numpy()
    gain = fb.gain.view(-1, k).cpu().numpy()
    cnt = fb.sel_count.cpu().numpy()
    stats = ReplayStats()
    same = 0
    for g in range(G):
        picks = sel[g, :lcnt[g]]
        replay_multi(oracle, okp, P, int(hp.grp_ptr[g]), int(sizes[g]), cl[g], k, picks, stats)
        if np.array_equal(picks, osel[g]):
            same += 1
            np.testing.assert_allclose(gain[g, :lcnt[g]], ogain[g], rtol=GAIN_REL, atol=GAIN_ABS, err_msg=str(g))
    assert same >= G - 2
    costs = [int(s) for s in sizes]
    ref = allocation.queue_allocate(ogain, costs, B)
    nd = _check_counts_near_cut(cnt, ref, ogain, costs, B)
    assert int(np.dot(cnt, sizes)) <= B
    print(f"groups {G}: replay {stats}; counts differing at the cut: {nd}; kept {np.dot(cnt, sizes)} of {B}")


def _valid_allocation(gain, lcnt, cnt, sizes, B):
    assert np.all(cnt >= 0) and np.all(cnt <= lcnt)
    assert int(np.dot(cnt, sizes)) <= B
    keys = _running_min_keys([gain[u, :lcnt[u]] for u in range(len(lcnt))])
    kept = [keys[u][cnt[u] - 1] for u in range(len(lcnt)) if cnt[u] > 0]
    dropped = [keys[u][cnt[u]] for u in range(len(lcnt)) if cnt[u] < lcnt[u]]
    if kept and dropped:
        assert min(kept) >= max(dropped)


@pytest.mark.parametrize("clustered", [False, True])
def test_groups_global_fp32_valid_and_close_to_fp64(env, clustered):
    """The register-resident FP32 supernodal path (<= 256 candidates, k <= 64) with
    decreases, at N = 2^16."""
    torch, sic, pipeline, h = env
    kp, hp = _groups_problem(env, 1 << 16, 2, 256, 64, clustered)
    sizes = np.diff(hp.grp_ptr).astype(int)
    B = int(32 * sizes.sum())
    dp = pipeline.DeviceProblem(hp)
    res = {}
    for name, prec, side in [("fp32", sic.SIC_FP32_MIXED, False), ("fp32_side", sic.SIC_FP32_MIXED, True),
                             ("fp64", sic.SIC_FP64, False)]:
        fb = pipeline.FactorBuilder(h, hp, prec, budget=B, side_fp64=side)
        fb.run(dp)
        h.sync()
        gain = fb.gain.view(-1, hp.k).cpu().numpy()
        lcnt, cnt = fb.local_count.cpu().numpy(), fb.sel_count.cpu().numpy()
        _valid_allocation(gain, lcnt, cnt, sizes, B)
        res[name] = float(fb.sum_logv.cpu()[0])
    even = pipeline.FactorBuilder(h, dataclasses.replace(hp, k=32), sic.SIC_FP32_MIXED)
    even.run(dp)
    h.sync()
    s_even = float(even.sum_logv.cpu()[0])
    print(f"clustered={clustered}: sum log v global fp32 {res['fp32']:.3f} fp32 + FP64 side state "
          f"{res['fp32_side']:.3f} fp64 {res['fp64']:.3f} even(32) {s_even:.3f}")
    assert res["fp32_side"] == pytest.approx(res["fp64"], rel=1e-4)
    assert res["fp32"] == pytest.approx(res["fp64"], rel=1e-3)
    assert max(res.values()) < s_even


@pytest.mark.parametrize("clustered,prec_name", [(False, "fp32"), (False, "fp64"), (True, "fp64")])
def test_columns_global_lowers_kl_at_scale(env, clustered, prec_name):
    """N = 2^16 single columns, 64 candidates, at most 32 picks: the global allocation of
    12 N nonzeros gives a lower sum log v (= 2 KL + logdet Theta) than 12 picks everywhere
    (FP32 selection with the decreases from the FP64 side state, and FP64 selection).  Not
    asserted: FP32 selection on the clustered cloud at nugget 1e-8, where the FP32 picks
    themselves go wrong (12 picks everywhere: sum log v 11.5 k above the FP64 selection's)
    and a greedy allocation over their erratic decreases can fall behind the even one."""
    torch, sic, pipeline, h = env
    kp, hp = _columns_problem(env, 1 << 16, 3, 64, 32, clustered)
    dp = pipeline.DeviceProblem(hp)
    B = 12 * hp.n
    prec = sic.SIC_FP32_MIXED if prec_name == "fp32" else sic.SIC_FP64
    own = pipeline.FactorBuilder(h, hp, prec, budget=B)
    own.run(dp)
    h.sync()
    s_own = float(own.sum_logv.cpu()[0])
    fb = pipeline.FactorBuilder(h, hp, prec, budget=B, side_fp64=True)
    fb.run(dp)
    h.sync()
    gain = fb.gain.view(-1, hp.k).cpu().numpy()
    lcnt, cnt = fb.local_count.cpu().numpy(), fb.sel_count.cpu().numpy()
    _valid_allocation(gain, lcnt, cnt, np.ones(hp.n, int), B)
    even = pipeline.FactorBuilder(h, dataclasses.replace(hp, k=12), prec)
    even.run(dp)
    h.sync()
    s_glob, s_even = float(fb.sum_logv.cpu()[0]), float(even.sum_logv.cpu()[0])
    print(f"clustered={clustered} {prec_name}: sum log v global (FP64 side state) {s_glob:.2f}, with the "
          f"selection's decreases {s_own:.2f}, even(12) {s_even:.2f}; "
          f"counts min {cnt.min()} max {cnt.max()}")
    assert s_glob < s_even and s_own < s_even
