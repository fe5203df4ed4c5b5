"""GPU partial selection for nonadjacent groups (Section 5.2, Appendix C.3) against the oracle.

Tolerances follow the parity tests (tests/parity.py): FP64 picks identical except at
near-ties of the oracle's decreases within 1e-10 relative (oracle replay); an FP32 pick
within 1e-3 relative of the oracle's best decrease plus the FP32 resolution of the two
picks' decreases, 2 E m (1/v_b + 1/v_c) with E as in tests/parity.py over the members' and the earlier
picks' pivot variances and v the pick's variance
given the members and earlier picks (each of the up to m member terms of the decrease is
a log-ratio of FP32 variances no smaller than v); the decreases of agreeing FP64 picks to
1e-9 relative plus 1e-12; the fill of the resulting pattern as in the parity tests (rows
identical, values 1e-8 of the column's largest, log v to 1e-9).
"""
import dataclasses

import numpy as np
import pytest

import synthetic
from parity import E32, REL32, TIE_BAND, ReplayStats, _replay, column_errors

pytestmark = pytest.mark.gpu

# (fraction of replayed steps that differ, worst decrease gap in nats) per precision
CAPS = {"fp64": (1e-3, 1e-9), "fp32": (0.02, 1e-3)}


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


def _problem(env, n, seed, n_cand, k, mmin=4, mmax=16):
    torch, sic, pipeline, h = env
    kp = sic.kernel(2, 3, 0.1, 1.0, 1e-6)
    return kp, pipeline.prepare_partial(synthetic.points(n, 2, seed), kp, n_cand, k, mmin, mmax)


def _var_given(oracle, okp, P, cond, j):
    """Variance of point j given the positions cond (dense FP64 solve)."""
    cond = [int(x) for x in cond]
    K = oracle.theta_matrix(okp, P, cond + [int(j)])
    c = len(cond)
    return float(K[c, c] - (K[:c, c] @ np.linalg.solve(K[:c, :c], K[:c, c]) if c else 0.0))


def _replay_partial(oracle, okp, hp, g, gpu_sel, stats, fp32):
    from oracle import partial
    mem = hp.members[hp.grp_ptr[g]:hp.grp_ptr[g + 1]]
    cand = hp.cand_idx[hp.cand_ptr[g]:hp.cand_ptr[g + 1]]
    def run(forced):
        return partial.select_partial(okp, hp.pts, mem, cand, hp.k, forced=forced if forced else None)

    def accept(j, r2, b, c, prefix):
        best, chosen = float(r2["best"][j]), float(r2["chosen"][j])
        gap = max(0.0, best - chosen)
        if not fp32:
            return best - chosen <= TIE_BAND * abs(best), gap, 0.0
        piv = oracle.pivot_variances(okp, hp.pts, [], list(mem) + list(prefix))[0]
        E = E32 * okp.variance * (1.0 + float(np.sum(np.sqrt(okp.variance / np.maximum(piv, 1e-300)))))
        vb = _var_given(oracle, okp, hp.pts, list(mem) + list(prefix), b)
        vc = _var_given(oracle, okp, hp.pts, list(mem) + list(prefix), c)
        delta = 2 * E * len(mem) * (1 / max(vb, 1e-300) + 1 / max(vc, 1e-300))
        return gap <= REL32 * best + delta, gap, delta

    _replay(run, gpu_sel, cand, stats, f"group {g}", accept)


@pytest.mark.parametrize("prec_name", ["fp64", "fp32"])
def test_partial_selection_matches_oracle(env, oracle_lib, prec_name):
    """N = 4096, groups of 4-16 members kept where the ordering puts them, 48 candidates
    (some between members), up to 12 picks; a sample of groups replayed by the oracle."""
    torch, sic, pipeline, h = env
    oracle = oracle_lib
    from oracle import partial
    kp, hp = _problem(env, 4096, 5, 48, 12)
    prec = sic.SIC_FP64 if prec_name == "fp64" else sic.SIC_FP32_MIXED
    dp = pipeline.DeviceProblem(hp)
    fb = pipeline.PartialFactorBuilder(h, hp, prec)
    fb.select(dp)
    h.sync()
    sels = fb.sel_lists()
    gain = fb.gain.view(-1, hp.k).cpu().numpy()
    okp = _okernel(oracle, kp)
    G = hp.n_units
    between = sum(int(any(hp.members[hp.grp_ptr[g]] < q < hp.members[hp.grp_ptr[g + 1] - 1] for q in sels[g]))
                  for g in range(G))
    assert between > 0  # picks between members: the case partial selection exists for
    stats = ReplayStats()
    same = 0
    sample = range(0, G, max(1, G // 40))
    for g in sample:
        _replay_partial(oracle, okp, hp, g, sels[g], stats, prec_name == "fp32")
        if prec_name == "fp64":
            mem = hp.members[hp.grp_ptr[g]:hp.grp_ptr[g + 1]]
            r = partial.select_partial(okp, hp.pts, mem, hp.cand_idx[hp.cand_ptr[g]:hp.cand_ptr[g + 1]], hp.k)
            if np.array_equal(r["sel"], sels[g]):
                same += 1
                ncond = [sum(int(i < q) for i in mem) for q in r["sel"]]
                np.testing.assert_allclose(gain[g, :len(sels[g])], r["decrease"] / np.maximum(ncond, 1),
                                           rtol=1e-9, atol=1e-12, err_msg=str(g))
    print(prec_name, f"groups {G}, with picks between members {between}; replay {stats}")
    stats.check(*CAPS[prec_name])
    if prec_name == "fp64":
        assert same >= len(sample) - 2


@pytest.mark.parametrize("per_column", [False, True])
def test_partial_fill_matches_oracle(env, oracle_lib, per_column):
    """The pattern of a partial selection (member i: later members + picks after i) filled in
    FP64 -- aggregated per group (one LDL^T of the group's members and picks) and column by
    column from the expanded lists -- against the oracle's dense per-column fill."""
    torch, sic, pipeline, h = env
    oracle = oracle_lib
    kp, hp = _problem(env, 4096, 6, 48, 12)
    dp = pipeline.DeviceProblem(hp)
    fb = pipeline.PartialFactorBuilder(h, hp, sic.SIC_FP64, per_column=per_column)
    fb.run(dp)
    h.sync()
    okp = _okernel(oracle, kp)
    sels = fb.sel_lists()
    cp = fb.col_ptr.cpu().numpy()
    nnz = int(cp[-1])
    ri, val, logv = fb.row_idx[:nnz].cpu().numpy(), fb.val[:nnz].cpu().numpy(), fb.logv.cpu().numpy()
    col = {}
    for g in range(hp.n_units):
        mem = hp.members[hp.grp_ptr[g]:hp.grp_ptr[g + 1]].tolist()
        for a, i in enumerate(mem):
            col[i] = mem[a + 1:] + [int(q) for q in sels[g] if q > i]
    assert sorted(col) == list(range(hp.n))
    worst = 0.0
    for i in range(0, hp.n, 7):
        rows, L, lv = oracle.fill_column(okp, hp.pts, i, col[i])
        a, b = cp[i], cp[i + 1]
        assert ri[a:b].tolist() == rows.tolist(), i
        e = column_errors(val[a:b], L)
        worst = max(worst, e)
        assert e <= 1e-8, (i, e)
        assert abs(logv[i] - lv) <= 1e-9, i
    assert nnz == sum(1 + len(v) for v in col.values())
    _, _, _, ologv = oracle.factor_columns(okp, hp.pts, [np.array(col[i], np.int32) for i in range(hp.n)])
    assert float(fb.sum_logv.cpu()[0]) == pytest.approx(float(ologv.sum()), rel=1e-9)
    print(f"fill (per column {per_column}): nnz {nnz}, worst column error {worst:.2e}")


def test_partial_beats_candidates_after_the_group(env):
    """The paper's observation behind partial selection: with the groups where the ordering
    puts them, forcing every candidate to lie after the whole group (so that the
    multiple-target selection applies) drops the candidates between members and gives a
    higher KL than partial selection over all of them -- here with fewer nonzeros, too.
    Renumbering the groups to be consecutive (this library's supernodal path) is reported
    beside them.  sum log v differences are 2 KL differences (logdet Theta does not depend on
    the ordering).  N = 2^16, k = 32, 128 candidates, groups of 8-32."""
    torch, sic, pipeline, h = env
    kp = sic.kernel(2, 3, 0.05, 1.0, 1e-6)
    pts = synthetic.points(1 << 16, 2, 9)
    k, C = 32, 128
    hp = pipeline.prepare_partial(pts, kp, C, k, 8, 32)
    ptr, idx = [0], []
    for g in range(hp.n_units):
        last = hp.members[hp.grp_ptr[g + 1] - 1]
        idx += [int(j) for j in hp.cand_idx[hp.cand_ptr[g]:hp.cand_ptr[g + 1]] if j > last]
        ptr.append(len(idx))
    hp_after = dataclasses.replace(hp, cand_ptr=np.array(ptr, np.int64), cand_idx=np.array(idx, np.int32))
    hp_renum = pipeline.prepare_groups(pts, kp, C, k, 8, 32)
    res = {}
    for name, p, B in [("partial", hp, pipeline.PartialFactorBuilder),
                       ("after_the_group", hp_after, pipeline.PartialFactorBuilder),
                       ("renumbered", hp_renum, pipeline.FactorBuilder)]:
        dp = pipeline.DeviceProblem(p)
        fb = B(h, p, sic.SIC_FP32_MIXED)
        fb.run(dp)
        h.sync()
        res[name] = (float(fb.sum_logv.cpu()[0]), int(fb.col_ptr[-1].item()))
    print("sum log v, nnz:", res)
    assert res["partial"][0] < res["after_the_group"][0] - 100.0
    assert res["partial"][1] <= res["after_the_group"][1]


def test_partial_errors_reported(env):
    torch, sic, pipeline, h = env
    kp, hp = _problem(env, 600, 7, 24, 8)
    dp = pipeline.DeviceProblem(hp)
    bad = dp.cand_idx.clone()
    g0 = int(hp.members[hp.grp_ptr[1]])
    bad[int(hp.cand_ptr[1])] = g0  # a candidate at the group's first member
    fb = pipeline.PartialFactorBuilder(h, hp, sic.SIC_FP64)
    sic.select_partial(h, dp.pts, kp, dp.grp_ptr, dp.members, dp.cand_ptr, bad, hp.max_cand, hp.max_m, hp.k,
                       sic.SIC_FP64, fb.sel_idx, fb.sel_count)
    with pytest.raises(sic.SicError):
        h.sync()
    with pytest.raises(sic.SicError):  # the factor cannot fit in shared memory
        sic.select_partial(h, dp.pts, kp, dp.grp_ptr, dp.members, dp.cand_ptr, dp.cand_idx, 4000, hp.max_m, hp.k,
                           sic.SIC_FP64, fb.sel_idx, fb.sel_count)
    fb.run(dp)
    h.sync()


def test_partial_no_groups(env):
    torch, sic, pipeline, h = env
    kp = sic.kernel(2, 3, 0.1, 1.0, 1e-6)
    pts = torch.from_numpy(synthetic.points(50, 2, 1)).cuda()
    gp = torch.zeros(1, dtype=torch.int64, device="cuda")
    z32 = torch.zeros(1, dtype=torch.int32, device="cuda")
    sic.select_partial(h, pts, kp, gp, gp, gp, z32, 8, 4, 4, sic.SIC_FP32_MIXED, z32, z32)
    h.sync()


def test_partial_full_size_sampled(env, oracle_lib):
    """The bench's partial-selection configuration: N = 2^18, groups of 8-64 kept where the
    ordering puts them, 256 candidates, k = 64, FP32; sampled groups replayed by the oracle
    (bands of the FP32 parity tests), the fill's sum of log v finite."""
    torch, sic, pipeline, h = env
    oracle = oracle_lib
    cfg = synthetic.PRESETS["cfg3_aggregated"]
    kp = sic.kernel(cfg["dim"], cfg["nu_x2"], cfg["length_scale"], cfg["variance"], cfg["nugget"])
    hp = pipeline.prepare_partial(synthetic.points(1 << 18, 2, cfg["seed"]), kp, 256, cfg["k"], cfg["m_min"],
                                  cfg["m_max"])
    dp = pipeline.DeviceProblem(hp)
    fb = pipeline.PartialFactorBuilder(h, hp, sic.SIC_FP32_MIXED)
    fb.run(dp)
    h.sync()
    sels = fb.sel_lists()
    okp = _okernel(oracle, kp)
    G = hp.n_units
    rng = np.random.default_rng(3)
    groups = sorted(set(rng.choice(G, 3, replace=False).tolist()) | {G - 1})
    stats = ReplayStats()
    for g in groups:
        _replay_partial(oracle, okp, hp, g, sels[g], stats, True)
    s = float(fb.sum_logv.cpu()[0])
    assert np.isfinite(s)
    print(f"partial full size: groups {G}, replay {stats}, sum log v {s:.1f}")
    stats.check(*CAPS["fp32"])
