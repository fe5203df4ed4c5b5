"""GPU tests of the learned proposal against the FP64 oracle (oracle/learned.py).

Tolerances: features are computed in FP32 (kernel values with the FP32 exponential), 2e-5; FP32 gradients
without BF16 rounding agree with the FP64 oracle to rel 1e-3 of the largest gradient
entry (FP32 accumulation over the batch); with BF16 rounding (as inference) the stated
BF16 tolerance is a relative L2 error of 3e-2 on the whole gradient; tensor-core scores
agree with the oracle's forward on BF16-rounded inputs and weights to 3e-2 of the
largest |score| (the hidden activations are rounded to BF16 on the way, and inference
evaluates GELU by its tanh form, within 1e-3 of the erf form).
"""
import numpy as np
import pytest

import synthetic
from oracle import learned as OL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_11648_gb300 import build
    build.build()
    from paper_2307_11648_gb300 import learned, pipeline, sic
    return torch, sic, pipeline, learned, sic.Handle(0)


def _bf16(x):
    import torch
    return torch.from_numpy(np.asarray(x, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _small_groups(env, n=4096, seed=11, C=192, k=24):
    torch, sic, pipeline, learned, h = env
    kp = sic.kernel(2, 3, 0.05, 1.0, 1e-6)
    pts = synthetic.points(n, 2, seed)
    return pipeline.prepare_groups(pts, kp, C, k, mmin=4, mmax=32)


def test_features_match_oracle(env, oracle_lib):
    torch, sic, pipeline, learned, h = env
    hp = _small_groups(env)
    dp = pipeline.DeviceProblem(hp)
    rows = int(hp.cand_ptr[-1])
    feat = torch.empty((rows, 8), dtype=torch.float32, device="cuda")
    sic.proposal_features(h, dp.pts, hp.kp, dp.grp_ptr, dp.cand_ptr, dp.cand_idx, feat)
    h.sync()
    F = feat.cpu().numpy()
    okp = oracle_lib.kernel(2, 3, 0.05, 1.0, 1e-6)
    gp = hp.grp_ptr
    for g in range(len(gp) - 1):
        g0, g1 = int(gp[g]), int(gp[g + 1])
        a, b = hp.cand_ptr[g], hp.cand_ptr[g + 1]
        cand = hp.cand_idx[a:b]
        ref = OL.features(okp, hp.pts, g0, g1 - g0, cand)
        # rows whose two nearest members are within FP32 resolution of each other may
        # name a different nearest member: skip their offset features f0, f1
        D = np.sort(np.sqrt(((hp.pts[cand][:, None, :] - hp.pts[g0:g1][None, :, :]) ** 2).sum(-1)), axis=1)
        amb = (D[:, 1] - D[:, 0] <= 1e-5 * D[:, 1]) if g1 - g0 > 1 else np.zeros(len(cand), bool)
        err = np.abs(F[a:b] - ref)
        err[amb, :2] = 0
        assert np.all(err <= 2e-5 * np.maximum(1.0, np.abs(ref))), g
    # the rows are written as 16-byte words: a buffer off that alignment is refused before any launch
    off = torch.empty(rows * 8 + 1, dtype=torch.float32, device="cuda")[1:].view(rows, 8)
    with pytest.raises(sic.SicError):
        sic.proposal_features(h, dp.pts, hp.kp, dp.grp_ptr, dp.cand_ptr, dp.cand_idx, off)


@pytest.mark.parametrize("bf16", [False, True])
def test_grads_and_loss_match_oracle(env, bf16):
    torch, sic, pipeline, learned, h = env
    B = 4096
    X = synthetic.normal(5, B * 8).reshape(B, 8).astype(np.float32)
    y = (synthetic.uniform(6, 3, B) < 0.1).astype(np.float32)
    P = learned.init_params(3)
    P[1024:1152] = 0.05
    P[17536:17664] = -0.02
    P[17792] = -1.0
    g = torch.zeros(P.size, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    ws = sic._ws(sic.mlp_train_workspace(B), "cuda")
    sic.mlp_grads(h, torch.from_numpy(P).cuda(), torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), 2.0, bf16,
                  g, loss, ws)
    h.sync()
    Pr = _bf16(P) if bf16 else P.astype(np.float64)
    Xr = _bf16(X) if bf16 else X.astype(np.float64)
    ref_g = OL.grads(Pr, Xr, y.astype(np.float64), 2.0)
    ref_l = OL.loss(Pr, Xr, y.astype(np.float64), 2.0)
    gg = g.cpu().numpy().astype(np.float64)
    if not bf16:
        assert np.allclose(gg, ref_g, rtol=1e-3, atol=1e-3 * np.abs(ref_g).max())
        assert float(loss.cpu()[0]) == pytest.approx(ref_l, rel=1e-5)
    else:
        rel = np.linalg.norm(gg - ref_g) / np.linalg.norm(ref_g)
        print("bf16 gradient relative L2 error", rel)
        assert rel <= 3e-2
        assert float(loss.cpu()[0]) == pytest.approx(ref_l, rel=1e-2)


@pytest.mark.parametrize("scale", [1.0, 4.0])
def test_tensor_core_scores_match_oracle(env, scale):
    """tcgen05 inference (128-row tiles) against the oracle's forward pass; scale 4 drives
    the hidden pre-activations over |z| ~ 4, where GELU is most nonlinear."""
    torch, sic, pipeline, learned, h = env
    rows = 5000  # not a multiple of 128: ragged last tile
    X = (synthetic.normal(8, rows * 8).reshape(rows, 8) * 0.7 * scale).astype(np.float32)
    P = learned.init_params(4)
    P[1024:1152] = 0.1
    P[1152:17536] *= scale
    P[17792] = 0.3
    s = torch.empty(rows, dtype=torch.float32, device="cuda")
    sic.proposal_score(h, torch.from_numpy(P).cuda(), torch.from_numpy(X).cuda(), s)
    h.sync()
    ref, _ = OL.forward(_bf16(P), _bf16(X))
    err = np.abs(s.cpu().numpy() - ref).max()
    print("tensor-core score max error", err, "max |s|", np.abs(ref).max(), "scale", scale)
    assert err <= 3e-2 * np.abs(ref).max()


def test_topk_and_labels_exact(env):
    torch, sic, pipeline, learned, h = env
    rng = np.random.default_rng(1)
    counts = np.array([0, 5, 256, 257, 300, 1024, 1000, 77, 4096])
    ptr = np.zeros(len(counts) + 1, np.int64)
    ptr[1:] = np.cumsum(counts)
    idx = rng.integers(0, 10 ** 6, ptr[-1]).astype(np.int32)
    score = np.round(synthetic.uniform(2, 4, ptr[-1]) * 50).astype(np.float32)  # many exact ties
    top = 256
    out_ptr = torch.empty(len(counts) + 1, dtype=torch.int64, device="cuda")
    out_idx = torch.empty(len(counts) * top, dtype=torch.int32, device="cuda")
    sic.proposal_topk(h, torch.from_numpy(ptr).cuda(), torch.from_numpy(idx).cuda(), torch.from_numpy(score).cuda(),
                      top, out_ptr, out_idx)
    h.sync()
    op = out_ptr.cpu().numpy()
    oi = out_idx.cpu().numpy()
    for g in range(len(counts)):
        a, b = ptr[g], ptr[g + 1]
        r = np.arange(b - a)
        keep = np.sort(np.lexsort((r, -score[a:b]))[:top])
        assert oi[op[g]:op[g + 1]].tolist() == idx[a:b][keep].tolist(), g
    # labels from a selection
    k = 6
    sel = np.full(len(counts) * k, -1, np.int32)
    cnt = np.zeros(len(counts), np.int32)
    for g in range(len(counts)):
        a, b = ptr[g], ptr[g + 1]
        take = idx[a:b][:: max(1, (b - a) // 4)][:k] if b > a else []
        sel[g * k:g * k + len(take)] = take
        cnt[g] = len(take)
    lab = torch.empty(ptr[-1], dtype=torch.float32, device="cuda")
    sic.proposal_labels(h, torch.from_numpy(ptr).cuda(), torch.from_numpy(idx).cuda(), torch.from_numpy(sel).cuda(),
                        torch.from_numpy(cnt).cuda(), k, lab)
    h.sync()
    L = lab.cpu().numpy()
    for g in range(len(counts)):
        a, b = ptr[g], ptr[g + 1]
        want = np.isin(idx[a:b], sel[g * k:g * k + cnt[g]]).astype(np.float32)
        assert np.array_equal(L[a:b], want)


def test_adamw_matches_oracle(env):
    torch, sic, pipeline, learned, h = env
    n = 1000
    p = synthetic.normal(1, n).astype(np.float32)
    gr = synthetic.normal(2, n).astype(np.float32) * 0.1
    P = torch.from_numpy(p.copy()).cuda()
    m = torch.zeros(n, device="cuda")
    v = torch.zeros(n, device="cuda")
    G = torch.from_numpy(gr).cuda()
    rp, rm, rv = p.astype(np.float64), np.zeros(n), np.zeros(n)
    for step in range(1, 4):
        sic.adamw_step(h, P, m, v, G, step, 1e-2, wd=1e-3)
        rp, rm, rv = OL.adamw_step(rp, rm, rv, gr.astype(np.float64), step, 1e-2, wd=1e-3)
    h.sync()
    assert np.allclose(P.cpu().numpy(), rp, rtol=1e-5, atol=1e-6)


def test_learned_proposal_gain(env):
    """Train on plain-greedy labels of two problems (seeds 1, 2), evaluate on seed 0 (the
    config-3 geometry scaled to N = 2^16: ell = 0.08 keeps ell / spacing as at 2^20; C =
    1024, k = 64, supernodes 8..64).  Reports the recall of the plain picks inside the 256
    kept candidates for the network and for plain distance order, and the KL gap
    (S_A - S_plain) / (S_plain - S_ref) with S = sum log v and a 2k-pick reference."""
    torch, sic, pipeline, learned, h = env
    import math
    n = 1 << 16
    kp = sic.kernel(2, 3, 0.02 * math.sqrt((1 << 20) / n), 1.0, 1e-6)

    def prob(seed, k=64):
        return pipeline.prepare_groups(synthetic.points(n, 2, seed), kp, 1024, k, 8, 64)

    train_probs = [prob(1), prob(2)]
    feat, label, n_sel = learned.training_set(h, train_probs)
    P, hist = learned.train(h, feat, label, epochs=3, batch=65536, lr=2e-3)
    print("training selections", n_sel, "loss", hist[0], "->", hist[-1])
    assert hist[-1][1] < hist[0][1]
    hp = prob(0)
    dp = pipeline.DeviceProblem(hp)
    res = {}
    for name, prec in [("plain64", sic.SIC_FP64), ("plain32", sic.SIC_FP32_MIXED)]:
        fb = pipeline.FactorBuilder(h, hp, prec)
        fb.run(dp)
        h.sync()
        res[name] = float(fb.sum_logv.cpu()[0])
        if name == "plain32":
            plain_sel = fb.sel_lists()
    ref_hp = pipeline.HostProblem(hp.pts, hp.kp, 128, hp.cand_ptr, hp.cand_idx, hp.grp_ptr, hp.order, hp.ell2)
    fr = pipeline.FactorBuilder(h, ref_hp, sic.SIC_FP32_MIXED)
    fr.run(dp)
    h.sync()
    res["ref"] = float(fr.sum_logv.cpu()[0])
    del fr
    prop = learned.Proposal(h, P, top=256)
    lb = learned.LearnedFactorBuilder(h, hp, prop)
    lb.run(dp)
    h.sync()
    res["learned"] = float(lb.sum_logv.cpu()[0])
    # distance baseline: the first 256 of each list
    cnt = np.minimum(np.diff(hp.cand_ptr), 256)
    dptr = np.zeros(len(cnt) + 1, np.int64)
    dptr[1:] = np.cumsum(cnt)
    didx = np.concatenate([hp.cand_idx[hp.cand_ptr[g]:hp.cand_ptr[g] + cnt[g]] for g in range(len(cnt))])
    dhp = pipeline.HostProblem(hp.pts, hp.kp, hp.k, dptr, didx, hp.grp_ptr, hp.order, hp.ell2)
    fd = pipeline.FactorBuilder(h, dhp, sic.SIC_FP32_MIXED)
    fd.run(pipeline.DeviceProblem(dhp))
    h.sync()
    res["distance"] = float(fd.sum_logv.cpu()[0])
    # recall of plain picks inside the kept lists
    op = lb.buf["out_ptr"].cpu().numpy()
    oi = lb.buf["out_idx"].cpu().numpy()
    hit_mlp = hit_dist = tot = 0
    for g in range(len(cnt)):
        picks = set(plain_sel[g].tolist())
        tot += len(picks)
        hit_mlp += len(picks & set(oi[op[g]:op[g + 1]].tolist()))
        hit_dist += len(picks & set(didx[dptr[g]:dptr[g + 1]].tolist()))
    base = res["plain64"] - res["ref"]
    gaps = {k: (res[k] - res["plain64"]) / base for k in ["plain32", "learned", "distance"]}
    print("sum log v", res, "KL gaps", gaps, f"recall mlp {hit_mlp / tot:.5f} distance {hit_dist / tot:.5f}")
    assert base > 0
    assert gaps["learned"] <= 0.01          # KL within 1% of plain greedy
    assert hit_mlp / tot >= 0.99


def _distance_problem(pipeline, hp, top):
    cnt = np.minimum(np.diff(hp.cand_ptr), top)
    ptr = np.zeros(len(cnt) + 1, np.int64)
    ptr[1:] = np.cumsum(cnt)
    idx = np.concatenate([hp.cand_idx[hp.cand_ptr[g]:hp.cand_ptr[g] + cnt[g]] for g in range(len(cnt))])
    return pipeline.HostProblem(hp.pts, hp.kp, hp.k, ptr, idx, hp.grp_ptr, hp.order, hp.ell2)


def test_learned_beats_distance_on_clustered_cloud(env):
    """Where the network earns its place: on an inhomogeneous cloud (half of the points crowded
    into a square of side 0.05, synthetic.clustered_points) the plain greedy's picks are not
    simply the nearest candidates, and at equal `top` the learned proposal keeps far more of
    what the plain greedy would pick than distance order does.  Config-3 kernel with ell
    scaled to N = 2^16, C = 1024, k = 64, supernodes 8..64; trained on two clustered clouds of
    other seeds; evaluated on seed 0 at top = 128 and 256.  Asserted: the learned KL gap is
    below the distance truncation's at both (measured at N = 2^18: 12.5 % against 32.7 % at
    128, 8.6 % against 18.7 % at 256 of the 2k-pick proxy)."""
    torch, sic, pipeline, learned, h = env
    import math
    n = 1 << 16
    kp = sic.kernel(2, 3, 0.02 * math.sqrt((1 << 20) / n), 1.0, 1e-6)

    def prob(seed, k=64):
        return pipeline.prepare_groups(synthetic.clustered_points(n, 2, seed), kp, 1024, k, 8, 64)

    feat, label, _ = learned.training_set(h, [prob(1), prob(2)])
    P, hist = learned.train(h, feat, label, epochs=3, batch=65536, lr=2e-3)
    del feat, label
    hp = prob(0)
    dp = pipeline.DeviceProblem(hp)
    S = {}

    def run(name, b, d=dp):
        b.run(d)
        h.sync()
        S[name] = float(b.sum_logv.cpu()[0])

    run("plain64", pipeline.FactorBuilder(h, hp, sic.SIC_FP64))
    run("ref", pipeline.FactorBuilder(h, pipeline.HostProblem(hp.pts, hp.kp, 128, hp.cand_ptr, hp.cand_idx,
                                                              hp.grp_ptr, hp.order, hp.ell2), sic.SIC_FP32_MIXED))
    gaps = {}
    for top in (128, 256):
        run(f"learned{top}", learned.LearnedFactorBuilder(h, hp, learned.Proposal(h, P, top=top)))
        dhp = _distance_problem(pipeline, hp, top)
        run(f"distance{top}", pipeline.FactorBuilder(h, dhp, sic.SIC_FP32_MIXED), pipeline.DeviceProblem(dhp))
        base = S["plain64"] - S["ref"]
        gaps[top] = ((S[f"learned{top}"] - S["plain64"]) / base, (S[f"distance{top}"] - S["plain64"]) / base)
    print("clustered: KL gaps (learned, distance) per top", gaps)
    for top, (gl, gd) in gaps.items():
        assert gl < gd, (top, gl, gd)


def test_training_checkpoint_resume(env, tmp_path):
    """Training interrupted after epoch 0 and resumed from its checkpoint ends with the same
    weights as an uninterrupted run (the kernels and the data order are deterministic)."""
    torch, sic, pipeline, learned, h = env
    B = 8192
    X = torch.from_numpy((synthetic.normal(11, 4 * B * 8).reshape(4 * B, 8) * 0.5).astype(np.float32)).cuda()
    y = torch.from_numpy((synthetic.uniform(12, 3, 4 * B) < 0.1).astype(np.float32)).cuda()
    full, _ = learned.train(h, X, y, epochs=2, batch=B, seed=5)
    ck = str(tmp_path / "proposal.pt")
    learned.train(h, X, y, epochs=2, batch=B, seed=5, checkpoint=ck, stop_after_epoch=0)
    resumed, _ = learned.train(h, X, y, epochs=2, batch=B, seed=5, checkpoint=ck)
    assert torch.equal(full, resumed)


def test_bounded_wait_reports_timeout(env):
    """A device wait that nothing satisfies gives up after its cap and reports
    SIC_ERR_TIMEOUT through sic_sync; the context stays usable afterwards."""
    torch, sic, pipeline, learned, h = env
    out = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    sic.selftest_wait_timeout(h, 1000, out)
    with pytest.raises(sic.SicError) as e:
        h.sync()
    assert e.value.code == sic.SIC_ERR_TIMEOUT and int(out.item()) == 0
    x = torch.ones(4, device="cuda")
    assert float((x * 2).sum().item()) == 8.0  # the context still works


def test_learned_step_in_cuda_graph(env):
    """The whole learned step (features, tensor-core scores, top-k, selection, nnz, fill,
    sum) captured in one CUDA graph replays to the eager result bit for bit."""
    torch, sic, pipeline, learned, h = env
    cfg = synthetic.PRESETS["cfg3_aggregated"]
    kp = sic.kernel(cfg["dim"], cfg["nu_x2"], cfg["length_scale"], cfg["variance"], cfg["nugget"])
    hp = pipeline.prepare_groups(synthetic.points(1 << 14, 2, 21), kp, 1024, 64, 8, 64)
    dp = pipeline.DeviceProblem(hp)
    lb = learned.LearnedFactorBuilder(h, hp, learned.Proposal(h, learned.init_params(3), top=256))
    lb.run(dp)
    h.sync()
    ref = [t.clone() for t in (lb.fb.sel_idx, lb.fb.sel_count, lb.fb.col_ptr, lb.fb.val, lb.fb.sum_logv)]
    for t in (lb.fb.sel_idx, lb.fb.val, lb.fb.sum_logv):
        t.zero_()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        lb.run(dp)
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        lb.run(dp)
    for t in (lb.fb.sel_idx, lb.fb.val, lb.fb.sum_logv):
        t.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    h.sync()
    nnz = int(ref[2][-1])
    got = (lb.fb.sel_idx, lb.fb.sel_count, lb.fb.col_ptr, lb.fb.val, lb.fb.sum_logv)
    for a, b in zip(ref[:3], got[:3]):
        assert torch.equal(a, b)
    assert torch.equal(ref[3][:nnz], got[3][:nnz])
    assert torch.equal(ref[4], got[4])


def test_guarded_build_falls_back_to_plain_greedy(env):
    """The plain greedy judges the learned path and replaces it when the KL gap exceeds the
    threshold: an untrained network keeping only 32 of 256 candidates is far off (large
    gap) and falls back; with a threshold above its measured gap the learned factor is kept.
    Either way the chosen factor is that builder's own output."""
    torch, sic, pipeline, learned, h = env
    kp = sic.kernel(2, 3, 0.05, 1.0, 1e-6)
    hp = pipeline.prepare_groups(synthetic.points(1 << 14, 2, 5), kp, 256, 16, 8, 32)
    dp = pipeline.DeviceProblem(hp)
    prop = learned.Proposal(h, learned.init_params(0), top=2 * hp.k)
    g = learned.GuardedBuild(h, hp, prop, max_gap=0.01)
    chosen = g.run(dp)
    print("untrained proposal KL gap", g.gap)
    assert g.gap > 0.01 and not g.use_learned and chosen is g.plain
    g2 = learned.GuardedBuild(h, hp, prop, max_gap=g.gap * 2 + 1.0)
    chosen2 = g2.run(dp)
    assert g2.use_learned and chosen2 is g2.learned.fb
    assert g2.gap == pytest.approx(g.gap, rel=1e-12)
    assert torch.equal(chosen2.val, g2.learned.fb.val)
