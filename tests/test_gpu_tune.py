"""GPU autotuning of the fill's launch split (sic_tune_build_factor, sic_tune_save/load).

The split only decides which launch fills which groups, and the worker count how many warps
share a group's work; every entry is computed by the same operations in the same order
either way, so the tuned fill must be bit-identical to the default one.
"""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_11648_gb300 import build
    build.build()
    from paper_2307_11648_gb300 import pipeline, sic
    return torch, sic, pipeline


def test_tuned_fill_is_identical_and_persists(env, tmp_path):
    torch, sic, pipeline = env
    h = sic.Handle(0)
    kp = sic.kernel(2, 3, 0.02, 1.0, 1e-6)
    hp = pipeline.prepare_groups(synthetic.points(1 << 16, 2, 3), kp, 256, 64)
    dp = pipeline.DeviceProblem(hp)
    fb = pipeline.FactorBuilder(h, hp, sic.SIC_FP32_MIXED)
    fb.run(dp)
    h.sync()
    ref = [t.clone() for t in (fb.col_ptr, fb.row_idx, fb.val, fb.logv, fb.sum_logv)]
    split = fb.tune(dp)
    h.sync()
    assert 1 <= split <= hp.max_m
    for a, b in zip(ref, (fb.col_ptr, fb.row_idx, fb.val, fb.logv, fb.sum_logv)):
        assert torch.equal(a, b)
    table = sic.tune_table(h)
    ops = {op: (a, b, v, ms) for op, a, b, v, ms in table}
    assert ops[1][:3] == (hp.k, hp.max_m, split) and ops[1][3] > 0.0
    assert ops[2][:2] == (hp.k, hp.max_m) and ops[2][2] in (256, 384)
    fb.fill(dp)  # later fills use the tuned split
    h.sync()
    assert torch.equal(ref[2], fb.val)
    path = tmp_path / "tune.txt"
    sic.tune_save(h, path)
    h2 = sic.Handle(0)
    sic.tune_load(h2, path)
    t2 = sic.tune_table(h2)
    assert [e[:4] for e in t2] == [e[:4] for e in table]
    assert [e[4] for e in t2] == pytest.approx([e[4] for e in table], abs=1e-5)
    # a malformed line is reported, the valid ones still load
    bad = tmp_path / "bad.txt"
    bad.write_text(path.read_text() + "1 2 three\n")
    h3 = sic.Handle(0)
    with pytest.raises(sic.SicError):
        sic.tune_load(h3, bad)
    assert [e[:4] for e in sic.tune_table(h3)] == [e[:4] for e in table]
    print("tuned split", split, "table", table)


SELECT_CASES = [  # (precision, candidates, k, largest group): which kernel and plans are tuned
    ("fp32", 100, 32, 16),   # register-resident kernel: 128 or 256 threads
    ("fp32", 200, 80, 16),   # generic kernel, state fits in shared memory: 256/512 threads x smem/workspace
    ("fp32", 400, 32, 32),   # generic kernel, 512 candidates bucket: 256/512 threads, workspace
    ("fp64", 192, 24, 32),   # generic FP64 kernel
]


@pytest.mark.parametrize("prec_name,n_cand,k,mmax", SELECT_CASES)
def test_tuned_selection_plan_gives_the_same_picks(env, tmp_path, prec_name, n_cand, k, mmax):
    """sic_tune_select_aggregated times every launch plan that gives the same picks (threads
    per CTA; shared memory or workspace) and keeps the fastest; the picks before tuning,
    during it (the final run) and after it (a later call with the tuned plan) are identical,
    and the choice survives sic_tune_save / sic_tune_load."""
    torch, sic, pipeline = env
    h = sic.Handle(0)
    kp = sic.kernel(2, 3, 0.05, 1.0, 1e-6)
    hp = pipeline.prepare_groups(synthetic.points(8192, 2, 13), kp, n_cand, k, mmin=4, mmax=mmax)
    dp = pipeline.DeviceProblem(hp)
    prec = sic.SIC_FP64 if prec_name == "fp64" else sic.SIC_FP32_MIXED
    U = hp.n_units
    ws = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")  # room for every workspace plan

    def select():
        si = torch.full((U * k,), -7, dtype=torch.int32, device="cuda")
        sc = torch.full((U,), -7, dtype=torch.int32, device="cuda")
        sic.select_aggregated(h, dp.pts, kp, dp.grp_ptr, dp.cand_ptr, dp.cand_idx, hp.max_cand, hp.max_m, k, prec,
                              si, sc, ws)
        h.sync()
        return si, sc

    si0, sc0 = select()
    si1 = torch.full_like(si0, -7)
    sc1 = torch.full_like(sc0, -7)
    choice = sic.tune_select_aggregated(h, dp.pts, kp, dp.grp_ptr, dp.cand_ptr, dp.cand_idx, hp.max_cand, hp.max_m,
                                        k, prec, si1, sc1, ws)
    h.sync()
    si2, sc2 = select()
    for si, sc in ((si1, sc1), (si2, sc2)):
        assert torch.equal(sc, sc0) and torch.equal(si, si0)
    table = [e for e in sic.tune_table(h) if e[0] == 3]
    assert len(table) == 1 and table[0][3] == choice
    assert table[0][1] == k + 256 * prec and table[0][2] == 128 * hp.max_cand + hp.max_m
    if prec_name == "fp32" and n_cand <= 128:
        assert choice in (128, 256)
    else:
        assert choice // 2 in (256, 512)
    path = tmp_path / "tune.txt"
    sic.tune_save(h, path)
    h2 = sic.Handle(0)
    sic.tune_load(h2, path)
    assert [e[:4] for e in sic.tune_table(h2)] == [e[:4] for e in sic.tune_table(h)]
    print(prec_name, n_cand, k, mmax, "plan", choice, "ms", table[0][4])
