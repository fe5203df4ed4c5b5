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
