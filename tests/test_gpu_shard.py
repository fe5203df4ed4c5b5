"""One factor built in slices on one GPU (each slice as a rank would build it), assembled
by the product's offset scan and placement, against the whole build: bit for bit.

The slices are the ranges of sic_prep_partition; each is built through the same entry
points a rank calls (selection on the slice's units, sic_factor_nnz_range /
sic_build_factor_range into the slice's own arrays, col_ptr again at the whole factor's
offsets).  The assembled col_ptr, row_idx, val, log v, the picks, and the fixed-order sum of
the gathered log v (sic_sum_fixed) must equal the whole build's exactly: every unit's
arithmetic is the same whichever slice it is in.  The slices themselves are checked against
the oracle by the whole build's parity tests.
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
    from paper_2307_11648_gb300 import learned, pipeline, shard, sic
    return torch, sic, pipeline, shard, learned, sic.Handle(0)


def _groups(pipeline, sic, n=1 << 16):
    kp = sic.kernel(2, 3, 0.02 * (2 ** 20 / n) ** 0.5, 1.0, 1e-6)
    return pipeline.prepare_groups(synthetic.points(n, 2, 5), kp, 1024, 64, 8, 64)


def _columns(pipeline, sic, n=20000):
    kp = sic.kernel(3, 5, 0.05 * (65536 / n) ** (1 / 3), 1.0, 1e-6)
    return pipeline.prepare_columns(synthetic.points(n, 3, 6), kp, 256, 32)


CASES = [("groups", "fp32", 2, False), ("groups", "fp32", 3, True), ("groups", "fp64", 2, False),
         ("columns", "fp32", 2, False), ("columns", "fp64", 5, False)]


@pytest.mark.parametrize("kind,prec_name,parts,use_learned", CASES)
def test_slices_match_whole_build(env, kind, prec_name, parts, use_learned):
    torch, sic, pipeline, shard, learned, h = env
    hp = _groups(pipeline, sic) if kind == "groups" else _columns(pipeline, sic)
    prec = sic.SIC_FP64 if prec_name == "fp64" else sic.SIC_FP32_MIXED
    prop = learned.Proposal(h, learned.init_params(0), top=256) if use_learned else None
    dp = pipeline.DeviceProblem(hp)
    whole = learned.LearnedFactorBuilder(h, hp, prop, prec) if use_learned else pipeline.FactorBuilder(h, hp, prec)
    whole.run(dp)
    h.sync()
    wfb = whole.fb if use_learned else whole
    nnz = int(wfb.col_ptr[-1].item())
    builders = [shard.ShardedFactorBuilder(h, hp, prec, r, parts, proposal=prop) for r in range(parts)]
    assert builders[0].u0 == 0 and builders[-1].u1 == hp.n_units
    assert all(b.u1 > b.u0 for b in builders)
    dps = [b.device_problem() for b in builders]
    for b, d in zip(builders, dps):
        b.run(d)
    h.sync()
    arrays, nnz_s, fixed = shard.assemble_local(h, hp, builders, dps)
    h.sync()
    assert nnz_s == nnz
    assert torch.equal(arrays["col_ptr"], wfb.col_ptr)
    assert torch.equal(arrays["row_idx"][:nnz], wfb.row_idx[:nnz])
    assert torch.equal(arrays["val"][:nnz], wfb.val[:nnz])
    assert torch.equal(arrays["logv"], wfb.logv)
    assert float(fixed[0]) == float(wfb.sum_logv[0])
    # the picks of every slice are the whole build's picks of the same units
    k = hp.k
    for b in builders:
        assert torch.equal(b.fb.sel_count, wfb.sel_count[b.u0:b.u1])
        assert torch.equal(b.fb.sel_idx.view(-1, k), wfb.sel_idx.view(-1, k)[b.u0:b.u1])
    # the slices' own sums add up to the whole sum up to rounding order
    s = sum(float(b.fb.sum_logv[0]) for b in builders)
    assert s == pytest.approx(float(wfb.sum_logv[0]), rel=1e-13)
    print(kind, prec_name, parts, "units per slice", [b.u1 - b.u0 for b in builders], "nnz", nnz)
