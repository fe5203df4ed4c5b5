"""CPU tests of one factor built in slices (Section 4: units are independent), without a GPU.

* sic_prep_partition (host code of libsic): contiguous, complete, and every part's cost
  within one unit's cost of the even share, under the cost model stated in include/sic.h
  (restated here from that statement);
* the gather over two gloo ranks: each rank's slice comes from the oracle (selection and
  dense fill of its units), the product's count exchange, offset scan and broadcasts
  assemble the whole factor, which must equal the oracle's one-piece factor exactly, with
  the all-reduced sum of log v equal to the slices' sums added.
"""
import os
import socket

import numpy as np
import pytest

import synthetic


@pytest.fixture(scope="module")
def sic():
    from paper_2307_11648_gb300 import build, sic as s
    build.build()
    return s


def _cost(cand_ptr, grp_ptr, k, max_cand):
    c = np.diff(cand_ptr).astype(np.float64)
    if max_cand > 0:
        c = np.minimum(c, max_cand)
    m = np.diff(grp_ptr).astype(np.float64) if grp_ptr is not None else np.ones_like(c)
    nn = k + m
    return c * (k * k + k * m + 0.5 * m * m) + 13.0 * (nn ** 3 / 6.0 + 0.5 * m * nn * nn)


@pytest.mark.parametrize("parts", [1, 2, 3, 8, 64])
@pytest.mark.parametrize("grouped", [False, True])
def test_partition_balanced_and_complete(sic, parts, grouped):
    rng = np.random.default_rng(parts)
    U = 5000
    cnt = rng.integers(0, 1025, U)
    cp = np.zeros(U + 1, np.int64)
    cp[1:] = np.cumsum(cnt)
    gp = None
    if grouped:
        gp = np.zeros(U + 1, np.int64)
        gp[1:] = np.cumsum(rng.integers(1, 65, U))
    for max_cand in (0, 256):
        b = sic.prep_partition(cp, gp, 64, parts, max_cand)
        assert b[0] == 0 and b[-1] == U and np.all(np.diff(b) >= 0)
        w = _cost(cp, gp, 64, max_cand)
        share = w.sum() / parts
        for r in range(parts):
            part = w[b[r]:b[r + 1]].sum()
            assert abs(part - share) <= w.max() * (1 + 1e-12), (r, part, share, w.max())


def test_partition_more_parts_than_units(sic):
    cp = np.array([0, 10, 20, 30], np.int64)
    b = sic.prep_partition(cp, None, 8, 6)
    assert b[0] == 0 and b[-1] == 3 and np.all(np.diff(b) >= 0)
    assert sorted(set(b.tolist())) == [0, 1, 2, 3]  # every unit in exactly one part


def test_rank_offsets():
    from paper_2307_11648_gb300 import shard
    assert shard.rank_offsets([5, 0, 7, 1]) == [0, 5, 5, 12]
    assert shard.rank_offsets([]) == []


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _problem():
    from paper_2307_11648_gb300 import pipeline, sic
    kp = sic.kernel(2, 3, 0.1, 1.0, 1e-6)
    return pipeline.prepare_groups(synthetic.points(600, 2, 3), kp, 48, 8, mmin=2, mmax=16)


def _oracle_slice(hp, u0, u1):
    """Selection and dense fill of units u0 .. u1-1 by the oracle, in the slice's own arrays."""
    import oracle
    kp = hp.kp
    okp = oracle.kernel(kp.dim, kp.nu_x2, kp.length_scale, kp.variance, kp.nugget)
    rows, vals, logv, cnts = [], [], [], []
    for g in range(u0, u1):
        g0, g1 = int(hp.grp_ptr[g]), int(hp.grp_ptr[g + 1])
        sel = oracle.select_multi(okp, hp.pts, g0, g1 - g0, hp.cand_idx[hp.cand_ptr[g]:hp.cand_ptr[g + 1]],
                                  hp.k)["sel"]
        for a in range(g1 - g0):
            r, L, lv = oracle.fill_member(okp, hp.pts, g0, g1 - g0, a, sel)
            rows.append(r)
            vals.append(L)
            logv.append(lv)
            cnts.append(len(r))
    cp = np.zeros(len(cnts) + 1, np.int64)
    cp[1:] = np.cumsum(cnts)
    return cp, np.concatenate(rows).astype(np.int32), np.concatenate(vals), np.array(logv)


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist

    from paper_2307_11648_gb300 import build, shard, sic
    build.build()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        hp = _problem()
        b = sic.prep_partition(hp.cand_ptr, hp.grp_ptr, hp.k, world)
        u0, u1 = int(b[rank]), int(b[rank + 1])
        col0, n_cols = int(hp.grp_ptr[u0]), int(hp.grp_ptr[u1] - hp.grp_ptr[u0])
        cp, ri, val, logv = _oracle_slice(hp, u0, u1)
        comm = shard.TorchComm()
        meta, offsets = shard.exchange_counts(comm, col0, n_cols, int(cp[-1]))
        sl = shard.Slice(col0, n_cols, int(cp[-1]), torch.from_numpy(cp + offsets[rank]), torch.from_numpy(ri),
                         torch.from_numpy(val), torch.from_numpy(logv),
                         torch.tensor([float(np.sum(logv))], dtype=torch.float64))
        whole, nnz, s = shard.gather_factor(comm, meta, offsets, sl, hp.n)
        out.put((rank, whole["col_ptr"].numpy(), whole["row_idx"][:nnz].numpy(), whole["val"][:nnz].numpy(),
                 whole["logv"].numpy(), float(s[0]), float(np.sum(logv)), (u0, u1)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_assemble_the_oracle_factor(sic):
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    hp = _problem()
    G = len(hp.grp_ptr) - 1
    assert res[0][7][0] == 0 and res[0][7][1] == res[1][7][0] and res[1][7][1] == G
    assert 0 < res[0][7][1] < G  # both ranks own units
    cp, ri, val, logv = _oracle_slice(hp, 0, G)   # the one-piece (1-rank) assembly
    for r in res:
        assert np.array_equal(r[1], cp)
        assert np.array_equal(r[2], ri)
        assert np.array_equal(r[3], val)
        assert np.array_equal(r[4], logv)
        assert r[5] == res[0][6] + res[1][6]       # the all-reduce adds the slices' sums
    assert res[0][5] == pytest.approx(float(np.sum(logv)), rel=1e-14)


def test_slice_problem_host_side(sic):
    """pipeline.slice_problem and the proposal's reduced problem on the host: the slice keeps the
    whole problem's points and launch bounds, rebased candidate lists and its column range."""
    from paper_2307_11648_gb300 import learned, pipeline
    hp = _problem()
    U = hp.n_units
    b = sic.prep_partition(hp.cand_ptr, hp.grp_ptr, hp.k, 3)
    cols = 0
    for r in range(3):
        sl = pipeline.slice_problem(hp, int(b[r]), int(b[r + 1]))
        assert sl.pts is hp.pts and sl.n_units == b[r + 1] - b[r]
        assert sl.col0 == hp.grp_ptr[b[r]] and sl.ncols == hp.grp_ptr[b[r + 1]] - hp.grp_ptr[b[r]]
        assert sl.sliced and (sl.max_cand, sl.max_m) == (hp.max_cand, hp.max_m)
        assert sl.cand_ptr[0] == 0
        assert np.array_equal(sl.cand_idx, hp.cand_idx[hp.cand_ptr[b[r]]:hp.cand_ptr[b[r + 1]]])
        red = learned.reduced_problem(sl, 16)
        assert red.max_cand == min(hp.max_cand, 16) and red.col0 == sl.col0 and red.ncols == sl.ncols
        cols += sl.ncols
    assert cols == hp.n and not pipeline.slice_problem(hp, 0, U).sliced
    cp = pipeline.prepare_columns(synthetic.points(300, 2, 4), hp.kp, 16, 4)
    sl = pipeline.slice_problem(cp, 100, 200)
    assert sl.targets.tolist() == list(range(100, 200)) and sl.col0 == 100 and sl.ncols == 100
