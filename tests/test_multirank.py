"""The multi-process timing of bench.py on CPU: two gloo ranks on 127.0.0.1 agree on the
max-over-ranks step time and pass the barrier (the sliced build's own collectives are
tested in test_shard.py); and the FLOP accounting of the bench's roofline lines."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    bench.barrier(ws)
    m = bench.max_over_ranks(10.0 + 5.0 * r, ws)
    out.put((r, ws, m))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_and_barrier():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2, 15.0), (1, 2, 15.0)]


def test_flop_accounting_small_case():
    import numpy as np

    import bench
    gp = np.array([0, 2, 5], np.int64)       # groups of 2 and 3
    cp = np.array([0, 10, 30], np.int64)     # 10 and 20 candidates
    k = 4
    # by hand: group 1: R=12, m=2 -> 12*2*1/2 = 12; steps 10*(4*3 + 4*2 + 12) = 320
    #          group 2: R=23, m=3 -> 23*3*2/2 = 69; steps 20*(12 + 12 + 12) = 720
    assert bench.select_flops(gp, cp, k) == 2.0 * (12 + 320 + 69 + 720)
    sc = np.array([4, 1])
    # group 1: n=6: 36 + (36 + 25)/2 = 66.5; group 2: n=4: 64/6 + (16 + 9 + 4)/2
    assert bench.fill_flops(gp, sc) == pytest.approx(2.0 * (216 / 6 + 30.5 + 64 / 6 + 14.5))


def test_single_target_flop_accounting_by_steps():
    """select_columns_flops against a step-by-step count of the same definition: at step t the
    left-looking dot over t earlier picks for the C candidate rows and the target's row, then 3C
    for the two downdates and the score (2 FLOPs per FMA)."""
    import numpy as np

    import bench
    cp = np.array([0, 7, 7, 19, 20], np.int64)  # 7, 0, 12 and 1 candidates
    sc = np.array([5, 0, 12, 1], np.int32)
    want = 0.0
    for C, picks in zip(np.diff(cp), sc):
        for t in range(picks):
            want += 2.0 * ((C + 1) * t + 3 * C)
    assert bench.select_columns_flops(cp, sc) == pytest.approx(want)
