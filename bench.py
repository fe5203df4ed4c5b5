"""Benchmark: factor columns per second for the supernodal sparse inverse-Cholesky build
(N = 2^20 points uniform in the unit square, Matern 3/2, length scale 0.02, nugget 1e-6,
supernodes of 8..64 targets, 1024 candidates and k = 64 picks per supernode).

Headline step (one pass of the whole device path over the prepared inputs):
  learned proposal (features -> BF16 tensor-core MLP -> top 256 of 1024 per supernode)
  -> FP32-mixed supernodal greedy selection on the survivors -> nnz scan
  -> FP64 KL-optimal fill -> sum of log conditional variances.
Timed alongside: the plain FP32-mixed and plain FP64 paths on all 1024 candidates, a
2k-pick reference factor for the KL gap (S_A - S_plain64) / (S_plain64 - S_ref) with
S = sum log v, and the plain distance truncation to 256 candidates.  Ordering /
candidate / grouping prep and the proposal's training are host / set-up work, timed and
reported separately.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl sic|reference]

Prints one JSON line (rank 0).  Under torchrun the ranks build ONE factor of the same
problem in slices of near-equal cost (strong scaling): each rank runs the step on its slice,
then the slices are gathered into the whole factor on every rank (the only collectives);
the max step time over ranks is used.  `--impl reference` times the CPU oracle (FP64, all
host cores) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic  # noqa: E402

METRIC = "factor columns/s at N=2^20,k=64 (learned+FP32 vs plain FP64); KL gap"
WORKLOAD = "cfg3_aggregated"
SMS = 152
SM_MAX_MHZ = 2070.0
FFMA_PER_SM_CLK = 128   # FP32 FMA lanes per SM per clock
DFMA_PER_SM_CLK = 2     # FP64 FMA per SM per clock on GB300 (1.26 TFLOP/s nominal at 2070 MHz)
# kernels of one learned step: k_features, k_mlp_tc, k_topk_counts + k_scan_one_block +
# k_topk_compact, k_agg_target_chol + k_agg_target_cols + k_select_agg_reg, k_nnz_count +
# k_scan_tile + k_scan_partials + k_scan_add, k_fill x 2 (two group-size classes) +
# k_sum_tiles + k_sum_final (plus one memset node)
LAUNCHES_PER_STEP = 16
# DRAM read + write bytes of the two k_fill launches, and of the selection's three launches
# (k_agg_target_chol, k_agg_target_cols, k_select_agg_reg), of one learned step at N = 2^19
# (22,423 supernodes), from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum);
# None where the kernel has changed since the capture
FILL_DRAM_BYTES_N2E19 = 16812544 + 256258560 + 9846272 + 117808640
SEL_DRAM_BYTES_N2E19 = 10139904 + 2321920 + 70493696 + 471795968 + 572655616 + 5679360
GROUPS_N2E19 = 22423


def measured_peak(key: str, fallback: float) -> float:
    """A peak from MEASURED_PEAKS.json (copy bandwidth, cuBLAS BF16), else the stated fallback."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))[key])
    except Exception:
        return fallback


# ------------------------------------------------------------- clocks ---

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        self.lines = []
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------ flop accounting ---

def select_flops(grp_ptr, cand_ptr, k) -> float:
    """Algorithmic FLOPs of the supernodal selection (2 per fused multiply-add): target
    columns R*m(m-1)/2 FMA (R = C + m rows), then per step t the two left-looking dot
    products C*t + C*(m + t), the two downdates and the score 3C; kernel evaluations
    not counted."""
    m = np.diff(grp_ptr).astype(np.float64)
    C = np.diff(cand_ptr).astype(np.float64)
    R = C + m
    return float(2.0 * np.sum(R * m * (m - 1) / 2.0 + C * (k * (k - 1) + k * m + 3.0 * k)))


def select_columns_flops(cand_ptr, sel_count) -> float:
    """Algorithmic FLOPs of the single-target selection (2 per FMA): per step t the
    left-looking dot over the t earlier picks for the C candidate rows and the target's row,
    (C + 1) t FMA, then the downdates of var and cov and the score, 3C; kernel evaluations
    not counted."""
    C = np.diff(cand_ptr).astype(np.float64)
    t = sel_count.astype(np.float64)
    return float(2.0 * np.sum((C + 1.0) * t * (t - 1.0) / 2.0 + 3.0 * C * t))


def fill_flops(grp_ptr, sel_count) -> float:
    """Algorithmic FP64 FLOPs of the fill (2 per FMA): Cholesky of the n x n reversed set
    n^3/6 and the m member back substitutions sum_a (n - a)^2 / 2, n = picks + m; the
    n(n+1)/2 kernel evaluations are not counted."""
    m = np.diff(grp_ptr).astype(np.float64)
    n = sel_count.astype(np.float64) + m
    back = np.array([np.sum((nn - np.arange(mm)) ** 2) / 2.0 for nn, mm in zip(n, m)])
    return float(2.0 * np.sum(n ** 3 / 6.0 + back))


# ------------------------------------------------------------- oracle ----

def _oracle_unit(okp, P, gp, cand_ptr, cand_idx, k, g):
    """One supernode through the oracle: FP64 two-factor greedy, then the dense fill of
    every member column.  Returns the member count."""
    import oracle
    g0, g1 = int(gp[g]), int(gp[g + 1])
    cand = cand_idx[cand_ptr[g]:cand_ptr[g + 1]]
    sel = oracle.select_multi(okp, P, g0, g1 - g0, cand, k)["sel"]
    for a in range(g1 - g0):
        oracle.fill_member(okp, P, g0, g1 - g0, a, sel)
    return g1 - g0


def oracle_batch(prob, groups, threads: int):
    """Run the CPU oracle on the given supernodes over `threads` host threads.
    Returns (columns, seconds)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    oracle.build()
    kd = prob["kernel"]
    okp = oracle.kernel(kd["dim"], kd["nu_x2"], kd["length_scale"], kd["variance"], kd["nugget"])
    P, gp, cp, ci, k = prob["pts"], prob["grp_ptr"], prob["cand_ptr"], prob["cand_idx"], int(prob["k"])
    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        cols = sum(ex.map(lambda g: _oracle_unit(okp, P, gp, cp, ci, k, g), groups, chunksize=4))
    return cols, time.perf_counter() - t0


def oracle_sample(prob, seconds: float, threads: int, seed: int = 0):
    """Time the CPU oracle on random supernodes of the problem for about `seconds`: a short
    calibration batch, then one batch sized to fill the rest.  Returns
    (columns/s, columns, groups, s) of the whole sample."""
    G = len(prob["grp_ptr"]) - 1
    order = np.random.default_rng(seed).permutation(G)
    first = order[:2 * threads]
    c0, t0 = oracle_batch(prob, first, threads)
    rest = int(max(0.0, seconds - t0) * len(first) / max(t0, 1e-9))
    second = order[len(first):len(first) + rest]
    c1, t1 = oracle_batch(prob, second, threads) if len(second) else (0, 0.0)
    return (c0 + c1) / (t0 + t1), c0 + c1, len(first) + len(second), t0 + t1


def proposal_gain_clustered(h, cfg, n, epochs):
    """Where the proposal network earns its place: a clustered cloud (half of the points in a
    square of side 0.05), the config-3 kernel with ell scaled to n points, a network trained on
    two clustered clouds of other seeds; KL gap (S_A - S_plain64) / (S_plain64 - S_ref) of the
    learned proposal and of distance truncation at top = 128 and 256."""
    import torch

    from paper_2307_11648_gb300 import learned, pipeline, sic
    ell = cfg["length_scale"] * math.sqrt(cfg["n"] / n)
    kp = sic.kernel(cfg["dim"], cfg["nu_x2"], ell, cfg["variance"], cfg["nugget"])

    def prob(seed, k=cfg["k"]):
        return pipeline.prepare_groups(synthetic.clustered_points(n, cfg["dim"], seed), kp, cfg["n_cand"], k,
                                       cfg["m_min"], cfg["m_max"])

    feat, label, _ = learned.training_set(h, [prob(1001), prob(1002)])
    params, _ = learned.train(h, feat, label, epochs=epochs, batch=65536, lr=2e-3, seed=0)
    del feat, label
    hp = prob(cfg["seed"])
    dp = pipeline.DeviceProblem(hp)
    S = {}

    def run(name, b, d=dp):
        b.run(d)
        h.sync()
        S[name] = float(b.sum_logv.cpu()[0])

    run("plain64", pipeline.FactorBuilder(h, hp, sic.SIC_FP64))
    run("plain32", pipeline.FactorBuilder(h, hp, sic.SIC_FP32_MIXED))
    run("ref", pipeline.FactorBuilder(h, dataclasses.replace(hp, k=2 * hp.k), sic.SIC_FP32_MIXED))
    out = {"n": n, "geometry": "clustered_points: half of the points in the centred square of side 0.05"}
    for top in (128, 256):
        run(f"learned{top}", learned.LearnedFactorBuilder(h, hp, learned.Proposal(h, params, top=top)))
        dhp = truncated(hp, top)
        run(f"distance{top}", pipeline.FactorBuilder(h, dhp, sic.SIC_FP32_MIXED), pipeline.DeviceProblem(dhp))
        base = S["plain64"] - S["ref"]
        out[f"top{top}"] = {"learned_kl_gap": (S[f"learned{top}"] - S["plain64"]) / base,
                            "distance_kl_gap": (S[f"distance{top}"] - S["plain64"]) / base}
    out["plain_fp32_kl_gap"] = (S["plain32"] - S["plain64"]) / (S["plain64"] - S["ref"])
    del dp
    torch.cuda.empty_cache()
    return out


def config1(h, timed, stream, oracle_s=3.0, naive_cols=4):
    """Config 1: N = 4096 points in the unit square (seed 0), Matern 3/2, ell = 0.1, nugget 1e-8,
    k = 16 of the 256 nearest later points per column, FP64.  The GPU build (selection + fill +
    sum of log v) as a CUDA graph; the oracle on all host cores and on one, on columns taken
    in order until about `oracle_s` seconds have passed (Cholesky-form greedy + dense fill);
    and the naive greedy (a fresh dense factorisation per candidate and step, O(C k^4)) on
    `naive_cols` columns."""
    import torch

    import oracle
    from paper_2307_11648_gb300 import pipeline, sic
    oracle.build()
    c = synthetic.PRESETS["cfg1_single_fp64"]
    kp = sic.kernel(c["dim"], c["nu_x2"], c["length_scale"], c["variance"], c["nugget"])
    hp = pipeline.prepare_columns(synthetic.points(c["n"], c["dim"], c["seed"]), kp, c["n_cand"], c["k"])
    dp = pipeline.DeviceProblem(hp)
    fb = pipeline.FactorBuilder(h, hp, sic.SIC_FP64)
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        fb.run(dp)
    stream.wait_stream(side)
    with torch.cuda.graph(g):
        fb.run(dp)
    g_ms, _, _ = timed([g.replay], 10, 3)
    okp = oracle.kernel(kp.dim, kp.nu_x2, kp.length_scale, kp.variance, kp.nugget)

    def col(i):
        sel = oracle.select_single(okp, hp.pts, i, hp.cand_idx[hp.cand_ptr[i]:hp.cand_ptr[i + 1]], hp.k)["sel"]
        oracle.fill_column(okp, hp.pts, i, sel)

    def rate(threads):
        from concurrent.futures import ThreadPoolExecutor
        done, t0 = 0, time.perf_counter()
        with ThreadPoolExecutor(threads) as ex:
            while time.perf_counter() - t0 < oracle_s and done < hp.n:
                batch = range(done, min(hp.n, done + 8 * threads))
                list(ex.map(col, batch))
                done = batch[-1] + 1
        return done / (time.perf_counter() - t0), done

    threads = os.cpu_count() or 1
    all_rate, all_cols = rate(threads)
    one_rate, one_cols = rate(1)
    t0 = time.perf_counter()
    for i in range(naive_cols):
        oracle.select_single_naive(okp, hp.pts, i, hp.cand_idx[hp.cand_ptr[i]:hp.cand_ptr[i + 1]], hp.k)
    naive_rate = naive_cols / (time.perf_counter() - t0)
    out = {"workload": "N=4096 uniform [0,1]^2 (seed 0), Matern 3/2, ell=0.1, nugget 1e-8, C=256, k=16, FP64",
           "gpu_graph_ms": g_ms, "gpu_columns_per_s": hp.n / (g_ms * 1e-3),
           "sum_logv": float(fb.sum_logv.cpu()[0]),
           "oracle_all_cores": {"columns_per_s": all_rate, "cores": threads, "sample_columns": all_cols},
           "oracle_one_core": {"columns_per_s": one_rate, "sample_columns": one_cols},
           "oracle_naive_one_core": {"columns_per_s": naive_rate, "sample_columns": naive_cols,
                                     "form": "O(C k^4): dense re-factorisation per candidate and step"}}
    del g, fb, dp
    return out


def host_problem_dict(hp):
    """The prepared inputs as plain arrays (what the oracle needs; no library objects)."""
    kp = hp.kp
    return {"pts": hp.pts, "grp_ptr": hp.grp_ptr, "cand_ptr": hp.cand_ptr, "cand_idx": hp.cand_idx, "k": hp.k,
            "kernel": {"dim": kp.dim, "nu_x2": kp.nu_x2, "length_scale": kp.length_scale,
                       "variance": kp.variance, "nugget": kp.nugget}}


def prepared_by_child(path: str):
    """The config-3 problem prepared (ordering, grouping, candidates: libsic host code) in a
    child process and handed over as an .npz, so that the process timing the oracle never
    loads libsic."""
    subprocess.check_call([sys.executable, os.path.join(ROOT, "bench.py"), "--prep-only", path])
    z = np.load(path)
    kd = {key: z["kernel_" + key].item() for key in ("dim", "nu_x2", "length_scale", "variance", "nugget")}
    return {"pts": z["pts"], "grp_ptr": z["grp_ptr"], "cand_ptr": z["cand_ptr"], "cand_idx": z["cand_idx"],
            "k": int(z["k"]), "kernel": kd}


# ---------------------------------------------------------------- main ---

def dist_env():
    return int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), int(
        os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def problem(cfg, seed, n=None):
    from paper_2307_11648_gb300 import pipeline, sic
    n = n or cfg["n"]
    ell = cfg["length_scale"] * math.sqrt(cfg["n"] / n)  # same ell / spacing as the full size
    kp = sic.kernel(cfg["dim"], cfg["nu_x2"], ell, cfg["variance"], cfg["nugget"])
    pts = synthetic.points(n, cfg["dim"], seed)
    return pipeline.prepare_groups(pts, kp, cfg["n_cand"], cfg["k"], cfg["m_min"], cfg["m_max"])


def cfg_single_seed(rank):
    return synthetic.PRESETS["cfg2_single_batched"]["seed"] + rank


def single_problem(n, seed):
    """The single-target workload: n points in the unit cube, Matern 5/2, 512 nearest
    later-ordered candidates per column, k = 32."""
    from paper_2307_11648_gb300 import pipeline, sic
    c = synthetic.PRESETS["cfg2_single_batched"]
    ell = c["length_scale"] * (c["n"] / n) ** (1.0 / c["dim"])  # same ell / spacing as the full size
    kp = sic.kernel(c["dim"], c["nu_x2"], ell, c["variance"], c["nugget"])
    return pipeline.prepare_columns(synthetic.points(n, c["dim"], seed), kp, c["n_cand"], c["k"])


def truncated(hp, top):
    """The same problem with every candidate list cut to its first `top` (nearest) entries."""
    from paper_2307_11648_gb300 import pipeline
    cnt = np.minimum(np.diff(hp.cand_ptr), top)
    ptr = np.zeros(len(cnt) + 1, np.int64)
    ptr[1:] = np.cumsum(cnt)
    idx = np.concatenate([hp.cand_idx[hp.cand_ptr[g]:hp.cand_ptr[g] + cnt[g]] for g in range(len(cnt))])
    return pipeline.HostProblem(hp.pts, hp.kp, hp.k, ptr, idx, hp.grp_ptr, hp.order, hp.ell2)


def pcg_comparison(h, cfg, params, n, nrhs=8, shift=1e-4, tol=1e-8, caps=None):
    """Config-5 style comparison: CG on (Theta + shift I) x = b, b ~ N(0, 1), with the factors of
    that matrix from the learned proposal, plain greedy and k nearest neighbours (first k
    candidates) as preconditioners, and without; FP32-entry matvec with compensated sums.
    caps: iteration cap per preconditioner ("learned", "conditional", "knn", "none"); 0 skips it."""
    import torch

    from paper_2307_11648_gb300 import learned, pipeline, sic
    ell = cfg["length_scale"] * math.sqrt(cfg["n"] / n)
    kp = sic.kernel(cfg["dim"], cfg["nu_x2"], ell, cfg["variance"], cfg["nugget"] + shift)
    hp = pipeline.prepare_groups(synthetic.points(n, cfg["dim"], cfg["seed"]), kp, cfg["n_cand"], cfg["k"],
                                 cfg["m_min"], cfg["m_max"])
    dp = pipeline.DeviceProblem(hp)
    B = torch.from_numpy(synthetic.normal(7, n * nrhs).reshape(n, nrhs)).cuda()
    ws = sic._ws(sic.pcg_workspace(n, nrhs), "cuda")
    out = {"n": n, "nrhs": nrhs, "tol": tol, "system": f"Theta (nugget {cfg['nugget']}) + {shift} I; factors of the "
           "same matrix; k=64, C=1024"}

    def solve(factor, cap):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its, rel = sic.pcg_solve(h, dp.pts, kp, 0.0, sic.SIC_FP32_MIXED, factor, B, torch.empty_like(B), tol, cap, ws)
        return its.tolist(), float(np.max(rel)), 1e3 * (time.perf_counter() - t0)

    def csc(fb):
        nnz = int(fb.col_ptr[-1].item())
        return (fb.col_ptr, fb.row_idx[:nnz].contiguous(), fb.val[:nnz].contiguous())

    caps = dict({"learned": 1000, "conditional": 1000, "knn": 1000, "none": 300}, **(caps or {}))
    out["caps"] = caps
    if caps["learned"]:
        lb = learned.LearnedFactorBuilder(h, hp, learned.Proposal(h, params, top=4 * cfg["k"]), sic.SIC_FP32_MIXED)
        lb.run(dp)
        out["learned"] = solve(csc(lb.fb), caps["learned"])
        del lb
    fb = pipeline.FactorBuilder(h, hp, sic.SIC_FP32_MIXED)
    fb.run(dp)
    if caps["conditional"]:
        out["conditional"] = solve(csc(fb), caps["conditional"])
    U, k = hp.n_units, hp.k
    sel = np.full((U, k), -1, np.int32)
    cnt = np.zeros(U, np.int32)
    for g in range(U):
        c = hp.cand_idx[hp.cand_ptr[g]:hp.cand_ptr[g + 1]][:k]
        sel[g, :len(c)] = c
        cnt[g] = len(c)
    fb.sel_idx.copy_(torch.from_numpy(sel.ravel()))
    fb.sel_count.copy_(torch.from_numpy(cnt))
    fb.fill(dp)
    if caps["knn"]:
        out["knn"] = solve(csc(fb), caps["knn"])
    if caps["none"]:
        out["none"] = solve(None, caps["none"])
    out["legend"] = "[iterations per right-hand side, max final relative residual, wall ms]; capped at 'caps'"
    return out


def run_reference(args, ws, rank):
    """The oracle arm: every step times the FP64 CPU oracle on a bounded random sample of the
    config-3 supernodes (about --ref-seconds of work on all host cores); ms_per_step is that
    sample's own wall time and value the sample's columns per second."""
    if rank != 0:
        return
    import tempfile
    with tempfile.TemporaryDirectory() as td:
        prob = prepared_by_child(os.path.join(td, "problem.npz"))
    threads = os.cpu_count() or 1
    G = len(prob["grp_ptr"]) - 1
    order = np.random.default_rng(0).permutation(G)
    # calibration (untimed): groups per second on this host, to size the steps
    c, t = oracle_batch(prob, order[:4 * threads], threads)
    per_step = max(threads, int(args.ref_seconds * 4 * threads / max(t, 1e-9)))
    pos = 4 * threads
    for _ in range(args.warmup):
        oracle_batch(prob, order[pos:pos + threads], threads)
        pos += threads
    step_s, cols_tot = [], 0
    for _ in range(args.steps):
        batch = np.take(order, np.arange(pos, pos + per_step), mode="wrap")
        pos += per_step
        cols, el = oracle_batch(prob, batch, threads)
        step_s.append(el)
        cols_tot += cols
    el_tot = sum(step_s)
    v = cols_tot / el_tot
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "columns/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el_tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "N=2^20 uniform [0,1]^2, Matern 3/2, ell=0.02, nugget 1e-6, supernodes 8..64, "
                                   "C=1024, k=64 (plain greedy, FP64 CPU oracle)", "groups": G,
                       "step": f"{per_step} random supernodes per step (a bounded sample of the {G})"},
            "cpu_baseline": {"value": v, "unit": "columns/s", "cores": threads, "kind": "oracle",
                             "sample": f"{per_step} random supernodes per step, FP64 two-factor greedy + dense fill "
                                       f"on all 1024 candidates ({cols_tot} columns over {args.steps} steps, "
                                       f"{el_tot:.1f} s); inputs prepared in a child process"},
            "e2e": {"value": v, "unit": "columns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_sharded(args, ws, rank, local, h, hp, proposal, timed, prep_s, train_s):
    """Multi-GPU step (strong scaling): the one N = 2^20 problem cut into `ws` slices of
    near-equal cost (sic_prep_partition); each rank runs the learned step (proposal ->
    FP32 selection -> FP64 fill) on its slice as one CUDA graph, then the slices are gathered
    into the whole factor on every rank (NCCL broadcasts into place, all-reduce of the sums
    of log v, fixed-order sum of the gathered log v).  The timed step is slice + gather; the
    max over ranks is used and value = N / step time."""
    import torch

    from paper_2307_11648_gb300 import shard, sic
    import torch.distributed as dist
    if not dist.is_initialized():  # --sharded on one GPU: a one-rank process group
        import socket
        sk = socket.socket()
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
        sk.close()
        dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    stream = torch.cuda.current_stream()
    comm = shard.TorchComm(device="cuda")
    sb = shard.ShardedFactorBuilder(h, hp, sic.SIC_FP32_MIXED, rank, ws, proposal=proposal)
    sdp = sb.device_problem()
    N = hp.n
    lb = sb.builder
    phases = {}
    graph = None
    if not sb.empty:
        rdp = lb._reduced_device(sdp)
        pr = lb.proposal
        sl_ms, ph, _ = timed([lambda: pr.features(sdp, lb.buf), lambda: pr.score(sdp, lb.buf),
                              lambda: pr.topk(sdp, lb.buf), lambda: lb.fb.select(rdp), lambda: lb.fb.fill(rdp)],
                             args.steps, args.warmup)
        phases = dict(zip(["features", "mlp", "topk", "select", "fill_and_kl"], ph))
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            lb.run(sdp)
        stream.wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            lb.run(sdp)
    res = {}

    def step():
        if graph is not None:
            graph.replay()
        res["out"] = sb.gather(sdp, comm)

    sampler = ClockSampler(local)
    t_ms, (slice_ms,), clocks = timed([lambda: graph.replay() if graph is not None else None], args.steps,
                                      args.warmup)
    t_ms, _, clocks = timed([step], args.steps, args.warmup, sampler)
    t_step = max_over_ranks(t_ms, ws)
    whole, nnz, s_red, s_fixed = res["out"]
    # end to end: this rank's inputs host -> device (points and its slice's lists), the step,
    # the gathered factor device -> host on rank 0
    loc = sb.local
    pin = {} if sb.empty else {key: torch.from_numpy(v).pin_memory() for key, v in
                               dict(pts=loc.pts, grp_ptr=loc.grp_ptr, cand_ptr=loc.cand_ptr,
                                    cand_idx=loc.cand_idx).items()}
    h2d_rank = sum(t.numel() * t.element_size() for t in pin.values())
    out_host = dict(col_ptr=torch.empty(N + 1, dtype=torch.int64).pin_memory(),
                    row_idx=torch.empty(nnz, dtype=torch.int32).pin_memory(),
                    val=torch.empty(nnz, dtype=torch.float64).pin_memory(),
                    sum_logv=torch.empty(1, dtype=torch.float64).pin_memory())

    def e2e_step():
        for key, t in pin.items():
            getattr(sdp, key).copy_(t, non_blocking=True)
        step()
        if rank == 0:
            w, nz, _, fx = res["out"]
            out_host["col_ptr"].copy_(w["col_ptr"], non_blocking=True)
            out_host["row_idx"].copy_(w["row_idx"][:nz], non_blocking=True)
            out_host["val"].copy_(w["val"][:nz], non_blocking=True)
            out_host["sum_logv"].copy_(fx, non_blocking=True)

    e_ms, _, _ = timed([e2e_step], max(args.steps, 3), 1)
    e_ms = max_over_ranks(e_ms, ws)
    h2d = sum(m[0] for m in comm.all_gather_ints([h2d_rank]))
    d2h = (N + 1) * 8 + nnz * 12 + 8
    # roofline of the dominant kernel on rank 0's slice (the FP64 fill)
    f64_peak = SMS * DFMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12
    roof = None
    if not sb.empty and phases:
        fill_tf = fill_flops(loc.grp_ptr, lb.fb.sel_count.cpu().numpy()) / (phases["fill_and_kl"] * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": "k_fill (FP64 fill, both launches) on rank 0's slice", "achieved": fill_tf,
                "peak": f64_peak, "unit": "TFLOP/s", "frac": fill_tf / f64_peak, "traffic": None,
                "peak_source": "152 SMs x 2 FP64 FMA/clk x 2 x 2070 MHz (derived from unit counts)"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": N / (t_step * 1e-3), "unit": "columns/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"N={N} uniform [0,1]^2 (seed {synthetic.PRESETS[WORKLOAD]['seed']}), Matern 3/2, "
                                   "ell=0.02, nugget 1e-6, supernodes 8..64, C=1024, k=64; one factor in "
                                   f"{ws} slices", "groups": hp.n_units, "nnz": nnz,
                       "path": "per rank: learned proposal (top 256) -> select_aggregated FP32 -> factor_nnz_range "
                               "-> build_factor_range FP64 on its slice; then gather (NCCL broadcasts), all-reduce "
                               "of sum log v, fixed-order sum",
                       "parallelism": f"{ws} slices of one factor (units {sb.bounds.tolist()})",
                       "l2": "inputs larger than L2"},
            "sum_logv": {"fixed_order": float(s_fixed[0]), "all_reduce": float(s_red[0])},
            "slice_ms_rank0": slice_ms, "phases_ms_rank0": phases,
            "roofline": roof,
            "e2e": {"value": N / (e_ms * 1e-3), "unit": "columns/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e_ms},
            "gpu_launches": (LAUNCHES_PER_STEP + 6) * args.steps,  # + the col_ptr scan at global offsets (4)
                                                                    # and the fixed-order sum (2)
            "clocks": clocks, "cpu_baseline": None,
            "setup_s": {"prep_host": prep_s, "train_proposal": train_s},
        }
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sic", choices=["sic", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--ref-seconds", type=float, default=5.0,
                    help="oracle seconds per step of the reference arm (and of the cpu_baseline sample x 2)")
    ap.add_argument("--prep-only", default="", help=argparse.SUPPRESS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--train-n", type=int, default=1 << 18, help="points per training problem")
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--case-only", type=int, default=0, metavar="N",
                    help="profiling case: one FP32-mixed supernodal factor build at N points, no timing")
    ap.add_argument("--case-top", type=int, default=0,
                    help="with --case-only: keep only the first TOP candidates of each list (the selection "
                         "kernel of the proposal path)")
    ap.add_argument("--case-mlp", action="store_true",
                    help="with --case-only: run the proposal (untrained network) and select on its top 256")
    ap.add_argument("--pcg-n", type=int, default=1 << 16, help="points of the preconditioning comparison (0: skip)")
    ap.add_argument("--pcg-only", type=int, default=0, metavar="N",
                    help="only the preconditioning comparison at N points (trained proposal), one JSON line")
    ap.add_argument("--pcg-caps", default="",
                    help="iteration caps, e.g. learned=1000,conditional=1000,knn=60,none=0 (0 skips)")
    ap.add_argument("--pcg-nrhs", type=int, default=8)
    ap.add_argument("--pcg-untrained", action="store_true",
                    help="with --pcg-only: the untrained network (a profiling case)")
    ap.add_argument("--case-global", action="store_true",
                    help="with --case-only: the learned step with a budget of 48 picks per supernode on average, "
                         "decreases from the FP64 side state, global allocation")
    ap.add_argument("--case-partial", action="store_true",
                    help="with --case-only: partial selection of nonadjacent groups (256 candidates) and its fill")
    ap.add_argument("--tune-save", default="", help="with --case-only: autotune the fill first, save the table here")
    ap.add_argument("--tune-load", default="", help="with --case-only: load a saved autotune table before the run")
    ap.add_argument("--single-n", type=int, default=1 << 16,
                    help="points of the single-target measurement (3-D, 512 candidates, k = 32; 0: skip)")
    ap.add_argument("--case-single", action="store_true",
                    help="with --case-only: one FP32-mixed single-target factor build (3-D, 512 candidates, k = 32)")
    ap.add_argument("--clustered-n", type=int, default=1 << 18,
                    help="points of the clustered-cloud comparison of the proposal against distance order (0: skip)")
    ap.add_argument("--cfg1", type=int, default=1, help="the config-1 line (FP64 path, oracle timings; 0: skip)")
    ap.add_argument("--sharded", action="store_true",
                    help="the multi-GPU path (one factor in slices, gathered) even on one GPU")
    ap.add_argument("--partial-n", type=int, default=1 << 18,
                    help="points of the partial-selection (nonadjacent groups) measurement (0: skip)")
    args = ap.parse_args()
    if args.prep_only:
        cfg = synthetic.PRESETS[WORKLOAD]
        d = host_problem_dict(problem(cfg, cfg["seed"]))
        kd = d.pop("kernel")
        np.savez(args.prep_only, **d, **{"kernel_" + key: v for key, v in kd.items()})
        return
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "sic" else "gloo")
    if args.impl == "reference":
        run_reference(args, ws, rank)
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    import torch

    from paper_2307_11648_gb300 import build, learned, pipeline, sic
    build.build()
    torch.cuda.set_device(local)
    cfg = synthetic.PRESETS[WORKLOAD]
    if args.case_only and args.case_single:
        h = sic.Handle(local)
        shp = single_problem(args.case_only, cfg_single_seed(0))
        fb = pipeline.FactorBuilder(h, shp, sic.SIC_FP32_MIXED)
        fb.run(pipeline.DeviceProblem(shp))
        # then the factor's two products with one right-hand side
        x = torch.ones(shp.n, dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        sums = []
        for op in (sic.SIC_OP_LT, sic.SIC_OP_L):
            sic.apply_factor(h, fb.col_ptr, fb.row_idx, fb.val, op, x, y)
            sums.append(float(y.sum().cpu()))
        h.sync()
        print(json.dumps({"case": args.case_only, "columns": shp.n, "sum_logv": float(fb.sum_logv.cpu()[0]),
                          "apply_sums": sums}))
        return
    if args.pcg_only:
        h = sic.Handle(local)
        if args.pcg_untrained:
            params = learned.init_params(0)
        else:
            train_probs = [problem(cfg, 1000 + i, args.train_n) for i in (1, 2)]
            feat, label, _ = learned.training_set(h, train_probs)
            params, _ = learned.train(h, feat, label, epochs=args.epochs, batch=65536, lr=2e-3, seed=0)
            del feat, label, train_probs
            torch.cuda.empty_cache()
        caps = {kv.split("=")[0]: int(kv.split("=")[1]) for kv in args.pcg_caps.split(",") if kv}
        p5 = synthetic.PRESETS["cfg5_pcg"]
        res = pcg_comparison(h, cfg, params, args.pcg_only, nrhs=args.pcg_nrhs, shift=p5["shift"], tol=p5["tol"],
                             caps=caps)
        res["trained"] = not args.pcg_untrained
        print(json.dumps({"pcg": res}))
        return
    if args.case_only and args.case_partial:
        h = sic.Handle(local)
        php = pipeline.prepare_partial(synthetic.points(args.case_only, 2, cfg["seed"]), sic.kernel(
            2, cfg["nu_x2"], cfg["length_scale"], cfg["variance"], cfg["nugget"]), 256, cfg["k"], cfg["m_min"],
            cfg["m_max"])
        fb = pipeline.PartialFactorBuilder(h, php, sic.SIC_FP32_MIXED)
        fb.run(pipeline.DeviceProblem(php))
        h.sync()
        print(json.dumps({"case": args.case_only, "groups": php.n_units, "sum_logv": float(fb.sum_logv.cpu()[0])}))
        return
    if args.case_only:
        # one FP32-mixed supernodal factor build at the requested size (for ncu captures)
        hp = problem(cfg, cfg["seed"], args.case_only)
        if args.case_top:
            hp = truncated(hp, args.case_top)
        h = sic.Handle(local)
        dp = pipeline.DeviceProblem(hp)
        if args.case_global:
            fb = learned.LearnedFactorBuilder(h, hp, learned.Proposal(h, learned.init_params(0), top=4 * cfg["k"]),
                                              budget=int(np.diff(hp.grp_ptr).sum()) * (3 * cfg["k"] // 4),
                                              side_fp64=True)
        elif args.case_mlp:
            fb = learned.LearnedFactorBuilder(h, hp, learned.Proposal(h, learned.init_params(0), top=4 * cfg["k"]))
        else:
            fb = pipeline.FactorBuilder(h, hp, sic.SIC_FP32_MIXED)
        if args.tune_load:
            sic.tune_load(h, args.tune_load)
        if args.tune_save:
            fb.tune(dp)
            h.sync()
            sic.tune_save(h, args.tune_save)
        fb.run(dp)
        h.sync()
        print(json.dumps({"case": args.case_only, "groups": hp.n_units, "sum_logv": float(fb.sum_logv.cpu()[0]),
                          "tune": sic.tune_table(h)}))
        return
    t0 = time.perf_counter()
    hp = problem(cfg, cfg["seed"])  # one problem; under torchrun every rank builds a slice of it
    prep_s = time.perf_counter() - t0
    h = sic.Handle(local)
    dp = pipeline.DeviceProblem(hp)
    stream = torch.cuda.current_stream()
    N = hp.n

    # ---- the proposal network: trained on plain-greedy labels of disjoint seeds
    t0 = time.perf_counter()
    train_probs = [problem(cfg, 1000 + i, args.train_n) for i in (1, 2)]
    feat, label, n_sel = learned.training_set(h, train_probs)
    params, hist = learned.train(h, feat, label, epochs=args.epochs, batch=65536, lr=2e-3, seed=0)
    del feat, label, train_probs
    torch.cuda.empty_cache()
    train_s = time.perf_counter() - t0
    proposal = learned.Proposal(h, params, top=4 * cfg["k"])

    def timed(phases, steps, warmup, sampler=None):
        """phases: list of callables issuing kernels on the stream; returns per-phase ms."""
        for _ in range(warmup):
            for f in phases:
                f()
        h.sync()
        barrier(ws)
        torch.cuda.synchronize()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(phases) + 1)] for _ in range(steps)]
        if sampler:
            sampler.start()
        for ev in evs:
            ev[0].record(stream)
            for i, f in enumerate(phases):
                f()
                ev[i + 1].record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop() if sampler else None
        h.sync()
        per = [[ev[i].elapsed_time(ev[i + 1]) for ev in evs] for i in range(len(phases))]
        total = evs[0][0].elapsed_time(evs[-1][-1])
        return total / steps, [statistics.mean(p) for p in per], clocks

    if ws > 1 or args.sharded:
        run_sharded(args, ws, rank, local, h, hp, proposal, timed, prep_s, train_s)
        h.close()
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()
        return

    # ---- headline: learned proposal + FP32-mixed selection + FP64 fill; the fill's launch
    # split is autotuned on this problem first (outside the timed region)
    lb = learned.LearnedFactorBuilder(h, hp, proposal, sic.SIC_FP32_MIXED)
    tuned_split = lb.tune(dp)
    h.sync()
    rdp = lb._reduced_device(dp)
    sampler = ClockSampler(local)
    pr = lb.proposal
    t_ms, (feat_ms, mlp_ms, topk_ms, sel_ms, fill_ms), clocks = timed(
        [lambda: pr.features(dp, lb.buf), lambda: pr.score(dp, lb.buf), lambda: pr.topk(dp, lb.buf),
         lambda: lb.fb.select(rdp), lambda: lb.fb.fill(rdp)], args.steps, args.warmup, sampler)
    prop_ms = feat_ms + mlp_ms + topk_ms
    eager_ms = max_over_ranks(t_ms, ws)
    # the same step captured once in a CUDA graph and replayed (one graph launch per step):
    # the headline time
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        lb.run(dp)
    stream.wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        lb.run(dp)
    g_ms, _, clocks = timed([graph.replay], args.steps, args.warmup, sampler)
    t_step = max_over_ranks(g_ms, ws)
    value = ws * N / (t_step * 1e-3)
    S = {"learned_fp32": float(lb.sum_logv.cpu()[0])}
    nnz = int(lb.col_ptr[-1].item())
    sel_count_learned = lb.fb.sel_count.cpu().numpy()

    # ---- plain FP32-mixed and plain FP64 on all candidates
    fb32 = pipeline.FactorBuilder(h, hp, sic.SIC_FP32_MIXED)
    p32_ms, (p32_sel, p32_fill), _ = timed([lambda: fb32.select(dp), lambda: fb32.fill(dp)], args.steps, 1)
    S["plain_fp32"] = float(fb32.sum_logv.cpu()[0])
    del fb32
    fb64 = pipeline.FactorBuilder(h, hp, sic.SIC_FP64)
    p64_ms, (p64_sel, p64_fill), _ = timed([lambda: fb64.select(dp), lambda: fb64.fill(dp)], args.fp64_steps, 1)
    p64_ms = max_over_ranks(p64_ms, ws)
    S["plain_fp64"] = float(fb64.sum_logv.cpu()[0])
    del fb64
    # ---- KL reference (2k picks from the same candidates) and distance truncation
    ref_hp = pipeline.HostProblem(hp.pts, hp.kp, 2 * cfg["k"], hp.cand_ptr, hp.cand_idx, hp.grp_ptr, hp.order,
                                  hp.ell2)
    fr = pipeline.FactorBuilder(h, ref_hp, sic.SIC_FP32_MIXED)
    fr.run(dp)
    h.sync()
    S["reference_2k"] = float(fr.sum_logv.cpu()[0])
    del fr
    top = 4 * cfg["k"]
    cnt = np.minimum(np.diff(hp.cand_ptr), top)
    dptr = np.zeros(len(cnt) + 1, np.int64)
    dptr[1:] = np.cumsum(cnt)
    didx = np.concatenate([hp.cand_idx[hp.cand_ptr[g]:hp.cand_ptr[g] + cnt[g]] for g in range(len(cnt))])
    dhp = pipeline.HostProblem(hp.pts, hp.kp, hp.k, dptr, didx, hp.grp_ptr, hp.order, hp.ell2)
    ddp = pipeline.DeviceProblem(dhp)
    fd = pipeline.FactorBuilder(h, dhp, sic.SIC_FP32_MIXED)
    d_ms, _, _ = timed([lambda: fd.run(ddp)], 2, 1)
    S["distance_fp32"] = float(fd.sum_logv.cpu()[0])
    del fd, ddp
    torch.cuda.empty_cache()
    # ---- the same network keeping only 2k = 128 candidates (the 128-thread selection kernel,
    # two supernodes per SM): not the configured 4k, reported beside it
    l128 = learned.LearnedFactorBuilder(h, hp, learned.Proposal(h, params, top=2 * cfg["k"]), sic.SIC_FP32_MIXED)
    l128_ms, _, _ = timed([lambda: l128.run(dp)], args.steps, 1)
    S["learned_top128_fp32"] = float(l128.sum_logv.cpu()[0])
    del l128
    torch.cuda.empty_cache()
    clustered = proposal_gain_clustered(h, cfg, args.clustered_n, args.epochs) if args.clustered_n else None
    # ---- global greedy allocation of nonzeros (Section 5.4): the learned step with the
    # nonzeros of 48 picks per supernode shared out by the global greedy (at most 64 per
    # supernode), against 48 picks everywhere
    kb = 3 * cfg["k"] // 4
    sizes = np.diff(hp.grp_ptr)
    budget = int(sizes.sum()) * kb
    lbg = learned.LearnedFactorBuilder(h, hp, proposal, sic.SIC_FP32_MIXED, budget=budget)
    grdp = lbg._reduced_device(dp)
    gstep_ms, (gprop_ms, gsel_ms, galloc_ms, gfill_ms), _ = timed(
        [lambda: lbg.propose(dp), lambda: lbg.fb.select_local(grdp), lambda: lbg.fb.allocate(grdp),
         lambda: lbg.fb.fill(grdp)], args.steps, args.warmup)
    S["learned_global_48"] = float(lbg.sum_logv.cpu()[0])
    gcnt = lbg.fb.sel_count.cpu().numpy()
    kept = int(np.dot(gcnt, sizes))
    del lbg
    # the same with the decreases from the FP64 side state of the FP32 picks
    lbs = learned.LearnedFactorBuilder(h, hp, proposal, sic.SIC_FP32_MIXED, budget=budget, side_fp64=True)
    srdp = lbs._reduced_device(dp)
    sstep_ms, _, _ = timed([lambda: lbs.run(dp)], args.steps, args.warmup)
    side_ms, _, _ = timed([lambda: lbs.fb.side_state(srdp)], args.steps, 1)
    S["learned_global_48_side_fp64"] = float(lbs.sum_logv.cpu()[0])
    del lbs
    lbe = learned.LearnedFactorBuilder(h, dataclasses.replace(hp, k=kb), proposal, sic.SIC_FP32_MIXED)
    lbe.run(dp)
    h.sync()
    S["learned_even_48"] = float(lbe.sum_logv.cpu()[0])
    del lbe
    torch.cuda.empty_cache()
    # algorithmic bytes of the allocation: every decrease read once, the counts read and
    # written, the group offsets read
    U = hp.n_units
    alloc_bytes = U * cfg["k"] * 8.0 + U * (4.0 + 4.0 + 8.0)
    hbm_peak = measured_peak("hbm_gbs", 6800.0)
    global_alloc = {
        "budget_nonzeros": budget, "kept_nonzeros": kept,
        "picks_per_group_min_max": [int(gcnt.min()), int(gcnt.max())],
        "ms_per_step": gstep_ms, "phases_ms": {"proposal": gprop_ms, "select_with_decreases": gsel_ms,
                                               "allocate": galloc_ms, "fill_and_kl": gfill_ms},
        "with_side_state_fp64": {"ms_per_step": sstep_ms, "side_state_ms": side_ms},
        "allocate_roofline": {"bound": "hbm", "achieved": alloc_bytes / (galloc_ms * 1e-3) / 1e9,
                              "peak": hbm_peak, "unit": "GB/s",
                              "frac": alloc_bytes / (galloc_ms * 1e-3) / 1e9 / hbm_peak,
                              "algorithmic_bytes": alloc_bytes},
    }
    # ---- partial selection for nonadjacent groups (Section 5.2): groups kept where the ordering
    # puts them, 256 candidates after each group's first member, FP32 selection, per-column fill
    partial = None
    if args.partial_n:
        php = pipeline.prepare_partial(synthetic.points(args.partial_n, 2, cfg["seed"] + rank), hp.kp, 256, cfg["k"],
                                       cfg["m_min"], cfg["m_max"])
        pdp = pipeline.DeviceProblem(php)
        pfb = pipeline.PartialFactorBuilder(h, php, sic.SIC_FP32_MIXED)
        p_ms, (psel_ms, pfill_ms), _ = timed([lambda: pfb.select(pdp), lambda: pfb.fill(pdp)], 2, 1)
        partial = {"n": args.partial_n, "groups": php.n_units, "candidates": 256, "k": cfg["k"],
                   "ms_per_step": p_ms, "select_ms": psel_ms, "fill_ms": pfill_ms,
                   "columns_per_s": args.partial_n / (p_ms * 1e-3), "sum_logv": float(pfb.sum_logv.cpu()[0]),
                   "nnz": int(pfb.col_ptr[-1].item())}
        del pfb, pdp, php
        torch.cuda.empty_cache()
    # ---- single-target selection (one column per unit), 3-D, 512 candidates, k = 32: FP32
    # mixed and FP64, each with the FP64 fill
    single = None
    if args.single_n:
        shp = single_problem(args.single_n, cfg_single_seed(rank))
        sdp = pipeline.DeviceProblem(shp)
        single = {"n": shp.n, "dim": shp.pts.shape[1], "candidates": int(np.diff(shp.cand_ptr).max()), "k": shp.k}
        unit_peaks = {"fp32": SMS * FFMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6,
                      "fp64": SMS * DFMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6}
        for name, prec, unit in [("fp32", sic.SIC_FP32_MIXED, "FP32 FFMA"), ("fp64", sic.SIC_FP64, "FP64 DFMA")]:
            peak = unit_peaks[name]
            sfb = pipeline.FactorBuilder(h, shp, prec)
            s_ms, (ssel_ms, sfill_ms), _ = timed([lambda: sfb.select(sdp), lambda: sfb.fill(sdp)], 3, 1)
            fl = select_columns_flops(shp.cand_ptr, sfb.sel_count.cpu().numpy())
            # the whole build (one persistent selection launch, the nnz scan, the fill) captured
            # once in a CUDA graph and replayed
            sg = torch.cuda.CUDAGraph()
            side = torch.cuda.Stream()
            side.wait_stream(stream)
            with torch.cuda.stream(side):
                sfb.run(sdp)
            stream.wait_stream(side)
            with torch.cuda.graph(sg):
                sfb.run(sdp)
            g_ms, _, _ = timed([sg.replay], 3, 1)
            del sg
            single[name] = {"ms_per_step": s_ms, "graph_ms_per_step": g_ms,
                            "graph_columns_per_s": shp.n / (g_ms * 1e-3), "select_ms": ssel_ms, "fill_ms": sfill_ms,
                            "columns_per_s": shp.n / (s_ms * 1e-3), "sum_logv": float(sfb.sum_logv.cpu()[0]),
                            "nnz": int(sfb.col_ptr[-1].item()),
                            "select_roofline": {"bound": "alu", "achieved": fl / (ssel_ms * 1e-3) / 1e12,
                                                "peak": peak / 1e12, "unit": "TFLOP/s",
                                                "frac": fl / (ssel_ms * 1e-3) / peak, "peak_of": unit}}
            del sfb
        del sdp, shp
        torch.cuda.empty_cache()
    cfg1 = config1(h, timed, stream) if args.cfg1 and rank == 0 else None
    base = S["plain_fp64"] - S["reference_2k"]
    kl_gap = {k: (S[k] - S["plain_fp64"]) / base for k in ["learned_fp32", "plain_fp32", "distance_fp32",
                                                           "learned_top128_fp32",
                                                           "learned_global_48", "learned_global_48_side_fp64",
                                                           "learned_even_48"]}

    # ---- end to end through the C-ABI with host buffers (pinned), copies in the region.
    # Every step copies its inputs host->device and its factor device->host.  Two device
    # slots: step i's input copy (one copy stream) and factor read-back (another) overlap
    # the neighbouring steps' compute on the compute stream.
    hpin = {k: torch.from_numpy(v).pin_memory() for k, v in
            dict(pts=hp.pts, grp_ptr=hp.grp_ptr, cand_ptr=hp.cand_ptr, cand_idx=hp.cand_idx).items()}
    out_host = dict(col_ptr=torch.empty(N + 1, dtype=torch.int64).pin_memory(),
                    row_idx=torch.empty(nnz, dtype=torch.int32).pin_memory(),
                    val=torch.empty(nnz, dtype=torch.float64).pin_memory(),
                    sum_logv=torch.empty(1, dtype=torch.float64).pin_memory())
    h2d = sum(t.numel() * t.element_size() for t in hpin.values())
    d2h = (N + 1) * 8 + nnz * 12 + 8
    dp2 = pipeline.DeviceProblem(hp)
    lb2 = learned.LearnedFactorBuilder(h, hp, proposal, sic.SIC_FP32_MIXED)
    slots = [(dp, lb), (dp2, lb2)]
    x_in, x_out = torch.cuda.Stream(), torch.cuda.Stream()

    def e2e_run(K):
        done, ev_in, ev_out = {}, {}, {}
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        x_in.wait_stream(stream)
        x_out.wait_stream(stream)
        for i in range(K):
            d, b = slots[i % 2]
            with torch.cuda.stream(x_in):
                if i >= 2:
                    x_in.wait_event(done[i - 2])  # the slot's inputs are no longer read
                for key in ("pts", "grp_ptr", "cand_ptr", "cand_idx"):
                    getattr(d, key).copy_(hpin[key], non_blocking=True)
                ev_in[i] = torch.cuda.Event()
                ev_in[i].record(x_in)
            stream.wait_event(ev_in[i])
            if i >= 2:
                stream.wait_event(ev_out[i - 2])  # the slot's factor has been read back
            b.run(d)
            done[i] = torch.cuda.Event()
            done[i].record(stream)
            with torch.cuda.stream(x_out):
                x_out.wait_event(done[i])
                out_host["col_ptr"].copy_(b.fb.col_ptr, non_blocking=True)
                out_host["row_idx"].copy_(b.fb.row_idx[:nnz], non_blocking=True)
                out_host["val"].copy_(b.fb.val[:nnz], non_blocking=True)
                out_host["sum_logv"].copy_(b.fb.sum_logv, non_blocking=True)
                ev_out[i] = torch.cuda.Event()
                ev_out[i].record(x_out)
        stream.wait_event(ev_out[K - 1])
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / K

    e2e_run(2)
    h.sync()
    barrier(ws)
    e2e_steps = max(args.steps, 8)  # amortises the pipeline's fill (first copy in) and drain (last copy out)
    e2e_ms = max_over_ranks(e2e_run(e2e_steps), ws)
    h.sync()
    if abs(float(out_host["sum_logv"][0]) - S["learned_fp32"]) > 1e-6 * abs(S["learned_fp32"]):
        raise RuntimeError("end-to-end result differs from the device-timed step")
    del dp2, lb2

    # ---- a10: the factor as a preconditioner, y = L^T x, L x and L L^T x (HBM-bound) on the
    # step's factor.  Algorithmic bytes per product: the factor once (12 B per nonzero + 8 B per
    # column pointer), x read once and y written once (8 B x nrhs per point each)
    hbm_peak = measured_peak("hbm_gbs", 6800.0)
    nnz_f = int(lb.col_ptr[-1].item())
    apply_res = {}
    gen = torch.Generator(device="cuda").manual_seed(0)
    for nrhs in (1, 8):
        X = torch.randn(N, nrhs, dtype=torch.float64, device="cuda", generator=gen)
        Y = torch.empty_like(X)
        wsa = sic._ws(sic.apply_factor_workspace(N, nrhs, sic.SIC_OP_LLT), "cuda")
        for name, op, passes in (("LT", sic.SIC_OP_LT, 1), ("L", sic.SIC_OP_L, 1), ("LLT", sic.SIC_OP_LLT, 2)):
            a_ms, _, _ = timed([lambda: sic.apply_factor(h, lb.col_ptr, lb.fb.row_idx, lb.fb.val, op, X, Y, wsa)],
                               5, 2)
            byts = passes * (12.0 * nnz_f + 8.0 * (N + 1) + 2 * 8.0 * nrhs * N)
            apply_res[f"{name}_nrhs{nrhs}"] = {"ms": a_ms, "gbs": byts / (a_ms * 1e-3) / 1e9,
                                               "frac": byts / (a_ms * 1e-3) / 1e9 / hbm_peak}
        del X, Y, wsa
    apply_res["peak_gbs"] = hbm_peak
    apply_res["nnz"] = nnz_f

    # ---- rooflines (ALU bound; peaks derived from unit counts and the maximum clock)
    rp = lb.rhp
    f32_peak = SMS * FFMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12
    f64_peak = SMS * DFMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12
    sel_tf = select_flops(rp.grp_ptr, rp.cand_ptr, hp.k) / (sel_ms * 1e-3) / 1e12
    rows = float(hp.cand_ptr[-1])
    mlp_tf = rows * 2.0 * (16 * 128 + 128 * 128 + 128) / (mlp_ms * 1e-3) / 1e12  # layer 1 padded to K = 16
    bf16_peak = measured_peak("bf16_tflops", 1900.0)
    fill_tf = fill_flops(hp.grp_ptr, sel_count_learned) / (fill_ms * 1e-3) / 1e12
    kernels = {
        "k_select_agg_reg (FP32, 256 candidates)": {"ms": sel_ms, "achieved_tflops": sel_tf, "peak_tflops": f32_peak,
                                                 "frac": sel_tf / f32_peak, "unit_peak": "FP32 FFMA"},
        "k_fill (FP64)": {"ms": fill_ms, "achieved_tflops": fill_tf, "peak_tflops": f64_peak,
                          "frac": fill_tf / f64_peak, "unit_peak": "FP64 DFMA"},
        "k_features": {"ms": feat_ms},
        "k_mlp_tc (BF16 tcgen05, TMEM)": {"ms": mlp_ms, "achieved_tflops": mlp_tf, "peak_tflops": bf16_peak,
                                        "frac": mlp_tf / bf16_peak, "unit_peak": "measured cuBLAS BF16 (burst)"},
        "top-k": {"ms": topk_ms},
    }
    if fill_ms >= sel_ms:
        # DRAM bytes of the two k_fill launches measured at N = 2^19, scaled by the supernode
        # count; the algorithmic bytes are the factor written (row index + value per nonzero),
        # col_ptr and log v, the points and the picks read
        traffic = FILL_DRAM_BYTES_N2E19 * hp.n_units / GROUPS_N2E19 if FILL_DRAM_BYTES_N2E19 else None
        roof = {"bound": "alu", "kernel": "k_fill (FP64 fill, both launches)", "achieved": fill_tf,
                "peak": f64_peak, "unit": "TFLOP/s", "frac": fill_tf / f64_peak, "traffic": traffic,
                "traffic_algorithmic": nnz * 12.0 + N * (8.0 + 8.0 + 8.0 * hp.pts.shape[1]) + hp.n_units * hp.k * 4.0,
                "peak_source": "152 SMs x 2 FP64 FMA/clk x 2 x 2070 MHz (derived from unit counts; a DFMA "
                               "throughput kernel saturates at 1.6 FMA/clk/SM = 1.0 TFLOP/s)",
                "achieved_of": "the LDL^T's and the back substitutions' multiply-adds (2 FLOPs each) per second, "
                               "FP64-equivalent: each panel's trailing update runs as exact integer products "
                               "with one FP64 addition per entry, the back substitutions in double-float "
                               "arithmetic on the FP32 pipe"}
    else:
        traffic = SEL_DRAM_BYTES_N2E19 * hp.n_units / GROUPS_N2E19 if SEL_DRAM_BYTES_N2E19 else None
        roof = {"bound": "alu", "kernel": "FP32 supernodal selection (k_agg_target_chol + k_agg_target_cols + "
                                          "k_select_agg_reg<256>)", "achieved": sel_tf, "peak": f32_peak,
                "unit": "TFLOP/s", "frac": sel_tf / f32_peak, "traffic": traffic,
                "peak_source": "152 SMs x 128 FP32 FMA/clk x 2 x 2070 MHz (derived; measured probe 75 TFLOP/s)"}

    pcg = None
    if args.pcg_n and rank == 0:
        pcg = pcg_comparison(h, cfg, params, args.pcg_n)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        v, cols, groups, el = oracle_sample(host_problem_dict(hp), 2 * args.ref_seconds, threads)
        cpu = {"value": v, "unit": "columns/s", "cores": threads, "kind": "oracle",
               "sample": f"{groups} random supernodes ({cols} columns), FP64 two-factor greedy + dense fill on all "
                         f"1024 candidates, {el:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "columns/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"N={N} uniform [0,1]^2 (seed {cfg['seed']}), Matern 3/2, ell=0.02, "
                                   f"nugget 1e-6, supernodes {cfg['m_min']}..{cfg['m_max']} (mean "
                                   f"{N / hp.n_units:.1f}), C=1024, k=64",
                       "path": f"learned proposal (top {top} of 1024) -> select_aggregated FP32 -> factor_nnz -> "
                               "build_factor FP64 -> sum log v",
                       "groups": hp.n_units, "nnz": nnz, "l2": "inputs larger than L2 (candidate lists "
                       f"{hp.cand_idx.nbytes / 2**20:.0f} MiB, features {int(hp.cand_ptr[-1]) * 32 / 2**20:.0f} MiB, "
                       f"factor {nnz * 12 / 2**20:.0f} MiB)",
                       "parallelism": "one GPU, the whole factor"},
            "kl_gap": kl_gap,
            "sum_logv": S,
            "fp64_plain": {"value": ws * N / (p64_ms * 1e-3), "unit": "columns/s", "ms_per_step": p64_ms,
                           "select_ms": p64_sel, "fill_ms": p64_fill},
            "fp32_plain": {"value": ws * N / (p32_ms * 1e-3), "unit": "columns/s", "ms_per_step": p32_ms,
                           "select_ms": p32_sel, "fill_ms": p32_fill},
            "distance_top256_fp32": {"value": ws * N / (d_ms * 1e-3), "unit": "columns/s", "ms_per_step": d_ms},
            "learned_top128_fp32": {"value": ws * N / (l128_ms * 1e-3), "unit": "columns/s", "ms_per_step": l128_ms,
                                    "note": "top 2k = 128 instead of the configured 4k (not the headline)"},
            "proposal_gain_clustered": clustered,
            "speedup_vs_fp64_plain": p64_ms / t_step,
            "timing": "CUDA graph of the whole step, replayed; phases_ms from the same launches issued "
                      "eagerly with events between phases",
            "eager_ms_per_step": eager_ms,
            "phases_ms": {"features": feat_ms, "mlp": mlp_ms, "topk": topk_ms, "select": sel_ms,
                          "fill_and_kl": fill_ms},
            "setup_s": {"prep_host": prep_s, "train_proposal": train_s, "train_selections": n_sel,
                        "train_loss": [hist[0][1], hist[-1][1]]},
            "kernels": kernels,
            "roofline": roof,
            "e2e": {"value": ws * N / (e2e_ms * 1e-3), "unit": "columns/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms, "steps": e2e_steps,
                    "pipelining": "two device slots; each step's input copy and factor read-back overlap the "
                                  "neighbouring steps' compute"},
            "autotune": {"fill_group_split": tuned_split, "table": sic.tune_table(h)},
            "gpu_launches": LAUNCHES_PER_STEP * args.steps,
            "clocks": clocks,
            "pcg": pcg,
            "global_allocation": global_alloc,
            "partial_selection": partial,
            "single_target": single,
            "config1": cfg1,
            "apply_factor": apply_res,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    h.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
