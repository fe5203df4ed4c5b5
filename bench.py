"""Benchmark: factor columns per second for the supernodal sparse inverse-Cholesky build
(N = 2^20 points uniform in the unit square, Matern 3/2, length scale 0.02, nugget 1e-6,
supernodes of 8..64 targets, 1024 candidates and k = 64 picks per supernode).

One step = the whole device path over the prepared inputs: supernodal greedy selection
(FP32-mixed, the headline; FP64 timed alongside) -> nnz scan -> FP64 KL-optimal fill ->
sum of log conditional variances.  Ordering / candidate / grouping prep is host set-up,
timed and reported separately.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl sic|reference]

Prints one JSON line (rank 0).  Under torchrun each rank builds its own problem
(seed = rank; weak scaling, no data-path collective) and the max step time over ranks
is used.  `--impl reference` times the CPU oracle (FP64, all host cores) on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
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
FFMA_PER_SM_CLK = 128          # FP32 FMA lanes per SM per clock (Blackwell SM)
SMS = 152
SM_MAX_MHZ = 2070.0


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "fallback": True}


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

def select_flops(hp) -> float:
    """Algorithmic FP32 FLOPs of the supernodal selection for the whole problem
    (2 per fused multiply-add): target columns R*m^2/2 FMA (R = C + m rows), then per
    step t the two left-looking dot products C*(t) + C*(m + t), the two downdates 2C and
    the score C (one division counted as one FMA); kernel evaluations not counted."""
    m = np.diff(hp.grp_ptr).astype(np.float64)
    C = np.diff(hp.cand_ptr).astype(np.float64)
    k = float(hp.k)
    R = C + m
    init = R * m * (m - 1) / 2.0
    steps = C * (k * (k - 1) + k * m + 3.0 * k)
    return float(2.0 * np.sum(init + steps))


# ------------------------------------------------------------- oracle ----

def oracle_sample(hp, seconds: float, threads: int):
    """Time the CPU oracle (FP64 two-factor greedy + per-member dense fill) on a sample
    of supernodes spread over the ordering until `seconds` have elapsed.  Returns
    (columns/s, columns done, groups done)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    oracle.build()
    kp = hp.kp
    okp = oracle.kernel(kp.dim, kp.nu_x2, kp.length_scale, kp.variance, kp.nugget)
    gp, P = hp.grp_ptr, hp.pts
    G = len(gp) - 1
    rng = np.random.default_rng(0)
    order = rng.permutation(G)

    def one(g):
        g0, g1 = int(gp[g]), int(gp[g + 1])
        cand = hp.cand_idx[hp.cand_ptr[g]:hp.cand_ptr[g + 1]]
        sel = oracle.select_multi(okp, P, g0, g1 - g0, cand, hp.k)["sel"]
        for a in range(g1 - g0):
            oracle.fill_member(okp, P, g0, g1 - g0, a, sel)
        return g1 - g0

    cols = groups = 0
    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        i = 0
        while time.perf_counter() - t0 < seconds and i < G:
            batch = order[i:i + 4 * threads]
            i += len(batch)
            cols += sum(ex.map(one, batch))
            groups += len(batch)
    el = time.perf_counter() - t0
    return cols / el, cols, groups, el


# ---------------------------------------------------------------- main ---

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


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


def run_reference(args, ws, rank):
    if rank != 0:
        return
    cfg = synthetic.PRESETS[WORKLOAD]
    from paper_2307_11648_gb300 import pipeline, sic
    kp = sic.kernel(cfg["dim"], cfg["nu_x2"], cfg["length_scale"], cfg["variance"], cfg["nugget"])
    pts = synthetic.points(cfg["n"], cfg["dim"], cfg["seed"])
    hp = pipeline.prepare_groups(pts, kp, cfg["n_cand"], cfg["k"], cfg["m_min"], cfg["m_max"])
    threads = os.cpu_count() or 1
    vals = []
    cols_tot = 0
    for _ in range(args.warmup):
        oracle_sample(hp, 2.0, threads)
    for _ in range(args.steps):
        v, cols, groups, el = oracle_sample(hp, args.ref_seconds, threads)
        vals.append(v)
        cols_tot += cols
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "columns/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * hp.n / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "N=2^20 uniform [0,1]^2, Matern 3/2, ell=0.02, nugget 1e-6, supernodes 8..64, "
                                   "C=1024, k=64", "groups": hp.n_units},
            "cpu_baseline": {"value": v, "unit": "columns/s", "cores": threads, "kind": "oracle",
                             "sample": f"random supernodes, {args.ref_seconds:.0f} s per step of FP64 two-factor "
                                       f"greedy + dense fill ({cols_tot} columns over {args.steps} steps)"},
            "e2e": {"value": v, "unit": "columns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sic", choices=["sic", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--ref-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=0, help="override N (smaller runs for profiling)")
    args = ap.parse_args()
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

    from paper_2307_11648_gb300 import build, pipeline, sic
    build.build()
    torch.cuda.set_device(local)
    cfg = dict(synthetic.PRESETS[WORKLOAD])
    if args.n:
        cfg["n"] = args.n
    kp = sic.kernel(cfg["dim"], cfg["nu_x2"], cfg["length_scale"], cfg["variance"], cfg["nugget"])
    t0 = time.perf_counter()
    pts = synthetic.points(cfg["n"], cfg["dim"], cfg["seed"] + rank)
    hp = pipeline.prepare_groups(pts, kp, cfg["n_cand"], cfg["k"], cfg["m_min"], cfg["m_max"])
    prep_s = time.perf_counter() - t0
    h = sic.Handle(local)
    dp = pipeline.DeviceProblem(hp)
    stream = torch.cuda.current_stream()
    N = hp.n

    def timed(fb, steps, warmup, sampler=None):
        for _ in range(warmup):
            fb.run(dp)
        h.sync()
        barrier(ws)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
                torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if sampler:
            sampler.start()
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for e0, e1, e2 in evs:
            e0.record(stream)
            fb.select(dp)
            e1.record(stream)
            fb.fill(dp)
            e2.record(stream)
        end.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop() if sampler else None
        h.sync()
        total_ms = start.elapsed_time(end)
        sel_ms = [a.elapsed_time(b) for a, b, _ in evs]
        fill_ms = [b.elapsed_time(c) for _, b, c in evs]
        return total_ms, sel_ms, fill_ms, clocks

    # ---- headline: FP32-mixed selection + FP64 fill
    fb32 = pipeline.FactorBuilder(h, hp, sic.SIC_FP32_MIXED)
    sampler = ClockSampler(local)
    total_ms, sel_ms, fill_ms, clocks = timed(fb32, args.steps, args.warmup, sampler)
    t_step = max_over_ranks(total_ms / args.steps, ws)
    value = ws * N / (t_step * 1e-3)
    sum_logv32 = float(fb32.sum_logv.cpu()[0])

    # ---- plain FP64 path (same pipeline, FP64 selection)
    fb64 = pipeline.FactorBuilder(h, hp, sic.SIC_FP64)
    t64, sel64, fill64, _ = timed(fb64, args.fp64_steps, 1)
    t64_step = max_over_ranks(t64 / args.fp64_steps, ws)
    sum_logv64 = float(fb64.sum_logv.cpu()[0])
    del fb64

    # ---- end to end through the C-ABI with host buffers (pinned), copies in the region
    hpin = {k: torch.from_numpy(v).pin_memory() for k, v in
            dict(pts=hp.pts, grp_ptr=hp.grp_ptr, cand_ptr=hp.cand_ptr, cand_idx=hp.cand_idx).items()}
    nnz_cap = fb32.nnz_cap
    out_host = dict(col_ptr=torch.empty(N + 1, dtype=torch.int64).pin_memory(),
                    row_idx=torch.empty(nnz_cap, dtype=torch.int32).pin_memory(),
                    val=torch.empty(nnz_cap, dtype=torch.float64).pin_memory(),
                    sum_logv=torch.empty(1, dtype=torch.float64).pin_memory())
    h2d = sum(t.numel() * t.element_size() for t in hpin.values())
    nnz = int(fb32.col_ptr[-1].item())
    d2h = (N + 1) * 8 + nnz * 12 + 8

    def e2e_step():
        dp.pts.copy_(hpin["pts"], non_blocking=True)
        dp.grp_ptr.copy_(hpin["grp_ptr"], non_blocking=True)
        dp.cand_ptr.copy_(hpin["cand_ptr"], non_blocking=True)
        dp.cand_idx.copy_(hpin["cand_idx"], non_blocking=True)
        fb32.run(dp)
        out_host["col_ptr"].copy_(fb32.col_ptr, non_blocking=True)
        out_host["row_idx"][:nnz].copy_(fb32.row_idx[:nnz], non_blocking=True)
        out_host["val"][:nnz].copy_(fb32.val[:nnz], non_blocking=True)
        out_host["sum_logv"].copy_(fb32.sum_logv, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    barrier(ws)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    s1.record(stream)
    torch.cuda.synchronize()
    h.sync()
    e2e_ms = max_over_ranks(s0.elapsed_time(s1) / args.steps, ws)

    # ---- roofline of the dominant kernel (FP32 selection; ALU bound)
    flops = select_flops(hp)
    sel_avg = statistics.mean(sel_ms)
    achieved = flops / (sel_avg * 1e-3) / 1e12
    peak_tf = SMS * FFMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12
    fill_avg = statistics.mean(fill_ms)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        v, cols, groups, el = oracle_sample(hp, args.ref_seconds, threads)
        cpu = {"value": v, "unit": "columns/s", "cores": threads, "kind": "oracle",
               "sample": f"{groups} random supernodes ({cols} columns), FP64 two-factor greedy + dense fill, "
                         f"{el:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "columns/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"N={N} uniform [0,1]^2 (seed {cfg['seed']}+rank), Matern 3/2, ell=0.02, "
                                   f"nugget 1e-6, supernodes {cfg['m_min']}..{cfg['m_max']} (mean "
                                   f"{N / hp.n_units:.1f}), C=1024, k=64; FP32-mixed selection, FP64 fill",
                       "groups": hp.n_units, "nnz": nnz, "l2": "inputs larger than L2 (candidate lists "
                       f"{hp.cand_idx.nbytes / 2**20:.0f} MiB, factor {nnz * 12 / 2**20:.0f} MiB)",
                       "parallelism": f"independent problems per rank ({ws})", "path": "select_aggregated(FP32) "
                       "-> factor_nnz -> build_factor(FP64) -> sum log v"},
            "fp64_plain": {"value": ws * N / (t64_step * 1e-3), "unit": "columns/s", "ms_per_step": t64_step,
                           "select_ms": statistics.mean(sel64), "fill_ms": statistics.mean(fill64)},
            "speedup_vs_fp64_plain": t64_step / t_step,
            "sum_logv": {"fp32_mixed": sum_logv32, "fp64_plain": sum_logv64,
                         "rel_diff": (sum_logv32 - sum_logv64) / abs(sum_logv64)},
            "phases_ms": {"select": sel_avg, "fill_and_kl": fill_avg, "prep_host_s": prep_s},
            "roofline": {"bound": "alu", "kernel": "k_select_agg<float>", "achieved": achieved,
                         "peak": peak_tf, "unit": "TFLOP/s", "frac": achieved / peak_tf, "traffic": None,
                         "peak_source": "152 SMs x 128 FP32 FMA/clk x 2 x 2070 MHz (derived, not measured)"},
            "e2e": {"value": ws * N / (e2e_ms * 1e-3), "unit": "columns/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
            "gpu_launches": 8 * args.steps,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    h.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
