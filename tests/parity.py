"""Parity helpers: compare the CUDA path's selections and factor with the oracle.

Selections are compared by *oracle replay*: run the oracle; at the first step where the
GPU picked differently, the oracle's own score of the GPU's pick must be within the
stated relative band of the oracle's best score at that step (a near-tie); the oracle
then continues from the GPU's pick.  Counts must match under the replayed prefix.
Returns the number of steps that needed the band, so tests can report it.
"""
import numpy as np


class ReplayStats:
    def __init__(self):
        self.steps = 0
        self.banded = 0
        self.worst = 0.0
        self.units = 0

    def __repr__(self):
        return (f"units={self.units} steps={self.steps} banded={self.banded} "
                f"({self.banded / max(1, self.steps):.2e}) worst_rel_gap={self.worst:.3e}")


def _replay(run, gpu_sel, cand, band, stats, what, abs_band=0.0):
    """run(forced) -> oracle dict with sel/best/chosen; forced lists indices into cand.
    A differing pick is accepted when best - chosen <= band * |best| + abs_band."""
    pos2idx = {int(p): i for i, p in enumerate(cand)}
    gpu_sel = [int(x) for x in gpu_sel]
    forced = []
    stats.units += 1
    stats.steps += len(gpu_sel)
    while True:
        r = run(forced)
        o = [int(x) for x in r["sel"]]
        j = len(forced)
        while j < min(len(o), len(gpu_sel)) and o[j] == gpu_sel[j]:
            j += 1
        if j == len(o) and j == len(gpu_sel):
            return
        if j >= len(gpu_sel) or j >= len(o):
            raise AssertionError(f"{what}: pick counts differ after replay: gpu {len(gpu_sel)} oracle {len(o)} "
                                 f"(gpu {gpu_sel}, oracle {o})")
        if gpu_sel[j] not in pos2idx:
            raise AssertionError(f"{what}: gpu pick {gpu_sel[j]} at step {j} is not a candidate")
        forced = [pos2idx[p] for p in gpu_sel[:j + 1]]
        r2 = run(forced)
        best, chosen = float(r2["best"][j]), float(r2["chosen"][j])
        gap = (best - chosen) / abs(best) if best != 0 else abs(best - chosen)
        stats.banded += 1
        stats.worst = max(stats.worst, gap)
        if best - chosen > band * abs(best) + abs_band:
            raise AssertionError(f"{what}: step {j} gpu picked {gpu_sel[j]} with oracle score {chosen!r}, "
                                 f"oracle best {best!r} (relative gap {gap:.3e} > {band:.1e})")


def replay_single(oracle, kp, P, target, cand, k, gpu_sel, band, stats, floor=None, abs_band=0.0):
    def run(forced):
        return oracle.select_single(kp, P, target, cand, k, floor=floor, forced=forced if forced else None)
    _replay(run, gpu_sel, cand, band, stats, f"column {target}", abs_band)


def replay_multi(oracle, kp, P, g0, m, cand, k, gpu_sel, band, stats, floor=None, abs_band=0.0):
    def run(forced):
        return oracle.select_multi(kp, P, g0, m, cand, k, floor=floor, forced=forced if forced else None)
    _replay(run, gpu_sel, cand, band, stats, f"group at {g0}", abs_band)


def column_errors(L_gpu, L_ref):
    """max |dL| / max |L_ref| over one column."""
    return float(np.max(np.abs(L_gpu - L_ref)) / max(np.max(np.abs(L_ref)), 1e-300))
