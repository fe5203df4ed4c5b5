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


def _replay(run, gpu_sel, cand, band, stats, what, abs_band=0.0, resolves=None):
    """run(forced) -> oracle dict with sel/best/chosen; forced lists indices into cand.
    A differing pick is accepted when best - chosen <= band * |best| + abs_band, or when
    resolves(prefix, oracle_pick, gpu_pick) says the two are not resolved apart."""
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
        if best - chosen > band * abs(best) + abs_band and not (resolves and resolves(gpu_sel[:j], o[j], gpu_sel[j])):
            raise AssertionError(f"{what}: step {j} gpu picked {gpu_sel[j]} with oracle score {chosen!r}, "
                                 f"oracle best {best!r} (relative gap {gap:.3e} > {band:.1e})")


def replay_single(oracle, kp, P, target, cand, k, gpu_sel, band, stats, floor=None, abs_band=0.0):
    def run(forced):
        return oracle.select_single(kp, P, target, cand, k, floor=floor, forced=forced if forced else None)
    _replay(run, gpu_sel, cand, band, stats, f"column {target}", abs_band)


def conditional_variances(oracle, kp, P, g0, m, S, j):
    """(var of j given S, var of j given P and S) in FP64 from dense solves."""
    S = [int(x) for x in S]
    tg = list(range(g0, g0 + m))
    K = oracle.theta_matrix(kp, P, tg + S + [int(j)])
    n0 = m + len(S)
    kj = K[-1, -1]
    v2 = kj - K[:n0, -1] @ np.linalg.solve(K[:n0, :n0], K[:n0, -1])
    if S:
        Ks = K[m:n0, m:n0]
        v1 = kj - K[m:n0, -1] @ np.linalg.solve(Ks, K[m:n0, -1])
    else:
        v1 = kj
    return float(v1), float(v2)


def replay_multi(oracle, kp, P, g0, m, cand, k, gpu_sel, band, stats, floor=None, abs_band=0.0, var_abs=0.0):
    """var_abs > 0: a differing pick is also accepted when the ratio scores var1 / var2 of
    the two picks cannot be told apart with every conditional variance known only to
    +-var_abs: (v1_c + E) / (v2_c - E) >= (v1_b - E) / (v2_b + E)."""
    def run(forced):
        return oracle.select_multi(kp, P, g0, m, cand, k, floor=floor, forced=forced if forced else None)

    def resolves(prefix, best_pick, gpu_pick):
        E = var_abs
        v1b, v2b = conditional_variances(oracle, kp, P, g0, m, prefix, best_pick)
        v1c, v2c = conditional_variances(oracle, kp, P, g0, m, prefix, gpu_pick)
        return v2c <= E or (v1c + E) / (v2c - E) >= (v1b - E) / (v2b + E)

    _replay(run, gpu_sel, cand, band, stats, f"group at {g0}", abs_band, resolves if var_abs > 0 else None)


def column_errors(L_gpu, L_ref):
    """max |dL| / max |L_ref| over one column."""
    return float(np.max(np.abs(L_gpu - L_ref)) / max(np.max(np.abs(L_ref)), 1e-300))
