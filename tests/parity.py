"""Parity helpers: compare the CUDA path's selections and factor with the oracle.

Selections are compared by *oracle replay*: run the oracle; at the first step where the
GPU picked differently, the oracle scores the GPU's pick in the same state (the same
earlier picks); if the pick is acceptable the oracle continues from it.  Counts must
match under the replayed prefix.

What is compared is each pick's decrease of the unit's objective, in nats of 2 KL
(eq. obj_chol: 2 KL = sum_i log v_i - logdet Theta), computed by the oracle in FP64:
  * single target (Section 3.1): D = log(v_t / v_{t+1}) = -log(1 - cov_j^2 / (var_j v_t)),
    v_t the target's conditional variance before the step;
  * supernode (Section 5.2, eq. greedy_mult): D = log(var_j|I / var_j|I,P), the decrease of
    logdet Theta_{PP|I}.
The gap of a differing pick is g = D(oracle best) - D(GPU pick) >= 0.

FP64 selections: a differing pick is a near-tie when the two scores agree to TIE_BAND
relative (1e-10); nothing else is accepted.

FP32 selections (the benchmark spec precision split: state in FP32): a differing pick is accepted
when g <= REL32 * D(best) + delta, where REL32 = 1e-3 is the stated relative band and
delta is what FP32 arithmetic cannot resolve in this state.  Derivation of delta (first
order): a new column u = n / sqrt(v) of a partial factor is formed from a numerator n known
to about 4 ulp of sigma^2 (the kernel entry's hardware exp, the dot product's roundings)
divided by the square root of its pivot's conditional variance v, so u's error is
amplified by sigma / sqrt(v); the downdate var -= u^2 then moves a variance by up to
2 |u| du <= 2 sigma du.  Summed over the columns (errors add, worst case):
    E = E32 sigma^2 (1 + sum over the factor's columns of sqrt(sigma^2 / v)),  E32 = 8 eps32,
the pivots v being the FP64 conditional variances of the earlier picks (and, for the
second factor of a supernode, of the targets first: its m target columns).  Then
  * single target: the score s = cov^2 / var of a candidate is known to
    E (2a + a^2) with a = |cov| / var, so two scores closer than E (2a_b + a_b^2 + 2a_c + a_c^2)
    cannot be ordered in FP32; in decrease units delta = log(1 + that / v_{t+1,b});
  * supernode: log var|I and log var|I,P are known to E1 / var|I and E2 / var|I,P (E1 over
    the picks' columns, E2 over the targets' and the picks' columns of the second factor), so
    delta = log((v1_c + E1)(v2_b + E2) / ((v2_c - E2)(v1_b - E1))) - log(v1_c v2_b / (v2_c v1_b))
    (the two decreases' intervals overlap), any pick being accepted once v2_c <= E2.
(a, v1, v2 and the pivots from dense FP64 solves.)  delta is tiny while the variances in
play are large and unbounded once a candidate's var|I,P approaches E2: on the finest
supernodes the targets nearly determine every candidate (var|I,P ~ 2 nugget), where FP32
cannot rank candidates at all; the aggregate bound on sum log v (the survey's FP32
tolerance, sum log v_FP32 <= sum log v_FP64 + 1e-3 KL_plain) is the check of what that costs.

Every test asserts the fraction of steps that needed acceptance and the worst gap
(ReplayStats.check), with caps stated in the test.
"""
import math

import numpy as np

TIE_BAND = 1e-10
E32 = 8 * 2.0 ** -24
REL32 = 1e-3
UNRESOLVED = 1e-3  # a step whose delta exceeds this many nats is not resolvable in FP32


class ReplayStats:
    def __init__(self):
        self.steps = 0
        self.banded = 0
        self.worst = 0.0        # largest gap g (nats)
        self.unresolved = 0     # accepted steps whose FP32 resolution delta > UNRESOLVED
        self.units = 0
        self.records = []       # (g, delta) of every differing step

    @property
    def frac(self):
        return self.banded / max(1, self.steps)

    def __repr__(self):
        return (f"units={self.units} steps={self.steps} banded={self.banded} ({self.frac:.2e}) "
                f"worst_gap={self.worst:.3e} nats unresolved={self.unresolved}")

    def check(self, max_frac, max_gap):
        """The stated caps of a test: fraction of steps that differ from the oracle's pick
        and the largest decrease gap among them."""
        assert self.frac <= max_frac, f"{self}: banded fraction above {max_frac}"
        assert self.worst <= max_gap, f"{self}: worst gap above {max_gap} nats"


def _replay(run, gpu_sel, cand, stats, what, accept):
    """run(forced) -> oracle dict with sel/best/chosen(/vtar); forced lists indices into cand.
    accept(j, r2, best_pick, gpu_pick, prefix) -> (ok, gap, delta) for a differing step j
    (r2: the oracle run forced through the GPU's pick j)."""
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
        ok, gap, delta = accept(j, r2, o[j], gpu_sel[j], gpu_sel[:j])
        stats.banded += 1
        stats.worst = max(stats.worst, gap)
        stats.records.append((gap, delta))
        if delta > UNRESOLVED:
            stats.unresolved += 1
        if not ok:
            raise AssertionError(f"{what}: step {j} gpu picked {gpu_sel[j]} (oracle best {o[j]}): decrease gap "
                                 f"{gap:.3e} nats above the accepted {delta:.3e} (+{REL32:g} relative)")


def _tie(best, chosen):
    return best - chosen <= TIE_BAND * abs(best)


def cond_single(oracle, kp, P, t, S, j):
    """(v_t, cov, var): the target's variance, its covariance with j and j's variance, all
    conditioned on the positions S, by dense FP64 solves."""
    S = [int(x) for x in S]
    K = oracle.theta_matrix(kp, P, S + [int(t), int(j)])
    s = len(S)
    if s:
        X = np.linalg.solve(K[:s, :s], K[:s, s:])
        A = K[s:, s:] - K[:s, s:].T @ X
    else:
        A = K[s:, s:]
    return float(A[0, 0]), float(A[0, 1]), float(A[1, 1])


def replay_single(oracle, kp, P, target, cand, k, gpu_sel, stats, fp32=False, floor=None):
    """Single-target replay; the oracle's scores are cov^2 / var and vtar[t] the target's
    variance before step t."""

    def run(forced):
        return oracle.select_single(kp, P, target, cand, k, floor=floor, forced=forced if forced else None)

    def accept(j, r2, b, c, prefix):
        best, chosen, vt = float(r2["best"][j]), float(r2["chosen"][j]), float(r2["vtar"][j])
        vb, vc = max(vt - best, 1e-300), max(vt - chosen, 1e-300)
        gap = max(0.0, math.log(vc / vb))
        if not fp32:
            return _tie(best, chosen), gap, 0.0
        piv, _ = oracle.pivot_variances(kp, P, [], prefix)
        E = E32 * kp.variance * (1.0 + float(np.sum(np.sqrt(kp.variance / np.maximum(piv, 1e-300)))))
        res = 0.0
        for q in (b, c):
            _, cov, var = cond_single(oracle, kp, P, target, prefix, q)
            a = abs(cov) / max(var, 1e-300)
            res += E * (2 * a + a * a)
        delta = math.log1p(res / vb)
        dbest = math.log(vt / vb)
        return gap <= REL32 * dbest + delta, gap, delta

    _replay(run, gpu_sel, cand, stats, f"column {target}", accept)


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


def replay_multi(oracle, kp, P, g0, m, cand, k, gpu_sel, stats, fp32=False, floor=None):
    """Supernode replay; the oracle's scores are var|I / var|I,P, the decrease their log."""

    def run(forced):
        return oracle.select_multi(kp, P, g0, m, cand, k, floor=floor, forced=forced if forced else None)

    def accept(j, r2, b, c, prefix):
        best, chosen = float(r2["best"][j]), float(r2["chosen"][j])
        gap = max(0.0, math.log(best / chosen))
        if not fp32:
            return _tie(best, chosen), gap, 0.0
        # pivots of the two factors: the picks given the earlier picks (first factor); the
        # targets given the earlier targets, then the picks given the targets and earlier picks
        piv1, piv2 = oracle.pivot_variances(kp, P, list(range(g0, g0 + m)), prefix)
        tdiag = np.diag(np.linalg.cholesky(oracle.theta_matrix(kp, P, list(range(g0, g0 + m))))) ** 2
        amp = lambda v: float(np.sum(np.sqrt(kp.variance / np.maximum(v, 1e-300))))  # noqa: E731
        E1 = E32 * kp.variance * (1.0 + amp(piv1))
        E2 = E32 * kp.variance * (1.0 + amp(tdiag) + amp(piv2))
        v1b, v2b = conditional_variances(oracle, kp, P, g0, m, prefix, b)
        v1c, v2c = conditional_variances(oracle, kp, P, g0, m, prefix, c)
        if v2c <= E2 or v1b <= E1:
            return True, gap, math.inf
        delta = (math.log((v1c + E1) * (v2b + E2) / ((v2c - E2) * (v1b - E1)))
                 - math.log(v1c * v2b / (v2c * v1b)))
        return gap <= REL32 * math.log(best) + delta, gap, delta

    _replay(run, gpu_sel, cand, stats, f"group at {g0}", accept)


def column_errors(L_gpu, L_ref):
    """max |dL| / max |L_ref| over one column."""
    return float(np.max(np.abs(L_gpu - L_ref)) / max(np.max(np.abs(L_ref)), 1e-300))
