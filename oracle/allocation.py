"""FP64 oracle of the global greedy allocation of nonzeros (Section 5.4) -- TEST INFRASTRUCTURE ONLY.

With a budget on the total number of off-diagonal nonzeros, the global greedy takes the next
sparsity entry from whichever unit (a column, or a supernode of m columns) lowers the KL
divergence (eq. obj_chol) the most per nonzero it adds.  A priority queue holds every unit's
best candidate, keyed by that exact decrease:

  * single column (Section 5.4.1, eq. global_obj): picking j lowers 2 KL by
    log Theta_{ii|I} - log Theta_{ii|I,j} = -log(1 - corr(y_i, y_j | I)^2); the local greedy's
    pick is the maximiser, one nonzero;
  * supernode of m targets P (Section 5.4.2): picking j lowers logdet Theta_{PP|I} by
    log Theta_{jj|I} - log Theta_{jj|I,P} (the multiple-target objective, eq. greedy_mult);
    it adds m nonzeros (one per member), so the key is that decrease / m.

The queue is popped until the budget is spent; popping a unit's entry changes only that
unit's candidate values, so the queue needs the unit's next best candidate only after a pop.
This oracle therefore runs each unit's local greedy (sic_oracle.c, FP64 Cholesky form) for up
to k picks and feeds the queue from that trajectory, one pick at a time, in the same order.

Readings where the paper leaves a choice (the same on the GPU):
  * a unit stops after k picks or when its local greedy ends (candidates exhausted);
  * equal keys pop the unit of lower index first;
  * the queue stops at the first pick whose nonzeros exceed what is left of the budget.

Pinned in tests/test_oracle_allocation.py against a brute-force global greedy that
re-evaluates every candidate of every unit by dense log-determinants after each pick, and
against an independent formulation of the queue's pop order.
"""
from __future__ import annotations

import heapq

import numpy as np

from . import select_multi, select_single


def queue_allocate(gains, costs, budget: int) -> np.ndarray:
    """Counts of leading picks that the global queue takes from each unit.

    gains[u] : the decreases (per nonzero) of unit u's successive picks, in pick order;
    costs[u] : nonzeros one pick of unit u adds (1 for a column, m for a supernode);
    budget   : total nonzeros available."""
    n = len(gains)
    counts = np.zeros(n, np.int32)
    heap = [(-float(gains[u][0]), u) for u in range(n) if len(gains[u]) > 0]
    heapq.heapify(heap)
    left = int(budget)
    while heap:
        _, u = heapq.heappop(heap)
        if costs[u] > left:
            break
        left -= int(costs[u])
        counts[u] += 1
        if counts[u] < len(gains[u]):
            heapq.heappush(heap, (-float(gains[u][counts[u]]), u))
    return counts


def column_gains(kp, pts, targets, cand_lists, k: int):
    """Local greedy trajectories of single columns: (picks, decreases) per column, where
    decrease t = log(v_t / v_{t+1}) and v_t is the target's variance after t picks."""
    sels, gains = [], []
    for c, cand in enumerate(cand_lists):
        tgt = int(targets[c]) if targets is not None else c
        r = select_single(kp, pts, tgt, cand, k)
        v = r["vtar"]
        sels.append(r["sel"])
        gains.append(np.log(v[:-1] / v[1:]))
    return sels, gains


def group_gains(kp, pts, grp_ptr, cand_lists, k: int):
    """Local greedy trajectories of supernodes: (picks, decreases per nonzero) per group,
    decrease t = log(Theta_{jj|I} / Theta_{jj|I,P}) / m for the t-th pick j."""
    sels, gains = [], []
    for g, cand in enumerate(cand_lists):
        g0, g1 = int(grp_ptr[g]), int(grp_ptr[g + 1])
        r = select_multi(kp, pts, g0, g1 - g0, cand, k)
        sels.append(r["sel"])
        gains.append(np.log(r["chosen"]) / (g1 - g0))
    return sels, gains


def select_columns_global(kp, pts, targets, cand_lists, k: int, budget: int):
    """Global greedy over single columns: (selections truncated to their counts, counts)."""
    sels, gains = column_gains(kp, pts, targets, cand_lists, k)
    counts = queue_allocate(gains, [1] * len(gains), budget)
    return [s[:c] for s, c in zip(sels, counts)], counts


def select_groups_global(kp, pts, grp_ptr, cand_lists, k: int, budget: int):
    """Global greedy over supernodes, nonzeros counted per member: (selections, counts)."""
    sels, gains = group_gains(kp, pts, grp_ptr, cand_lists, k)
    costs = [int(grp_ptr[g + 1] - grp_ptr[g]) for g in range(len(gains))]
    counts = queue_allocate(gains, costs, budget)
    return [s[:c] for s, c in zip(sels, counts)], counts
