"""Orchestration of libsic calls into a whole factor build (no arithmetic here).

`Problem` holds the prepared inputs (points in elimination order, candidate lists,
optional supernodes) resident on the device; `FactorBuilder` owns the output and
scratch buffers and issues, on one stream, the sequence

    select (per column or per supernode) -> nnz scan -> FP64 fill + sum of log v

every step of which is a libsic kernel.  With a nonzero budget (Section 5.4) the
selection also reports each pick's KL decrease and the global greedy allocation keeps
a prefix of every unit's picks before the fill.  Buffers are allocated once, so a build can
be replayed (and captured in a CUDA graph) without allocation.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass

import numpy as np

from . import sic


@dataclass
class HostProblem:
    pts: np.ndarray          # n x dim, elimination order
    kp: sic.Kernel
    k: int
    cand_ptr: np.ndarray     # int64, units + 1
    cand_idx: np.ndarray     # int32
    grp_ptr: np.ndarray | None = None  # int64, groups + 1 (None: single columns)
    order: np.ndarray | None = None    # old point index per position (for reference)
    ell2: np.ndarray | None = None
    members: np.ndarray | None = None  # nonadjacent groups: member positions (grp_ptr indexes it)
    col0: int = 0                      # a slice of a larger factor: its first column ...
    n_cols: int | None = None          # ... and its column count (None: all n columns)
    targets: np.ndarray | None = None  # single columns of a slice: their positions (int32)
    bounds: tuple | None = None        # (max_cand, max_m) of the whole problem, kept by a slice so
                                       # that its launches take the whole build's shapes

    @property
    def n(self):
        return self.pts.shape[0]

    @property
    def ncols(self):
        """Columns of the factor this problem builds (all n, or a slice's)."""
        return self.n if self.n_cols is None else self.n_cols

    @property
    def sliced(self):
        return self.col0 != 0 or self.ncols != self.n

    @property
    def n_units(self):
        return len(self.cand_ptr) - 1

    @property
    def max_cand(self):
        if self.bounds is not None:
            return self.bounds[0]
        return int(np.max(np.diff(self.cand_ptr))) if self.n_units else 0

    @property
    def max_m(self):
        if self.bounds is not None:
            return self.bounds[1]
        return 1 if self.grp_ptr is None else int(np.max(np.diff(self.grp_ptr)))

    @property
    def kc(self):
        """Longest single-column list of a nonadjacent-group pattern: later members + picks."""
        return self.max_m - 1 + self.k

    def h2d_bytes(self):
        b = self.pts.nbytes + self.cand_ptr.nbytes + self.cand_idx.nbytes
        if self.grp_ptr is not None:
            b += self.grp_ptr.nbytes
        return b


def prepare_columns(points: np.ndarray, kp: sic.Kernel, n_cand: int, k: int, n_threads: int = 0) -> HostProblem:
    """Reverse-maximin order + later-ordered candidate lists (libsic host prep)."""
    order, ell2 = sic.prep_maximin(points, n_threads)
    P = np.ascontiguousarray(points[order])
    ptr, idx = sic.prep_candidates_columns(P, n_cand, n_threads)
    return HostProblem(P, kp, k, ptr, idx, None, order, ell2)


def prepare_groups(points: np.ndarray, kp: sic.Kernel, n_cand: int, k: int, mmin: int = 8, mmax: int = 64,
                   lam: float = 1.5, n_threads: int = 0) -> HostProblem:
    """Reverse-maximin order, supernodes (Section 6.1 rule on the 2k nearest later points,
    renumbered to be consecutive) and group candidate lists."""
    order, ell2 = sic.prep_maximin(points, n_threads)
    P = np.ascontiguousarray(points[order])
    members, gp = sic.prep_groups(P, ell2, 2 * k, lam, mmin, mmax, n_threads)
    P2 = np.ascontiguousarray(P[members])
    ptr, idx = sic.prep_candidates_groups(P2, gp, n_cand, n_threads)
    return HostProblem(P2, kp, k, ptr, idx, gp, order[members], ell2[members])


def prepare_partial(points: np.ndarray, kp: sic.Kernel, n_cand: int, k: int, mmin: int = 8, mmax: int = 64,
                    lam: float = 1.5, n_threads: int = 0) -> HostProblem:
    """Reverse-maximin order and the Section 6.1 groups kept where they fall in the ordering
    (nonadjacent, no renumbering), with candidates after each group's first member
    (Section 5.1.1): the input of partial selection."""
    order, ell2 = sic.prep_maximin(points, n_threads)
    P = np.ascontiguousarray(points[order])
    members, gp = sic.prep_groups(P, ell2, 2 * k, lam, mmin, mmax, n_threads)
    ptr, idx = sic.prep_candidates_partial(P, members, gp, n_cand, n_threads)
    return HostProblem(P, kp, k, ptr, idx, gp, order, ell2, members)


def slice_problem(hp: HostProblem, u0: int, u1: int) -> HostProblem:
    """Units u0 .. u1-1 of hp as a problem of their own (a slice of hp's factor, Section 4:
    units are independent): the same points, the units' candidate lists (offsets from 0) and
    their columns col0 .. col0 + n_cols - 1 (for single columns, targets u0 .. u1-1)."""
    cp = hp.cand_ptr[u0:u1 + 1]
    ptr = np.ascontiguousarray(cp - cp[0])
    idx = np.ascontiguousarray(hp.cand_idx[int(cp[0]):int(cp[-1])])
    bounds = (hp.max_cand, hp.max_m)
    if hp.grp_ptr is None:
        return dataclasses.replace(hp, cand_ptr=ptr, cand_idx=idx, col0=int(u0), n_cols=int(u1 - u0),
                                   targets=np.arange(u0, u1, dtype=np.int32), bounds=bounds)
    gp = np.ascontiguousarray(hp.grp_ptr[u0:u1 + 1])
    return dataclasses.replace(hp, cand_ptr=ptr, cand_idx=idx, grp_ptr=gp, col0=int(gp[0]),
                               n_cols=int(gp[-1] - gp[0]), bounds=bounds)


class DeviceProblem:
    def __init__(self, hp: HostProblem, device="cuda"):
        import torch
        self.hp = hp
        self.device = device
        self.pts = torch.from_numpy(hp.pts).to(device)
        self.cand_ptr = torch.from_numpy(hp.cand_ptr).to(device)
        idx = hp.cand_idx if hp.cand_idx.size else np.zeros(1, np.int32)  # never a NULL pointer
        self.cand_idx = torch.from_numpy(idx).to(device)
        self.grp_ptr = torch.from_numpy(hp.grp_ptr).to(device) if hp.grp_ptr is not None else None
        self.members = torch.from_numpy(hp.members).to(device) if hp.members is not None else None
        self.targets = torch.from_numpy(hp.targets).to(device) if hp.targets is not None else None


class FactorBuilder:
    """Preallocated outputs + scratch for building the factor of one problem.

    budget=None: every unit keeps its (up to) k greedy picks.  budget=B: at most B
    off-diagonal nonzeros shared out by the global greedy allocation (a supernode's pick
    costs one nonzero per member); `local_count` then holds the local greedy's counts and
    `sel_count` the allocated ones, which the fill uses.  side_fp64=True takes the picks'
    decreases from the FP64 side state (exact in FP64 whatever the selection's precision)
    instead of from the selection's own arithmetic."""

    def __init__(self, h: sic.Handle, hp: HostProblem, prec: int, device="cuda", nnz_cap: int | None = None,
                 budget: int | None = None, side_fp64: bool = False):
        import torch
        self.h, self.hp, self.prec, self.budget, self.side_fp64 = h, hp, prec, budget, side_fp64
        self.select_plan = None
        n, U, k = hp.n, hp.n_units, hp.k
        dev = device
        self.sel_idx = torch.empty(U * k, dtype=torch.int32, device=dev)
        self.sel_count = torch.empty(U, dtype=torch.int32, device=dev)
        self.local_count = self.sel_count
        self.gain = None
        if budget is not None:
            self.local_count = torch.empty(U, dtype=torch.int32, device=dev)
            self.gain = torch.empty(U * k, dtype=torch.float64, device=dev)
            self.ws_alloc = sic._ws(sic.allocate_global_workspace(U, k), dev)
        nc = hp.ncols
        self.col_ptr = torch.empty(nc + 1, dtype=torch.int64, device=dev)
        # capacity: every column holds at most (its group's later members) + k + 1 entries
        if nnz_cap is None:
            if hp.grp_ptr is None:
                nnz_cap = nc * (k + 1)
            else:
                m = np.diff(hp.grp_ptr)
                nnz_cap = int(np.sum(m * (m + 1) // 2 + m * k))
        self.nnz_cap = nnz_cap
        self.row_idx = torch.empty(nnz_cap, dtype=torch.int32, device=dev)
        self.val = torch.empty(nnz_cap, dtype=torch.float64, device=dev)
        self.logv = torch.empty(nc, dtype=torch.float64, device=dev)
        self.sum_logv = torch.zeros(1, dtype=torch.float64, device=dev)
        if hp.grp_ptr is None:
            self.ws_sel = None
        else:
            self.ws_sel = sic._ws(sic.select_aggregated_workspace(h, U, hp.max_cand, hp.max_m, k, prec), dev)
        self.ws_nnz = sic._ws(sic.factor_nnz_workspace(nc), dev)
        self.ws_fill = sic._ws(sic.build_factor_workspace(nc), dev)

    def select(self, dp: DeviceProblem, stream=None):
        self.select_local(dp, stream)
        if self.budget is not None:
            self.allocate(dp, stream)

    def select_local(self, dp: DeviceProblem, stream=None):
        """Every unit's greedy picks (and, with a budget, their KL decreases)."""
        hp = self.hp
        own = None if self.side_fp64 else self.gain
        if hp.grp_ptr is None:
            sic.select_columns(self.h, dp.pts, hp.kp, dp.cand_ptr, dp.cand_idx, hp.max_cand, hp.k, self.prec,
                               self.sel_idx, self.local_count, targets=getattr(dp, "targets", None), stream=stream,
                               gain=own)
        else:
            sic.select_aggregated(self.h, dp.pts, hp.kp, dp.grp_ptr, dp.cand_ptr, dp.cand_idx, hp.max_cand, hp.max_m,
                                  hp.k, self.prec, self.sel_idx, self.local_count, self.ws_sel, stream=stream,
                                  gain=own)
        if self.gain is not None and self.side_fp64:
            self.side_state(dp, stream)

    def side_state(self, dp: DeviceProblem, stream=None):
        """The picks' exact FP64 decreases (sic_side_state_fp64) into `gain`."""
        hp = self.hp
        sic.side_state_fp64(self.h, dp.pts, hp.kp, self.sel_idx, self.local_count, hp.k, grp_ptr=dp.grp_ptr,
                            max_m=hp.max_m, gain=self.gain, stream=stream)

    def allocate(self, dp: DeviceProblem, stream=None):
        """Global greedy allocation of the budget over the units' picks (Section 5.4)."""
        sic.allocate_global(self.h, self.gain, self.local_count, self.hp.k, self.budget, self.sel_count,
                            self.ws_alloc, grp_ptr=dp.grp_ptr, stream=stream)

    def fill(self, dp: DeviceProblem, stream=None):
        hp = self.hp
        if hp.sliced:
            sic.factor_nnz_range(self.h, dp.grp_ptr, self.sel_count, hp.col0, hp.ncols, 0, self.col_ptr,
                                 self.ws_nnz, stream=stream)
            sic.build_factor_range(self.h, dp.pts, hp.kp, dp.grp_ptr, hp.max_m, self.sel_idx, self.sel_count, hp.k,
                                   hp.col0, hp.ncols, self.col_ptr, 0, self.row_idx, self.val, self.logv,
                                   self.sum_logv, self.ws_fill, stream=stream)
            return
        sic.factor_nnz(self.h, dp.grp_ptr, self.sel_count, hp.n, self.col_ptr, self.ws_nnz, stream=stream)
        sic.build_factor(self.h, dp.pts, hp.kp, dp.grp_ptr, hp.max_m, self.sel_idx, self.sel_count, hp.k,
                         self.col_ptr, self.row_idx, self.val, self.logv, self.sum_logv, self.ws_fill, stream=stream)

    def col_ptr_from(self, dp: DeviceProblem, base: int, out, stream=None):
        """out[0 .. ncols] = this build's column pointers with offsets starting at `base` (the
        entries of the slices before it): the slice's part of the whole factor's col_ptr."""
        hp = self.hp
        sic.factor_nnz_range(self.h, dp.grp_ptr, self.sel_count, hp.col0, hp.ncols, base, out, self.ws_nnz,
                             stream=stream)

    def run(self, dp: DeviceProblem, stream=None):
        self.select(dp, stream)
        self.fill(dp, stream)

    def tune(self, dp: DeviceProblem, stream=None) -> int:
        """Tune the supernodal selection's launch plan (groups only), select, then tune the
        fill's launch split on this problem (both kept in the handle for later calls with the
        same sizes); returns the chosen split (the selection's plan: `select_plan`)."""
        hp = self.hp
        if hp.grp_ptr is not None:
            self.select_plan = sic.tune_select_aggregated(self.h, dp.pts, hp.kp, dp.grp_ptr, dp.cand_ptr, dp.cand_idx,
                                                          hp.max_cand, hp.max_m, hp.k, self.prec, self.sel_idx,
                                                          self.local_count, self.ws_sel, stream=stream)
        self.select(dp, stream)
        sic.factor_nnz(self.h, dp.grp_ptr, self.sel_count, hp.n, self.col_ptr, self.ws_nnz, stream=stream)
        return sic.tune_build_factor(self.h, dp.pts, hp.kp, dp.grp_ptr, hp.max_m, self.sel_idx, self.sel_count, hp.k,
                                     self.col_ptr, self.row_idx, self.val, self.logv, self.sum_logv, self.ws_fill,
                                     stream=stream)

    def sel_lists(self):
        si = self.sel_idx.view(-1, self.hp.k).cpu().numpy()
        sc = self.sel_count.cpu().numpy()
        return [si[u, :sc[u]].copy() for u in range(len(sc))]

    def csc(self):
        cp = self.col_ptr.cpu().numpy()
        nnz = int(cp[-1])
        return cp, self.row_idx[:nnz].cpu().numpy(), self.val[:nnz].cpu().numpy(), self.logv.cpu().numpy()


class PartialFactorBuilder:
    """Nonadjacent groups: partial selection (Section 5.2, Appendix C.3) and the KL-optimal
    FP64 fill of its pattern -- aggregated per group (one LDL^T of the group's members and
    picks, latest first) or, with per_column=True, one factorisation per column."""

    def __init__(self, h: sic.Handle, hp: HostProblem, prec: int, device="cuda", per_column: bool = False):
        import torch
        assert hp.members is not None and hp.grp_ptr is not None
        self.h, self.hp, self.prec, self.per_column = h, hp, prec, per_column
        n, G, k, kc = hp.n, hp.n_units, hp.k, hp.kc
        dev = device
        self.sel_idx = torch.empty(G * k, dtype=torch.int32, device=dev)
        self.sel_count = torch.empty(G, dtype=torch.int32, device=dev)
        self.gain = torch.empty(G * k, dtype=torch.float64, device=dev)
        self.col_sel = torch.empty(n * kc if per_column else 1, dtype=torch.int32, device=dev)
        self.col_count = torch.zeros(n, dtype=torch.int32, device=dev)
        self.col_ptr = torch.empty(n + 1, dtype=torch.int64, device=dev)
        m = np.diff(hp.grp_ptr)
        self.nnz_cap = int(np.sum(m * (m + 1) // 2 + m * k))
        self.row_idx = torch.empty(self.nnz_cap, dtype=torch.int32, device=dev)
        self.val = torch.empty(self.nnz_cap, dtype=torch.float64, device=dev)
        self.logv = torch.empty(n, dtype=torch.float64, device=dev)
        self.sum_logv = torch.zeros(1, dtype=torch.float64, device=dev)
        self.ws_nnz = sic._ws(sic.factor_nnz_workspace(n), dev)
        self.ws_fill = sic._ws(sic.build_factor_workspace(n), dev)

    def select(self, dp: DeviceProblem, stream=None):
        hp = self.hp
        sic.select_partial(self.h, dp.pts, hp.kp, dp.grp_ptr, dp.members, dp.cand_ptr, dp.cand_idx, hp.max_cand,
                           hp.max_m, hp.k, self.prec, self.sel_idx, self.sel_count, gain=self.gain, stream=stream)

    def fill(self, dp: DeviceProblem, stream=None):
        hp = self.hp
        if self.per_column:
            sic.partial_columns(self.h, hp.n, dp.grp_ptr, dp.members, self.sel_idx, self.sel_count, hp.k, hp.kc,
                                self.col_sel, self.col_count, stream=stream)
            sic.factor_nnz(self.h, None, self.col_count, hp.n, self.col_ptr, self.ws_nnz, stream=stream)
            sic.build_factor(self.h, dp.pts, hp.kp, None, 1, self.col_sel, self.col_count, hp.kc, self.col_ptr,
                             self.row_idx, self.val, self.logv, self.sum_logv, self.ws_fill, stream=stream)
            return
        sic.partial_columns(self.h, hp.n, dp.grp_ptr, dp.members, self.sel_idx, self.sel_count, hp.k, hp.kc,
                            None, self.col_count, stream=stream)
        sic.factor_nnz(self.h, None, self.col_count, hp.n, self.col_ptr, self.ws_nnz, stream=stream)
        sic.build_factor_partial(self.h, dp.pts, hp.kp, dp.grp_ptr, dp.members, hp.max_m, self.sel_idx,
                                 self.sel_count, hp.k, self.col_ptr, self.row_idx, self.val, self.logv,
                                 self.sum_logv, self.ws_fill, stream=stream)

    def run(self, dp: DeviceProblem, stream=None):
        self.select(dp, stream)
        self.fill(dp, stream)

    def sel_lists(self):
        si = self.sel_idx.view(-1, self.hp.k).cpu().numpy()
        sc = self.sel_count.cpu().numpy()
        return [si[u, :sc[u]].copy() for u in range(len(sc))]
