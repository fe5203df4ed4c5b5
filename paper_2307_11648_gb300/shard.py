"""One factor built in slices, one slice per rank (one process per GPU).

The factor's columns (or supernodes) are independent of one another (Section 4: each
column's selection and values need only the points), so the units are cut into contiguous
ranges of near-equal estimated cost (sic_prep_partition) and every rank, holding all the
points, builds its range:

    select + fill of the rank's units into the rank's own arrays (libsic kernels)
    -> exchange of the slices' (first column, columns, entries)         [collective]
    -> offsets of the slices' entries: an exclusive scan over the ranks (host)
    -> the slice's part of the whole factor's col_ptr: the nnz scan again, offsets starting
       at the rank's base (sic_factor_nnz_range)
    -> gather of col_ptr, row_idx, val and log v into whole-factor arrays on every rank,
       one broadcast per rank and array straight into place                [collective]
    -> sum of log v: an all-reduce of the slices' sums                   [collective]
       and, on the device, the fixed-order sum over the gathered log v (sic_sum_fixed),
       bit-identical to one build of the whole factor.

No exchange happens during selection or fill; the collectives run once, at the end.  The
communicator is torch.distributed (NCCL between GPUs, gloo on CPU).  Nothing here does
arithmetic of the method: it moves buffers and calls libsic.
"""
from __future__ import annotations

from dataclasses import dataclass

from . import pipeline, sic


def rank_offsets(nnz):
    """Exclusive scan over ranks: the first entry of every slice in the whole factor."""
    out, run = [], 0
    for x in nnz:
        out.append(run)
        run += int(x)
    return out


class TorchComm:
    """The collectives of the sliced build over a torch.distributed process group: tensors
    live on the GPU for NCCL, on the host for gloo."""

    def __init__(self, group=None, device=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        if device is None:
            device = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
        self.device = device

    def all_gather_ints(self, vals):
        import torch
        t = torch.tensor([int(v) for v in vals], dtype=torch.int64, device=self.device)
        out = [torch.empty_like(t) for _ in range(self.world)]
        self.dist.all_gather(out, t, group=self.group)
        return [[int(x) for x in o.cpu().tolist()] for o in out]

    def broadcast_(self, t, src):
        self.dist.broadcast(t, src=self.dist.get_global_rank(self.group, src) if self.group else src,
                            group=self.group)

    def all_reduce_sum_(self, t):
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)


@dataclass
class Slice:
    """One rank's piece of the factor: columns col0 .. col0 + n_cols - 1 with nnz entries;
    col_ptr (n_cols + 1) at offsets of the whole factor, row_idx / val (nnz), logv
    (n_cols) and the slice's sum of log v (one FP64)."""
    col0: int
    n_cols: int
    nnz: int
    col_ptr: object
    row_idx: object
    val: object
    logv: object
    sum_logv: object


def exchange_counts(comm, col0: int, n_cols: int, nnz: int):
    """Every rank's (col0, n_cols, nnz) and the offset of every slice's first entry."""
    meta = comm.all_gather_ints([col0, n_cols, nnz])
    return meta, rank_offsets([m[2] for m in meta])


def check_cover(meta, n: int):
    """The slices must cover the columns 0 .. n-1 in rank order without gaps or overlaps."""
    c = 0
    for r, (c0, nc, _) in enumerate(meta):
        if c0 != c or nc < 0:
            raise ValueError(f"slice of rank {r} starts at column {c0}, expected {c}")
        c += nc
    if c != n:
        raise ValueError(f"slices cover {c} columns of {n}")


def whole_arrays(meta, n: int, device):
    """Empty whole-factor arrays for the slices described by meta."""
    import torch
    nnz = sum(m[2] for m in meta)
    return dict(col_ptr=torch.empty(n + 1, dtype=torch.int64, device=device),
                row_idx=torch.empty(max(nnz, 1), dtype=torch.int32, device=device),
                val=torch.empty(max(nnz, 1), dtype=torch.float64, device=device),
                logv=torch.empty(max(n, 1), dtype=torch.float64, device=device)), nnz


def slice_views(whole, c0: int, nc: int, off: int, nz: int):
    """The places of one slice's arrays inside the whole-factor arrays."""
    return dict(col_ptr=whole["col_ptr"][c0:c0 + nc + 1], row_idx=whole["row_idx"][off:off + nz],
                val=whole["val"][off:off + nz], logv=whole["logv"][c0:c0 + nc])


def place(whole, meta, offsets, r: int, sl: Slice):
    """Copy slice r's arrays into their places (one process holding every slice)."""
    c0, nc, nz = meta[r]
    for key, dst in slice_views(whole, c0, nc, offsets[r], nz).items():
        if dst.numel():
            dst.copy_(getattr(sl, key)[:dst.numel()])


def gather_factor(comm, meta, offsets, sl: Slice, n: int):
    """Whole-factor arrays on every rank from every rank's slice (one broadcast per rank and
    array, into place) and the all-reduced sum of log v.  Returns (arrays, nnz, sum_logv)."""
    import torch
    check_cover(meta, n)
    whole, nnz = whole_arrays(meta, n, comm.device)
    for r in range(comm.world):
        c0, nc, nz = meta[r]
        views = slice_views(whole, c0, nc, offsets[r], nz)
        if r == comm.rank:
            place(whole, meta, offsets, r, sl)
        for dst in views.values():
            if dst.numel():
                comm.broadcast_(dst, r)
    s = sl.sum_logv.reshape(1).to(device=comm.device, dtype=torch.float64).clone()
    comm.all_reduce_sum_(s)
    return whole, nnz, s


class ShardedFactorBuilder:
    """This rank's slice of one factor: the units bounds[rank] .. bounds[rank+1]-1 of the
    partition into `world` slices, built with the plain FactorBuilder or, given a proposal,
    the learned path; gather() assembles the whole factor on every rank."""

    def __init__(self, h: sic.Handle, hp: pipeline.HostProblem, prec: int, rank: int, world: int, proposal=None,
                 device="cuda"):
        import torch
        self.h, self.hp, self.rank, self.world, self.dev = h, hp, rank, world, device
        self.bounds = sic.prep_partition(hp.cand_ptr, hp.grp_ptr, hp.k, world,
                                         proposal.top if proposal is not None else 0)
        u0, u1 = int(self.bounds[rank]), int(self.bounds[rank + 1])
        self.u0, self.u1 = u0, u1
        self.empty = u1 == u0
        if self.empty:
            col0 = int(hp.grp_ptr[u0]) if hp.grp_ptr is not None else u0
            self.local = None
            self.col0, self.n_cols = col0, 0
            self.builder = self.fb = None
            return
        self.local = pipeline.slice_problem(hp, u0, u1)
        self.col0, self.n_cols = self.local.col0, self.local.ncols
        if proposal is not None:
            from . import learned
            self.builder = learned.LearnedFactorBuilder(h, self.local, proposal, prec, device)
            self.fb = self.builder.fb
        else:
            self.builder = self.fb = pipeline.FactorBuilder(h, self.local, prec, device)
        self.gcol_ptr = torch.empty(self.n_cols + 1, dtype=torch.int64, device=device)

    def device_problem(self):
        return None if self.empty else pipeline.DeviceProblem(self.local, self.dev)

    def run(self, dp, stream=None):
        if not self.empty:
            self.builder.run(dp, stream)

    def local_nnz(self) -> int:
        return 0 if self.empty else int(self.fb.col_ptr[-1].item())

    def slice(self, dp, base: int, stream=None) -> Slice:
        """This rank's Slice with col_ptr at the whole factor's offsets (base = the entries of
        the slices before it)."""
        import torch
        if self.empty:
            cp = torch.full((1,), base, dtype=torch.int64, device=self.dev)
            z = torch.zeros(0, dtype=torch.float64, device=self.dev)
            return Slice(self.col0, 0, 0, cp, torch.zeros(0, dtype=torch.int32, device=self.dev), z, z,
                         torch.zeros(1, dtype=torch.float64, device=self.dev))
        self.fb.col_ptr_from(dp, base, self.gcol_ptr, stream)
        nnz = self.local_nnz()
        return Slice(self.col0, self.n_cols, nnz, self.gcol_ptr, self.fb.row_idx[:nnz], self.fb.val[:nnz],
                     self.fb.logv, self.fb.sum_logv)

    def gather(self, dp, comm, stream=None):
        """Whole factor on every rank: (arrays, nnz, all-reduced sum of log v,
        fixed-order sum of the gathered log v on the device)."""
        import torch
        meta, offsets = exchange_counts(comm, self.col0, self.n_cols, self.local_nnz())
        sl = self.slice(dp, offsets[comm.rank], stream)
        whole, nnz, s = gather_factor(comm, meta, offsets, sl, self.hp.ncols)
        fixed = torch.empty(1, dtype=torch.float64, device=whole["logv"].device)
        if whole["logv"].is_cuda:
            ws = sic._ws(sic.build_factor_workspace(self.hp.ncols), whole["logv"].device)
            sic.sum_fixed(self.h, whole["logv"], fixed, ws, stream)
        else:
            fixed = None
        return whole, nnz, s, fixed


def assemble_local(h, hp: pipeline.HostProblem, builders, dps, device="cuda", stream=None):
    """Every slice built in this one process (e.g. all ranges on one GPU): the same count
    exchange, offsets, col_ptr at global offsets and placement as gather(), without a
    communicator.  Returns (arrays, nnz, fixed-order sum of log v)."""
    import torch
    meta = [[b.col0, b.n_cols, b.local_nnz()] for b in builders]
    offsets = rank_offsets([m[2] for m in meta])
    check_cover(meta, hp.ncols)
    whole, nnz = whole_arrays(meta, hp.ncols, device)
    for r, (b, dp) in enumerate(zip(builders, dps)):
        place(whole, meta, offsets, r, b.slice(dp, offsets[r], stream))
    fixed = torch.empty(1, dtype=torch.float64, device=device)
    ws = sic._ws(sic.build_factor_workspace(hp.ncols), device)
    sic.sum_fixed(h, whole["logv"], fixed, ws, stream)
    return whole, nnz, fixed
