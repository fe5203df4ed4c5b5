"""Learned candidate proposal: orchestration of libsic's proposal kernels.

A small MLP (8 features -> 128 -> 128 -> 1) scores each supernode's candidates; only
the `top` best per group go to the exact greedy selection.  The network is trained on
the GPU with libsic's own forward/backward and AdamW kernels, on labels produced by the
plain greedy selection (1 if a candidate was picked) of training problems whose seeds
differ from the evaluation problem.  Everything arithmetic runs in libsic; this module
only allocates buffers, batches rows and loops.
"""
from __future__ import annotations

import dataclasses
import math
import time

import numpy as np

import synthetic

from . import pipeline, sic

N_FEAT = 8
HIDDEN = 128


def init_params(seed: int = 0) -> np.ndarray:
    """Xavier-uniform weights (drawn from the seeded generator), zero biases; flat layout
    W1 [8][128] at 0, b1 at 1024, W2 [128][128] at 1152, b2 at 17536, w3 at 17664, b3 at
    17792 (include/sic.h)."""
    n = sic.mlp_param_count()
    p = np.zeros(n, np.float32)
    u = synthetic.uniform(seed, 77, n) * 2.0 - 1.0
    for off, rows, cols in [(0, N_FEAT, HIDDEN), (1152, HIDDEN, HIDDEN), (17664, HIDDEN, 1)]:
        a = math.sqrt(6.0 / (rows + cols))
        p[off:off + rows * cols] = (u[off:off + rows * cols] * a).astype(np.float32)
    return p


class Proposal:
    """Scores candidates with the MLP and keeps the `top` best per group."""

    def __init__(self, h: sic.Handle, params, top: int = 256, device="cuda"):
        import torch
        self.h = h
        self.top = top
        self.params = params if isinstance(params, torch.Tensor) else torch.from_numpy(params).to(device)
        self.device = device

    def buffers(self, hp: pipeline.HostProblem):
        import torch
        rows = int(hp.cand_ptr[-1])
        G = hp.n_units
        dev = self.device
        return dict(feat=torch.empty((max(rows, 1), N_FEAT), dtype=torch.float32, device=dev),
                    score=torch.empty(max(rows, 1), dtype=torch.float32, device=dev),
                    out_ptr=torch.empty(G + 1, dtype=torch.int64, device=dev),
                    out_idx=torch.empty(max(G * self.top, 1), dtype=torch.int32, device=dev))

    def features(self, dp, buf, stream=None):
        hp = dp.hp
        rows = int(hp.cand_ptr[-1])
        sic.proposal_features(self.h, dp.pts, hp.kp, dp.grp_ptr, dp.cand_ptr, dp.cand_idx, buf["feat"][:rows], stream)

    def score(self, dp, buf, stream=None):
        rows = int(dp.hp.cand_ptr[-1])
        sic.proposal_score(self.h, self.params, buf["feat"][:rows], buf["score"][:rows], stream)

    def topk(self, dp, buf, stream=None):
        sic.proposal_topk(self.h, dp.cand_ptr, dp.cand_idx, buf["score"], self.top, buf["out_ptr"], buf["out_idx"],
                          stream)

    def run(self, dp: pipeline.DeviceProblem, buf, stream=None):
        """features -> scores -> per-group top-k; fills buf['out_ptr'], buf['out_idx']."""
        self.features(dp, buf, stream)
        self.score(dp, buf, stream)
        self.topk(dp, buf, stream)


def reduced_problem(hp: pipeline.HostProblem, top: int) -> pipeline.HostProblem:
    """Host-side description of the reduced problem (sizes only; the lists live on the device)."""
    cnt = np.minimum(np.diff(hp.cand_ptr), top)
    ptr = np.zeros(len(cnt) + 1, np.int64)
    ptr[1:] = np.cumsum(cnt)
    bounds = None if hp.bounds is None else (min(hp.bounds[0], top), hp.bounds[1])
    return dataclasses.replace(hp, cand_ptr=ptr, cand_idx=np.zeros(max(int(ptr[-1]), 1), np.int32), bounds=bounds)


class LearnedFactorBuilder:
    """proposal (features -> MLP -> top-k) -> exact greedy on the survivors -> FP64 fill
    (with a nonzero budget: the global greedy allocation before the fill)."""

    def __init__(self, h: sic.Handle, hp: pipeline.HostProblem, proposal: Proposal, prec=sic.SIC_FP32_MIXED,
                 device="cuda", budget: int | None = None, side_fp64: bool = False):
        import torch
        self.h, self.hp, self.proposal = h, hp, proposal
        self.buf = proposal.buffers(hp)
        self.rhp = reduced_problem(hp, proposal.top)
        self.fb = pipeline.FactorBuilder(h, self.rhp, prec, device, budget=budget, side_fp64=side_fp64)
        self.rdp = None

    def _reduced_device(self, dp):
        if self.rdp is None or self.rdp.pts is not dp.pts:
            class _R:
                pass
            r = _R()
            r.hp, r.pts, r.grp_ptr, r.targets = self.rhp, dp.pts, dp.grp_ptr, getattr(dp, "targets", None)
            r.cand_ptr, r.cand_idx = self.buf["out_ptr"], self.buf["out_idx"]
            self.rdp = r
        return self.rdp

    def propose(self, dp, stream=None):
        self.proposal.run(dp, self.buf, stream)

    def select(self, dp, stream=None):
        self.propose(dp, stream)
        self.fb.select(self._reduced_device(dp), stream)

    def fill(self, dp, stream=None):
        self.fb.fill(self._reduced_device(dp), stream)

    def run(self, dp, stream=None):
        self.select(dp, stream)
        self.fill(dp, stream)

    def tune(self, dp, stream=None) -> int:
        """Propose, then tune the fill's launch split on the reduced problem (kept in the handle)."""
        self.propose(dp, stream)
        return self.fb.tune(self._reduced_device(dp), stream)

    @property
    def sum_logv(self):
        return self.fb.sum_logv

    @property
    def col_ptr(self):
        return self.fb.col_ptr

    @property
    def nnz_cap(self):
        return self.fb.nnz_cap

    def sel_lists(self):
        return self.fb.sel_lists()


class GuardedBuild:
    """The learned path judged by the plain greedy, which is also its fallback.

    run(dp) builds the factor with the learned proposal and with plain greedy selection on
    all candidates, and a reference factor with 2k picks from the same candidates; the KL gap
    (S_learned - S_plain) / (S_plain - S_ref), S = sum of log v (the same proxy as the
    benchmark's: logdet Theta cancels in both differences, and S_ref >= logdet Theta makes the
    denominator a lower bound of 2 KL(plain), so the gap is overstated, never understated).
    If the gap is at most `max_gap` the learned factor is kept, else the plain one.  `chosen`
    names the builder whose outputs (col_ptr, row_idx, val, logv, sum_logv) hold the factor.
    The audit costs a plain and a 2k build; use it once per geometry and kernel, then keep
    the decision (`use_learned`)."""

    def __init__(self, h: sic.Handle, hp: pipeline.HostProblem, proposal: Proposal, max_gap: float = 0.01,
                 prec=sic.SIC_FP32_MIXED, device="cuda"):
        import dataclasses
        self.max_gap = max_gap
        self.learned = LearnedFactorBuilder(h, hp, proposal, prec, device)
        self.plain = pipeline.FactorBuilder(h, hp, prec, device)
        self.ref = pipeline.FactorBuilder(h, dataclasses.replace(hp, k=2 * hp.k), prec, device)
        self.h = h
        self.gap = None
        self.use_learned = None

    def run(self, dp: pipeline.DeviceProblem, stream=None):
        for b in (self.learned, self.plain, self.ref):
            b.run(dp, stream)
        self.h.sync(stream)
        s_l, s_p, s_r = (float(b.sum_logv.cpu()[0]) for b in (self.learned, self.plain, self.ref))
        den = s_p - s_r
        self.gap = (s_l - s_p) / den if den > 0 else float("inf")
        self.use_learned = bool(self.gap <= self.max_gap)
        return self.chosen

    @property
    def chosen(self):
        return self.learned.fb if self.use_learned else self.plain


# ----------------------------------------------------------------- training --

def training_set(h: sic.Handle, problems, prec=sic.SIC_FP32_MIXED, device="cuda"):
    """Features and plain-greedy labels of every candidate of every group of the problems."""
    import torch
    feats, labels = [], []
    n_sel = 0
    for hp in problems:
        dp = pipeline.DeviceProblem(hp, device)
        fb = pipeline.FactorBuilder(h, hp, prec, device)
        fb.select(dp)
        rows = int(hp.cand_ptr[-1])
        f = torch.empty((rows, N_FEAT), dtype=torch.float32, device=device)
        y = torch.empty(rows, dtype=torch.float32, device=device)
        sic.proposal_features(h, dp.pts, hp.kp, dp.grp_ptr, dp.cand_ptr, dp.cand_idx, f)
        sic.proposal_labels(h, dp.cand_ptr, dp.cand_idx, fb.sel_idx, fb.sel_count, hp.k, y)
        h.sync()
        n_sel += int(fb.sel_count.sum().item())
        feats.append(f)
        labels.append(y)
        del fb, dp
    return torch.cat(feats), torch.cat(labels), n_sel


def save_checkpoint(path, P, m, v, step, epoch, seed):
    """Weights, AdamW moments, step and data-order state (the epoch and seed fix the shuffles)."""
    import torch
    torch.save({"params": P.cpu(), "m": m.cpu(), "v": v.cpu(), "step": step, "epoch": epoch, "seed": seed}, path)


def train(h: sic.Handle, feat, label, params=None, epochs: int = 3, batch: int = 65536, lr: float = 2e-3,
          wd: float = 1e-4, pos_weight: float = 2.0, seed: int = 0, bf16: bool = True, log=None,
          checkpoint: str | None = None, stop_after_epoch: int | None = None):
    """AdamW training of the proposal network with libsic's kernels.  Returns (params, history).

    With `checkpoint`, the state is saved after every epoch and, if the file exists at the
    start, training resumes from it (same result as an uninterrupted run: the per-epoch
    shuffles depend only on the seed and the epoch).  `stop_after_epoch` ends the run early
    (used to test resumption)."""
    import os

    import torch
    dev = feat.device
    n = feat.shape[0]
    P = torch.from_numpy(init_params(seed) if params is None else params).to(dev)
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    g = torch.zeros_like(P)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    ws = sic._ws(sic.mlp_train_workspace(batch), dev)
    hist = []
    step = 0
    ep0 = 0
    if checkpoint and os.path.exists(checkpoint):
        ck = torch.load(checkpoint)
        P.copy_(ck["params"].to(dev))
        m.copy_(ck["m"].to(dev))
        v.copy_(ck["v"].to(dev))
        step, ep0 = int(ck["step"]), int(ck["epoch"]) + 1
        assert int(ck["seed"]) == seed
    t0 = time.perf_counter()
    for ep in range(ep0, epochs):
        perm = np.argsort(synthetic.uniform(seed + 1000 + ep, 91, n), kind="stable")
        perm_t = torch.from_numpy(perm).to(dev)
        for b0 in range(0, n - batch + 1, batch):
            idx = perm_t[b0:b0 + batch]
            xb = feat.index_select(0, idx).contiguous()
            yb = label.index_select(0, idx).contiguous()
            sic.mlp_grads(h, P, xb, yb, pos_weight, bf16, g, loss, ws)
            step += 1
            sic.adamw_step(h, P, m, v, g, step, lr, wd=wd)
            if step % 50 == 1:
                hist.append((step, float(loss.item())))
                if log:
                    log(f"epoch {ep} step {step} loss {hist[-1][1]:.5f} ({time.perf_counter() - t0:.1f}s)")
        if checkpoint:
            h.sync()
            save_checkpoint(checkpoint, P, m, v, step, ep, seed)
        if stop_after_epoch is not None and ep >= stop_after_epoch:
            break
    h.sync()
    hist.append((step, float(loss.item())))
    return P, hist
