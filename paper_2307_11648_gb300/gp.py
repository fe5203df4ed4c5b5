"""Directed GP regression (Section 3) on the GPU through libsic.

For each target point: greedy conditional selection of k of its C nearest training
points (sic_select_columns on the stacked point set, targets first, so that the
training points are the "later" positions), then the FP64 posterior mean and variance
of the latent process from the picked observations (sic_gp_predict).
"""
from __future__ import annotations

import numpy as np

from . import sic


class DirectedGP:
    """Training points x_train (n x dim), observations y_train (n); kp's nugget is the
    observation-noise variance."""

    def __init__(self, h: sic.Handle, kp: sic.Kernel, x_train, y_train, n_cand: int = 128, k: int = 32,
                 prec: int = sic.SIC_FP64, device="cuda"):
        self.h, self.kp, self.k, self.n_cand, self.prec, self.device = h, kp, k, n_cand, prec, device
        self.x_train = np.ascontiguousarray(x_train, dtype=np.float64)
        self.y_train = np.ascontiguousarray(y_train, dtype=np.float64)

    def select(self, x_test):
        """Stacked points, candidate lists and the picks (device tensors) for x_test."""
        import torch
        x_test = np.ascontiguousarray(x_test, dtype=np.float64)
        nt = x_test.shape[0]
        pts = np.vstack([x_test, self.x_train])
        ptr, idx = sic.prep_candidates_targets(pts, nt, self.n_cand)
        dev = self.device
        d = dict(pts=torch.from_numpy(pts).to(dev), ptr=torch.from_numpy(ptr).to(dev),
                 idx=torch.from_numpy(idx if idx.size else np.zeros(1, np.int32)).to(dev),
                 targets=torch.arange(nt, dtype=torch.int32, device=dev),
                 sel_idx=torch.empty(max(nt, 1) * self.k, dtype=torch.int32, device=dev),
                 sel_count=torch.empty(max(nt, 1), dtype=torch.int32, device=dev))
        max_cand = int(np.max(np.diff(ptr))) if nt else 0
        sic.select_columns(self.h, d["pts"], self.kp, d["ptr"], d["idx"], max(max_cand, 1), self.k, self.prec,
                           d["sel_idx"], d["sel_count"], targets=d["targets"])
        return d

    def predict(self, x_test):
        """(mean, var) at x_test as device FP64 tensors."""
        import torch
        d = self.select(x_test)
        nt = d["targets"].numel()
        y = torch.zeros(d["pts"].shape[0], dtype=torch.float64, device=self.device)
        y[nt:] = torch.from_numpy(self.y_train).to(self.device)
        mean = torch.empty(nt, dtype=torch.float64, device=self.device)
        var = torch.empty(nt, dtype=torch.float64, device=self.device)
        sic.gp_predict(self.h, d["pts"], self.kp, d["targets"], d["sel_idx"], d["sel_count"], self.k, y, mean, var)
        self.last = d
        return mean, var
