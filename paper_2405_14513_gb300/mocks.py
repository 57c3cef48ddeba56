"""Many mocks through one plan: per-bin mean and scatter of B_l^m.

The paper validates the estimator with the mean and standard deviation of
B_l^m over independent realisations (Sec. III.B); covariance studies need
the same over many more.  `run_mocks` generates seeded synthetic fields on
the device, estimates them `batch` at a time through one captured CUDA graph
(every stage one launch for the whole batch), and folds each batch's output
into running FP64 statistics on the device (``estimator_stats_update``,
Welford's update; empty bins are skipped).
"""
from __future__ import annotations

import numpy as np

from . import api, synth


class MomentStats:
    """Running count, mean and squared deviations of a plan's output, per
    element (out_shape(1)[1:]), on the device."""

    def __init__(self, shape, device="cuda"):
        import torch
        self.shape = tuple(shape)
        n = int(np.prod(self.shape))
        self.count = torch.zeros(n, dtype=torch.int64, device=device)
        self.mean_ = torch.zeros(n, dtype=torch.float64, device=device)
        self.m2 = torch.zeros(n, dtype=torch.float64, device=device)

    def update(self, out, stream=None):
        """Fold the fields of out [k][...] (CUDA float64) in."""
        api.stats_update(out, self.count, self.mean_, self.m2, stream=stream)

    def numpy(self):
        """(count, mean, standard deviation) as host arrays of the output's
        shape; mean and deviation are NaN where fewer than 1 / 2 values."""
        c = self.count.cpu().numpy().reshape(self.shape)
        m = self.mean_.cpu().numpy().reshape(self.shape)
        s2 = self.m2.cpu().numpy().reshape(self.shape)
        with np.errstate(invalid="ignore", divide="ignore"):
            mean = np.where(c > 0, m, np.nan)
            std = np.where(c > 1, np.sqrt(s2 / np.maximum(c - 1, 1)), np.nan)
        return c, mean, std


def run_mocks(plan, seeds, batch: int, beta: float = 0.5, device="cuda", stream=None) -> MomentStats:
    """Estimate the seeded fields synth.make_field_torch(plan.n_g, plan.box_len,
    seed, beta) for every seed, `batch` per launch (batch <= plan.max_batch),
    and return their statistics.  Full batches replay one captured estimate;
    a last partial batch runs as a plain estimate."""
    import torch
    if not 1 <= batch <= plan.max_batch:
        raise ValueError("batch must be in [1, plan.max_batch]")
    dt = torch.float64 if plan.precision == "fp64" else torch.float32
    ng = plan.n_g
    fields = torch.empty((batch, ng, ng, ng), dtype=dt, device=device)
    ws = plan.workspace(batch, device=device)
    out = torch.empty(plan.out_shape(batch), dtype=torch.float64, device=device)
    stats = MomentStats(plan.out_shape(1)[1:], device=device)
    s = stream if stream is not None else torch.cuda.current_stream(device)
    graph = plan.graph(fields, ws, out, stream=s)
    seeds = list(seeds)
    try:
        with torch.cuda.stream(s):
            for i in range(0, len(seeds), batch):
                chunk = seeds[i:i + batch]
                for j, seed in enumerate(chunk):
                    fields[j].copy_(synth.make_field_torch(ng, plan.box_len, seed, beta=beta, device=device))
                if len(chunk) == batch:
                    graph.launch(stream=s)
                    stats.update(out, stream=s)
                else:
                    k = len(chunk)
                    part = plan.estimate(fields[:k], ws, out=out[:k], stream=s)
                    stats.update(part, stream=s)
        s.synchronize()
    finally:
        graph.close()
    return stats
