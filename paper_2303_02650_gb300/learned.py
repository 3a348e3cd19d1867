"""Driver of the learned warm start: training data from the descent itself, Adam training, and
the paired evaluation against the plain descent.  Calls the C ABI only (pecc_features,
pecc_targets, pecc_descend, pecc_mlp_train_step, pecc_warm_start); no arithmetic here.

A sample is (features of a circle at a random initial layout, the displacement the plain FP32
descent gives that circle over its first T sweeps, in the circle's frame).
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import pecc


def descent_samples(n, R, seed, T=50, target="window", **cfg):
    """Features and targets of the circles of the instances (n[], R[]) from one random start.
    target "window": every circle's displacement over the first T sweeps of the plain FP32 descent;
    "final": the displacement to the layout the whole descent (FP32 + polish) ends at, for the
    circles of the instances that end converged (E <= e_tol) only.
    cfg: further settings of the descent that makes the targets (k_batches, step_max, ...)."""
    if target == "window":
        with pecc.Context(n, precision=pecc.FP32, max_iter=T, stall_window=0, **cfg) as c:
            c.set_radius(R)
            c.init_random(seed)
            x0 = c.get_positions()
            feat = c.features()
            c.descend()
            tgt = c.targets(x0)
        return feat, tgt
    with pecc.Context(n, precision=pecc.FP32_POLISH64, **cfg) as c:
        c.set_radius(R)
        c.init_random(seed)
        x0 = c.get_positions()
        feat = c.features()
        _, status = c.descend()
        tgt = c.targets(x0)
    keep = (status == 0).cpu().numpy()
    off = np.concatenate([[0], np.cumsum(n)])
    parts = [(int(off[q]), int(off[q + 1])) for q in range(len(n)) if keep[q]]
    idx = torch.cat([torch.arange(a, b, device=feat.device) for a, b in parts])
    return feat.index_select(0, idx).contiguous(), tgt.index_select(0, idx).contiguous()


def train(mlp, manifest, rounds=8, T=50, steps=20, lr=1e-3, seed=1000, log=None, target="window", **cfg):
    """rounds x (fresh descent samples of the manifest's instances, `steps` full-batch Adam steps).
    cfg: settings of the descent the targets come from (those the warm start will precede)."""
    n, R = manifest
    losses = []
    rows = 0
    for r in range(rounds):
        feat, tgt = descent_samples(n, R, seed + r, T, target, **cfg)
        rows += feat.shape[0]
        for s in range(steps):
            loss = mlp.train_step(feat, tgt, lr)
        losses.append(float(loss.item()))
        if log:
            log(f"round {r}: rows {feat.shape[0]} loss {losses[-1]:.5f}")
    return losses, rows


def solve(n, R, seed, mlp=None, warm_rounds=2, max_move=0.25, **cfg):
    """Init + (warm start) + descent + feasibility; returns outcome arrays and device ms."""
    with pecc.Context(n, **cfg) as c:
        c.set_radius(R)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        c.init_random(seed)
        a.record()
        acc = c.warm_start(mlp, warm_rounds, max_move) if mlp is not None else None
        iters, status = c.descend()
        feas, mo = c.check_feasible()
        b.record()
        torch.cuda.synchronize()
        return dict(iters=iters.cpu().numpy(), status=status.cpu().numpy(), feasible=feas.cpu().numpy(),
                    ms=a.elapsed_time(b), accepted=None if acc is None else acc.cpu().numpy())


def gain(mlp, manifest, seed, warm_rounds=2, max_move=0.25, **cfg):
    """Paired comparison on the same instances and seeds: plain descent vs warm start + descent."""
    n, R = manifest
    plain = solve(n, R, seed, None, **cfg)
    warm = solve(n, R, seed, mlp, warm_rounds, max_move, **cfg)
    return dict(plain_feasible=int(plain["feasible"].sum()), warm_feasible=int(warm["feasible"].sum()),
                plain_iters=float(plain["iters"].mean()), warm_iters=float(warm["iters"].mean()),
                plain_ms=plain["ms"], warm_ms=warm["ms"],
                accepted_rounds=float(warm["accepted"].mean()), instances=int(n.size))
