"""Training data and training loop for the Laplacian-weight surrogate.

Stencils come from jittered grid patches (one patch per stencil, jitter
amplitude U(0, 0.3 h) per patch): the library's kNN picks the 25 nearest
nodes of each patch centre, the library's FP64 solver gives the exact
weights (PHS r^5 + degree-4 monomials), the library's feature kernel the
scaled offsets, and mm_surrogate_targets the weights in scaled units,
w_s = w * s^2 (the targets); the output scaling is fitted on the GPU.
Training runs the library's BF16 forward/backward kernels and Adam.
"""
from __future__ import annotations

import math

import torch

import nodesets as NS

from . import binding as B


def make_stencils(ctx: B.Context, count: int, seed: int, n: int = 25):
    """Patch node set + CSR stencils of the `count` patch centres (rows
    0..count-1).  Returns (pts, row_ptr, col) on the GPU."""
    ns = NS.patches(count, seed=seed)
    pts = torch.from_numpy(ns.pts).cuda()
    rp = torch.arange(count + 1, dtype=torch.int64, device="cuda") * n
    col = torch.empty(count * n, dtype=torch.int32, device="cuda")
    ctx.knn_stencils(pts, [(0, count, n, col)], method=B.KNN_GRID)
    return pts, rp, col


def make_dataset(ctx: B.Context, count: int, seed: int, n: int = 25, k: int = 5, m: int = 4):
    """Features X [count, 2n] (FP32) and scaled FP64 Laplacian weights T
    [count, n] (as FP32 targets and FP64), all on the GPU."""
    pts, rp, col = make_stencils(ctx, count, seed, n)
    vals = torch.zeros(count * n, dtype=torch.float64, device="cuda")
    status = torch.empty(count, dtype=torch.int32, device="cuda")
    ctx.rbffd_weights(B.LAP, k, m, pts, rp, col, [vals], row_begin=0, row_end=count, n_max=n,
                      precision=B.FP64, status=status)
    x = torch.empty((count, 2 * n), dtype=torch.float32, device="cuda")
    s = torch.empty(count, dtype=torch.float64, device="cuda")
    B.stencil_features(ctx, pts, rp, col, 0, count, n, x, s)
    t = torch.empty((count, n), dtype=torch.float32, device="cuda")
    B.surrogate_targets(ctx, rp, 0, count, n, vals, s, 2, t)
    ok = status == B.ST_OK
    return {"x": x[ok].contiguous(), "t": t[ok].contiguous(), "pts": pts, "row_ptr": rp, "col": col,
            "status": status}


def train(net: B.MLP, x: torch.Tensor, t: torch.Tensor, epochs: int = 4, batch: int = 4096,
          lr: float = 2e-3, lr_final: float = 1e-4, seed: int = 0, log_every: int = 0):
    """Adam with cosine-decayed learning rate over shuffled minibatches;
    returns the per-step losses (read back once at the end)."""
    net.fit_output_scaling(t)
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    N = x.shape[0]
    steps_per_epoch = max(1, N // batch)
    total = epochs * steps_per_epoch
    losses = torch.zeros(total, dtype=torch.float32, device="cuda")
    step = 0
    for ep in range(epochs):
        perm = torch.randperm(N, device="cuda", generator=g)
        for b in range(steps_per_epoch):
            idx = perm[b * batch:(b + 1) * batch]
            xb = x.index_select(0, idx).contiguous()
            tb = t.index_select(0, idx).contiguous()
            frac = step / max(1, total - 1)
            cur = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * frac))
            net.train_step(xb, tb, cur, losses[step:step + 1])
            step += 1
    return losses.cpu().numpy()
