"""Fitting Htex textures to target lookup values (texture optimisation).

The lookup is linear in the stored texels, so its gradient is exact and
cheap: ``htex_lookup_backward`` scatters dL/dvalue times the blend weights
into a pool-shaped texel gradient (queries sorted by halfedge range, so the
scatter-adds stay in L2).  ``fit`` runs Adam on the FP32 pool's own values
in place with ``htex_textures_adam_step`` (an FP32 pool holds them
exactly, so no separate master copy is kept), which also clears the
gradient in the same pass.  The
lookups, their adjoint and the optimiser step all run in libhtex's kernels.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

from . import LOOKUP_BIN, Textures, lookup, lookup_backward


@dataclass
class FitResult:
    losses: list = field(default_factory=list)
    seconds: float = 0.0
    steps: int = 0

    @property
    def ratio(self) -> float:
        return self.losses[-1] / self.losses[0] if self.losses else float("nan")


def fit(tex: Textures, batches, steps: int = 200, lr: float = 0.05, init=None) -> FitResult:
    """Adam on the texels of an FP32 asset so that lookups match targets.

    ``batches(step)`` returns (queries int32 [n, 4] CUDA, targets float32
    [n, channels] CUDA).  Loss: mean squared error over queries and channels.
    ``init``: optional FP32 CUDA tensor with the starting pool (zeros when
    None).  Returns the per-step losses."""
    import torch
    if tex.dtype != "f32":
        raise ValueError("fit needs an FP32 asset (the master copy is written as stored values)")
    start = (init if init is not None else
             torch.zeros(tex.pool_elements, dtype=torch.float32, device="cuda"))
    tex.write_pool(start)
    grad = torch.zeros(tex.pool_elements, dtype=torch.float32, device="cuda")
    m = torch.zeros_like(grad)
    v = torch.zeros_like(grad)
    res = FitResult()
    losses = torch.empty(steps, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.no_grad():
        for step in range(steps):
            q, target = batches(step)
            out = lookup(tex, q)
            diff = out - target
            n = diff.numel()
            losses[step] = diff.double().pow(2).sum() / n
            lookup_backward(tex, q, (2.0 / n) * diff, grad_texels=grad, flags=LOOKUP_BIN)
            tex.adam_step(None, grad, m, v, step + 1, lr)
    torch.cuda.synchronize()
    res.seconds = time.perf_counter() - t0
    res.steps = steps
    res.losses = losses.cpu().tolist()
    return res
