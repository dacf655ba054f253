"""Fitting Htex textures to target lookup values (texture optimisation).

The lookup is linear in the stored texels, so its gradient is exact and
cheap: ``htex_lookup_backward`` scatters dL/dvalue times the blend weights
into a pool-shaped texel gradient.  ``fit`` runs Adam on an FP32 master copy
of the pool, writing it into the resident textures before every forward
pass (``htex_textures_write_pool``).  The lookups and their adjoint run in
libhtex's kernels; the optimiser step is torch's fused Adam.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

from . import Textures, lookup, lookup_backward


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
    master = (init.clone() if init is not None else
              torch.zeros(tex.pool_elements, dtype=torch.float32, device="cuda")).requires_grad_(True)
    opt = torch.optim.Adam([master], lr=lr, fused=True)
    res = FitResult()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for step in range(steps):
        q, target = batches(step)
        with torch.no_grad():
            tex.write_pool(master.detach())
            out = lookup(tex, q)
            diff = out - target
            n = diff.numel()
            res.losses.append(diff.pow(2).sum().item() / n)
            grad = lookup_backward(tex, q, (2.0 / n) * diff)
        master.grad = grad
        opt.step()
        opt.zero_grad(set_to_none=True)
    torch.cuda.synchronize()
    res.seconds = time.perf_counter() - t0
    res.steps = steps
    with torch.no_grad():
        tex.write_pool(master.detach())
    return res
