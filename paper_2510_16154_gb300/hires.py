"""High-resolution control transfer (Section 4.3): a control eps* optimised on an image is
applied to a higher-resolution version of the same image by one forward sweep.

The control only sees positions in the unit square (the spatial term eps_x/2 |x_j - x_i|^2
uses coordinates in [0, 1]^2), so eps* carries over unchanged.  The interaction window is
given in pixels, so its radius is scaled by the resolution factor (R_hi = factor R) to keep
the same neighbourhood in the unit square; the normalisation 1/M follows the larger window.
Marshalling only: the sweep runs in libagents.so.
"""
from __future__ import annotations

import torch

from . import _lib as lib


def transfer_radius(radius: int, factor: float) -> int:
    return max(1, int(round(radius * factor)))


def apply_control(eps, img_hi: torch.Tensor, radius_lo: int, factor: float, params_lo=None,
                  stream=None) -> torch.Tensor:
    """c(T) of the agent system on img_hi [H, W, C] (float32 CUDA) under the control eps
    [T, 2] (float64, host or device), window radius round(factor * radius_lo).  Other
    parameters (dt, E, normalisation) are taken from params_lo when given."""
    H, W, C = img_hi.shape
    T = int(eps.shape[0])
    p = lib.agents_default_params(H, W, C, transfer_radius(radius_lo, factor), T)
    if params_lo is not None:
        p.dt, p.norm_mode = params_lo.dt, params_lo.norm_mode
        for k in range(2):
            p.eps_lo[k], p.eps_hi[k] = params_lo.eps_lo[k], params_lo.eps_hi[k]
    out = torch.empty_like(img_hi)
    with lib.Context(p, img_hi.contiguous(), stream) as ctx:
        lib.agents_forward(ctx.handle, eps, out, store=False)
        torch.cuda.synchronize(img_hi.device)
    return out
