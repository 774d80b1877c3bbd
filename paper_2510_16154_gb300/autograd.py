"""Differentiable forward sweep: ``torch.autograd.Function`` over the C ABI.

``flow(context, eps, c0)`` returns the final colour field c(T; eps, c0) of the agent
dynamics (Eq. MAsystem, explicit Euler); its backward pass is the library's exact
discrete adjoint (``agents_flow_backward``): for an upstream gradient g = dL/dc(T) it
runs the reverse sweep from lambda(T) = -g and returns dL/deps^n = -dt D^n and
dL/dc0 = -lambda(0) (Section 3.1: the adjoint of Eq. opt_system-b), the sign changes and
the dt scaling done on the device.  Long horizons use
the context's checkpointing (``traj_mode = k``: every k-th state is kept and the others
are recomputed segment by segment during the backward pass, k ~ sqrt(T)).

Marshalling only: every forward step and adjoint step runs in ``libagents.so``.
A context stores one trajectory, so each forward must be followed by its backward before
the context runs another stored forward; a stale backward raises.
"""
from __future__ import annotations

import torch

from . import _lib as lib


class FlowContext:
    """A library context bound to torch's current CUDA stream, for use with ``flow``."""

    def __init__(self, params, c0: torch.Tensor):
        if not (c0.is_cuda and c0.dtype == torch.float32 and c0.is_contiguous()):
            raise TypeError("c0 must be a contiguous float32 CUDA tensor")
        self.params = params
        self.stream = torch.cuda.current_stream(c0.device)
        self.ctx = lib.Context(params, c0, self.stream)
        self.generation = 0

    @property
    def handle(self):
        return self.ctx.handle

    def close(self):
        self.ctx.close()


class AgentsFlow(torch.autograd.Function):
    @staticmethod
    def forward(fctx, eps: torch.Tensor, c0: torch.Tensor, context: FlowContext):
        p = context.params
        if eps.dtype != torch.float64 or tuple(eps.shape) != (p.nsteps, 2):
            raise TypeError(f"eps must be float64 of shape ({p.nsteps}, 2)")
        eps_c = eps.detach().contiguous()
        c0_c = c0.detach().contiguous()
        lib.agents_set_image(context.handle, c0_c)
        cT = torch.empty_like(c0_c)
        lib.agents_forward(context.handle, eps_c, cT, store=True)
        context.generation += 1
        fctx.generation = context.generation
        fctx.context = context
        fctx.save_for_backward(eps_c)
        return cT

    @staticmethod
    def backward(fctx, grad_cT: torch.Tensor):
        context = fctx.context
        if context.generation != fctx.generation:
            raise RuntimeError("the context ran another stored forward sweep since this one; "
                               "its trajectory is gone")
        (eps,) = fctx.saved_tensors
        g = grad_cT.to(torch.float32).contiguous()
        grad_eps = torch.empty(eps.shape, dtype=torch.float64, device=eps.device) \
            if fctx.needs_input_grad[0] else None
        grad_c0 = torch.empty_like(g) if fctx.needs_input_grad[1] else None
        lib.agents_flow_backward(context.handle, eps, g, grad_eps, grad_c0)
        return grad_eps, grad_c0, None


def flow(context: FlowContext, eps: torch.Tensor, c0: torch.Tensor) -> torch.Tensor:
    """c(T; eps, c0), differentiable in eps (float64 [T, 2]) and c0 (float32 [H, W, C])."""
    return AgentsFlow.apply(eps, c0, context)
