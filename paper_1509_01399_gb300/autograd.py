"""torch.autograd form of the forward solve.

``hyb_trace(sigma, mesh, sources, nsteps, dt)`` returns the recorded trace
of the forward solve with coefficient a = 1 + sigma on the unknown voxels
(the conductivity of Eq. (2.3) written as a perturbation of the background
a = 1).  Its backward is the library's exact discrete adjoint followed by
the gradient accumulation of Eq. (gradient1): for a loss L(trace) the
incoming grad_trace is the cotangent dL/dtrace and the returned grad_sigma is
dL/da = dL/dsigma.  With a checkpointing mesh (ckpt_every = C) the forward
keeps full fields every C steps and the backward recomputes each segment.

The mesh holds the state of its last forward, so a mesh must not run another
forward between this function's forward and its backward; that is checked.
"""
from __future__ import annotations

import torch

from . import hyb as H


class _HybTrace(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sigma, mesh, sources, nsteps, dt):
        a = (1.0 + sigma.detach().to(torch.float64)).contiguous()
        trace = mesh.forward(a, sources, nsteps, dt)
        ctx.mesh = mesh
        ctx.generation = mesh._generation
        ctx.sigma_dtype = sigma.dtype
        ctx.save_for_backward(a)
        return trace

    @staticmethod
    def backward(ctx, grad_trace):
        mesh = ctx.mesh
        if getattr(mesh, "_generation", None) != ctx.generation:
            raise RuntimeError("the mesh ran another forward before this backward")
        (a,) = ctx.saved_tensors
        mesh.adjoint(grad_trace.contiguous())
        g = mesh.gradient(a, 0.0, 1.0)
        return g.to(ctx.sigma_dtype), None, None, None, None


def hyb_trace(sigma: torch.Tensor, mesh: "H.HybMesh", sources, nsteps: int, dt: float) -> torch.Tensor:
    """Differentiable trace [n_src, nsteps + 1, obs_stride] of the forward
    solve at a = 1 + sigma."""
    return _HybTrace.apply(sigma, mesh, sources, nsteps, dt)
