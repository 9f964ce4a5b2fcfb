"""torch.autograd.Function for the FTCS run u(0), r -> u(K).

Forward: the library's synchronous run (or the replay of a recorded
asynchronous run's delay trace).  Backward: the hand-written adjoint
(heat1d_vjp): checkpoints every C steps, recompute, transposed stencil marched
back through the same trace.  Gradients flow to u(0) and to r; the two
Dirichlet entries of u(0) get zero gradient.
"""
from __future__ import annotations

import torch

from . import heat1d


class Heat1dRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, r, K, c1=0.0, cN=0.0, trace=None, segments=0, q=3, ckpt_every=128):
        rv = float(r)
        opts = {}
        if segments:
            opts["segments"] = int(segments)
        if trace is not None:
            opts["q"] = int(q)
        dt = "float64" if u0.dtype == torch.float64 else "float32"
        with heat1d.Heat1d(u0.numel(), rv, c1, cN, dtype=dt, **opts) as h:
            h.set_u(u0.detach())
            if trace is None:
                h.run_sync(int(K))
            else:
                h.replay(int(K), trace)
            h.sync()
            uK = h.get_u()
        ctx.save_for_backward(u0.detach())
        ctx.cfg = (rv, int(K), c1, cN, trace, opts, dt, int(ckpt_every), torch.is_tensor(r))
        return uK

    @staticmethod
    def backward(ctx, grad_uK):
        (u0,) = ctx.saved_tensors
        rv, K, c1, cN, trace, opts, dt, C, r_is_tensor = ctx.cfg
        with heat1d.Heat1d(u0.numel(), rv, c1, cN, dtype=dt, **opts) as h:
            h.set_u(u0)
            g, gr = h.vjp(K, grad_uK.contiguous(), trace=trace, ckpt_every=C)
        grad_u0 = g.to(u0.dtype) if ctx.needs_input_grad[0] else None
        grad_r = None
        if ctx.needs_input_grad[1] and r_is_tensor:
            grad_r = torch.tensor(gr, dtype=torch.float64, device=u0.device)
        return grad_u0, grad_r, None, None, None, None, None, None, None


def heat1d_run(u0, r, K, c1=0.0, cN=0.0, trace=None, segments=0, q=3, ckpt_every=128):
    """u(K) as a differentiable function of u0 (CUDA tensor) and r (float or
    0-dim tensor)."""
    return Heat1dRun.apply(u0, r, K, c1, cN, trace, segments, q, ckpt_every)
