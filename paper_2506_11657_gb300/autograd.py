"""torch.autograd.Function over the C ABI: d_t b_z as a differentiable function of log sigma.

Forward: tem_grid_set_sigma(exp(log_sigma)) + tem_forward (solutions kept).
Backward: tem_adjoint with the incoming gradient dphi/dd, returning dphi/dlog sigma
(Sec. 4: the Jacobian-transpose product through the shifted solves).
All arithmetic runs in libtem.so; this module only moves arrays.

The kept solutions belong to the conductivity of their forward call.  When another forward
has changed the grid's conductivity before this backward (two loss terms on one grid, a line
search), the library refuses the stale state; backward then sets this call's conductivity
again and repeats the forward solve before the adjoint.  The state stays alive with the graph,
so backward may run more than once (retain_graph).
"""
from __future__ import annotations

import numpy as np
import torch

from . import tem


class TEMForward(torch.autograd.Function):
    """d = TEMForward.apply(log_sigma, model): log_sigma (nz*ny*nx) FP64 -> d (n_rx, K) FP64."""

    @staticmethod
    def forward(ctx, log_sigma, grid, loop_xy, z_loop, rx, shifts, c, options):
        ls = log_sigma.detach().to("cpu", torch.float64).numpy().ravel().copy()
        grid.set_sigma(np.exp(ls))
        res = tem.forward(grid, loop_xy, z_loop, rx, shifts, c, options, keep_state=True)
        ctx.state = res.state
        ctx.args = (grid, loop_xy, z_loop, rx, shifts, c, options, ls)
        ctx.shape = log_sigma.shape
        return torch.from_numpy(res.d.copy()).to(log_sigma.device)

    @staticmethod
    def backward(ctx, grad_d):
        g = grad_d.detach().to("cpu", torch.float64).numpy()
        try:
            grad = ctx.state.adjoint(g)
        except tem.TEMError as e:
            if e.code != tem.TEM_EINVAL:
                raise
            grid, loop_xy, z_loop, rx, shifts, c, options, ls = ctx.args
            grid.set_sigma(np.exp(ls))
            ctx.state.close()
            ctx.state = tem.forward(grid, loop_xy, z_loop, rx, shifts, c, options, keep_state=True).state
            grad = ctx.state.adjoint(g)
        out = torch.from_numpy(grad).reshape(ctx.shape).to(grad_d.device)
        return out, None, None, None, None, None, None, None


def tem_forward_logsigma(log_sigma, grid, loop_xy, z_loop, rx, shifts, c, options=None):
    """Convenience wrapper: differentiable d_t b_z for a log-conductivity tensor."""
    opt = options if options is not None else tem.default_options()
    return TEMForward.apply(log_sigma, grid, loop_xy, z_loop, rx, shifts, c, opt)
