"""The constrained step as a differentiable PyTorch function.

``ConstrainedStep.apply(ctx, x, quat, f_nc, eta)`` runs one aLENS_step on
copies of (x, quat) and returns (x', quat') with x' unwrapped (x + h U_t);
its backward calls the library's hand-written adjoint (aLENS_step_adjoint)
for dL/dx, dL/dquat (unit-quaternion tangent space), dL/dF_nc and dL/deta.
``eta`` is a 0-dim float64 tensor: the viscosity, which the function sets on
the context before the step.  The forward keeps a copy of the parameters it
ran with (viscosity, dt, precision, tolerance ...), and the backward runs the
adjoint under that copy, then puts back whatever parameters the context held
when the backward began: a context may run other forwards, with other
parameters, between a forward and its backward.  Both passes run in the
library's kernels; this module only marshals tensors.
"""
from __future__ import annotations

import torch

from . import Context, Params

__all__ = ["ConstrainedStep", "constrained_step"]


class ConstrainedStep(torch.autograd.Function):
    @staticmethod
    def forward(fctx, actx: Context, x, quat, f_nc, eta):
        p = Params.from_buffer_copy(actx.params)
        p.viscosity = float(eta)
        actx.set_params(p)
        x0, q0, f0 = x.detach().contiguous(), quat.detach().contiguous(), f_nc.detach().contiguous()
        xw, qw = x0.clone(), q0.clone()
        vel = torch.empty((x.shape[0], 6), dtype=torch.float64, device=x.device)
        pairs = torch.empty((actx.max_pairs, 3), dtype=torch.int32, device=x.device)
        gamma = torch.empty(actx.max_pairs, dtype=torch.float64, device=x.device)
        info = actx.step(xw, qw, f0, pairs_out=pairs, gamma_out=gamma, vel_out=vel)
        m = info.n_pairs
        xn = x0 + p.dt * vel[:, :3]
        fctx.actx = actx
        fctx.params = Params.from_buffer_copy(p)
        fctx.save_for_backward(x0, q0, f0, pairs[:m].clone(), gamma[:m].clone())
        return xn, qw

    @staticmethod
    def backward(fctx, g_xn, g_qn):
        x0, q0, f0, pairs, gamma = fctx.saved_tensors
        gxn = None if g_xn is None else g_xn.contiguous().to(torch.float64)
        gqn = None if g_qn is None else g_qn.contiguous().to(torch.float64)
        actx = fctx.actx
        now = Params.from_buffer_copy(actx.params)
        actx.set_params(Params.from_buffer_copy(fctx.params))
        try:
            gx, gq, gf, geta, _ = actx.step_adjoint(x0, q0, f0, pairs, gamma, gxn, gqn)
        finally:
            actx.set_params(now)
        return None, gx, gq, gf, torch.tensor(geta, dtype=torch.float64, device=x0.device)


def constrained_step(actx: Context, x, quat, f_nc, eta):
    """(x', quat') of one constrained step, differentiable in all four inputs."""
    return ConstrainedStep.apply(actx, x, quat, f_nc, eta)
