"""torch.autograd bridge of the chemgb integrator.

IntegrateFn.apply(T0, Y0, p, theta, handle, opts, cap) integrates every cell
over opts.dt on the GPU (cg_integrate_ckpt) and returns (T, Y, status);
backward runs the discrete adjoint (cg_integrate_adjoint) and returns
dL/dT0, dL/dY0 and dL/dtheta, where theta [nr, 3] holds (ln A, b, Ea) of
every reaction in the mechanism's reaction order. The derivative is the one
of the integrator's converged stage equations with the accepted steps frozen
to those of the forward pass. Marshalling only: the computation is in the
CUDA library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import chemgb as cg


def _sync_theta(handle, theta: torch.Tensor):
    a = theta.detach().to("cpu", torch.float64).numpy().reshape(handle.nr, 3)
    if not np.array_equal(a, handle.arr):
        cg.cg_mech_set_arrhenius(handle, a)


class IntegrateFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, T0, Y0, p, theta, handle, opts, cap):
        if handle.nr:
            _sync_theta(handle, theta)
        N = T0.shape[0]
        dev = T0.device
        T = T0.detach().clone().contiguous()
        Y = Y0.detach().clone().contiguous()
        ckpt = torch.empty((N, cap, handle.n + 1), dtype=torch.float64, device=dev)
        ckpt_n = torch.empty(N, dtype=torch.int32, device=dev)
        status = torch.empty(N, dtype=torch.int32, device=dev)
        cg.cg_integrate_ckpt(handle, opts, T, Y, p.detach().contiguous(), ckpt, ckpt_n, status)
        ctx.save_for_backward(ckpt, ckpt_n)
        ctx.handle, ctx.opts = handle, opts
        ctx.theta = theta.detach().clone()
        ctx.theta_device = theta.device
        ctx.mark_non_differentiable(status)
        return T, Y, status

    @staticmethod
    def backward(ctx, gT, gY, _gstatus):
        ckpt, ckpt_n = ctx.saved_tensors
        h = ctx.handle
        if h.nr:
            _sync_theta(h, ctx.theta)
        N = ckpt.shape[0]
        dev = ckpt.device
        gT = torch.zeros(N, dtype=torch.float64, device=dev) if gT is None else gT.contiguous()
        gY = torch.zeros((h.ns, N), dtype=torch.float64, device=dev) if gY is None else gY.contiguous()
        dT0 = torch.empty(N, dtype=torch.float64, device=dev)
        dY0 = torch.empty((h.ns, N), dtype=torch.float64, device=dev)
        dtheta = torch.empty((h.nr, 3), dtype=torch.float64, device=dev)
        cg.cg_integrate_adjoint(h, ctx.opts, ckpt, ckpt_n, gT, gY, dT0, dY0,
                                dtheta if h.nr else None)
        return dT0, dY0, None, dtheta.to(ctx.theta_device), None, None, None


def integrate(handle, opts, T0, Y0, p, theta=None, cap: int = 256):
    """Differentiable integration of N cells: T0 [N], Y0 [ns, N], p [N]
    (pressure, or density at constant volume) on the GPU; theta [nr, 3]
    defaults to the mechanism's current parameters (not differentiated)."""
    if theta is None:
        theta = torch.as_tensor(handle.arr, dtype=torch.float64)
    return IntegrateFn.apply(T0, Y0, p, theta, handle, opts, cap)
