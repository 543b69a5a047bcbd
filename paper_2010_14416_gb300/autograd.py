"""torch.autograd.Function over the discrete adjoint (swe_adjoint).

PyTorch provides the autograd frame and device memory; the forward run,
loss and reverse sweep all run in libswe's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import capi


class SWEAdjoint(torch.autograd.Function):
    """loss = SWEAdjoint.apply(manning, bathy, mesh, state, nsteps, gauges, target, cfl, checkpoint_every)

    manning, bathy: [n_cells] FP64 tensors (caller cell order) -- the
    differentiable inputs.  mesh: an FP64 capi.Mesh built on the same
    triangles; state: (h, hu, hv) initial arrays.  The loss is
    sum_k (h[gauges[k]] after nsteps - target[k])^2 with the time steps of the
    run held fixed in the gradient.  The mesh's state advances by nsteps."""

    @staticmethod
    def forward(ctx, manning, bathy, mesh, state, nsteps, gauges, target, cfl=0.9, checkpoint_every=50):
        mesh.set_fields(bathy=bathy.detach().cpu().numpy(), manning=manning.detach().cpu().numpy())
        mesh.set_state(*state)
        dev = manning.device
        if dev.type == "cuda":
            gm = torch.empty_like(manning, dtype=torch.float64)
            gz = torch.empty_like(bathy, dtype=torch.float64)
            loss, _, _, dts = mesh.adjoint(nsteps, gauges, target, cfl, checkpoint_every, out=(gm, gz))
        else:
            loss, gm_np, gz_np, dts = mesh.adjoint(nsteps, gauges, target, cfl, checkpoint_every)
            gm, gz = torch.from_numpy(gm_np), torch.from_numpy(gz_np)
        ctx.save_for_backward(gm, gz)
        ctx.dts = dts
        return torch.tensor(loss, dtype=torch.float64, device=dev)

    @staticmethod
    def backward(ctx, grad_loss):
        gm, gz = ctx.saved_tensors
        return grad_loss * gm, grad_loss * gz, None, None, None, None, None, None, None
