"""torch.autograd view of the load path: reaction curve as a differentiable
function of the ICNN weights.

``reaction = GDLoadPath.apply(theta, handle)`` sets the weights theta = [theta_psi |
theta_yield] (FP64, host or CUDA tensor) on the handle, restarts the path from the
undeformed state and runs every load step (gd_run_load_path); the backward pass
is the library's discrete adjoint through the whole path with history
(gd_backward, checkpointed every ``checkpoint_every`` steps).  The reaction curve
comes back as an FP64 tensor on theta's device.  Argument marshalling only: the
path and its adjoint run in the CUDA library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class GDLoadPath(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, handle: "B.Handle") -> torch.Tensor:
        meta = handle.meta
        n_psi, n_y = meta["n_psi"], meta["n_yield"]
        if theta.numel() != n_psi + n_y:
            raise ValueError(f"theta has {theta.numel()} entries, the handle's networks {n_psi + n_y}")
        th = theta.detach().to(torch.float64).contiguous()
        B.gd_set_params(handle, th[:n_psi] if n_psi else None, th[n_psi:] if n_y else None)
        n = meta["n_nodes"] * meta["ndof"]
        B.gd_set_state(handle, np.zeros(n), np.zeros((meta["n_elems"], meta["nq"])), 0)
        reac, _ = B.gd_run_load_path(handle)
        ctx.handle = handle
        ctx.generation = handle.generation
        ctx.device = theta.device
        return torch.as_tensor(np.array(reac), dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(ctx, grad_reaction: torch.Tensor):
        if ctx.handle.generation != ctx.generation:
            raise RuntimeError("the handle ran another path or changed its weights or state after this forward; "
                               "its adjoint would belong to that path")
        g = grad_reaction.detach().to(torch.float64).cpu().numpy()
        d_theta = B.gd_backward(ctx.handle, g)
        return torch.as_tensor(d_theta, dtype=torch.float64, device=ctx.device), None


def reaction_curve(theta: torch.Tensor, handle: "B.Handle") -> torch.Tensor:
    """Differentiable reaction curve of the handle's load path at weights theta."""
    return GDLoadPath.apply(theta, handle)
