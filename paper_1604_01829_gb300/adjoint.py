"""Differentiable drag through the hand-written adjoint (torch.autograd).

``terminal_velocity(gamma, beads, make_lattice, ...)`` returns J, the mean
velocity over the last steps of a colloid pulled by a constant force, as a
torch scalar whose gradient with respect to the bead friction gamma and the
body-frame bead offsets comes from ``lb_adjoint_drag`` (the reverse pass of
the CUDA library, include/lb.h). The drag is xi = F_ext / J (Eq. (stokesflow)
of Ustach & Faller, arXiv:1604.01829, read for a driven colloid), so
calibrating a raspberry's hydrodynamic radius against a target drag is a
gradient-based fit of gamma or of the bead offsets.
"""
from __future__ import annotations

import numpy as np
import torch


class _DragAdjoint(torch.autograd.Function):
    @staticmethod
    def forward(ctx, gamma, beads, make_lattice, nsteps, window, axis, checkpoints):
        L = make_lattice(float(gamma.detach().cpu()), beads.detach().cpu().numpy().astype(np.float64))
        try:
            J, dg, ds = L.lb_adjoint_drag(nsteps, window, body=0, axis=axis, checkpoints=checkpoints)
        finally:
            L.close()
        nb = beads.shape[0]
        ctx.save_for_backward(torch.tensor(dg, dtype=torch.float64),
                              torch.from_numpy(np.ascontiguousarray(ds[:nb])))
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        dg, ds = ctx.saved_tensors
        return gJ * dg, gJ * ds.to(gJ.dtype), None, None, None, None, None


def terminal_velocity(gamma: torch.Tensor, beads: torch.Tensor, make_lattice, nsteps: int, window: int,
                      axis: int = 2, checkpoints: int = 0) -> torch.Tensor:
    """J(gamma, beads). make_lattice(gamma, beads) must return a fresh
    ``lb.LB`` whose body 0 carries exactly these beads (translation-only or
    fixed bodies, kT = 0); the call consumes it."""
    return _DragAdjoint.apply(gamma, beads, make_lattice, nsteps, window, axis, checkpoints)
