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


def calibrate(target_drag: float, F_ext: float, make_lattice, beads, gamma0: float, nsteps: int, window: int,
              param: str = "gamma", axis: int = 2, checkpoints: int = 0, iters: int = 8, rtol: float = 1e-10):
    """Fit the bead friction gamma (param="gamma") or a uniform scale of the
    bead offsets (param="scale", the raspberry's size at fixed gamma) so that
    the drag xi = F_ext / J of the pulled colloid equals target_drag: Newton
    iterations on xi(p) - target with dxi/dp from the adjoint (for the scale,
    dxi/ds summed against the offsets). This is the calibration of a
    raspberry's hydrodynamic radius against a target drag (e.g. 6 pi eta R).
    Returns (p, xi, history)."""
    b0 = torch.as_tensor(np.asarray(beads, dtype=np.float64))
    p = float(gamma0 if param == "gamma" else 1.0)
    hist = []
    for _ in range(iters):
        if param == "gamma":
            g = torch.tensor(p, dtype=torch.float64, requires_grad=True)
            b = b0.clone()
            J = terminal_velocity(g, b, make_lattice, nsteps, window, axis, checkpoints)
            xi = F_ext / J
            xi.backward()
            dxi = g.grad.item()
        elif param == "scale":
            g = torch.tensor(float(gamma0), dtype=torch.float64)
            sc = torch.tensor(p, dtype=torch.float64, requires_grad=True)
            b = b0 * sc
            J = terminal_velocity(g, b, make_lattice, nsteps, window, axis, checkpoints)
            xi = F_ext / J
            xi.backward()
            dxi = sc.grad.item()
        else:
            raise ValueError("param must be 'gamma' or 'scale'")
        hist.append((p, xi.item()))
        step = (xi.item() - target_drag) / dxi
        p -= step
        if abs(step) <= rtol * abs(p):
            break
    return p, hist[-1][1], hist
