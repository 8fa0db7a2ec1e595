"""Raspberry construction on the GPU (Sec. 2.1 and the SI section "Details for
ellipsoidal raspberry construction" of Ustach & Faller, arXiv:1604.01829).

A filled two-layer raspberry is a set of shells (outer hydrodynamic shell,
inner shell 0.5 further in, fill shells every unit further in, one bead per
unit area each) plus a line of core beads along the longest axis. Every
shell is relaxed on its ellipsoid by lb_relax_shells (harmonic pull to the
nearest surface point plus WCA between the shell's beads, damped leapfrog),
all shells of all requested raspberries in one launch. This module only
plans the shells and marshals arrays; the relaxation runs in the CUDA
library.
"""
from __future__ import annotations

import math

import numpy as np

from . import lb
from . import workloads as W


def build_raspberries(specs, steps=200000, seed=0, density=1.0, inner_offset=0.5, fill=True,
                      k_surface=1000.0, sigma=1.4, epsilon=0.1, dt=1e-3, eta=1000.0, precision=32,
                      stream=None):
    """Body-frame bead positions of one raspberry per (a, b, c) in specs.

    Each shell starts from seeded, roughly evenly spread points
    (workloads.spread_shell_start, nearest pairs ~0.65 apart at unit
    density). Defaults: the paper's WCA sigma and epsilon, damping and time
    step (eta dt = 1: steepest descent with step dt^2 = 1e-6, small enough for
    the closest starting pairs), k = 1000, and 2e5 of the paper's ~1e7 steps.
    Returns a list of [n, 3] arrays."""
    axes, starts, owner = [], [], []
    for r, (a, b, c) in enumerate(specs):
        for s, ((sa, sb, sc), n) in enumerate(W.raspberry_shells(a, b, c, density, inner_offset, fill)):
            axes.append((sa, sb, sc))
            starts.append(W.spread_shell_start(sa, sb, sc, n, seed=seed * 1000003 + 1009 * r + s))
            owner.append(r)
    relaxed = lb.lb_relax_shells(np.array(axes), starts, steps, k_surface=k_surface, sigma=sigma,
                                 epsilon=epsilon, dt=dt, eta=eta, precision=precision, project_final=True,
                                 stream=stream)
    out = []
    for r, (a, b, c) in enumerate(specs):
        parts = [x for x, o in zip(relaxed, owner) if o == r]
        if fill:
            ax = int(np.argmax([a, b, c]))
            m = int(math.floor(max(a, b, c) - min(a, b, c)))
            core = np.zeros((2 * m + 1, 3))
            core[:, ax] = np.arange(-m, m + 1, dtype=np.float64)
            parts.append(core)
        out.append(np.concatenate(parts, axis=0))
    return out
