"""Ellipsoidal raspberry construction, plain FP64 (test infrastructure only).

TEST INFRASTRUCTURE ONLY: tests/, the smoke check and the benchmark's CPU
baseline leg may import this module; the CUDA library never does, and this
module shares no code with it.

Ustach & Faller (arXiv:1604.01829) build a raspberry's surface shell in an
MD-style scheme (Sec. 2.1; SI "Details for ellipsoidal raspberry
construction"):

* every surface bead is pulled towards the nearest point r_s of the surface by
  a harmonic potential U = k |r - r_s|^2 (Eq. (harmonic_sphere) for a sphere);
* r_s follows from the normal condition r - r_s = (t/2) grad S(r_s), which
  gives x = x_s (t/a^2 + 1), ... (Eq. (xtoxs)); inserted into the surface
  equation (Eq. (ellsurfacecoords)) this is F(t) = 0, solved by bisection for
  the largest root (Eq. (bisection));
* the surface beads repel each other pairwise with a WCA potential;
* the beads are integrated with a damped leapfrog (damping eta = 1000, WCA
  sigma = 1.4, epsilon = 0.1, dt = 0.001 in the paper).

Readings of what the paper leaves open or prints garbled:

* Eq. (bisection) as printed has "+1" inside each square, which contradicts
  Eq. (xtoxs); the function used is
  F(t) = (x a/(t + a^2))^2 + (y b/(t + b^2))^2 + (z c/(t + c^2))^2 - 1.
  F decreases for t > -min(a^2, b^2, c^2); the root is bracketed by
  t_lo = -m^2 + m |x_m| (m the smallest semi-axis, x_m the bead's coordinate
  along it; the largest such coordinate among equal smallest axes), where
  the term of that axis alone is 1, and t_hi = a_max |r|, where F <= 0. The
  paper stops at |F| < 1e-6; here the bracket is halved 64 times (to FP64
  resolution of its width), which meets that tolerance.
* The spring constant k is not given: k = 1000 by default.
* The damped leapfrog with unit mass: v <- (1 - eta dt) v + dt F(r),
  r <- r + dt v. With the paper's eta dt = 1 this is steepest descent with
  step dt^2.
* Optionally (the default of the CUDA entry point) every bead is finally
  replaced by its nearest surface point, so the hydrodynamic sites lie on the
  surface.
"""
from __future__ import annotations

import math

import numpy as np

WCA_CUT = 2.0 ** (1.0 / 6.0)
BISECTION_HALVINGS = 64


def bisection_function(t, r, axes):
    """F(t) of Eq. (bisection), read without the printed '+1' (see above)."""
    r = np.asarray(r, dtype=np.float64)
    axes = np.asarray(axes, dtype=np.float64)
    return float(np.sum((r * axes / (t + axes * axes)) ** 2) - 1.0)


def surface_point(r, axes):
    """Nearest point r_s of the ellipsoid surface to r and the parameter t
    (Eqs. (xtoxs), (bisection)), by bisection on the bracket above."""
    r = np.asarray(r, dtype=np.float64)
    axes = np.asarray(axes, dtype=np.float64)
    m = float(np.min(axes))
    tied = [k for k in range(3) if axes[k] == m]
    xm = max(abs(float(r[k])) for k in tied)
    lo = -m * m + m * xm
    hi = float(np.max(axes)) * float(np.linalg.norm(r))
    if hi < lo:
        hi = lo
    for _ in range(BISECTION_HALVINGS):
        mid = 0.5 * (lo + hi)
        if bisection_function(mid, r, axes) > 0.0:
            lo = mid
        else:
            hi = mid
    t = 0.5 * (lo + hi)
    den = t + axes * axes
    # den > 0 unless the bracket collapsed onto t_lo = -m^2 (a bead on the
    # medial set inside, where the nearest point is not unique): that
    # component is then 0
    rs = np.where(den > 0.0, r * axes * axes / np.where(den > 0.0, den, 1.0), 0.0)
    return rs, t


def wca_force(d, sigma, epsilon):
    """Force on bead i from bead j, d = r_i - r_j: WCA (Lennard-Jones cut and
    shifted at its minimum 2^(1/6) sigma, purely repulsive)."""
    r2 = float(np.dot(d, d))
    if r2 >= (WCA_CUT * sigma) ** 2:
        return np.zeros(3)
    s6 = (sigma * sigma / r2) ** 3
    return 24.0 * epsilon * (2.0 * s6 * s6 - s6) / r2 * np.asarray(d, dtype=np.float64)


def wca_energy(r2, sigma, epsilon):
    if r2 >= (WCA_CUT * sigma) ** 2:
        return 0.0
    s6 = (sigma * sigma / r2) ** 3
    return 4.0 * epsilon * (s6 * s6 - s6) + epsilon


def surface_points(X, axes):
    """surface_point for every row of X at once (the same bisection, the
    bracket halved for all beads together)."""
    X = np.asarray(X, dtype=np.float64).reshape(-1, 3)
    axes = np.asarray(axes, dtype=np.float64)
    m = float(np.min(axes))
    tied = [k for k in range(3) if axes[k] == m]
    xm = np.max(np.abs(X[:, tied]), axis=1)
    lo = -m * m + m * xm
    hi = float(np.max(axes)) * np.linalg.norm(X, axis=1)
    hi = np.maximum(hi, lo)
    for _ in range(BISECTION_HALVINGS):
        mid = 0.5 * (lo + hi)
        F = np.sum((X * axes / (mid[:, None] + axes * axes)) ** 2, axis=1) - 1.0
        pos = F > 0.0
        lo = np.where(pos, mid, lo)
        hi = np.where(pos, hi, mid)
    t = 0.5 * (lo + hi)
    den = t[:, None] + axes * axes
    return np.where(den > 0.0, X * axes * axes / np.where(den > 0.0, den, 1.0), 0.0)


def forces(X, axes, k, sigma, epsilon):
    """Total force on every bead: harmonic pull to its nearest surface point
    (-2k (r - r_s)) plus the WCA forces of all other beads of the shell."""
    X = np.asarray(X, dtype=np.float64).reshape(-1, 3)
    F = -2.0 * k * (X - surface_points(X, axes))
    d = X[:, None, :] - X[None, :, :]                 # d[i, j] = r_i - r_j
    r2 = (d * d).sum(-1)
    np.fill_diagonal(r2, np.inf)
    near = r2 < (WCA_CUT * sigma) ** 2
    r2n = np.where(near, r2, 1.0)
    s6 = (sigma * sigma / r2n) ** 3
    fm = np.where(near, 24.0 * epsilon * (2.0 * s6 * s6 - s6) / r2n, 0.0)
    return F + (fm[:, :, None] * d).sum(axis=1)


def energy(X, axes, k, sigma, epsilon):
    """Harmonic plus pairwise WCA energy of a shell."""
    X = np.asarray(X, dtype=np.float64).reshape(-1, 3)
    U = k * float(((X - surface_points(X, axes)) ** 2).sum())
    for i in range(len(X)):
        for j in range(i + 1, len(X)):
            d = X[i] - X[j]
            U += wca_energy(float(np.dot(d, d)), sigma, epsilon)
    return U


def relax_shell(X0, axes, steps, k=1000.0, sigma=1.4, epsilon=0.1, dt=1e-3, eta=1000.0,
                project_final=True):
    """Damped-leapfrog relaxation of one shell from positions X0 (zero initial
    velocity, unit mass), then optionally each bead onto its surface point."""
    X = np.array(X0, dtype=np.float64).reshape(-1, 3)
    V = np.zeros_like(X)
    for _ in range(int(steps)):
        F = forces(X, axes, k, sigma, epsilon)
        V = (1.0 - eta * dt) * V + dt * F
        X = X + dt * V
    if project_final:
        X = surface_points(X, axes)
    return X


def nearest_neighbour_distances(X):
    X = np.asarray(X, dtype=np.float64)
    d = np.sqrt(((X[:, None, :] - X[None, :, :]) ** 2).sum(-1))
    np.fill_diagonal(d, math.inf)
    return d.min(axis=1)
