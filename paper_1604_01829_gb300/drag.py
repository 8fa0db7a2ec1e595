"""Drag measurements on the CUDA path, through the C ABI (Sec. 2.3-2.4 and
Sec. 2.8 of Ustach & Faller, arXiv:1604.01829).

* pulled_drag: a raspberry pulled by a constant force through a periodic
  box, with the opposite force spread over the fluid so the total momentum
  stays zero; xi(L) = F / (V - mean fluid velocity) at steady state.
* unbounded: xi_0 from xi(L) at several box sizes by Hasimoto's law,
  1/xi(L) = 1/xi_0 - 2.837/(6 pi eta L) + c3/L^3 (Eq. (hasimoto) in its drag
  form; the 1/L coefficient fixed, c3 fitted).
* pore_drag: the drag of a raspberry translating along the axis of a
  periodic cylindrical pore through fluid at rest far away, at a radial
  offset from the axis (Sec. 2.8, the confinement geometry; the axial
  direction z^p of Sec. 3.3). The periodic pore cannot hold a sphere moving
  through a fluid at rest directly, so two runs are superposed (Stokes flow
  is linear): (A) the sphere pulled by F with no force on the fluid, (B) a
  free sphere in fluid driven by a uniform force density;
  U = U_A - (Q_A/Q_B) U_B is the sphere's velocity when the net flux Q
  through the pore vanishes, and xi = F / U.
* pore_radial_drag: the same raspberry moving radially towards the wall
  (the x^p direction of Sec. 3.3), whose momentum the walls take up.
* spin_drag: rotational drag xi_r = -T / omega of a raspberry held in place
  and spinning at omega in a periodic box.

Everything here only drives the library (steps, body state, conservation
sums); the arithmetic of the step is the library's.
"""
from __future__ import annotations

import math

import numpy as np

from . import lb

HASIMOTO = 2.837
BGK1 = dict(collision=0, tau=1.0)     # nu = 1/6: short viscous times, Re << 1


def pulled_drag(L, beads, mass, axis=0, F=1e-3, gamma=0.3, precision=64, params=None, X=None):
    """xi(L) of a translation-only raspberry pulled along `axis` in a periodic
    L^3 box with the compensating force on the fluid, after the viscous
    transient (1.5 L^2 steps), averaged over 10 samples 0.03 L^2 apart."""
    params = dict(BGK1 if params is None else params)
    Fe = [0.0, 0.0, 0.0]
    Fe[axis] = F
    h = lb.LB(L, L, L, precision=precision, gamma_bead=gamma, compensate_force=1, **params)
    try:
        X = [L / 2 + 0.13, L / 2 - 0.21, L / 2 + 0.07] if X is None else X
        h.lb_add_raspberry(beads, X, mass=mass, inertia=(mass,) * 3, F_ext=Fe, fixed=2)
        h.lb_step(int(1.5 * L * L))
        rel = []
        for _ in range(10):
            h.lb_step(max(1, int(0.03 * L * L)))
            m, p = h.lb_conservation()
            rel.append(h.lb_get_body(0)["V"][axis] - p[axis] / m)
    finally:
        h.close()
    return F / float(np.mean(rel))


def unbounded(xis, Ls, eta):
    """xi_0 from pulled drags xi(L) (Hasimoto slope fixed, L^-3 term fitted)."""
    x = 1.0 / np.asarray(Ls, float)
    y = 1.0 / np.asarray(xis, float) + HASIMOTO / (6 * math.pi * eta) * x
    c = np.linalg.lstsq(np.stack([np.ones_like(x), x ** 3], axis=1), y, rcond=None)[0]
    return 1.0 / c[0]


def pore_flux_radius(nx, nz, R, eta, g=1e-6, precision=64, params=None, steps=6000):
    """Hydrodynamic radius of the staircase pore: R_h with the Poiseuille
    flux pi g R_h^4 / (8 eta) of a fluid driven by the force density g."""
    params = dict(BGK1 if params is None else params)
    h = lb.LB(nx, nx, nz, precision=precision, body_force=(0, 0, g), **params)
    try:
        h.lb_set_pore(R, 2)
        h.lb_step(steps)
        P = []
        for _ in range(20):
            h.lb_step(100)
            P.append(h.lb_conservation()[1][2])
    finally:
        h.close()
    return (8 * eta * (float(np.mean(P)) / nz) / (math.pi * g)) ** 0.25


def pore_drag(nx, nz, R, beads, mass, offset=0.0, F=1e-3, g=1e-6, gamma=0.3, precision=64, params=None,
              steps=6000, samples=20, every=100):
    """xi of a raspberry moving along the axis of a z pore (radius R, box
    nx x nx x nz) at radial distance `offset` from the axis (along x),
    through fluid at rest far away (superposition of runs A and B above)."""
    params = dict(BGK1 if params is None else params)

    def run(Fz, gz):
        h = lb.LB(nx, nx, nz, precision=precision, gamma_bead=gamma, body_force=(0, 0, gz), **params)
        try:
            h.lb_set_pore(R, 2)
            h.lb_add_raspberry(beads, [nx / 2 + offset, nx / 2, nz / 2 + 0.3], mass=mass, inertia=(1e3,) * 3,
                               F_ext=(0, 0, Fz), fixed=2)
            h.lb_step(steps)
            U, P = [], []
            for _ in range(samples):
                h.lb_step(every)
                P.append(h.lb_conservation()[1][2])
                U.append(h.lb_get_body(0)["V"][2])
        finally:
            h.close()
        return float(np.mean(U)), float(np.mean(P))

    UA, PA = run(F, 0.0)
    UB, PB = run(0.0, g)
    return F / (UA - PA / PB * UB)


def pore_radial_drag(nx, nz, R, beads, mass, offset=0.0, F=1e-4, gamma=0.3, precision=64, params=None,
                     steps=6000, samples=20, every=100):
    """xi of a raspberry at radial distance `offset` from the axis of a z pore
    moving radially outwards (towards the wall, the x^p direction of Sec.
    3.3): pulled by F along x with no force on the fluid, whose momentum the
    walls take up, so at steady state xi = F / V_x. F is small so that the
    colloid moves by < 0.1 lattice units during the run."""
    params = dict(BGK1 if params is None else params)
    h = lb.LB(nx, nx, nz, precision=precision, gamma_bead=gamma, **params)
    try:
        h.lb_set_pore(R, 2)
        h.lb_add_raspberry(beads, [nx / 2 + offset, nx / 2, nz / 2 + 0.3], mass=mass, inertia=(1e3,) * 3,
                           F_ext=(F, 0, 0), fixed=2)
        h.lb_step(steps)
        U = []
        for _ in range(samples):
            h.lb_step(every)
            U.append(h.lb_get_body(0)["V"][0])
    finally:
        h.close()
    return F / float(np.mean(U))


def spin_drag(L, beads, omega=1e-4, axis=2, gamma=0.3, precision=64, params=None):
    """Rotational drag of a raspberry held in place (fixed = 1) and spinning
    at omega about `axis` at the centre of a periodic L^3 box:
    xi_r = -T_axis / omega at steady state (after 1.2 L^2 steps, mean of 5
    samples 0.02 L^2 apart)."""
    params = dict(BGK1 if params is None else params)
    h = lb.LB(L, L, L, precision=precision, gamma_bead=gamma, **params)
    try:
        h.lb_add_raspberry(beads, [L / 2 + 0.13, L / 2 - 0.21, L / 2 + 0.07], fixed=1)
        w = [0.0, 0.0, 0.0]
        w[axis] = omega
        h.lb_set_body_state(0, w=tuple(w))
        h.lb_step(int(1.2 * L * L))
        T = []
        for _ in range(5):
            h.lb_step(max(1, int(0.02 * L * L)))
            T.append(h.lb_forces(0)[1][axis])
    finally:
        h.close()
    return -float(np.mean(T)) / omega


def bohlin(lam):
    """Centreline wall correction K(lambda) of a sphere in a cylinder
    (Bohlin 1960 / Haberman & Sayre 1958)."""
    return 1.0 / (1 - 2.10444 * lam + 2.08877 * lam ** 3 - 0.94813 * lam ** 5 - 1.372 * lam ** 6
                  + 3.87 * lam ** 8 - 4.19 * lam ** 10)
