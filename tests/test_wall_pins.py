"""Pins of the oracle's repulsive pore-wall beads (Sec. 2.3 of Ustach &
Faller, arXiv:1604.01829: beads around the pore surface, purely repulsive
WCA interaction with the colloid beads, sigma = r_r + r_p): the force is
minus the gradient of the energy, both vanish beyond 2^(1/6) sigma, the
WCA values at sigma, the ring symmetry on the axis, and the periodic image
along the axis."""
import math

import numpy as np
import pytest

from oracle import oracle as O

EPS, RP, RR, SP, R = 2e-3, 2.5, 0.5, 2.0, 7.5
SIGMA = RP + RR
RCUT = 2 ** (1 / 6) * SIGMA


def _lattice(n=(20, 20, 16), axis=2, R=R, spacing=SP):
    o = O.OracleLB(*n, collision=0, tau=1.0)
    o.set_pore(R, axis)
    o.set_pore_beads(R, axis, spacing, RP, RR, EPS)
    return o


def _wall_beads(n=(20, 20, 16), axis=2, R=R, spacing=SP):
    """The wall-bead positions as the oracle's documented lattice places them."""
    a1, a2 = (1, 2) if axis == 0 else ((0, 2) if axis == 1 else (0, 1))
    Rc = R + RP
    nth = max(3, round(2 * math.pi * Rc / spacing))
    nrow = max(1, round(n[axis] / spacing))
    out = []
    for k in range(nrow):
        for j in range(nth):
            p = np.zeros(3)
            p[a1] = 0.5 * n[a1] + Rc * math.cos(2 * math.pi * j / nth)
            p[a2] = 0.5 * n[a2] + Rc * math.sin(2 * math.pi * j / nth)
            p[axis] = (k + 0.5) * n[axis] / nrow
            out.append(p)
    return np.array(out)


def test_force_is_minus_the_gradient_of_the_energy():
    o = _lattice()
    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(20):
        ang = rng.uniform(0, 2 * math.pi)
        rad = rng.uniform(R + RP - RCUT + 0.05, R + RP - SIGMA * 0.92)
        r = np.array([10 + rad * math.cos(ang), 10 + rad * math.sin(ang), rng.uniform(0, 16)])
        F = o.wall_force(r)
        G = np.array([(o.wall_energy(r + h * e) - o.wall_energy(r - h * e)) / (2 * h) for e in np.eye(3)])
        assert np.allclose(F, -G, rtol=1e-5, atol=1e-9 * max(1.0, np.abs(F).max())), (r, F, -G)


def test_energy_and_force_vanish_beyond_the_cutoff_and_are_continuous():
    o = _lattice()
    walls = _wall_beads()
    # a point just outside every cutoff sphere, and the same point moved to 1e-7 inside one
    p = walls[5]
    direction = np.array([10.0, 10.0, p[2]]) - p
    direction /= np.linalg.norm(direction)
    out = p + (RCUT + 1e-9) * direction
    dmin = np.min(np.linalg.norm(walls - out, axis=1))
    if dmin >= RCUT:
        assert o.wall_energy(out) == 0.0 and np.all(o.wall_force(out) == 0.0)
    near = p + (RCUT - 1e-7) * direction
    assert 0.0 < o.wall_energy(near) < 1e-12 * EPS * 1e6


def test_wca_values_at_sigma():
    """At distance sigma from one wall bead (and beyond the cutoff of all
    others) U = epsilon and |F| = 24 epsilon / sigma, pointing away."""
    o = _lattice(spacing=6.0)            # wall beads far apart
    walls = _wall_beads(spacing=6.0)
    p = walls[0]
    direction = np.array([10.0, 10.0, p[2]]) - p
    direction /= np.linalg.norm(direction)
    r = p + SIGMA * direction
    assert np.sort(np.linalg.norm(walls - r, axis=1))[1] > RCUT
    assert o.wall_energy(r) == pytest.approx(EPS, rel=1e-12)
    F = o.wall_force(r)
    assert np.linalg.norm(F) == pytest.approx(24 * EPS / SIGMA, rel=1e-12)
    assert np.dot(F, direction) > 0


def test_ring_symmetry_on_the_axis():
    """A narrow pore (every wall bead of the nearest rings within the
    cutoff of the axis): on the axis, at a ring's height, the forces cancel."""
    Rn = 0.5
    o = O.OracleLB(12, 12, 12, collision=0, tau=1.0)
    o.set_pore(Rn, 2)
    o.set_pore_beads(Rn, 2, SP, RP, RR, EPS)
    r = np.array([6.0, 6.0, 0.5 * 12 / round(12 / SP)])
    F = o.wall_force(r)
    single = 24 * EPS / SIGMA
    assert o.wall_energy(r) > 0
    assert np.abs(F).max() <= 1e-12 * single


def test_periodic_image_along_the_axis():
    o = _lattice()
    r = np.array([10 + 6.9, 10.3, 0.4])
    assert np.allclose(o.wall_force(r), o.wall_force(r + np.array([0, 0, 16.0])), rtol=1e-12, atol=1e-18)
    assert np.allclose(o.wall_force(r), o.wall_force(r - np.array([0, 0, 48.0])), rtol=1e-12, atol=1e-18)
