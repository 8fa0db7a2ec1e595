"""Geometric resistance factors of ellipsoids of revolution (test
infrastructure only: the expected values of the physics tests of the CUDA
path; only ``tests/`` imports this module).

Ustach & Faller (arXiv:1604.01829) compare the transport of ellipsoidal
raspberries with closed forms given in their SI:

* lab frame (SI, "Perrin factors for lab-frame transport of ellipsoids"):
  A(phi) = a / R_eff,t (Eq. (a_phi)) and B(phi) = (a / R_eff,r)^3
  (Eq. (b_phi)), phi = a / b for semi-axes (a, b = c);
* body-frame translation (SI, "Happel-Brenner factors"): E, F for prolate
  and G, H for oblate ellipsoids, R_eff / c along the singular axis and
  along the degenerate axes (Eqs. (happelbrenner_e) to (happelbrenner_h));
* body-frame rotation (SI, "Perrin factors for body-frame rotation"):
  I, J (prolate) and K, L (oblate) = (R_eff,r / c)^3 about the singular and
  the degenerate axes, with the radii of Eq. (r_rot_a) built from the
  integrals P and Q (Eqs. (P), (Q)).

R_eff,t is the radius of the sphere with the same Stokes friction
(xi = 6 pi eta R), R_eff,r the one with the same rotational friction
(xi_r = 8 pi eta R^3).

Reading: Eq. (happelbrenner_h) as printed has (2 phi^2 - 3) in front of the
arcsine, which makes H negative for every oblate phi; the factor below uses
(3 - 2 phi^2), the sign for which H agrees with the Oberbeck friction
integrals and tends to 1 for a sphere.
"""
from __future__ import annotations

import math

from scipy.integrate import quad


def perrin_A(phi: float) -> float:
    """Lab-frame translation factor a / R_eff,t, Eq. (a_phi)."""
    if phi == 1.0:
        return 1.0
    r = math.sqrt(abs(1.0 - phi ** -2))
    if phi < 1.0:
        return math.atan(math.sqrt(phi ** -2 - 1.0)) / r
    return math.log(phi + math.sqrt(phi * phi - 1.0)) / r


def perrin_B(phi: float) -> float:
    """Lab-frame rotation factor (a / R_eff,r)^3, Eq. (b_phi)."""
    p2 = phi ** -2
    return (1.0 + 3.0 * p2 * perrin_A(phi)) / (2.0 * p2 * (1.0 + p2))


def happel_brenner_E(phi: float) -> float:
    """Prolate (phi > 1), translation along the singular axis: R_eff / c,
    Eq. (happelbrenner_e)."""
    if phi == 1.0:
        return 1.0
    s = math.sqrt(phi * phi - 1.0)
    den = -2.0 * phi / (phi * phi - 1.0) + (2.0 * phi * phi - 1.0) / s ** 3 * math.log((phi + s) / (phi - s))
    return 8.0 / 3.0 / den


def happel_brenner_F(phi: float) -> float:
    """Prolate, translation along a degenerate axis, Eq. (happelbrenner_f)."""
    if phi == 1.0:
        return 1.0
    s = math.sqrt(phi * phi - 1.0)
    den = phi / (phi * phi - 1.0) + (2.0 * phi * phi - 3.0) / s ** 3 * math.log(phi + s)
    return 8.0 / 3.0 / den


def happel_brenner_G(phi: float) -> float:
    """Oblate (phi < 1), translation along the singular axis,
    Eq. (happelbrenner_g)."""
    if phi == 1.0:
        return 1.0
    s = math.sqrt(1.0 - phi * phi)
    den = 2.0 * phi / (1.0 - phi * phi) + (2.0 - 4.0 * phi * phi) / s ** 3 * math.atan(s / phi)
    return 8.0 / 3.0 / den


def happel_brenner_H(phi: float) -> float:
    """Oblate, translation along a degenerate axis, Eq. (happelbrenner_h)
    with the arcsine coefficient read as (3 - 2 phi^2) (module docstring)."""
    if phi == 1.0:
        return 1.0
    s = math.sqrt(1.0 - phi * phi)
    den = -phi / (1.0 - phi * phi) + (3.0 - 2.0 * phi * phi) / s ** 3 * math.asin(s)
    return 8.0 / 3.0 / den


def rotation_PQ(a: float, c: float) -> tuple[float, float]:
    """The integrals P and Q of Eqs. (P) and (Q) for semi-axes (a, c = b), by
    adaptive quadrature over [0, inf)."""
    P = quad(lambda s: 1.0 / ((c * c + s) * (a * a + s) ** 1.5), 0.0, math.inf, epsabs=0.0, epsrel=1e-13,
             limit=400)[0]
    Q = quad(lambda s: 1.0 / ((c * c + s) ** 2 * math.sqrt(a * a + s)), 0.0, math.inf, epsabs=0.0,
             epsrel=1e-13, limit=400)[0]
    return P, Q


def rotation_radii(a: float, c: float) -> tuple[float, float]:
    """Rotational effective radii about the singular axis a and about a
    degenerate axis, Eq. (r_rot_a) (first and second form)."""
    P, Q = rotation_PQ(a, c)
    r_singular = (2.0 / (3.0 * Q)) ** (1.0 / 3.0)
    r_degenerate = (2.0 / 3.0 * (a * a + c * c) / (a * a * P + c * c * Q)) ** (1.0 / 3.0)
    return r_singular, r_degenerate


def perrin_rotation(phi: float) -> tuple[float, float]:
    """(R_eff,x^b,r / c)^3 and (R_eff,y^b z^b,r / c)^3 for a = phi, c = 1:
    I and J for a prolate ellipsoid (Eqs. (dr_bf_i), (dr_bf_j)), K and L for
    an oblate one (Eqs. (dr_bf_k), (dr_bf_l))."""
    rs, rd = rotation_radii(phi, 1.0)
    return rs ** 3, rd ** 3
