"""Pins of the resistance-factor formulas (SI of Ustach & Faller,
arXiv:1604.01829: Perrin lab-frame factors, Happel-Brenner body-frame
translation factors, Perrin body-frame rotation factors) against routes that
do not use them: the Oberbeck friction integrals of a triaxial ellipsoid,
Perrin's closed-form rotational frictions of spheroids, the sphere limit and
the relations between lab-frame and body-frame factors."""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import factors as Fc

PROLATE = [1.25, 2.0, 3.0, 6.0]
OBLATE = [0.2, 0.5, 0.8]


def _oberbeck(a, b, c):
    """chi = int ds / Delta and alpha_i = int ds / ((a_i^2 + s) Delta) with
    Delta = sqrt((a^2+s)(b^2+s)(c^2+s)); Stokes friction along axis i is
    16 pi eta / (chi + a_i^2 alpha_i), rotational friction about axis i is
    16 pi eta (a_j^2 + a_k^2) / (3 (a_j^2 alpha_j + a_k^2 alpha_k))."""
    D = lambda s: math.sqrt((a * a + s) * (b * b + s) * (c * c + s))
    kw = dict(epsabs=0.0, epsrel=1e-13, limit=400)
    chi = quad(lambda s: 1.0 / D(s), 0.0, math.inf, **kw)[0]
    al = [quad(lambda s, x=x: 1.0 / ((x * x + s) * D(s)), 0.0, math.inf, **kw)[0] for x in (a, b, c)]
    ax = (a, b, c)
    xt = [16 * math.pi / (chi + ax[i] ** 2 * al[i]) for i in range(3)]
    xr = [16 * math.pi * (ax[j] ** 2 + ax[k] ** 2) / (3 * (ax[j] ** 2 * al[j] + ax[k] ** 2 * al[k]))
          for (j, k) in ((1, 2), (2, 0), (0, 1))]
    return xt, xr                     # per unit viscosity


@pytest.mark.parametrize("phi", [1.0, 1 - 1e-4, 1 + 1e-4])
def test_sphere_limit_of_every_factor(phi):
    vals = [Fc.perrin_A(phi), Fc.perrin_B(phi), *Fc.perrin_rotation(phi)]
    vals += [Fc.happel_brenner_E(phi), Fc.happel_brenner_F(phi)] if phi >= 1 else \
        [Fc.happel_brenner_G(phi), Fc.happel_brenner_H(phi)]
    assert np.allclose(vals, 1.0, atol=1e-3), vals


@pytest.mark.parametrize("phi", PROLATE + OBLATE)
def test_translation_factors_match_oberbeck_integrals(phi):
    xt, _ = _oberbeck(phi, 1.0, 1.0)
    R = [x / (6 * math.pi) for x in xt]            # Stokes radii, c = 1
    if phi > 1:
        got = [Fc.happel_brenner_E(phi), Fc.happel_brenner_F(phi)]
    else:
        got = [Fc.happel_brenner_G(phi), Fc.happel_brenner_H(phi)]
    assert np.allclose(got, [R[0], R[1]], rtol=1e-9), (got, R)
    # lab frame: the orientation average is the harmonic mean of the frictions
    R_lab = 3.0 / sum(1.0 / r for r in R)
    assert Fc.perrin_A(phi) == pytest.approx(phi / R_lab, rel=1e-9)


@pytest.mark.parametrize("phi", PROLATE + OBLATE)
def test_rotation_factors_match_jeffery_and_perrin_closed_forms(phi):
    _, xr = _oberbeck(phi, 1.0, 1.0)
    R3 = [x / (8 * math.pi) for x in xr]
    I, J = Fc.perrin_rotation(phi)
    assert [I, J] == pytest.approx([R3[0], R3[1]], rel=1e-9)
    # Perrin's closed forms for a spheroid (a, b = c = 1)
    a, b = phi, 1.0
    if a > b:
        e = math.sqrt(a * a - b * b)
        S = 2.0 * math.log((a + e) / b) / e
    else:
        e = math.sqrt(b * b - a * a)
        S = 2.0 * math.atan(e / a) / e
    xs = 32.0 * math.pi / 3.0 * (a * a - b * b) * b * b / (2.0 * a - b * b * S)
    xd = 32.0 * math.pi / 3.0 * (a ** 4 - b ** 4) / ((2.0 * a * a - b * b) * S - 2.0 * a)
    assert [I, J] == pytest.approx([xs / (8 * math.pi), xd / (8 * math.pi)], rel=1e-8)
    # lab frame: harmonic mean of the three rotational frictions
    assert Fc.perrin_B(phi) == pytest.approx(phi ** 3 / 3.0 * (1.0 / I + 2.0 / J), rel=1e-9)


def test_printed_oblate_degenerate_factor_has_the_wrong_sign():
    """With the arcsine coefficient as printed, (2 phi^2 - 3), H would be
    negative; the reading (3 - 2 phi^2) is what the friction integrals give
    (checked above)."""
    phi = 0.5
    s = math.sqrt(1 - phi * phi)
    printed = 8 / 3 / (-phi / (1 - phi * phi) + (2 * phi * phi - 3) / s ** 3 * math.asin(s))
    assert printed < 0 < Fc.happel_brenner_H(phi)


def test_prolate_drag_ratio_values():
    """Tabulated-style values for the drag anisotropy of a 3:1 prolate
    spheroid: F/E = xi_perp / xi_par = 1.2301 (Oberbeck integrals above)."""
    assert Fc.happel_brenner_F(3.0) / Fc.happel_brenner_E(3.0) == pytest.approx(1.23008, rel=1e-4)
