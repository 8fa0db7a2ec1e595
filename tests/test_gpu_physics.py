"""Physics of the CUDA path itself (beyond parity), measured through the C
ABI against closed forms of Stokes flow:

* the Hasimoto finite-size law for the drag of a raspberry in a periodic box
  (Sec. 2.4, Eq. (hasimoto)), with the protocol of the oracle pin;
* the drag anisotropy of a prolate raspberry, xi_perp / xi_par = F / E of
  the Happel-Brenner factors (SI, Eqs. (happelbrenner_e), (happelbrenner_f)),
  and its rotational drag anisotropy against Perrin's spheroid factors
  (SI, Eqs. (dr_bf_i), (dr_bf_j));
* the drag of a sphere on the axis of a cylindrical pore (Sec. 2.8, the
  confinement geometry) against the centreline wall-correction series of
  Bohlin (1960) / Haberman & Sayre (1958), K(lambda) = 1 / (1 - 2.10444
  lambda + 2.08877 lambda^3 - 0.94813 lambda^5 - 1.372 lambda^6 + 3.87
  lambda^8 - 4.19 lambda^10), whose leading term is the 1 + 2.104 lambda of
  the Faxen-type expansion;
* the Stokes-flow resistance set-up (Sec. 2.3, Eq. (stokesflow)): a fixed
  raspberry between moving walls gives, extrapolated in the box size, the
  same unbounded drag as a pulled raspberry in a periodic box extrapolated
  by Hasimoto's law.

* the fluctuating fluid: node velocity variance kT/rho0 per component and the
  stationary variance 3 rho0 kT b_k of every non-conserved mode;
* resistance against the designed radius (Sec. 3.2): linear, through a
  renormalised radius offset from R by a constant, for translation and
  rotation; and against the bead friction (Sec. 3.1): rising to a plateau,
  the bead friction in series with the hydrodynamic resistance.

The drag runs: BGK tau = 1 (nu = 1/6), FP64, deterministic fluid (kT = 0)."""
import math

import numpy as np
import pytest

from helpers import observe
from oracle import factors as Fc
from paper_1604_01829_gb300 import workloads as Wl

pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1604_01829_gb300 import build
    build.build()


def _drag_cuda(L, g=1e-6):
    from paper_1604_01829_gb300 import lb
    h = lb.LB(L, L, L, precision=64, collision=0, tau=1.0, gamma_bead=0.3, body_force=(g, 0, 0))
    h.lb_add_raspberry(Wl.sphere_raspberry(2.0), [L / 2 + 0.13, L / 2 - 0.21, L / 2 + 0.07], fixed=1)
    h.lb_step(int(1.5 * L * L))
    us = []
    for k in range(3):
        m, p = h.lb_conservation()
        us.append(p[0] / m)
        if k < 2:
            h.lb_step(int(0.6 * L * L))
    h.close()
    U1, U2, U3 = us
    return g * L ** 3 / ((U1 * U3 - U2 * U2) / (U1 + U3 - 2 * U2))


def test_hasimoto_slope_on_the_cuda_path():
    """FP64 CUDA path, L = 16-40, raspberry R = 2: same protocol and bound
    as the oracle pin (mean momentum sampled after the viscous transient,
    steady mean flow by Aitken extrapolation, 1/L coefficient fitted with the
    L^-3 term free)."""
    Ls = np.array([16, 20, 24, 32, 40], float)
    xi = np.array([_drag_cuda(int(L)) for L in Ls])
    x = 1.0 / Ls
    A = np.stack([np.ones_like(x), x, x ** 3], axis=1)
    b = np.linalg.lstsq(A, 1.0 / xi, rcond=None)[0][1]
    eta = 0.5 / 3.0
    assert abs(b / (-2.837 / (6 * math.pi * eta)) - 1) < 0.02, (xi, b)
    assert np.all(np.diff(xi) < 0)


ETA = 1.0 / 6.0
HASIMOTO = -2.837 / (6 * math.pi * ETA)


def _pulled_drag(L, beads, mass, axis, F=1e-3):
    """Drag of a translation-only raspberry pulled by F along `axis` in a
    periodic L^3 box with the compensating force on the fluid (BGK tau = 1,
    gamma = 0.3, FP64; paper_1604_01829_gb300.drag.pulled_drag)."""
    from paper_1604_01829_gb300 import drag as D
    return D.pulled_drag(L, beads, mass, axis, F)


def _unbounded(xis, Ls):
    """xi_0 by Hasimoto's law (slope fixed, L^-3 term fitted)."""
    from paper_1604_01829_gb300 import drag as D
    return D.unbounded(xis, Ls, ETA)


def test_prolate_drag_anisotropy_matches_happel_brenner():
    """A 3:1 prolate raspberry (semi-axes 9, 3, 3) pulled along its long and
    along a short body axis, L = 48-80, extrapolated to infinite dilution:
    xi_perp / xi_par within 4 % of F(3) / E(3) = 1.230 (measured 1.207; the
    raspberry surface is a shell of beads, not a smooth spheroid)."""
    beads = Wl.ellipsoid_raspberry(9.0, 3.0, 3.0)
    mass = 4.0 / 3.0 * math.pi * 81.0
    Ls = [48, 64, 80]
    par = _unbounded([_pulled_drag(L, beads, mass, 0) for L in Ls], Ls)
    perp = _unbounded([_pulled_drag(L, beads, mass, 1) for L in Ls], Ls)
    expect = Fc.happel_brenner_F(3.0) / Fc.happel_brenner_E(3.0)
    assert perp > par
    assert abs(perp / par / expect - 1) < 0.04, (par, perp, perp / par, expect)


def test_prolate_rotational_drag_anisotropy_matches_perrin():
    """The same 3:1 prolate raspberry held in place and spinning about its
    long axis and about a short one (L = 64; the rotational drag changes by
    < 0.3 % from L = 48 to 80): xi_r,perp / xi_r,par within 4 % of Perrin's
    spheroid value J / I = 3.129 (SI, Eqs. (dr_bf_i), (dr_bf_j); measured
    3.169), and the two short axes agree (rotational symmetry of the bead
    shell about the long axis)."""
    from paper_1604_01829_gb300 import drag as D
    beads = Wl.ellipsoid_raspberry(9.0, 3.0, 3.0)
    par = D.spin_drag(64, beads, axis=0)
    perp_y = D.spin_drag(64, beads, axis=1)
    perp_z = D.spin_drag(64, beads, axis=2)
    I, J = Fc.perrin_rotation(3.0)
    observe("rot_anisotropy_vs_perrin", abs(perp_y / par / (J / I) - 1))
    assert abs(perp_y / perp_z - 1) < 1e-3, (perp_y, perp_z)
    assert abs(perp_y / par / (J / I) - 1) < 0.04, (par, perp_y, perp_y / par, J / I)


def test_pore_drag_enhancement_across_radial_offsets():
    """The confinement workload's drag readout (Sec. 2.8 and Sec. 3.3): a
    sphere raspberry (R = 4) in a periodic pore (R_pore = 20, 48 x 48 x 96,
    halfway bounce-back) at d = 0, 0.2, 0.4, 0.6 R_pore from the axis,
    deterministic, FP64 and FP32 (deviation storage); enhancement
    S = xi_pore / xi_0, xi_0 from the periodic-box extrapolation of the same
    raspberry (paper_1604_01829_gb300.drag).

    * Axial motion (z^p): on the axis S is within 2 % of Bohlin's K(lambda)
      (lambda = a / R_h, a = xi_0 / (6 pi eta), R_h the pore radius seen by
      Poiseuille flow) and beyond its leading term 1 + 2.104 lambda. Off the
      axis S first falls and then rises towards the wall: Sec. 3.3 states that
      the reference values for this direction have their minimum at an
      off-centre position (the pressure force is largest at the centre, the
      lubrication force at the wall), a minimum the paper's own simulations
      did not capture. Measured on GB300: 1.600, 1.588, 1.568, 1.614.
    * Radial motion towards the wall (x^p, head-on): S rises monotonically
      with the offset, as Sec. 3.3 describes, and on the axis it is below the
      axial value (a sphere on the axis is hindered less moving across the
      pore than along it).
    * FP32 gives the FP64 values within 2e-4.
    The off-axis values themselves (Happel-Brenner / Higdon-Muldowney) are
    not available here: parity unpinned beyond these shapes."""
    from paper_1604_01829_gb300 import drag as D
    beads = Wl.sphere_raspberry(4.0)
    mass = 4.0 / 3.0 * math.pi * 64.0
    R, nx, nz = 20.0, 48, 96
    R_h = D.pore_flux_radius(nx, nz, R, ETA)
    assert abs(R_h - R) < 0.05, R_h                          # halfway wall at R
    Ls = [32, 48, 64, 80]
    xi0 = D.unbounded([D.pulled_drag(L, beads, mass, 0) for L in Ls], Ls, ETA)
    lam = xi0 / (6 * math.pi * ETA) / R_h
    offs = [0.0, 0.2, 0.4, 0.6]
    Sz = {p: np.array([D.pore_drag(nx, nz, R, beads, mass, offset=b * R, precision=p) / xi0 for b in offs])
          for p in (64, 32)}
    Sx = {p: np.array([D.pore_radial_drag(nx, nz, R, beads, mass, offset=b * R, precision=p) / xi0 for b in offs])
          for p in (64, 32)}
    print("lambda", lam, "Bohlin", D.bohlin(lam), "Sz64", Sz[64], "Sz32", Sz[32], "Sx64", Sx[64], "Sx32", Sx[32])
    assert abs(Sz[64][0] / D.bohlin(lam) - 1) < 0.02, (Sz[64][0], lam, D.bohlin(lam))
    assert Sz[64][0] > 1 + 2.104 * lam
    for p in (64, 32):
        kmin = int(np.argmin(Sz[p]))
        assert 0 < kmin < len(offs) - 1, (p, Sz[p])         # off-centre minimum of the axial drag
        assert np.all(np.diff(Sx[p]) > 0), (p, Sx[p])       # head-on: rising towards the wall
        assert Sx[p][0] < Sz[p][0], (p, Sx[p], Sz[p])
    rel = max(np.abs(Sz[32] / Sz[64] - 1).max(), np.abs(Sx[32] / Sx[64] - 1).max())
    observe("S32_vs_S64", rel)
    assert rel < 2e-4, rel


def test_stokes_flow_set_up_gives_the_unbounded_drag():
    """Eq. (stokesflow): a fixed sphere raspberry (R = 2) at the centre of a
    cubic box whose +y and -y walls move at U along z; the steady summed bead
    force is xi_S(L) U. Fitting xi_S(L) = xi_0 (1 - c / L) over L = 32, 48, 64
    gives xi_0 within 1 % of the pulled-body value extrapolated with
    Hasimoto's law (measured: 0.1 %); xi_S grows with L toward it."""
    from paper_1604_01829_gb300 import lb
    beads = Wl.sphere_raspberry(2.0)
    U = 1e-3
    Ls = [32, 48, 64]
    xs = []
    for L in Ls:
        h = lb.LB(L, L, L, precision=64, collision=0, tau=1.0, gamma_bead=0.3)
        h.lb_set_channel_walls((0, 0, U), (0, 0, U))
        h.lb_add_raspberry(beads, [L / 2 + 0.13, L / 2 - 0.21, L / 2 + 0.07], fixed=1)
        T = int(12 * L * L / (ETA * math.pi ** 2))        # 12 e-folds of the slowest channel mode
        h.lb_step(T)
        F, _ = h.lb_forces(0)
        h.close()
        xs.append(F[2] / U)
    assert np.all(np.diff(xs) > 0)
    A = np.stack([np.ones(3), -1.0 / np.asarray(Ls, float)], axis=1)
    xi0_stokes = np.linalg.lstsq(A, np.asarray(xs), rcond=None)[0][0]
    mass = 4.0 / 3.0 * math.pi * 8.0
    xi0_pulled = _unbounded([_pulled_drag(L, beads, mass, 0) for L in Ls], Ls)
    assert abs(xi0_stokes / xi0_pulled - 1) < 0.01, (xs, xi0_stokes, xi0_pulled)


@pytest.mark.parametrize("precision", [64, 32])
def test_fluctuating_fluid_thermalises_on_the_cuda_path(precision):
    """Fluctuating MRT (Sec. 1.1, stochastic mode; 16-bit Philox variates) on
    the CUDA path: after a warm-up the node velocity variance per component is
    kT/rho0, and every non-conserved mode k has the stationary variance
    3 rho0 kT b_k (b_k the mode norm). The mode basis and norms are the
    oracle's (Gram-Schmidt of the DSL polynomials)."""
    from oracle import oracle as O
    from paper_1604_01829_gb300 import lb
    kT, L = 1e-4, 24
    rates = dict(collision=1, gamma_shear=-0.5, gamma_bulk=-0.3, gamma_odd=0.0, gamma_even=0.0)
    h = lb.LB(L, L, L, precision=precision, kT=kT, seed=4242, **rates)
    M, _, b = O.mrt_tables()
    c = np.array(O.lattice()[0], dtype=np.float64)
    h.lb_step(400)
    u2, mv = [], []
    for _ in range(40):
        h.lb_step(7)
        f = h.lb_get_populations()
        rho = f.sum(axis=0)
        u = (c.T @ f) / rho
        u2.append(((u - u.mean(axis=1, keepdims=True)) ** 2).mean(axis=1))
        m = M @ f
        mv.append((m[4:] ** 2).mean(axis=1))
    h.close()
    u2 = np.mean(u2, axis=0)
    assert np.all(np.abs(u2 / kT - 1.0) < 0.03), u2 / kT
    ratio = np.mean(mv, axis=0) / (3.0 * kT * b[4:])
    assert np.all(np.abs(ratio - 1.0) < 0.03), ratio


def _spin_drag(L, beads, omega=1e-4):
    """Rotational drag of a raspberry held in place and spinning at omega
    about z in a periodic L^3 box (paper_1604_01829_gb300.drag.spin_drag)."""
    from paper_1604_01829_gb300 import drag as D
    return D.spin_drag(L, beads, omega)


def test_resistance_grows_with_radius_through_a_renormalised_radius():
    """Sec. 3.2 (Fig. radius): the translational resistance of filled
    raspberries is linear in the designed radius R, and the rotational one in
    R^3, through a hydrodynamic radius offset from R by a constant (the LB
    renormalisation of the bead radius). On the CUDA path, R = 2, 3, 4 at
    gamma = 0.3 (lattice units, BGK tau = 1): xi_t extrapolated to infinite
    dilution (Hasimoto, two box sizes) lies on a line within 1 % with a slope
    within 5 % of 6 pi eta; the translational radius xi_t / (6 pi eta) and the
    rotational radius (xi_r / (8 pi eta))^(1/3) differ from R by offsets that
    vary by less than 0.05 between radii and are below half a grid spacing."""
    Rs = np.array([2.0, 3.0, 4.0])
    xi_t, xi_r = [], []
    for R in Rs:
        beads = Wl.sphere_raspberry(R)
        mass = 4.0 / 3.0 * math.pi * R ** 3
        Ls = [int(4 * R + 12), int(6 * R + 16)]
        xi_t.append(_unbounded([_pulled_drag(L, beads, mass, 2) for L in Ls], Ls))
        xi_r.append(_spin_drag(int(6 * R + 10), beads))
    xi_t, xi_r = np.array(xi_t), np.array(xi_r)
    a, b = np.polyfit(Rs, xi_t, 1)
    res = np.abs(np.polyval([a, b], Rs) / xi_t - 1).max()
    dt = xi_t / (6 * math.pi * ETA) - Rs
    dr = (xi_r / (8 * math.pi * ETA)) ** (1.0 / 3.0) - Rs
    info = dict(xi_t=xi_t, xi_r=xi_r, slope_ratio=a / (6 * math.pi * ETA), offset_t=dt, offset_r=dr)
    assert res < 0.01, info
    assert abs(a / (6 * math.pi * ETA) - 1) < 0.05, info
    for d in (dt, dr):
        assert np.ptp(d) < 0.05 and np.abs(d).max() < 0.5, info


def test_resistance_rises_with_bead_friction_towards_a_plateau():
    """Sec. 3.1 (Fig. friction_trans, the Stokes-flow half): the colloid's
    translational resistance rises with the bead friction towards a plateau.
    R = 2.5 in a 24^3 box, gamma = 0.025 ... 0.4 (lattice units; the explicit
    coupling of this bead density becomes unstable near 0.8). The bead
    friction acts in series with the hydrodynamic resistance (as in the
    effective friction of a point particle in LB, 1/xi_eff = 1/xi_bead +
    1/(g a eta)), so 1/xi is linear in 1/gamma (within 2 %), with a positive
    intercept: the plateau xi_inf, which the largest gamma approaches within
    20 %."""
    beads = Wl.sphere_raspberry(2.5)
    mass = 4.0 / 3.0 * math.pi * 2.5 ** 3
    from paper_1604_01829_gb300 import lb
    gam = np.array([0.025, 0.05, 0.1, 0.2, 0.4])
    xi = []
    for g in gam:
        h = lb.LB(24, 24, 24, precision=64, collision=0, tau=1.0, gamma_bead=float(g), compensate_force=1)
        h.lb_add_raspberry(beads, [12.13, 11.79, 12.07], mass=mass, inertia=(mass,) * 3, F_ext=(0, 0, 1e-3), fixed=2)
        h.lb_step(900)
        rel = []
        for _ in range(5):
            h.lb_step(20)
            m, p = h.lb_conservation()
            rel.append(h.lb_get_body(0)["V"][2] - p[2] / m)
        h.close()
        xi.append(1e-3 / float(np.mean(rel)))
    xi = np.array(xi)
    assert np.all(np.diff(xi) > 0), xi
    B, A = np.polyfit(1.0 / gam, 1.0 / xi, 1)
    fit = A + B / gam
    assert np.abs(fit * xi - 1).max() < 0.02, (xi, A, B)
    assert A > 0 and B > 0, (A, B)
    assert xi[-1] > 0.8 / A, (xi, 1.0 / A)
