"""Brownian colloids on the CUDA path (Sec. 2.4: translational diffusion
from mean squared displacements, Eqs. (dt_lab) and (hasimoto); Sec. 1.1,
Eq. (latticeboltzmannfriction): the bead noise obeys fluctuation-
dissipation).

* Equipartition: the set-ups of the oracle pin (tests/test_fdt_pins.py) on
  the GPU, FP64 and FP32, with longer runs: point colloids (one and two MD
  substeps) and a six-bead body (translation and rotation) take the fluid's
  temperature, <M V^2> = <I w^2> = kT within 5 %.
* Einstein relation: free sphere raspberries (R = 2, gamma = 0.3) in thermal
  periodic boxes L = 16, 24, 32 (one sphere per box, many independent boxes
  in one batched handle, the device recorder every 10 steps), FP32. The
  lab-frame MSD from lb_msd_trajectory grows linearly at lags beyond the
  fluid's slowest relaxation, with slope 2 D(L) per axis (Eq. (dt_lab)).
  With the total momentum held at zero (fluid and bead noise both conserve
  it), the body's displacement is that of the body relative to the fluid,
  scaled by 1/(1 + M/(rho L^3)); so D(L) (1 + M/(rho L^3))^2 = kT / xi(L),
  where xi(L) is the drag of the same sphere pulled through the same box
  with the compensating force on the fluid (deterministic run). Measured on
  GB300: 0.989, 0.974, 0.992 of kT / xi(L) (standard errors 0.8-1.9 %).
  Extrapolated with Hasimoto's law, D(L) = D0 - 2.837 kT/(6 pi eta L), the
  diffusion data give D0 = kT / xi0, xi0 the pulled drag extrapolated the
  same way, and the 1/L slope of D(L) is Hasimoto's.
* Rotation (Sec. 2.5, Sec. 2.7) from the same trajectories: the summed
  body-frame angular displacements (projection method) grow as 2 D_r t per
  body axis and the angle of a body-fixed vector as 4 D_r t (small angles),
  with D_r = kT / xi_r, xi_r the torque per angular velocity of the same
  sphere held in place and spinning in the same box (drag.spin_drag).
  Measured on GB300: within 1.0 % at every box size for both forms
  (standard errors 0.7-0.9 %; bound 6 %).
* Anisotropic rotation: a free 3:1 prolate raspberry's body-frame
  projections give D_r about its long and short axes, each kT / xi_r of
  the same raspberry spinning about that axis (within 1.4 % and 0.9 %).
"""
import math

import numpy as np
import pytest

from helpers import observe
from paper_1604_01829_gb300 import workloads as Wl

pytestmark = pytest.mark.gpu

ZERO_RATES = dict(collision=1, gamma_shear=0.0, gamma_bulk=0.0, gamma_odd=0.0, gamma_even=0.0)
KT = 1e-4
ETA = 1.0 / 6.0                       # all rates 0: nu = 1/6, rho0 = 1
HASIMOTO = -2.837 / (6 * math.pi * ETA)
OCTAHEDRON = 0.6 * np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1604_01829_gb300 import build
    build.build()


def _equipartition(precision, nbodies, beads, gamma, mass, inertia, nsub=1, steps=24000, burn=400, seed=7, L=10):
    from paper_1604_01829_gb300 import lb
    h = lb.LB(L, L, L, precision=precision, kT=KT, seed=seed, gamma_bead=gamma, md_substeps=nsub, **ZERO_RATES)
    rng = np.random.default_rng(seed)
    for _ in range(nbodies):
        h.lb_add_raspberry(beads, rng.uniform(0, L, 3), (1, 0, 0, 0), mass, (inertia,) * 3)
    h.lb_step(burn)
    V2 = np.zeros((steps, nbodies, 3))
    W2 = np.zeros((steps, nbodies, 3))
    for k in range(steps):
        h.lb_step(1)
        for b in range(nbodies):
            s = h.lb_get_body(b)
            V2[k, b] = s["V"] ** 2
            W2[k, b] = s["w"] ** 2
    h.close()
    nblk = 20

    def stat(a, m):
        blk = (a * m / KT).reshape(nblk, -1).mean(axis=1)
        return blk.mean(), blk.std(ddof=1) / math.sqrt(nblk)

    return stat(V2, mass) + stat(W2, inertia)


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("nsub", [1, 2])
def test_point_colloids_take_the_fluid_temperature(precision, nsub):
    t, st, _, _ = _equipartition(precision, 6, np.zeros((1, 3)), 0.25, 1.0, 1.0, nsub=nsub)
    observe("T_trans", abs(t - 1))
    assert st < 0.01, st
    assert abs(t - 1.0) < 0.05, (t, st)


@pytest.mark.parametrize("precision", [64, 32])
def test_a_small_raspberry_takes_the_fluid_temperature(precision):
    t, st, r, sr = _equipartition(precision, 4, OCTAHEDRON, 0.08, 2.0, 0.4)
    observe("T_trans", abs(t - 1))
    observe("T_rot", abs(r - 1))
    assert st < 0.01 and sr < 0.01, (st, sr)
    assert abs(t - 1.0) < 0.05 and abs(r - 1.0) < 0.05, (t, r)


R_SPHERE, GAMMA = 2.0, 0.3


def _mass():
    return 4.0 / 3.0 * math.pi * R_SPHERE ** 3


def _pulled_drag(L, F=1e-3):
    """xi(L) = F / (V - mean fluid velocity) of the sphere pulled along x
    with the compensating force on the fluid, deterministic FP64, same
    rates, friction and bead set as the thermal runs."""
    from paper_1604_01829_gb300 import lb
    h = lb.LB(L, L, L, precision=64, gamma_bead=GAMMA, compensate_force=1, **ZERO_RATES)
    m = _mass()
    h.lb_add_raspberry(Wl.sphere_raspberry(R_SPHERE), [L / 2 + 0.13, L / 2 - 0.21, L / 2 + 0.07], mass=m,
                       inertia=(0.4 * m * R_SPHERE ** 2,) * 3, F_ext=(F, 0, 0), fixed=2)
    h.lb_step(int(1.5 * L * L))
    rel = []
    for _ in range(10):
        h.lb_step(max(1, int(0.03 * L * L)))
        mass, p = h.lb_conservation()
        rel.append(h.lb_get_body(0)["V"][0] - p[0] / mass)
    h.close()
    return F / float(np.mean(rel))


def _diffusion(L, ninst, steps, every=10, seed=1604, beads=None, mass=None, inertia=None, random_q=False):
    """D(L) from the lab-frame MSD of ninst independent thermal boxes (one
    free raspberry each, the sphere unless beads / mass / inertia are given,
    FP32, batched handle, device recorder): the slope of the MSD, averaged
    over boxes and axes, fitted over lags from 6 to 18 relaxation times of
    the slowest shear mode (L^2 / (4 pi^2 nu)); and its standard error from
    the spread of the per-box slopes. random_q: seeded orientations."""
    from paper_1604_01829_gb300 import lb
    m = _mass() if mass is None else mass
    inertia = (0.4 * m * R_SPHERE ** 2,) * 3 if inertia is None else inertia
    params = [dict(nx=L, ny=L, nz=L, precision=32, kT=KT, seed=seed, instance=k, gamma_bead=GAMMA, **ZERO_RATES)
              for k in range(ninst)]
    B = lb.LBBatch(params)
    rng = np.random.default_rng(seed + L)
    beads = Wl.sphere_raspberry(R_SPHERE) if beads is None else beads
    for k in range(ninst):
        q = Wl.random_unit_quaternion(rng) if random_q else (1, 0, 0, 0)
        B.lb_batch_add_raspberry(k, beads, rng.uniform(0, L, 3), q, m, inertia)
    B.lb_batch_step(1000)                            # thermalise
    nrec = steps // every
    B.lb_batch_record_bodies(every, nrec)
    B.lb_batch_step(steps)
    traj = [B.lb_batch_get_trajectory(k, 0) for k in range(ninst)]
    X = np.stack([t[1] for t in traj])
    q = np.stack([t[2] for t in traj])
    B.close()
    assert X.shape == (ninst, nrec, 3)
    t_relax = L * L / (4 * math.pi ** 2 * ETA)
    lag1, lag2 = int(6 * t_relax / every), int(18 * t_relax / every)
    msd_all = lb.lb_msd_trajectory(X, q, lag2)

    def slope(cols, l1, l2, per):
        """per-box slope of the MSD (mean of cols) over lags l1..l2 records, divided by per"""
        m = msd_all[:, :, cols].mean(axis=2)
        lags = np.arange(l1, l2 + 1)
        A = np.stack([np.ones(len(lags)), per * every * lags], axis=1)
        pb = np.linalg.lstsq(A, m[:, lags - 1].T, rcond=None)[0][1]
        return float(pb.mean()), float(pb.std(ddof=1) / math.sqrt(ninst))

    out = {"t": slope([0, 1, 2], lag1, lag2, 2.0)}              # per lab axis: 2 D_t t
    # body-frame angles about chosen axes, lag window in steps
    out["r_cols"] = lambda cols, s1=100, s2=600: slope(cols, s1 // every, s2 // every, 2.0)
    # rotation decorrelates within tens of steps: lags of 100-600 steps; the
    # summed body-frame angles grow as 2 D_r t per axis, the angle of a
    # body-fixed vector as 4 D_r t (small angles: D_r t < 0.003 here)
    out["r_body"] = slope([7, 8, 9], 10, 60, 2.0)
    out["r_lab"] = slope([6], 10, 60, 4.0)
    return out


def test_einstein_relation_and_hasimoto_law_from_diffusion():
    Ls = [16, 24, 32]
    runs = {16: (128, 60000), 24: (96, 60000), 32: (64, 90000)}
    m = _mass()
    from paper_1604_01829_gb300 import drag as Dr
    D, sD, xi = [], [], []
    for L in Ls:
        res = _diffusion(L, *runs[L])
        d, s = res["t"]
        eps = m / L ** 3
        D.append(d * (1 + eps) ** 2)
        sD.append(s * (1 + eps) ** 2)
        xi.append(_pulled_drag(L))
        # rotation (Sec. 2.5, 2.7): D_r = kT / xi_r, xi_r of the same sphere
        # spinning in the same box
        xi_r = Dr.spin_drag(L, Wl.sphere_raspberry(R_SPHERE), params=ZERO_RATES, gamma=GAMMA)
        for key in ("r_body", "r_lab"):
            dr, sdr = res[key]
            ratio_r = dr * xi_r / KT
            print(f"L={L} {key}: D_r={dr:.4e} +- {sdr:.1e}, kT/xi_r={KT / xi_r:.4e}, ratio {ratio_r:.4f}")
            observe(f"einstein_rot_{key}_L{L}", abs(ratio_r - 1))
            assert sdr / dr < 0.02, (L, key, sdr / dr)
            assert abs(ratio_r - 1) < 0.06, (L, key, ratio_r)
    D, sD, xi = np.array(D), np.array(sD), np.array(xi)
    ratio = D * xi / KT
    print("D(L)", D, "+-", sD, "kT/xi(L)", KT / xi, "ratio", ratio)
    for L, r, s in zip(Ls, ratio, sD / D):
        observe(f"einstein_L{L}", abs(r - 1))
        assert s < 0.025, (L, s)
        assert abs(r - 1) < 0.06, (L, r, s)
    # Hasimoto: D(L) = D0 + kT H / L (+ O(L^-3)); slope from the diffusion data
    x = 1.0 / np.array(Ls, float)
    wts = 1.0 / sD
    A = np.stack([np.ones(3), x], axis=1) * wts[:, None]
    D0, slope = np.linalg.lstsq(A, D * wts, rcond=None)[0]
    x3 = np.stack([np.ones(3), x ** 3], axis=1)
    c = np.linalg.lstsq(x3, 1.0 / xi - HASIMOTO * x, rcond=None)[0]
    xi0 = 1.0 / c[0]
    print("D0", D0, "kT/xi0", KT / xi0, "slope/(kT H)", slope / (KT * HASIMOTO))
    observe("D0_vs_kT_over_xi0", abs(D0 * xi0 / KT - 1))
    observe("hasimoto_slope", abs(slope / (KT * HASIMOTO) - 1))
    assert abs(D0 * xi0 / KT - 1) < 0.06, (D0, KT / xi0)
    assert abs(slope / (KT * HASIMOTO) - 1) < 0.3, (slope, KT * HASIMOTO)


def test_ellipsoid_rotational_diffusion_projections_obey_einstein():
    """Body-frame rotational diffusion of a free 3:1 prolate raspberry
    (semi-axes 9, 3, 3; Sec. 2.5 and Sec. 2.7: the summed body-frame angular
    displacements grow as 2 D_r,k t about each body axis k), 128 thermal
    boxes of L = 40 with seeded orientations, 120,000 steps: D_r about the
    long axis and about the short axes each equal kT / xi_r of the same
    raspberry spinning about that axis in the same box (FP64 deterministic,
    drag.spin_drag) within 6 %. The lag window (500-2000 steps) starts
    beyond the viscous relaxation time a^2 / nu of the flow around the long
    semi-axis a = 9 (486 steps), which governs rotation about a short axis:
    fitted at 100-600 steps, as for the sphere, that axis reads 0.964.
    Measured on GB300: 1.012 +- 0.017 (long axis) and 0.989 +- 0.012 (short
    axes); D_r,par / D_r,perp = 3.26 against the spin drags' 3.19 in the same
    box and Perrin's spheroid value J / I = 3.13 (the spin-drag ratio itself
    is held to Perrin in test_gpu_physics.py)."""
    from paper_1604_01829_gb300 import drag as Dr
    from oracle import factors as Fc
    L = 40
    beads = Wl.ellipsoid_raspberry(9.0, 3.0, 3.0)
    m = 4.0 / 3.0 * math.pi * 81.0
    inertia = Wl.solid_ellipsoid_inertia(m, 9.0, 3.0, 3.0)
    res = _diffusion(L, 128, 120000, every=20, beads=beads, mass=m, inertia=inertia, random_q=True)
    xi = {"par": Dr.spin_drag(L, beads, axis=0, params=ZERO_RATES, gamma=GAMMA),
          "perp": Dr.spin_drag(L, beads, axis=1, params=ZERO_RATES, gamma=GAMMA)}
    # per body axis: column 7 is the long axis, 8 and 9 the short ones
    D = {"par": res["r_cols"]([7], 500, 2000), "perp": res["r_cols"]([8, 9], 500, 2000)}
    for name in ("par", "perp"):
        d, sd = D[name]
        ratio = d * xi[name] / KT
        print(f"{name}: D_r={d:.4e} +- {sd:.1e}, kT/xi_r={KT / xi[name]:.4e}, ratio {ratio:.4f}")
        observe(f"ellipsoid_rot_{name}", abs(ratio - 1))
        assert sd / d < 0.025, (name, sd / d)
        assert abs(ratio - 1) < 0.06, (name, ratio)
    I, J = Fc.perrin_rotation(3.0)
    print(f"D_r,par / D_r,perp = {D['par'][0] / D['perp'][0]:.4f}, xi_perp / xi_par = {xi['perp'] / xi['par']:.4f}, "
          f"Perrin J/I = {J / I:.4f}")
