"""Seeded synthetic inputs shaped like the paper's workloads.

This module only generates inputs (bead sets, body placements, lattice sizes,
initial perturbations). It holds none of the LB or coupling arithmetic, so
both the CUDA path and the CPU oracle may use it.

Raspberry bead sets follow Sec. 2.1 of Ustach & Faller (arXiv:1604.01829):
an outer hydrodynamic shell at the design surface, an inner shell 0.5 length
units further in, and interior filling beads. The paper relaxes beads by a
long MD run (SI Sec. "Details for ellipsoidal raspberry construction"); here
the shells are deterministic stand-ins at its density of one bead per unit
area: golden-angle (Fibonacci) points on spheres, and area-uniform points
thinned by farthest-point selection on ellipsoids.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GOLDEN = math.pi * (3.0 - math.sqrt(5.0))


def fibonacci_sphere(n: int, radius: float) -> np.ndarray:
    """n golden-angle points on a sphere of the given radius."""
    if n <= 0:
        return np.zeros((0, 3))
    if n == 1:
        return np.zeros((1, 3))
    k = np.arange(n) + 0.5
    z = 1.0 - 2.0 * k / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = GOLDEN * np.arange(n)
    return radius * np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def sphere_raspberry(R: float, density: float = 1.0, inner_offset: float = 0.5,
                     fill: bool = True) -> np.ndarray:
    """Filled two-layer spherical raspberry (Sec. 2.1): shells at R, R-0.5,
    then interior shells every unit down to the centre."""
    radii = [R]
    if inner_offset > 0 and R - inner_offset > 0.25:
        radii.append(R - inner_offset)
    if fill:
        r = R - inner_offset - 1.0
        while r > 0.25:
            radii.append(r)
            r -= 1.0
    pts = [fibonacci_sphere(max(1, int(round(4.0 * math.pi * r * r * density))), r) for r in radii]
    if fill:
        pts.append(np.zeros((1, 3)))
    return np.concatenate(pts, axis=0)


def ellipsoid_area(a: float, b: float, c: float, n: int = 256) -> float:
    """Surface area of an ellipsoid by midpoint quadrature in (theta, phi)."""
    th = (np.arange(n) + 0.5) * math.pi / n
    ph = (np.arange(2 * n) + 0.5) * math.pi / n
    T, P = np.meshgrid(th, ph, indexing="ij")
    st, ct, sp, cp = np.sin(T), np.cos(T), np.sin(P), np.cos(P)
    # |d r/d theta x d r/d phi| for r = (a st cp, b st sp, c ct)
    nx = b * c * st * st * cp
    ny = a * c * st * st * sp
    nz = a * b * st * ct
    dA = np.sqrt(nx * nx + ny * ny + nz * nz)
    return float(dA.sum() * (math.pi / n) * (math.pi / n))


def _ellipsoid_shell(a, b, c, n, rng):
    """n roughly evenly spread points on the ellipsoid (x/a)^2+(y/b)^2+(z/c)^2=1."""
    if n <= 0:
        return np.zeros((0, 3))
    m = max(10 * n, 200)
    # area-uniform candidates: map sphere points, accept by the local area ratio
    cand = []
    gmax = max(b * c, a * c, a * b)
    while sum(len(x) for x in cand) < m:
        v = rng.standard_normal((2 * m, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        g = np.sqrt((b * c * v[:, 0]) ** 2 + (a * c * v[:, 1]) ** 2 + (a * b * v[:, 2]) ** 2)
        keep = rng.random(2 * m) < g / gmax
        cand.append(v[keep] * np.array([a, b, c]))
    P = np.concatenate(cand)[:m]
    # farthest-point selection
    sel = [0]
    d = np.linalg.norm(P - P[0], axis=1)
    for _ in range(1, n):
        k = int(np.argmax(d))
        sel.append(k)
        d = np.minimum(d, np.linalg.norm(P - P[k], axis=1))
    return P[sel]


def ellipsoid_raspberry(a: float, b: float, c: float, density: float = 1.0,
                        inner_offset: float = 0.5, fill: bool = True,
                        seed: int = 0) -> np.ndarray:
    """Filled two-layer ellipsoidal raspberry with semi-axes (a, b, c) along the
    body x, y, z axes (Sec. 2.1: inner shell (a-0.5, b-0.5, c-0.5))."""
    rng = np.random.default_rng(seed)
    pts = []
    for (sa, sb, sc), n in raspberry_shells(a, b, c, density, inner_offset, fill):
        pts.append(_ellipsoid_shell(sa, sb, sc, n, rng))
    if fill:
        # a line of core beads along the longest axis, unit spacing
        ax = int(np.argmax([a, b, c]))
        reach = max(a, b, c) - (min(a, b, c))
        m = int(math.floor(reach))
        core = np.zeros((2 * m + 1, 3))
        core[:, ax] = np.arange(-m, m + 1, dtype=np.float64)
        pts.append(core)
    return np.concatenate(pts, axis=0)


def raspberry_shells(a: float, b: float, c: float, density: float = 1.0, inner_offset: float = 0.5,
                     fill: bool = True) -> list:
    """(semi-axes, bead count) of every shell of a filled two-layer raspberry
    (Sec. 2.1): the outer shell, the inner shell inner_offset further in, fill
    shells every unit further in; round(area x density) beads each."""
    shells = [(a, b, c)]
    if inner_offset > 0 and min(a, b, c) - inner_offset > 0.25:
        shells.append((a - inner_offset, b - inner_offset, c - inner_offset))
    if fill:
        k = inner_offset + 1.0
        while min(a, b, c) - k > 0.25:
            shells.append((a - k, b - k, c - k))
            k += 1.0
    return [((sa, sb, sc), max(1, int(round(ellipsoid_area(sa, sb, sc) * density)))) for (sa, sb, sc) in shells]


def random_shell_start(a: float, b: float, c: float, n: int, seed: int, spread: float = 0.0) -> np.ndarray:
    """Seeded starting positions for a shell relaxation: n uniformly random
    directions u mapped to (a u_x, b u_y, c u_z) on the ellipsoid (not
    area-uniform: the relaxation evens them out), each scaled by
    1 + spread U(-1, 1)."""
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    scale = 1.0 + spread * rng.uniform(-1.0, 1.0, size=(n, 1))
    return u * np.array([a, b, c]) * scale


def spread_shell_start(a: float, b: float, c: float, n: int, seed: int, jitter: float = 0.0) -> np.ndarray:
    """Seeded, roughly evenly spread starting positions for a shell
    relaxation (area-uniform candidates thinned by farthest-point selection,
    so no two beads start very close), each scaled radially by
    1 + jitter U(-1, 1)."""
    rng = np.random.default_rng(seed)
    P = _ellipsoid_shell(a, b, c, n, rng)
    return P * (1.0 + jitter * rng.uniform(-1.0, 1.0, size=(n, 1)))


def solid_ellipsoid_inertia(mass: float, a: float, b: float, c: float) -> np.ndarray:
    """Principal moments of a uniform solid ellipsoid."""
    return mass * np.array([b * b + c * c, a * a + c * c, a * a + b * b]) / 5.0


def random_unit_quaternion(rng) -> np.ndarray:
    """Uniformly distributed rotation (normalised 4-D Gaussian)."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    if q[0] < 0:
        q = -q
    return q


@dataclass
class Body:
    beads: np.ndarray
    X: np.ndarray
    q: np.ndarray
    mass: float
    inertia: np.ndarray
    F_ext: np.ndarray = field(default_factory=lambda: np.zeros(3))
    T_ext: np.ndarray = field(default_factory=lambda: np.zeros(3))
    fixed: int = 0          # 0 free, 1 held, 2 translation only
    axes: tuple | None = None  # semi-axes (a, b, c) of an ellipsoidal raspberry


@dataclass
class Workload:
    """One lattice instance with its parameters and bodies (lattice units)."""
    name: str
    nx: int
    ny: int
    nz: int
    params: dict
    bodies: list
    pore: tuple | None = None   # (radius, axis)
    steps: int = 1

    @property
    def nodes(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def nbeads(self) -> int:
        return int(sum(len(b.beads) for b in self.bodies))


def mrt_rates(nu: float, bulk: float | None = None, odd: float = 0.0, even: float = 0.0) -> dict:
    """Relaxation parameters for kinematic viscosity nu: gamma_shear = (6nu-1)/(6nu+1)."""
    gs = (6.0 * nu - 1.0) / (6.0 * nu + 1.0)
    return dict(gamma_shear=gs, gamma_bulk=gs if bulk is None else bulk,
                gamma_odd=odd, gamma_even=even)


# Unit system of Sec. 2.3: M0 = 100 amu, sigma = 1 nm, epsilon = kB 298 K,
# t0 = 6.352 ps; water density 6.004 M0/sigma^3; LB step 0.02 t0 on a grid of
# 1 sigma. One lattice mass unit is rho a^3 = 6.004 M0.
RHO_PAPER = 6.004        # M0 / sigma^3
DT_LB_PAPER = 0.02       # t0
A_GRID_PAPER = 1.0       # sigma


AMU_KG = 1.66053906660e-27
KB_J_PER_K = 1.380649e-23
M0_KG = 100.0 * AMU_KG
SIGMA_M = 1e-9
EPS_J = KB_J_PER_K * 298.0


def t0_seconds() -> float:
    """Time unit t0 = sigma sqrt(M0 / epsilon) of Sec. 2.3."""
    return SIGMA_M * math.sqrt(M0_KG / EPS_J)


def density_to_paper_units(rho_kg_m3: float) -> float:
    """kg/m^3 -> M0/sigma^3."""
    return rho_kg_m3 * SIGMA_M ** 3 / M0_KG


def kinematic_viscosity_to_paper_units(nu_m2_s: float) -> float:
    """m^2/s -> sigma^2/t0."""
    return nu_m2_s * t0_seconds() / SIGMA_M ** 2


def friction_to_si(xi_paper: float) -> float:
    """M0/t0 -> kg/s."""
    return xi_paper * M0_KG / t0_seconds()


def paper_gamma_to_lattice(xi_bead: float) -> float:
    """Bead friction xi_bead in M0/t0 (Sec. 2.3, Sec. 3.1) -> lattice units
    (mass rho a^3, time dt_LB): xi dt_LB / (rho a^3)."""
    return xi_bead * DT_LB_PAPER / (RHO_PAPER * A_GRID_PAPER ** 3)


# Viscosity of the paper's scaled runs: nu = 0.8 sigma^2/t0 with an LB step of
# 0.02 t0 on a 1 nm grid (Sec. 2.3) -> 0.016 in lattice units.
NU_PAPER = 0.8 * 0.02


def sphere_32(seed: int = 1605, gamma: float = 20.0, R: float = 3.0, L: int = 32) -> Workload:
    """32^3 periodic FP64 BGK tau = 1, one filled sphere R = 3 at the box centre
    plus a seeded sub-cell offset, body force 1e-4 along z on the colloid."""
    rng = np.random.default_rng(seed)
    beads = sphere_raspberry(R)
    X = np.array([L / 2.0] * 3) + rng.random(3)
    mass = (4.0 / 3.0) * math.pi * R ** 3
    inertia = np.full(3, 0.4 * mass * R * R)
    b = Body(beads, X, np.array([1.0, 0, 0, 0]), mass, inertia, F_ext=np.array([0, 0, 1e-4]))
    params = dict(collision=0, tau=1.0, rho0=1.0, kT=0.0, gamma_bead=paper_gamma_to_lattice(gamma), seed=seed,
                  compensate_force=1, precision=64)
    return Workload("sphere_32^3_bgk_fp64", L, L, L, params, [b], None, 200)


def pore_48(offset_frac: float = 0.0, precision: int = 32, kT: float = 1e-4, seed: int = 1606,
            gamma: float = 20.0) -> Workload:
    """48x48x96 cylindrical pore R = 20 along z (axis at the box centre),
    MRT nu = 0.016 with fluctuations, sphere R = 4 at radial offset
    offset_frac * R_pore."""
    rng = np.random.default_rng(seed)
    beads = sphere_raspberry(4.0)
    X = np.array([24.0 + offset_frac * 20.0, 24.0, 48.0]) + 0.1 * rng.random(3)
    mass = (4.0 / 3.0) * math.pi * 4.0 ** 3
    b = Body(beads, X, np.array([1.0, 0, 0, 0]), mass, np.full(3, 0.4 * mass * 16.0))
    params = dict(collision=1, rho0=1.0, kT=kT, gamma_bead=paper_gamma_to_lattice(gamma), seed=2,
                  precision=precision, compensate_force=0, **mrt_rates(NU_PAPER))
    return Workload(f"pore_48x48x96_R20_off{offset_frac:.1f}", 48, 48, 96, params, [b], (20.0, 2), 5000)


def ellipsoids_256(n_bodies: int = 64, L: int = 256, seed: int = 1607, kT: float = 1e-4,
                   gamma: float = 20.0, precision: int = 32) -> Workload:
    """256^3 periodic box, FP32 MRT with fluctuations, n prolate ellipsoidal
    raspberries (aspect 2-4, semi-axes 2-8) at seeded non-overlapping positions
    and uniformly random orientations."""
    rng = np.random.default_rng(seed)
    bodies = []
    placed = []
    tries = 0
    while len(bodies) < n_bodies:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place the bodies")
        aspect = rng.uniform(2.0, 4.0)
        b_ax = rng.uniform(2.0, min(4.0, 8.0 / aspect))
        a_ax = aspect * b_ax
        X = rng.random(3) * L
        ok = True
        for (Y, ay) in placed:
            d = np.abs(X - Y)
            d = np.minimum(d, L - d)
            if np.linalg.norm(d) <= a_ax + ay + 1.0:
                ok = False
                break
        if not ok:
            continue
        placed.append((X, a_ax))
        beads = ellipsoid_raspberry(a_ax, b_ax, b_ax, seed=int(rng.integers(1 << 30)))
        mass = (4.0 / 3.0) * math.pi * a_ax * b_ax * b_ax
        bodies.append(Body(beads, X, random_unit_quaternion(rng), mass,
                           solid_ellipsoid_inertia(mass, a_ax, b_ax, b_ax), axes=(a_ax, b_ax, b_ax)))
    params = dict(collision=1, rho0=1.0, kT=kT, gamma_bead=paper_gamma_to_lattice(gamma), seed=seed, precision=precision,
                  compensate_force=0, **mrt_rates(NU_PAPER))
    return Workload(f"ellipsoids{n_bodies}_{L}^3_mrt_kT", L, L, L, params, bodies, None, 2000)


def ellipsoid_adjoint_96(seed: int = 1609, precision: int = 32) -> Workload:
    """96^3 periodic, deterministic, one prolate ellipsoid aspect 1:3 (b = 5,
    a = 15) under constant force along its long axis."""
    beads = ellipsoid_raspberry(15.0, 5.0, 5.0, seed=seed)
    mass = (4.0 / 3.0) * math.pi * 15 * 25
    # pulled along its long (body x) axis with the orientation held
    b = Body(beads, np.array([48.0, 48.0, 48.0]), np.array([1.0, 0, 0, 0]), mass,
             solid_ellipsoid_inertia(mass, 15, 5, 5), F_ext=np.array([1e-3, 0, 0]), fixed=2)
    params = dict(collision=1, rho0=1.0, kT=0.0, gamma_bead=paper_gamma_to_lattice(20.0), seed=seed, precision=precision,
                  compensate_force=1, **mrt_rates(NU_PAPER))
    return Workload("ellipsoid_adjoint_96^3", 96, 96, 96, params, [b], None, 3000)


def batched_instances(n: int = 256, seed: int = 1608, precision: int = 32) -> list:
    """n independent instances of uneven size: half cubic periodic boxes with
    edge 24..64, half cylindrical pores with radius 8..28 (L_xy = 2R + 4,
    L_z = 48), each holding one sphere (R 2..5) or prolate ellipsoid (aspect
    1.5..3) at a seeded offset. Deterministic MRT at nu = 0.016."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        if k % 2 == 0:
            L = int(rng.integers(24, 65))
            dims = (L, L, L)
            pore = None
        else:
            R = int(rng.integers(8, 29))
            Lxy = 2 * R + 4
            dims = (Lxy, Lxy, 48)
            pore = (float(R), 2)
        size = rng.uniform(2.0, 5.0)
        if pore is not None:
            size = min(size, pore[0] - 3.0)
        if rng.random() < 0.5:
            beads = sphere_raspberry(size)
            mass = (4.0 / 3.0) * math.pi * size ** 3
            inertia = np.full(3, 0.4 * mass * size * size)
        else:
            asp = rng.uniform(1.5, 3.0)
            bb = size / asp ** (1.0 / 3.0)
            aa = asp * bb
            if pore is not None:
                aa = min(aa, pore[0] - 2.0)
            beads = ellipsoid_raspberry(aa, bb, bb, seed=int(rng.integers(1 << 30)))
            mass = (4.0 / 3.0) * math.pi * aa * bb * bb
            inertia = solid_ellipsoid_inertia(mass, aa, bb, bb)
        centre = np.array(dims, dtype=np.float64) / 2.0
        off = rng.uniform(-1.0, 1.0, 3)
        X = centre + off
        q = random_unit_quaternion(rng) if pore is None else np.array([1.0, 0, 0, 0])
        body = Body(beads, X, q, mass, inertia, F_ext=np.array([0.0, 0.0, 1e-4]))
        params = dict(collision=1, rho0=1.0, kT=0.0, gamma_bead=paper_gamma_to_lattice(20.0), seed=seed + k,
                      precision=precision, compensate_force=1 if pore is None else 0,
                      **mrt_rates(NU_PAPER))
        out.append(Workload(f"instance{k}", *dims, params, [body], pore, 1000))
    return out
