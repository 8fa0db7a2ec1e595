"""Pins of the FP64 CPU oracle against what the physics and the mathematics
fix, independently of the oracle's own formulas (CPU only).

Each test names the property and the passage of Ustach & Faller
(arXiv:1604.01829) or the textbook fact it rests on. Together they are
chosen so that a dropped term, a wrong sign, a wrong index or a transposed
operand anywhere in the oracle fails at least one of them.
"""
import ctypes
import math

import numpy as np
import pytest

from oracle import oracle as O

NQ = 19


# ----------------------------------------------------------------- lattice tables

def test_d3q19_isotropy_and_opposites():
    """Sec. 1.1 lattice (read as D3Q19): weights sum to one, odd moments
    vanish, second moment c_s^2 I with c_s^2 = 1/3, fourth moment isotropic
    (c_s^4 (dd + dd + dd)); opposite links are negatives."""
    c, w, opp = O.lattice()
    assert c.shape == (19, 3)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.abs(np.einsum("i,ia->a", w, c)).max() < 1e-16
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(3) / 3.0, atol=1e-16)
    assert np.abs(np.einsum("i,ia,ib,ic->abc", w, c, c, c)).max() < 1e-16
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c), iso, atol=1e-16)
    assert all((c[opp[i]] == -c[i]).all() for i in range(19))
    assert len({tuple(v) for v in c}) == 19


def test_mrt_basis_orthogonal_with_hand_derived_norms():
    """The moment basis is orthogonal under sum_i w_i e_k e_l, and the norms
    b_k match a hand derivation from the polynomial values on the 19 links."""
    c, w, _ = O.lattice()
    M, Minv, b = O.mrt_tables()
    G = np.einsum("ki,i,li->kl", M, w, M)
    assert np.abs(G - np.diag(np.diag(G))).max() < 1e-14
    hand = np.array([1, 1 / 3, 1 / 3, 1 / 3, 2 / 3, 4 / 3, 4 / 9, 1 / 9, 1 / 9, 1 / 9,
                     2 / 3, 2 / 3, 2 / 3, 2 / 9, 2 / 9, 2 / 9, 2, 4 / 3, 4 / 9])
    assert np.allclose(np.diag(G), hand, atol=1e-14)
    assert np.allclose(b, hand, atol=1e-14)
    assert np.linalg.matrix_rank(M) == 19
    assert np.allclose(Minv @ M, np.eye(19), atol=1e-13)
    # the inverse of an orthogonal basis is w_i e_k(c_i) / b_k
    assert np.allclose(Minv, (w[:, None] * M.T) / hand[None, :], atol=1e-13)
    # moments 1..3 are the momentum, 0 the density
    assert np.allclose(M[0], 1.0) and np.allclose(M[1:4], c.T)


def test_equilibrium_moments_exact():
    """Second-order equilibrium: density, momentum and momentum flux
    rho/3 I + rho u u are exact on D3Q19, and all ghost moments vanish."""
    c, w, _ = O.lattice()
    M, _, _ = O.mrt_tables()
    rng = np.random.default_rng(3)
    for _ in range(5):
        rho = 1.0 + 0.1 * rng.standard_normal()
        u = 0.05 * rng.standard_normal(3)
        feq = O.equilibrium(rho, u)
        assert abs(feq.sum() - rho) < 1e-14
        assert np.allclose(feq @ c, rho * u, atol=1e-15)
        Pi = np.einsum("i,ia,ib->ab", feq, c, c)
        assert np.allclose(Pi, rho / 3 * np.eye(3) + rho * np.outer(u, u), atol=1e-15)
        assert np.abs((M @ feq)[10:]).max() < 1e-15


# ------------------------------------------------------------------- collision

def _params(**kw):
    return O.make_params(4, 4, 4, **kw)


@pytest.mark.parametrize("kind", ["bgk", "mrt", "mrt_noise"])
def test_collision_conserves_mass_and_adds_force(kind):
    """Collision keeps the density and adds exactly F to the momentum (Guo
    forcing), with or without thermal noise (noise lives on the 15
    non-conserved modes only)."""
    c, _, _ = O.lattice()
    rng = np.random.default_rng(11)
    if kind == "bgk":
        p = _params(collision=0, tau=0.7)
    else:
        p = _params(collision=1, gamma_shear=-0.4, gamma_bulk=0.2, gamma_odd=0.3, gamma_even=-0.1,
                    kT=1e-3 if kind == "mrt_noise" else 0.0, seed=99)
    for t in range(5):
        f = O.equilibrium(1.0, [0.01, -0.02, 0.03]) * (1 + 0.05 * rng.standard_normal(19))
        F = 1e-3 * rng.standard_normal(3)
        fo = O.collide_node(p, f, F, node_id=t, step=7)
        assert abs(fo.sum() - f.sum()) < 1e-15
        assert np.allclose(fo @ c, f @ c + F, atol=1e-16)


def test_bgk_equals_mrt_with_equal_rates():
    """BGK (population space, one time scale) and MRT (explicit 19x19 moment
    transform) are different code paths; with every non-conserved rate set to
    1 - 1/tau they must agree to round-off, forcing included."""
    rng = np.random.default_rng(5)
    for tau in (0.55, 0.8, 1.0, 1.7):
        g = 1.0 - 1.0 / tau
        pb = _params(collision=0, tau=tau)
        pm = _params(collision=1, gamma_shear=g, gamma_bulk=g, gamma_odd=g, gamma_even=g)
        for _ in range(4):
            f = O.equilibrium(1.0, 0.03 * rng.standard_normal(3)) * (1 + 0.1 * rng.standard_normal(19))
            F = 1e-3 * rng.standard_normal(3)
            assert np.allclose(O.collide_node(pb, f, F), O.collide_node(pm, f, F), atol=1e-15, rtol=0)


def test_mrt_relaxes_each_mode_at_its_rate():
    """With F = 0 and no noise, a perturbation along basis vector k decays
    by exactly its rate g_k (non-equilibrium moment scaling)."""
    M, Minv, _ = O.mrt_tables()
    rates = dict(gamma_shear=-0.3, gamma_bulk=0.45, gamma_odd=0.15, gamma_even=-0.6)
    p = _params(collision=1, **rates)
    gk = [0, 0, 0, 0, 0.45] + [-0.3] * 5 + [0.15] * 6 + [-0.6] * 3
    feq = O.equilibrium(1.0, [0, 0, 0])
    for k in range(4, 19):
        e = np.zeros(19)
        e[k] = 1e-4
        f = feq + Minv @ e
        m_out = M @ O.collide_node(p, f, np.zeros(3))
        # at u = 0 the perturbation moves no conserved quantity, so m_eq is unchanged
        assert abs(m_out[k] - gk[k] * 1e-4) < 1e-15, k
        others = np.delete(m_out - M @ feq, [k])
        assert np.abs(others).max() < 1e-15


# ---------------------------------------------------------------------- Philox

def _curand():
    for name in ("libcurand.so", "libcurand.so.10", "/usr/local/cuda/lib64/libcurand.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


def test_philox_matches_curand_host_generator():
    """Philox4x32-10 written from Salmon et al. (SC'11) reproduces the
    cuRAND library's own host-side Philox4x32-10 stream: output block b of
    seed s is the bijection applied to counter (0, 0, b, 0) under key
    (s_lo, s_hi)."""
    cr = _curand()
    if cr is None:
        pytest.skip("libcurand not available")
    for seed in (0, 1, 0x0123456789ABCDEF, 2 ** 32, 2 ** 64 - 1):
        gen = ctypes.c_void_p()
        assert cr.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
        try:
            assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
            n = 64
            buf = (ctypes.c_uint32 * n)()
            assert cr.curandGenerate(gen, buf, n) == 0
        finally:
            cr.curandDestroyGenerator(gen)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for blk in range(n // 4):
            assert O.philox([0, 0, blk, 0], key) == list(buf[4 * blk:4 * blk + 4]), (seed, blk)


def test_unit_uniform_variates():
    """Noise variates: uniform on (-sqrt3, sqrt3), zero mean, unit variance,
    no lag correlation across consecutive counters; extremes map exactly."""
    assert abs(O.unit_uniform(0) - math.sqrt(12) * (0.5 / 2 ** 32 - 0.5)) < 1e-15
    assert abs(O.unit_uniform(2 ** 32 - 1) + O.unit_uniform(0)) < 1e-15
    xs = []
    for i in range(20000):
        xs.extend(O.philox([i, 3, 1, 0], [7, 9]))
    v = np.array([O.unit_uniform(x) for x in xs])
    assert abs(v.mean()) < 0.01
    assert abs(v.var() - 1.0) < 0.01
    assert np.abs(v).max() < math.sqrt(3)
    hist, _ = np.histogram(v, bins=20, range=(-math.sqrt(3), math.sqrt(3)))
    exp = len(v) / 20
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < 45  # 19 dof, p ~ 1e-3
    a = v.reshape(-1, 4)
    assert abs(np.corrcoef(a[:-1, 0], a[1:, 0])[0, 1]) < 0.03
    assert abs(np.corrcoef(a[:, 0], a[:, 1])[0, 1]) < 0.03


def test_unit_uniform16_variates_exact_moments():
    """Fluid-noise variates from 16 bits: over all 65536 values the mean is 0
    and the variance 1 - 2^-32 exactly (discrete uniform on a centred grid),
    the extremes are mirror images, and the two halves of one Philox word
    are uncorrelated."""
    assert abs(O.unit_uniform16(0) - math.sqrt(12) * (0.5 / 65536 - 0.5)) < 1e-15
    assert abs(O.unit_uniform16(65535) + O.unit_uniform16(0)) < 1e-15
    v = np.array([O.unit_uniform16(h) for h in range(65536)])
    assert abs(v.sum()) < 1e-9
    assert abs((v * v).mean() - (1.0 - 2.0 ** -32)) < 1e-12
    assert np.all(np.diff(v) > 0)
    words = []
    for i in range(20000):
        words.extend(O.philox([i, 5, 0, 1], [3, 8]))
    hi = np.array([O.unit_uniform16(w >> 16) for w in words])
    lo = np.array([O.unit_uniform16(w & 0xFFFF) for w in words])
    assert abs(np.corrcoef(hi, lo)[0, 1]) < 0.02
    assert abs(hi.var() - 1.0) < 0.02 and abs(lo.var() - 1.0) < 0.02


# ------------------------------------------------------------ fluid dynamics pins

def _shear_wave_rate(nu_expected, **kw):
    ny = 32
    L = O.OracleLB(2, ny, 2, **kw)
    k = 2 * math.pi / ny
    A = 1e-4
    f = np.zeros((19, L.N))
    for idx in range(L.N):
        y = (idx // 2) % ny
        f[:, idx] = O.equilibrium(1.0, [A * math.sin(k * (y + 0.5)), 0, 0])
    L.set_populations(f)

    def amp():
        _, u = L.node_velocity()
        ys = (np.arange(L.N) // 2) % ny
        return 2 * np.mean(u[:, 0] * np.sin(k * (ys + 0.5)))

    L.step(40)
    a0 = amp()
    L.step(200)
    a1 = amp()
    rate = -math.log(a1 / a0) / 200
    return rate, nu_expected * k * k


@pytest.mark.parametrize("case", ["bgk", "mrt"])
def test_shear_wave_decays_at_nu_k2(case):
    """Sec. 1.1: LB recovers Navier-Stokes; a transverse shear wave decays at
    rate nu k^2 with nu = (tau - 1/2)/3, i.e. (1 + g_s)/(6 (1 - g_s))."""
    if case == "bgk":
        tau = 0.8
        rate, exp = _shear_wave_rate((tau - 0.5) / 3, collision=0, tau=tau)
    else:
        gs = -0.5
        rate, exp = _shear_wave_rate((1 + gs) / (6 * (1 - gs)), collision=1, gamma_shear=gs,
                                     gamma_bulk=0.3, gamma_odd=0.2, gamma_even=0.1)
    assert abs(rate / exp - 1) < 0.01


def _channel_mask(nx, ny, nz):
    mask = np.zeros((nz, ny, nx), np.uint8)
    mask[:, 0, :] = 1
    mask[:, ny - 1, :] = 1
    return mask.reshape(-1)


def test_plane_poiseuille_exact_with_halfway_bounce_back():
    """Sec. 1.1 bounce-back at boundary nodes: with two-relaxation-time
    rates of magic product (tau+ - 1/2)(tau- - 1/2) = 3/16 the halfway
    bounce-back channel reproduces the parabola u = g/(2 nu) (y - y0)(y1 - y)
    with walls half-way between fluid and wall nodes, to round-off; the
    amplitude pins the force term and the viscosity."""
    nx, ny, nz = 2, 10, 2
    g = 1e-5
    gs = -1.0 / 7.0           # tau+ = 7/8, nu = 1/8
    L = O.OracleLB(nx, ny, nz, collision=1, gamma_shear=gs, gamma_bulk=gs, gamma_odd=0.0,
                   gamma_even=gs, body_force=(g, 0, 0))
    L.set_mask(_channel_mask(nx, ny, nz))
    L.step(6000)
    _, u = L.node_velocity()
    u = u.reshape(nz, ny, nx, 3)
    yc = np.arange(ny) + 0.5
    exact = g / (2 * 0.125) * (yc - 1.0) * (ny - 1.0 - yc)
    assert np.abs(u[0, 1:-1, 0, 0] - exact[1:-1]).max() < 1e-9 * exact.max()
    assert np.abs(u[:, 1:-1, :, 1:]).max() < 1e-14
    mass, _ = L.conservation()
    assert abs(mass - nx * nz * (ny - 2)) < 1e-10


def test_cylinder_poiseuille_flux():
    """Sec. 2.3 pore: halfway bounce-back on a staircase cylinder carries the
    Hagen-Poiseuille flux pi R^4 g / (8 nu rho) of the radius that has the
    staircase's cross-section, to within the staircase error (a few percent
    at R = 8-10)."""
    g = 1e-6
    tau = 1.0
    nu = (tau - 0.5) / 3
    for R in (8.0, 10.0):
        n = int(2 * R + 4)
        L = O.OracleLB(n, n, 2, collision=0, tau=tau, body_force=(0, 0, g))
        L.set_pore(R, axis=2)
        L.step(int(6 * R * R / nu))
        _, u = L.node_velocity()
        fluid = L.mask == 0
        area = fluid.sum() / 2
        # the fluid cross-section approximates pi R^2
        assert abs(area / (math.pi * R * R) - 1) < 0.05
        flux = u[fluid, 2].sum() / 2   # per z-layer
        R_eff = math.sqrt(area / math.pi)
        exact = math.pi * R_eff ** 4 * g / (8 * nu)
        assert abs(flux / exact - 1) < 0.04, R


def test_pore_mask_geometry():
    """Sec. 2.3: boundary nodes half a grid spacing outside the wall; along a
    lattice axis the first wall node centre sits at R + 1/2."""
    n = 48
    m = O.pore_mask(n, n, 4, 20.0, 2).reshape(4, n, n)
    row = m[0, n // 2, :]      # y centre 24.5 -> distance 0.5 in y
    xs = np.arange(n) + 0.5 - n / 2
    # centres with sqrt(dx^2 + 0.25) >= 20 are walls
    assert (row == (xs * xs + 0.25 >= 400)).all()
    assert (m[0] == m[3]).all()
    # axis along x: the mask depends on (y, z) only
    mx = O.pore_mask(6, 10, 10, 3.0, 0).reshape(10, 10, 6)
    assert (mx == mx[:, :, :1]).all()


def test_equipartition_of_fluctuating_mrt():
    """Sec. 1.1 stochastic LB: with noise on the non-conserved modes the
    node velocity variance approaches kT/rho0 per component and each ghost
    mode's variance approaches 3 rho kT b_k."""
    kT = 1e-4
    L = O.OracleLB(8, 8, 8, collision=1, gamma_shear=-0.5, gamma_bulk=-0.2, gamma_odd=0.0,
                   gamma_even=0.0, kT=kT, seed=1234)
    L.step(100)
    us = []
    for _ in range(60):
        L.step(5)
        _, u = L.node_velocity(with_force=False)
        us.append(u - u.mean(axis=0))
    u = np.concatenate(us)
    var = (u * u).mean(axis=0)
    # 512 nodes with zero total momentum: one degree of freedom per component is removed
    assert np.allclose(var / (kT * (1 - 1 / 512)), 1.0, atol=0.03)
    M, _, b = O.mrt_tables()
    m = M @ L.populations()
    ghost_var = m[16:].var(axis=1)
    assert np.allclose(ghost_var / (3 * kT * b[16:]), 1.0, atol=0.2)


# -------------------------------------------------------------- rigid body pins

def test_rotation_matrix_and_quaternion_product():
    """Rotation by a unit quaternion is orthogonal with det 1 (the SI matrix
    has a sign typo in its (3,1) entry; the Hamilton form is used) and the
    quaternion product composes rotations."""
    rng = np.random.default_rng(2)
    for _ in range(10):
        q1 = rng.standard_normal(4); q1 /= np.linalg.norm(q1)
        q2 = rng.standard_normal(4); q2 /= np.linalg.norm(q2)
        R1, R2 = O.rotation(q1), O.rotation(q2)
        assert np.allclose(R1.T @ R1, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R1) - 1) < 1e-14
        assert np.allclose(O.rotation(O.quat_mul(q1, q2)), R1 @ R2, atol=1e-14)
    # 90 degrees about z maps x to y
    s = math.sqrt(0.5)
    assert np.allclose(O.rotation([s, 0, 0, s]) @ [1, 0, 0], [0, 1, 0], atol=1e-15)


def _free_top_drift(scale):
    L = O.OracleLB(4, 4, 4, collision=0, tau=1.0, gamma_bead=0.0)
    I = np.array([1.0, 2.0, 3.0])
    w0 = scale * np.array([0.02, 0.01, -0.015])
    L.add_raspberry(np.zeros((1, 3)), [2, 2, 2], [1, 0, 0, 0], 1.0, I, w=w0)
    B = L.body(0)
    L0 = O.rotation(B["q"]) @ (I * B["w"])
    E0 = 0.5 * (I * w0 * w0).sum()
    worst = 0.0
    for _ in range(10):
        L.step(int(100 / scale))
        B = L.body(0)
        Lt = O.rotation(B["q"]) @ (I * B["w"])
        worst = max(worst, np.linalg.norm(Lt - L0) / np.linalg.norm(L0))
        assert abs(np.linalg.norm(B["q"]) - 1) < 1e-14
    E = 0.5 * (I * B["w"] * B["w"]).sum()
    return worst, abs(E / E0 - 1)


def test_free_rigid_body_conserves_angular_momentum():
    """Sec. 2.3 rotation integrator with no coupling (gamma = 0): the lab
    angular momentum R I w of an asymmetric top and its energy stay constant
    to the integrator's error, and that error is second order (halving the
    angular velocity over the same total angle quarters it), as for the
    velocity-Verlet rotation schemes the paper cites."""
    d1, e1 = _free_top_drift(1.0)
    d2, e2 = _free_top_drift(0.5)
    assert d1 < 2e-4 and e1 < 2e-4
    assert 3.0 < d1 / d2 < 5.0


def test_torque_free_symmetric_spin_and_drift():
    """A body spinning about a principal axis keeps w; a free body drifts at
    constant V (velocity Verlet with zero force)."""
    L = O.OracleLB(8, 8, 8, collision=0, tau=1.0, gamma_bead=0.0)
    L.add_raspberry(np.zeros((1, 3)), [2.25, 2.5, 2.75], mass=2.0, inertia=(1, 1, 1),
                    V=(0.01, 0, -0.02), w=(0, 0, 0.05))
    L.step(50)
    B = L.body(0)
    assert np.allclose(B["X"], [2.25 + 0.5, 2.5, 2.75 - 1.0], atol=1e-13)
    assert np.allclose(B["w"], [0, 0, 0.05], atol=1e-16)
    ang = 2 * math.atan2(B["q"][3], B["q"][0])
    assert abs(ang - 50 * 0.05) < 1e-12


# ------------------------------------------------------------------ coupling pins

def test_interpolation_exact_for_linear_field_and_drag_sign():
    """Eq. (latticeboltzmannfriction): u(r) interpolated between the 8
    nearest nodes is exact for a linear velocity field (trilinear weights sum
    to one and reproduce coordinates), and F = -gamma (v - u)."""
    n = 12
    L = O.OracleLB(n, n, n, collision=0, tau=1.0, gamma_bead=0.01)
    a = np.array([1e-3, -2e-3, 5e-4])
    B = np.array([[1e-4, 2e-5, -3e-5], [0, -1e-4, 2e-5], [4e-5, 1e-5, 5e-5]])
    f = np.zeros((19, L.N))
    for idx in range(L.N):
        x, y, z = idx % n, (idx // n) % n, idx // (n * n)
        f[:, idx] = O.equilibrium(1.0, a + B @ (np.array([x, y, z]) + 0.5))
    L.set_populations(f)
    beads = np.array([[0.3, -0.7, 1.1], [-1.45, 0.25, 0.0], [0.0, 0.0, 0.0]])
    X = np.array([5.37, 6.01, 5.5])
    V = np.array([1e-3, 1e-3, -1e-3])
    L.add_raspberry(beads, X, fixed=True, V=V)
    L.step(1)
    Fb = L.bead_forces(0)
    for k in range(3):
        r = X + beads[k]
        u = a + B @ r
        assert np.allclose(Fb[k], -0.01 * (V - u), atol=1e-17, rtol=1e-12)


def test_coupling_momentum_exchange_is_exact():
    """Momentum balance of one step in a periodic box: the fluid gains
    -sum F_bead plus the uniform force density times the node count."""
    n = 10
    g = np.array([1e-6, 0, 2e-6])
    L = O.OracleLB(n, n, n, collision=1, gamma_shear=-0.3, gamma_bulk=-0.3, gamma_odd=0.0,
                   gamma_even=0.0, gamma_bead=0.05, body_force=tuple(g))
    rng = np.random.default_rng(0)
    beads = rng.uniform(-2, 2, (40, 3))
    L.add_raspberry(beads, [5.2, 4.9, 5.1], [0.9, 0.1, 0.3, 0.2] / np.linalg.norm([0.9, 0.1, 0.3, 0.2]),
                    mass=30.0, inertia=(10, 12, 14), V=(1e-3, -2e-3, 5e-4), w=(1e-3, 0, -1e-3))
    for _ in range(5):
        _, p0 = L.conservation()
        L.step(1)
        _, p1 = L.conservation()
        Fb = L.bead_forces(0).sum(axis=0)
        assert np.allclose(p1 - p0, -Fb + g * L.N, atol=1e-13, rtol=1e-11)
        assert np.allclose(L.body(0)["F"], Fb, atol=1e-18, rtol=1e-13)


def test_total_momentum_invariant_with_free_colloid_and_compensation():
    """Driven free colloid with the compensating fluid force: the total
    momentum sum(j) + M V + F_last/2 (velocity-Verlet bookkeeping) is
    invariant, and mass is conserved."""
    from paper_1604_01829_gb300 import workloads as W
    n = 16
    sph = W.sphere_raspberry(2.0)
    L = O.OracleLB(n, n, n, collision=0, tau=1.0, gamma_bead=W.paper_gamma_to_lattice(20.0),
                   compensate_force=1)
    L.add_raspberry(sph, [8.3, 7.9, 8.1], mass=33.5, inertia=(53.6,) * 3, F_ext=(0, 0, 1e-3))
    m0, p0 = L.conservation()
    for _ in range(6):
        L.step(25)
        m, p = L.conservation()
        B = L.body(0)
        Ptot = p + 33.5 * B["V"] + 0.5 * B["F_last"]
        assert abs(m - m0) < 1e-10
        # the colloid alone has taken F_ext t ~ 0.15 of momentum from the drive
        assert np.abs(Ptot).max() < 1e-12
    assert B["V"][2] > 0  # the colloid moves along the applied force


@pytest.mark.parametrize("nsub", [2, 3])
def test_md_substeps_conserve_momentum(nsub):
    """MD substeps (Sec. 2.3: two MD steps per LB step in the paper): the
    bodies move nsub times per LB step with dt = 1/nsub and the fluid receives
    each substep's bead forces times dt, so sum(j) + M V + dt F_last / 2 is
    invariant with the compensating drive, and mass is conserved."""
    from paper_1604_01829_gb300 import workloads as W
    n = 14
    sph = W.sphere_raspberry(2.0)
    L = O.OracleLB(n, n, n, collision=0, tau=1.0, gamma_bead=W.paper_gamma_to_lattice(20.0),
                   compensate_force=1, md_substeps=nsub)
    L.add_raspberry(sph, [7.3, 6.9, 7.1], [0.9, 0.3, 0.1, -0.2], mass=33.5, inertia=(53.6,) * 3,
                    F_ext=(0, 0, 1e-3), T_ext=(2e-4, 0, 0))
    m0, _ = L.conservation()
    for _ in range(4):
        L.step(20)
        m, p = L.conservation()
        B = L.body(0)
        Ptot = p + 33.5 * B["V"] + 0.5 / nsub * B["F_last"]
        assert abs(m - m0) < 1e-10
        assert np.abs(Ptot).max() < 1e-12
    assert B["V"][2] > 0


def test_md_substeps_give_the_same_steady_drag():
    """The MD time step does not change the steady drag of a pulled colloid:
    terminal velocities with one and with two MD substeps per LB step agree
    within 1 % (the paper takes two MD steps per LB step, Sec. 2.3; one or
    two give the same hydrodynamics)."""
    from paper_1604_01829_gb300 import workloads as W
    n = 12
    sph = W.sphere_raspberry(2.0)
    V = {}
    for nsub in (1, 2):
        L = O.OracleLB(n, n, n, collision=0, tau=1.0, gamma_bead=W.paper_gamma_to_lattice(50.0),
                       compensate_force=1, md_substeps=nsub)
        L.add_raspberry(sph, [6.2, 5.9, 6.1], mass=33.5, inertia=(53.6,) * 3, F_ext=(1e-4, 0, 0), fixed=2)
        L.step(1500)
        v1 = L.body(0)["V"][0]
        L.step(100)
        V[nsub] = L.body(0)["V"][0]
        assert abs(V[nsub] / v1 - 1) < 2e-3        # steady
    assert abs(V[2] / V[1] - 1) < 0.01, V


def test_spinning_colloid_is_slowed_by_the_fluid():
    """Torque sign: a colloid spinning in quiescent fluid receives a torque
    opposing its angular velocity, and the fluid picks up angular momentum."""
    from paper_1604_01829_gb300 import workloads as W
    n = 16
    sph = W.sphere_raspberry(3.0)
    L = O.OracleLB(n, n, n, collision=0, tau=1.0, gamma_bead=0.05)
    L.add_raspberry(sph, [8, 8, 8], mass=113.0, inertia=(407.0,) * 3, w=(0, 0, 1e-3))
    L.step(3)
    B = L.body(0)
    assert B["T"][2] < 0 and abs(B["T"][0]) < 1e-3 * abs(B["T"][2])
    assert np.linalg.norm(B["F"]) < 1e-3 * abs(B["T"][2])
    w_before = B["w"][2]
    L.step(20)
    assert 0 < L.body(0)["w"][2] < w_before


def test_wall_nodes_absorb_spread_force_and_keep_mass():
    """Beads next to the pore wall: corners that are wall nodes carry u = 0
    and take no spread force; the fluid mass is still exactly conserved."""
    n = 16
    L = O.OracleLB(n, n, 4, collision=1, gamma_shear=-0.2, gamma_bulk=-0.2, gamma_odd=0.0,
                   gamma_even=0.0, gamma_bead=0.05)
    L.set_pore(6.0, axis=2)
    beads = np.array([[5.6, 0.0, 0.0], [0.0, -5.8, 0.3], [3.0, 3.0, 0.0]])
    L.add_raspberry(beads, [8, 8, 2], fixed=True, V=(0, 0, 1e-3))
    m0, _ = L.conservation()
    L.step(10)
    m1, _ = L.conservation()
    assert abs(m1 - m0) < 1e-12
    Fn = L.Fnode.reshape(3, -1)
    assert np.abs(Fn[:, L.mask == 1]).max() == 0.0
    assert np.abs(Fn).max() > 0


# --------------------------------------------------------------- adjoint pins

@pytest.mark.parametrize("kind", ["bgk", "mrt"])
def test_collision_adjoint_matches_finite_differences(kind):
    """Reverse of one node's collision (oracle adjoint) against central
    differences of the oracle collision, for f and for the force."""
    kw = dict(collision=0, tau=0.8) if kind == "bgk" else dict(
        collision=1, gamma_shear=-0.4, gamma_bulk=0.2, gamma_odd=0.3, gamma_even=-0.1)
    p = _params(**kw)
    rng = np.random.default_rng(1)
    f = O.equilibrium(1.0, [0.02, -0.01, 0.03]) * (1 + 0.05 * rng.standard_normal(19))
    F = 1e-3 * rng.standard_normal(3)
    lam = rng.standard_normal(19)
    lf, lF = O.collide_node_adjoint(p, f, F, lam)
    h = 1e-6
    fd = np.array([(O.collide_node(p, f + h * e, F) - O.collide_node(p, f - h * e, F)) @ lam / (2 * h)
                   for e in np.eye(19)])
    fdF = np.array([(O.collide_node(p, f, F + h * e) - O.collide_node(p, f, F - h * e)) @ lam / (2 * h)
                    for e in np.eye(3)])
    assert np.abs(lf - fd).max() <= 1e-8 * np.abs(fd).max()
    assert np.abs(lF - fdF).max() <= 1e-8 * np.abs(fdF).max()


def _adjoint_case(gamma, pore=False):
    from paper_1604_01829_gb300 import workloads as W
    kw = dict(collision=1, gamma_shear=-0.3, gamma_bulk=-0.3, gamma_odd=0.0, gamma_even=0.0,
              gamma_bead=gamma, compensate_force=0 if pore else 1)
    L = O.OracleLB(12, 12, 12, **kw)
    if pore:
        L.set_pore(5.5, axis=2)
    L.add_raspberry(W.sphere_raspberry(2.0), [6.3, 5.9, 6.1], mass=40.0, inertia=(60, 60, 60),
                    F_ext=(0, 0, 2e-3), fixed=2)
    L.step(5)
    return L


@pytest.mark.parametrize("pore", [False, True])
def test_drag_adjoint_matches_finite_differences(pore):
    """Gradient of J = mean pulled-body velocity over the last steps with
    respect to gamma and to bead offsets, from the oracle's reverse pass,
    against central differences of the oracle forward (no bead crosses a
    cell face under the perturbation)."""
    g0 = 0.1
    base = _adjoint_case(g0, pore)
    run = base.clone()
    J, dg, ds = run.adjoint_drag(30, 10)
    assert J > 0
    h = 1e-6
    Jp = base.clone()
    Jp.p.gamma_bead = g0 + h
    Jm = base.clone()
    Jm.p.gamma_bead = g0 - h
    fd = (Jp.adjoint_drag(30, 10)[0] - Jm.adjoint_drag(30, 10)[0]) / (2 * h)
    assert abs(dg - fd) <= 1e-6 * abs(fd)
    for (k, a) in [(0, 0), (5, 2), (40, 1)]:
        vals = []
        for d in (1e-5, -1e-5):
            c = base.clone()
            c.bodies[0]["s"] = c.bodies[0]["s"].copy()
            c.bodies[0]["s"][k, a] += d
            P = base._packed
            c._pack()
            for key in ("X", "V", "q", "w", "F_last", "T_last"):
                c._packed[key][:] = P[key]
            vals.append(c.adjoint_drag(30, 10)[0])
        fd = (vals[0] - vals[1]) / 2e-5
        assert abs(ds[k, a] - fd) <= 2e-5 * abs(fd) + 1e-12, (k, a, ds[k, a], fd)
    # the pass advances the state exactly like plain steps
    plain = base.clone()
    plain.step(30)
    assert np.array_equal(plain.populations(), run.populations())


# ------------------------------------------------------------- Hasimoto pin

def _mean_flow_drag(L, R=1.5, gamma=0.3, g=1e-6):
    """Drag of a fixed raspberry in a periodic box driven by a uniform force
    density g: xi = g N / U_inf, where the mean fluid velocity approaches its
    steady value U_inf as a single exponential once the viscous transient
    (~L^2/nu) has gone; U_inf from three equally spaced samples (Aitken)."""
    from paper_1604_01829_gb300 import workloads as W
    o = O.OracleLB(L, L, L, collision=0, tau=1.0, gamma_bead=gamma, body_force=(g, 0, 0))
    o.add_raspberry(W.sphere_raspberry(R), [L / 2 + 0.13, L / 2 - 0.21, L / 2 + 0.07], fixed=1)
    o.step(int(1.5 * L * L))
    us = []
    for k in range(3):
        rho, u = o.node_velocity()
        us.append((rho * u[:, 0]).sum() / rho.sum())
        if k < 2:
            o.step(int(0.6 * L * L))
    U1, U2, U3 = us
    return g * L ** 3 / ((U1 * U3 - U2 * U2) / (U1 + U3 - 2 * U2))


def test_hasimoto_finite_size_slope():
    """Sec. 2.4, Eq. (hasimoto) in drag form (the printed '6 rho eta' read as
    6 pi eta): for a periodic array of drag centres 1/xi(L) = 1/xi_0 -
    2.837/(6 pi eta L) + O(L^-3), whatever the raspberry's permeability (the
    bead friction only sets xi_0). Fitted over L = 12-24 with the next
    (L^-3) term free, the 1/L coefficient matches -2.837/(6 pi eta) with
    eta = rho0 (tau - 1/2)/3."""
    Ls = np.array([12, 16, 20, 24])
    xi = np.array([_mean_flow_drag(int(L)) for L in Ls])
    x = 1.0 / Ls
    A = np.stack([np.ones_like(x), x, x ** 3], axis=1)
    a, b, c = np.linalg.lstsq(A, 1.0 / xi, rcond=None)[0]
    eta = 1.0 * (1.0 - 0.5) / 3.0
    assert abs(b / (-2.837 / (6 * math.pi * eta)) - 1) < 0.02
    assert np.all(np.diff(xi) < 0)   # drag falls towards infinite dilution
