"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same
seeded inputs, element by element.

Tolerances (written here, derived in the design notes):
  FP64 populations: |f_gpu - f_oracle| <= 1e-12 w_i rho0 after the stated
  steps (summation order and FMA contraction differ; atomics reorder the
  bead-force sums);
  FP32 storage of f - w_i rho0: <= 1e-5 w_i rho0 for populations, and
  1e-5 relative for bead forces, body force and torque (FP32 rounding of
  deviations of order 1e-2 w_i rho0 over tens of steps; the worst errors
  these tests have shown on GB300 are 1.4e-7 for populations and 1.7e-6 for
  body torques).
Sizes span several 4x4x4 force tiles and several thread blocks with a ragged
tail in every direction; odd and even step counts exercise both AA parities.
"""
import math

import numpy as np
import pytest

from helpers import Pair, W19, observe, perturbed_populations
from paper_1604_01829_gb300 import workloads as Wl

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1604_01829_gb300 import build
    build.build()


MRT = dict(collision=1, gamma_shear=-0.45, gamma_bulk=-0.2, gamma_odd=0.3, gamma_even=-0.1)


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("case", ["bgk", "mrt", "mrt_noise"])
@pytest.mark.parametrize("steps", [1, 2, 7])
def test_periodic_fluid(precision, case, steps):
    nx, ny, nz = 37, 13, 10
    params = dict(collision=0, tau=0.8) if case == "bgk" else dict(MRT)
    if case == "mrt_noise":
        params.update(kT=1e-4, seed=0xABCDEF0123)
    params["body_force"] = (1e-5, -2e-5, 3e-6)
    P = Pair(nx, ny, nz, precision=precision, **params)
    P.set_populations(perturbed_populations(P.N, seed=3))
    P.step(steps)
    assert P.pop_error() <= TOL[precision]


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("axis", [2, 0])
def test_pore_bounce_back(precision, axis):
    n_ax, n_cross = 9, 22
    dims = [n_cross, n_cross, n_cross]
    dims[axis] = n_ax
    params = dict(MRT, body_force=tuple(1e-5 if a == axis else 0.0 for a in range(3)))
    P = Pair(*dims, precision=precision, pore=(8.3, axis), **params)
    P.set_populations(perturbed_populations(P.N, seed=5))
    for _ in range(3):
        P.step(3)
        assert P.pop_error() <= TOL[precision]
    mg, _ = P.gpu.lb_conservation()
    mo, _ = P.orc.conservation()
    # FP32 deviations carry ~1e-7 relative rounding of O(1e-2) deviations
    assert abs(mg - mo) <= (1e-11 if precision == 64 else 1e-8) * mo


@pytest.mark.parametrize("precision", [64, 32])
def test_free_raspberry_periodic(precision):
    L = 24
    params = dict(collision=0, tau=0.9, gamma_bead=Wl.paper_gamma_to_lattice(100.0),
                  compensate_force=1, body_force=(0, 2e-6, 0))
    P = Pair(L, L, L + 3, precision=precision, **params)
    P.set_populations(perturbed_populations(P.N, amp=0.005, u_amp=0.005, seed=7))
    beads = Wl.sphere_raspberry(3.0)
    q = [0.9, 0.2, -0.3, 0.1]
    b = P.add_body(beads, [11.3, 12.7, 13.1], q, mass=113.0, inertia=(400, 420, 440),
                   F_ext=(1e-3, 0, -5e-4), T_ext=(0, 1e-3, 0), V=(1e-3, -2e-3, 5e-4), w=(1e-3, 2e-3, -1e-3))
    for k in range(4):
        P.step(3 if k % 2 == 0 else 2)
        assert P.pop_error() <= TOL[precision]
        e = P.body_errors(b)
        tb = 1e-11 if precision == 64 else 1e-5
        assert e["bead"] <= tb and e["F"] <= tb and e["T"] <= tb, e
        assert e["X"] <= tb and e["V"] <= tb * 1e-2 and e["q"] <= tb and e["w"] <= tb * 1e-2, e
    # spread force field of the last step
    Fg = P.gpu.lb_get_node_force()
    Fo = P.orc.Fnode.reshape(3, -1)
    assert np.abs(Fg - Fo).max() <= (1e-12 if precision == 64 else 1e-5) * np.abs(Fo).max()


@pytest.mark.parametrize("precision", [64, 32])
def test_external_forces_set_between_steps_and_read_back_together(precision):
    """lb_set_external_forces between steps (all or the first bodies, with and
    without torques; with the compensating fluid force) against the oracle's
    set_external; lb_forces_all (every body in one read) equals lb_forces
    body by body."""
    params = dict(MRT, kT=1e-4, seed=13, gamma_bead=Wl.paper_gamma_to_lattice(50.0), compensate_force=1)
    P = Pair(24, 20, 18, precision=precision, **params)
    P.set_populations(perturbed_populations(P.N, seed=14))
    sph = Wl.sphere_raspberry(2.0)
    ell = Wl.ellipsoid_raspberry(3.0, 1.5, 1.5, seed=3)
    P.add_body(sph, [6.2, 5.1, 4.3], mass=34.0, inertia=(50, 50, 50), F_ext=(1e-3, 0, 0))
    P.add_body(ell, [16.7, 13.2, 11.1], q=[0.9, 0.1, -0.2, 0.3], mass=30.0, inertia=(10, 40, 40),
               F_ext=(0, 5e-4, 0), T_ext=(0, 0, 1e-3))
    P.add_body(sph, [8.8, 15.5, 13.9], mass=34.0, inertia=(50, 50, 50))
    rng = np.random.default_rng(2)
    tb = 1e-11 if precision == 64 else 1e-5
    for n, nset, with_T in ((1, 3, True), (2, 2, False), (3, 3, True), (4, 1, True)):
        F = rng.normal(scale=1e-3, size=(nset, 3))
        T = rng.normal(scale=1e-3, size=(nset, 3)) if with_T else None
        P.gpu.lb_set_external_forces(F, T)
        for b in range(nset):
            P.orc.set_external(b, F_ext=F[b], T_ext=T[b] if with_T else np.zeros(3))
        P.step(n)
        assert P.pop_error() <= TOL[precision]
        Fa, Ta = P.gpu.lb_forces_all()
        for b in range(3):
            Fb, Tb = P.gpu.lb_forces(b)
            assert np.array_equal(Fa[3 * b:3 * b + 3], Fb) and np.array_equal(Ta[3 * b:3 * b + 3], Tb)
            e = P.body_errors(b)
            assert e["bead"] <= tb and e["F"] <= tb and e["T"] <= tb and e["X"] <= tb, (n, b, e)


@pytest.mark.parametrize("precision", [64, 32])
def test_step_io_equals_the_three_calls(precision):
    """lb_step_io (external forces in, steps, every body's totals out, one
    library call) leaves the same state and returns the same totals as
    lb_set_external_forces + lb_step + lb_forces_all on a twin handle, to the
    rounding of the atomics that sum bead forces in an unspecified order
    (FP64 1e-11, FP32 1e-5 of the largest value); F_ext None keeps the
    forces, no output arrays skips the read-back; wrong arrays are refused
    before the call."""
    from paper_1604_01829_gb300 import lb
    params = dict(MRT, kT=1e-4, seed=21, gamma_bead=Wl.paper_gamma_to_lattice(50.0), compensate_force=1)
    sph = Wl.sphere_raspberry(2.0)
    ell = Wl.ellipsoid_raspberry(3.0, 1.5, 1.5, seed=3)
    hs = []
    for _ in range(2):
        h = lb.LB(20, 18, 16, precision=precision, **params)
        h.lb_add_raspberry(sph, [6.2, 5.1, 4.3], mass=34.0, inertia=(50, 50, 50), F_ext=(1e-3, 0, 0))
        h.lb_add_raspberry(ell, [13.7, 11.2, 9.1], [0.9, 0.1, -0.2, 0.3], 30.0, (10, 40, 40))
        hs.append(h)
    A, B = hs
    rng = np.random.default_rng(5)
    Fa, Ta, Fb, Tb = (np.zeros(6) for _ in range(4))
    tol = 1e-11 if precision == 64 else 1e-5

    def close(a, b):
        d = float(np.abs(a - b).max() / max(np.abs(a).max(), 1e-30))
        observe("step_io", d)
        return d <= tol

    for n, set_forces in ((1, True), (3, False), (2, True), (1, True)):
        F = rng.normal(scale=1e-3, size=6)
        T = rng.normal(scale=1e-3, size=6)
        if set_forces:
            A.lb_set_external_forces(F, T)
        A.lb_step(n)
        A.lb_forces_all(Fa, Ta)
        B.lb_step_io(F if set_forces else None, T if set_forces else None, Fb, Tb, n)
        assert close(Fa, Fb) and close(Ta, Tb), n
    B.lb_step_io(None, None, None, None, 2)
    A.lb_step(2)
    fa, fb = A.lb_get_populations(), B.lb_get_populations()
    assert float((np.abs(fa - fb).max(axis=1) / W19).max()) <= tol
    for b in range(2):
        sa, sb = A.lb_get_body(b), B.lb_get_body(b)
        assert all(close(sa[k], sb[k]) for k in ("X", "q")), b
    with pytest.raises(ValueError):
        B.lb_step_io(np.zeros(5), None, Fb, Tb)
    with pytest.raises(ValueError):
        B.lb_step_io(None, None, np.zeros(6, dtype=np.float32), Tb)
    A.close()
    B.close()


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("nsub", [2, 3])
def test_md_substeps_match_oracle(precision, nsub):
    """MD substeps per LB step (the paper's MD step is half the LB step):
    bodies move and couple nsub times per LB step with dt = 1/nsub, bead noise
    per substep; a free ellipsoid and a fixed sphere in a thermal pore, odd and
    even step counts, eager steps and graph replay, with the recorder."""
    params = dict(MRT, kT=1e-4, seed=88, gamma_bead=Wl.paper_gamma_to_lattice(50.0), md_substeps=nsub)
    P = Pair(26, 26, 20, precision=precision, pore=(11.0, 2), **params)
    P.add_body(Wl.sphere_raspberry(2.5), [13 + 6.9, 13.4, 6.0], fixed=True, V=(0, 0, 1e-3))
    ell = Wl.ellipsoid_raspberry(4.0, 2.0, 2.0, seed=3)
    m = 4.0 / 3.0 * math.pi * 16.0
    P.add_body(ell, [11.5, 12.2, 14.7], [0.8, 0.1, 0.5, -0.2], mass=m,
               inertia=tuple(Wl.solid_ellipsoid_inertia(m, 4.0, 2.0, 2.0)), F_ext=(0, 0, 2e-3), T_ext=(1e-3, 0, 0))
    P.gpu.lb_record_bodies(2, 20)
    tb = 1e-11 if precision == 64 else 1e-5
    for n in (3, 2, 5):
        P.step(n)
        assert P.pop_error() <= TOL[precision]
        for b in range(2):
            e = P.body_errors(b)
            assert e["bead"] <= tb and e["F"] <= tb and e["T"] <= tb and e["X"] <= tb, (n, b, e)
    steps, X, q = P.gpu.lb_get_trajectory(1)
    assert list(steps) == [2, 4, 6, 8, 10]
    assert np.array_equal(X[-1], P.gpu.lb_get_body(1)["X"])


@pytest.mark.parametrize("precision", [64, 32])
def test_raspberry_in_pore_with_noise(precision):
    """Thermal MRT fluid, bead noise, a fixed sphere near the pore wall (some
    corners are wall nodes) and a free ellipsoid."""
    params = dict(MRT, kT=1e-4, seed=77, gamma_bead=Wl.paper_gamma_to_lattice(50.0))
    P = Pair(26, 26, 20, precision=precision, pore=(11.0, 2), **params)
    sph = Wl.sphere_raspberry(2.5)
    P.add_body(sph, [13 + 7.2, 13.4, 6.0], fixed=True, V=(0, 0, 1e-3))
    ell = Wl.ellipsoid_raspberry(4.0, 2.0, 2.0, seed=3)
    P.add_body(ell, [11.5, 12.2, 14.7], [0.8, 0.1, 0.5, -0.2], mass=60.0, inertia=(30, 90, 90),
               F_ext=(0, 0, 2e-3))
    for _ in range(3):
        P.step(3)
        assert P.pop_error() <= TOL[precision]
        for b in range(2):
            e = P.body_errors(b)
            tb = 1e-11 if precision == 64 else 1e-5
            assert e["bead"] <= tb and e["F"] <= tb and e["T"] <= tb, (b, e)


def test_conservation_matches_oracle_and_is_exact():
    params = dict(MRT, kT=1e-4, seed=5)
    P = Pair(20, 18, 16, precision=64, **params)
    P.set_populations(perturbed_populations(P.N, seed=9))
    m0, p0 = P.gpu.lb_conservation()
    mo, po = P.orc.conservation()
    assert abs(m0 - mo) <= 1e-12 * mo and np.abs(p0 - po).max() <= 1e-12
    P.step(11)
    m1, p1 = P.gpu.lb_conservation()
    assert abs(m1 - m0) <= 1e-12 * m0
    assert np.abs(p1 - p0).max() <= 1e-13 * m0


@pytest.mark.parametrize("steps", [0, 3, 4])
def test_fp32_periodic_conservation_matches_oracle(steps):
    """FP32 deviations in a periodic box take the one-pass plane-sum
    reduction (mass and momentum from the slots, the momentum sign flipped
    on odd step counts): equal to the oracle's FP64 sums within the FP32
    storage rounding, on even and odd step counts."""
    params = dict(MRT, kT=1e-4, seed=15)
    P = Pair(20, 18, 16, precision=32, **params)
    P.set_populations(perturbed_populations(P.N, seed=3))
    P.step(steps)
    m, p = P.gpu.lb_conservation()
    mo, po = P.orc.conservation()
    assert abs(m - mo) <= 1e-9 * mo
    assert np.abs(p - po).max() <= 2e-5 * np.sqrt(P.N) * 1e-2


def test_sample_populations_matches_full_readback():
    P = Pair(17, 9, 6, precision=32, **MRT)
    P.set_populations(perturbed_populations(P.N, seed=2))
    P.gpu.lb_step(3)
    full = P.gpu.lb_get_populations()
    idx = np.array([0, 5, P.N - 1, 123, 456])
    s = P.gpu.lb_sample_populations(idx)
    assert np.array_equal(s, full[:, idx].T)


def test_errors_are_reported_not_raised_in_the_library():
    from paper_1604_01829_gb300 import lb
    with pytest.raises(lb.LBError) as ei:
        lb.LB(8, 8, 8, collision=0, tau=0.4)
    assert ei.value.status == lb.LB_ERR_ARG
    with pytest.raises(lb.LBError):
        lb.LB(8, 8, 8, collision=0, tau=1.0, kT=1e-4)
    g = lb.LB(8, 8, 8)
    with pytest.raises(lb.LBError) as ei:
        g.lb_set_pore(3.0, axis=5)
    assert ei.value.status == lb.LB_ERR_ARG
    g.lb_step(1)
    with pytest.raises(lb.LBError) as ei:
        g.lb_set_pore(3.0, axis=2)
    assert ei.value.status == lb.LB_ERR_STATE
    with pytest.raises(lb.LBError):
        g.lb_sample_populations([8 ** 3])


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("case", ["bgk", "mrt_noise"])
@pytest.mark.parametrize("steps", [1, 4, 7])
def test_fp32_kernel_variants(variant, case, steps):
    """Plain and TMA-staged collide kernels (nx a multiple of 4, periodic)
    against the oracle; rows of 36 nodes, 9 x 7 rows."""
    params = dict(collision=0, tau=0.7) if case == "bgk" else dict(MRT, kT=1e-4, seed=99)
    params["body_force"] = (2e-5, 1e-5, -1e-5)
    P = Pair(36, 9, 7, precision=32, **params)
    P.gpu.lb_set_kernel_variant(variant)
    P.set_populations(perturbed_populations(P.N, seed=17))
    P.step(steps)
    assert P.pop_error() <= TOL[32]


@pytest.mark.parametrize("precision", [64, 32])
def test_checkpoint_resume(precision):
    """A checkpoint taken at an odd step count and loaded into a fresh handle
    with the same parameters and bodies resumes the run: without bodies bit
    for bit (the noise is counter-based), with a body up to the order of the
    bead-force atomics. A checkpoint of another lattice is refused."""
    from paper_1604_01829_gb300 import lb
    params = dict(MRT, kT=1e-4, seed=21, gamma_bead=Wl.paper_gamma_to_lattice(50.0), precision=precision)
    f0 = perturbed_populations(40 * 20 * 18, seed=5)
    q = np.array([0.9, 0.2, -0.3, 0.1]) / np.linalg.norm([0.9, 0.2, -0.3, 0.1])
    ell = Wl.ellipsoid_raspberry(4.0, 2.0, 2.0, seed=2)
    m = 4.0 / 3.0 * math.pi * 16.0

    def make(with_body):
        g = lb.LB(40, 20, 18, **params)
        if with_body:
            g.lb_add_raspberry(ell, [20.3, 9.7, 8.8], q, m, tuple(Wl.solid_ellipsoid_inertia(m, 4.0, 2.0, 2.0)),
                               (1e-3, 0, 0))
        return g

    for with_body in (False, True):
        a = make(with_body)
        a.lb_set_populations(f0)
        a.lb_step(7)
        ck = a.lb_checkpoint_save()
        a.lb_step(6)
        b = make(with_body)
        b.lb_checkpoint_load(ck)
        b.lb_step(6)
        fa, fb = a.lb_get_populations(), b.lb_get_populations()
        assert a.lb_info()["step"] == b.lb_info()["step"] == 13
        if not with_body:
            assert np.array_equal(fa, fb)
        else:
            d = (np.abs(fa - fb).max(axis=1) / W19).max()
            assert d <= (1e-13 if precision == 64 else 1e-6), d
            xa, xb = a.lb_get_body(0)["X"], b.lb_get_body(0)["X"]
            assert np.abs(xa - xb).max() <= (1e-12 if precision == 64 else 1e-7)
        other = lb.LB(40, 20, 16, **params)
        with pytest.raises(lb.LBError) as e:
            other.lb_checkpoint_load(ck)
        assert e.value.status == lb.LB_ERR_STATE
        for g in (a, b, other):
            g.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_run_to_run_nondeterminism_is_bounded(precision):
    """The same coupled run twice: bead forces are summed onto nodes and bodies
    by atomics in arbitrary order, so results may differ in the last bits;
    over 20 steps the populations stay within 1e-14 w_i (FP64) / 1e-6 w_i
    (FP32) of each other. The fluid alone (no atomics, counter-based noise)
    repeats bit for bit."""
    from paper_1604_01829_gb300 import lb
    params = dict(MRT, kT=1e-4, seed=31, gamma_bead=Wl.paper_gamma_to_lattice(50.0), precision=precision)
    f0 = perturbed_populations(48 * 20 * 18, seed=8)
    ell = Wl.ellipsoid_raspberry(4.0, 2.0, 2.0, seed=3)
    m = 4.0 / 3.0 * math.pi * 16.0
    q = np.array([0.8, 0.1, 0.5, -0.2]) / np.linalg.norm([0.8, 0.1, 0.5, -0.2])

    def run(with_body):
        g = lb.LB(48, 20, 18, **params)
        g.lb_set_populations(f0)
        if with_body:
            g.lb_add_raspberry(ell, [22.6, 9.3, 8.1], q, m, tuple(Wl.solid_ellipsoid_inertia(m, 4.0, 2.0, 2.0)),
                               (1e-3, 5e-4, 0))
        g.lb_step(20)
        f = g.lb_get_populations()
        g.close()
        return f

    assert np.array_equal(run(False), run(False))
    d = (np.abs(run(True) - run(True)).max(axis=1) / W19).max()
    assert d <= (1e-14 if precision == 64 else 1e-6), d


def test_bounded_wait_runs_out_and_is_reported():
    """Failure detection without a fault: the TMA-staged kernel's stage waits
    get a limit (16 SM cycles) far below the copy latency, so they run out; the
    blocks stop once their copies in flight have landed and the next
    synchronising call returns LB_ERR_TIMEOUT, once. The context stays usable:
    with the default limit and the state restored, further steps match the
    oracle."""
    from paper_1604_01829_gb300 import lb
    P = Pair(64, 24, 20, precision=32, **dict(MRT, kT=1e-4, seed=5))
    P.set_populations(perturbed_populations(P.N, seed=3))
    P.gpu.lb_set_kernel_variant(2)
    P.gpu.lb_set_wait_limit(16)
    P.step(1)
    with pytest.raises(lb.LBError) as e:
        P.gpu.lb_conservation()
    assert e.value.status == lb.LB_ERR_TIMEOUT
    P.gpu.lb_conservation()                                   # reported once
    with pytest.raises(lb.LBError):
        P.gpu.lb_set_wait_limit(-1)
    P.gpu.lb_set_wait_limit(0)
    P.gpu.lb_set_populations(P.orc.populations())             # the oracle's state after the same step
    P.step(4)
    assert P.pop_error() <= TOL[32]
    m, _ = P.gpu.lb_conservation()
    m_orc = float(P.orc.populations().sum())
    assert abs(m / m_orc - 1.0) < 1e-6


@pytest.mark.parametrize("stages,ctas", [(2, 1), (3, 2), (6, 1)])
def test_tma_ring_depths_with_coupling(stages, ctas):
    """TMA-staged kernel with bead forces in flagged tiles, several ring
    depths and persistent grids; rows of 64 nodes (several rows per CTA)."""
    # explicit coupling is stable for N gamma / M well below 2 (here ~0.2)
    params = dict(MRT, kT=1e-4, seed=5, gamma_bead=Wl.paper_gamma_to_lattice(50.0), compensate_force=1)
    P = Pair(64, 12, 10, precision=32, **params)
    P.gpu.lb_set_kernel_variant(2, stages, ctas)
    ell = Wl.ellipsoid_raspberry(4.0, 2.0, 2.0, seed=8)
    P.add_body(ell, [30.3, 6.1, 5.2], [0.7, 0.3, -0.5, 0.4], mass=120.0, inertia=(60, 180, 180),
               F_ext=(1e-3, 0, 0))
    for _ in range(3):
        P.step(3)
        assert P.pop_error() <= TOL[32]
        e = P.body_errors(0)
        assert e["bead"] <= 1e-5 and e["F"] <= 1e-5, e


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("spacing,R,rp,rs,off", [(2.0, 7.5, 2.5, 2.0, 4.9), (0.9, 7.5, 2.5, 2.0, 4.9),
                                                 (2.0, 3.0, 4.0, 1.5, 0.9)])
def test_pore_wall_beads_match_oracle(precision, spacing, R, rp, rs, off):
    """Repulsive pore-wall beads (WCA, Sec. 2.3) on a sphere raspberry pushed
    towards the wall of a z pore: body force, torque and trajectory as the
    oracle's sum over every wall bead (the GPU sums a window around the
    nearest one). Dense wall beads and a narrow pore with a wide cutoff."""
    params = dict(MRT, kT=1e-4, seed=31, gamma_bead=Wl.paper_gamma_to_lattice(50.0))
    P = Pair(20, 20, 16, precision=precision, pore=(R, 2), **params)
    P.gpu.lb_set_pore_beads(spacing, rp, 0.5, 2e-3)
    P.orc.set_pore_beads(R, 2, spacing, rp, 0.5, 2e-3)
    P.add_body(Wl.sphere_raspberry(rs), [10 + off, 10.3, 7.1], mass=34.0, inertia=(50, 50, 50),
               F_ext=(2e-3, 0, 0))
    # the wall beads do act on some of the colloid beads at this position
    X = np.array([10 + off, 10.3, 7.1]) + Wl.sphere_raspberry(rs)
    assert max(np.linalg.norm(P.orc.wall_force(x)) for x in X) > 1e-4
    for _ in range(3):
        P.step(3)
        assert P.pop_error() <= TOL[precision]
        e = P.body_errors(0)
        tb = 1e-11 if precision == 64 else 1e-5
        assert e["bead"] <= tb and e["F"] <= tb and e["T"] <= tb and e["X"] <= tb, e


def test_pore_beads_need_a_pore():
    from paper_1604_01829_gb300 import lb
    g = lb.LB(8, 8, 8)
    with pytest.raises(lb.LBError) as ei:
        g.lb_set_pore_beads(2.0, 2.5, 0.5, 1e-3)
    assert ei.value.status == lb.LB_ERR_STATE
    g.lb_set_pore(3.0, 2)
    with pytest.raises(lb.LBError) as ei:
        g.lb_set_pore_beads(-1.0, 2.5, 0.5, 1e-3)
    assert ei.value.status == lb.LB_ERR_ARG


@pytest.mark.parametrize("precision", [64, 32])
def test_step_pairs_replayed_from_a_graph(precision):
    """lb_step with four or more steps replays eight-step and step-pair CUDA
    graphs (odd starting counts take one step eagerly first, a leftover odd
    step runs eagerly): a pore with wall beads, a free ellipsoid, thermal
    noise and the recorder; the graphs are rebuilt after the wall beads and
    the recorder change."""
    params = dict(MRT, kT=1e-4, seed=61, gamma_bead=Wl.paper_gamma_to_lattice(50.0))
    P = Pair(22, 22, 18, precision=precision, pore=(9.5, 2), **params)
    P.set_populations(perturbed_populations(P.N, seed=6))
    P.gpu.lb_set_pore_beads(2.0, 2.5, 0.5, 1e-3)
    P.orc.set_pore_beads(9.5, 2, 2.0, 2.5, 0.5, 1e-3)
    ell = Wl.ellipsoid_raspberry(4.0, 2.0, 2.0, seed=2)
    P.add_body(ell, [11.3, 11.8, 9.2], [0.9, 0.2, -0.3, 0.1], mass=80.0, inertia=(40, 120, 120),
               F_ext=(1e-3, 5e-4, 0))
    P.gpu.lb_record_bodies(3, 50)
    tb = 1e-11 if precision == 64 else 1e-5
    for n in (9, 6, 4, 5, 16):
        if n == 4:
            P.gpu.lb_set_pore_beads(2.5, 2.5, 0.5, 2e-3)
            P.orc.set_pore_beads(9.5, 2, 2.5, 2.5, 0.5, 2e-3)
            P.gpu.lb_record_bodies(2, 50)
        P.step(n)
        assert P.pop_error() <= TOL[precision]
        e = P.body_errors(0)
        assert e["bead"] <= tb and e["F"] <= tb and e["X"] <= tb, (n, e)
    steps, X, q = P.gpu.lb_get_trajectory(0)          # recorder restarted at step 15, every 2
    assert list(steps) == list(range(16, 42, 2))
    assert np.array_equal(X[-1], P.gpu.lb_get_body(0)["X"])


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("nsteps", [(1, 2, 3), (5, 4)])
def test_channel_walls_match_oracle(precision, nsteps):
    """Moving walls at y = -1/2 and ny - 1/2 (the Stokes-flow set-up) with
    different tangential velocities, thermal MRT fluid, a free sphere whose
    beads reach beyond the lower wall plane's first node row; eager steps
    and graph-replayed step pairs."""
    params = dict(MRT, kT=1e-4, seed=19, gamma_bead=Wl.paper_gamma_to_lattice(50.0))
    P = Pair(14, 12, 10, precision=precision, **params)
    ulo, uhi = (1e-3, 0.0, -5e-4), (-2e-3, 0.0, 1e-3)
    P.gpu.lb_set_channel_walls(ulo, uhi)
    P.orc.set_channel_walls(ulo, uhi)
    P.set_populations(perturbed_populations(P.N, seed=9))
    P.add_body(Wl.sphere_raspberry(2.0), [6.3, 2.4, 4.8], mass=34.0, inertia=(50, 50, 50), F_ext=(0, -1e-3, 0))
    tb = 1e-11 if precision == 64 else 1e-5
    for n in nsteps:
        P.step(n)
        assert P.pop_error() <= TOL[precision]
        e = P.body_errors(0)
        assert e["bead"] <= tb and e["F"] <= tb and e["X"] <= tb, (n, e)
    m, _ = P.gpu.lb_conservation()
    mo, _ = P.orc.conservation()
    assert abs(m - mo) <= (1e-12 if precision == 64 else 1e-8) * mo


def test_channel_walls_exclude_a_pore():
    from paper_1604_01829_gb300 import lb
    g = lb.LB(8, 8, 8)
    g.lb_set_pore(3.0, 2)
    with pytest.raises(lb.LBError) as ei:
        g.lb_set_channel_walls((0, 0, 1e-3), (0, 0, 1e-3))
    assert ei.value.status == lb.LB_ERR_STATE
    h = lb.LB(8, 8, 8)
    with pytest.raises(lb.LBError) as ei:
        h.lb_set_channel_walls((0, 1e-3, 0), (0, 0, 0))
    assert ei.value.status == lb.LB_ERR_ARG


def test_kernel_variant_rejects_unsupported_shapes():
    from paper_1604_01829_gb300 import lb
    g = lb.LB(37, 8, 8, precision=32)
    with pytest.raises(lb.LBError):
        g.lb_set_kernel_variant(2)
    g64 = lb.LB(36, 8, 8, precision=64)
    with pytest.raises(lb.LBError):
        g64.lb_set_kernel_variant(2)
