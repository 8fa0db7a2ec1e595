"""Trajectory recorder and GPU mean-squared-displacement analysis
(lb_record_bodies, lb_get_trajectory, lb_batch_*, lb_msd_trajectory):
records equal the body states read back at those steps and the oracle's
bodies; the GPU MSD equals the oracle analysis of the same trajectory
(Sec. 2.4-2.7 of Ustach & Faller, arXiv:1604.01829)."""
import numpy as np
import pytest

from helpers import Pair, perturbed_populations
from oracle import analysis as A
from paper_1604_01829_gb300 import workloads as Wl

pytestmark = pytest.mark.gpu

MRT = dict(collision=1, gamma_shear=-0.45, gamma_bulk=-0.2, gamma_odd=0.3, gamma_even=-0.1)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1604_01829_gb300 import build
    build.build()


def _synthetic(nb, n, seed):
    """Random-walk centres and a random walk of orientations (small random
    rotations per record, some large enough to test the angle range)."""
    rng = np.random.default_rng(seed)
    X = np.cumsum(rng.normal(scale=0.3, size=(nb, n, 3)), axis=1) + 10.0
    q = np.zeros((nb, n, 4))
    for b in range(nb):
        cur = rng.normal(size=4)
        cur /= np.linalg.norm(cur)
        for k in range(n):
            q[b, k] = cur
            d = np.concatenate([[1.0], rng.normal(scale=0.08 if k % 50 else 0.6, size=3)])
            d /= np.linalg.norm(d)
            w1, x1, y1, z1 = cur
            w2, x2, y2, z2 = d
            cur = np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                            w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])
    return X, q


@pytest.mark.parametrize("nb,n,lags", [(1, 40, 39), (3, 300, 60)])
def test_msd_matches_oracle_analysis(nb, n, lags):
    from paper_1604_01829_gb300 import lb
    X, q = _synthetic(nb, n, seed=nb)
    p_ref = (0.2, -0.7, 0.4)
    got = lb.lb_msd_trajectory(X, q, lags, p_ref)
    for b in range(nb):
        ref = A.msd(X[b], q[b], lags, p_ref)
        # sums of positive terms in another order: 1e-12; summed angles: 1e-10
        assert np.allclose(got[b, :, 0:6], ref[:, 0:6], rtol=1e-12, atol=0)
        assert np.allclose(got[b, :, 6:10], ref[:, 6:10], rtol=1e-10, atol=1e-22)


def test_msd_rejects_bad_arguments():
    from paper_1604_01829_gb300 import lb
    X, q = _synthetic(1, 10, seed=3)
    with pytest.raises(lb.LBError) as ei:
        lb.lb_msd_trajectory(X, q, 10)
    assert ei.value.status == lb.LB_ERR_ARG
    with pytest.raises(lb.LBError):
        lb.lb_msd_trajectory(X, q, 3, p_ref=(0, 0, 0))


@pytest.mark.parametrize("precision", [64, 32])
def test_recorder_matches_body_states_and_oracle(precision):
    """Thermal MRT fluid with a free ellipsoid and a free sphere; one record
    every 3 steps in a ring of 7, stepped in uneven chunks. Each record is
    bit-identical to the body state read back after that step, and matches
    the oracle's body within the parity tolerance."""
    params = dict(MRT, kT=1e-4, seed=12, gamma_bead=Wl.paper_gamma_to_lattice(50.0), compensate_force=1)
    P = Pair(24, 20, 18, precision=precision, **params)
    P.set_populations(perturbed_populations(P.N, seed=2))
    ell = Wl.ellipsoid_raspberry(4.0, 2.0, 2.0, seed=6)
    P.add_body(ell, [11.2, 9.7, 8.1], [0.9, 0.2, -0.3, 0.1], mass=80.0, inertia=(40, 120, 120),
               F_ext=(1e-3, 0, 0), V=(1e-3, 0, 0), w=(0, 1e-3, 2e-3))
    P.add_body(Wl.sphere_raspberry(2.0), [4.3, 14.2, 12.6], mass=34.0, inertia=(50, 50, 50),
               F_ext=(0, -1e-3, 5e-4))
    every, cap = 3, 7
    P.gpu.lb_step(2)
    P.orc.step(2)
    P.gpu.lb_record_bodies(every, cap)
    expect = {}
    step = 2
    for chunk in (1, 3, 5, 2, 4, 6, 3, 3, 1):
        for _ in range(chunk):
            P.step(1)
            step += 1
            if step % every == 0:
                for b in range(2):
                    g = P.gpu.lb_get_body(b)
                    expect[(step, b)] = (g["X"].copy(), g["q"].copy(), P.orc.body(b))
    for b in range(2):
        steps, X, q = P.gpu.lb_get_trajectory(b)
        want = sorted(s for (s, bb) in expect if bb == b)[-cap:]
        assert list(steps) == want
        for k, s in enumerate(steps):
            Xg, qg, o = expect[(s, b)]
            assert np.array_equal(X[k], Xg) and np.array_equal(q[k], qg)
            tol = 1e-11 if precision == 64 else 1e-5
            assert np.abs(X[k] - o["X"]).max() <= tol * 10 and np.abs(q[k] - o["q"]).max() <= tol, (s, b)
    # turning it off and on restarts the ring
    P.gpu.lb_record_bodies(0)
    assert len(P.gpu.lb_get_trajectory(0)[0]) == 0
    P.gpu.lb_record_bodies(2, 5)
    P.gpu.lb_step(5)
    want = [2 * k for k in range(step // 2 + 1, (step + 5) // 2 + 1)]
    assert list(P.gpu.lb_get_trajectory(1)[0]) == want


def test_recorder_rejects_a_lattice_without_bodies():
    from paper_1604_01829_gb300 import lb
    g = lb.LB(8, 8, 8)
    with pytest.raises(lb.LBError) as ei:
        g.lb_record_bodies(5, 10)
    assert ei.value.status == lb.LB_ERR_ARG


def test_batched_recorder_with_graph_replays_and_autotune():
    """Two instances with bodies and one without; steps replayed from the
    two-step graph, odd eager steps and an autotune in between: every record
    equals the body state read back after that step."""
    from paper_1604_01829_gb300 import lb
    g = Wl.paper_gamma_to_lattice(50.0)
    sph = Wl.sphere_raspberry(2.0)
    cases = [dict(nx=16, ny=16, nz=12, precision=32, seed=1, gamma_bead=g, kT=1e-4, **MRT),
             dict(nx=12, ny=10, nz=9, precision=32, seed=2, kT=1e-4, **MRT),
             dict(nx=20, ny=14, nz=14, precision=32, seed=3, gamma_bead=g, kT=1e-4, compensate_force=1, **MRT)]
    B = lb.LBBatch(cases)
    B.lb_batch_add_raspberry(0, sph, [8.2, 7.9, 6.1], [1, 0, 0, 0], 34.0, (50, 50, 50), (0, 0, 1e-3), None, False)
    B.lb_batch_add_raspberry(2, sph, [5.2, 7.1, 6.6], [1, 0, 0, 0], 34.0, (50, 50, 50), (1e-3, 0, 0), None, False)
    B.lb_batch_add_raspberry(2, sph, [14.6, 6.4, 8.1], [0.8, 0.6, 0, 0], 34.0, (50, 50, 50), None, None, False)
    every, cap = 2, 50
    B.lb_batch_record_bodies(every, cap)
    expect = {}
    step = 0

    def snapshot():
        for (i, b) in ((0, 0), (2, 0), (2, 1)):
            st = B.lb_batch_get_body(i, b)
            expect[(step, i, b)] = (st["X"].copy(), st["q"].copy())

    for k, chunk in enumerate((2, 4, 1, 3, 6, 2)):
        if k == 3:
            B.lb_batch_autotune(2)          # trial steps on a snapshot, restored
        if chunk % 2:                       # single eager steps
            for _ in range(chunk):
                B.lb_batch_step(1)
                step += 1
                if step % every == 0:
                    snapshot()
        else:                               # even step count from an even step: graph replays
            B.lb_batch_step(chunk)
            step += chunk
            snapshot()
    for (i, b) in ((0, 0), (2, 0), (2, 1)):
        steps, X, q = B.lb_batch_get_trajectory(i, b)
        assert len(steps) == step // every
        assert list(steps) == list(range(every, step + 1, every))
        for kk, s in enumerate(steps):
            if (s, i, b) in expect:
                Xg, qg = expect[(s, i, b)]
                assert np.array_equal(X[kk], Xg) and np.array_equal(q[kk], qg), (s, i, b)


@pytest.mark.parametrize("axis", [2, 0])
def test_pore_msd_matches_oracle(axis):
    """Binned pore-frame MSD of a random walk inside a pore: equal to the
    oracle's analysis of the same trajectory (bins decided identically:
    exact counts; sums to 1e-12)."""
    from paper_1604_01829_gb300 import lb
    rng = np.random.default_rng(7 + axis)
    shape = (40, 40, 60) if axis == 2 else (60, 40, 40)
    n, R = 600, 15.0
    X = np.empty((n, 3))
    X[0] = [s / 2 + 0.3 for s in shape]
    for k in range(1, n):
        X[k] = X[k - 1] + rng.normal(scale=0.5, size=3)
    got, cnt = lb.lb_pore_msd(X, shape, axis, R, 6, 40)
    ref, rcnt = A.pore_msd(X, shape, axis, R, 6, 40)
    assert np.array_equal(cnt, rcnt)
    assert np.allclose(got, ref, rtol=1e-12, atol=0)


def test_pore_msd_of_a_recorded_confined_trajectory():
    """A thermal sphere raspberry in a pore with repulsive wall beads, its
    centre recorded on the GPU every 5 steps, analysed by lb_pore_msd and by
    the oracle analysis: same result; and the colloid stays inside the pore."""
    from paper_1604_01829_gb300 import lb
    params = dict(MRT, kT=1e-3, seed=44, gamma_bead=Wl.paper_gamma_to_lattice(50.0), precision=32)
    h = lb.LB(24, 24, 32, **params)
    h.lb_set_pore(9.0, 2)
    h.lb_set_pore_beads(2.0, 2.5, 0.5, 1e-3)
    h.lb_add_raspberry(Wl.sphere_raspberry(2.0), [12.0 + 3.0, 12.0, 16.0], mass=34.0, inertia=(50, 50, 50),
                       F_ext=(5e-4, 0, 0))
    h.lb_record_bodies(5, 400)
    h.lb_step(2000)
    steps, X, q = h.lb_get_trajectory(0)
    assert len(steps) == 400
    r = np.hypot(X[:, 0] - 12, X[:, 1] - 12)
    assert r.max() < 9.0 - 2.0                         # the wall beads keep the sphere inside
    got, cnt = lb.lb_pore_msd(X, (24, 24, 32), 2, 9.0, 3, 20)
    ref, rcnt = A.pore_msd(X, (24, 24, 32), 2, 9.0, 3, 20)
    assert np.array_equal(cnt, rcnt)
    assert np.allclose(got, ref, rtol=1e-12, atol=0)
