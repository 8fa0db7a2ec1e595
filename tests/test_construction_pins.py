"""Pins of the raspberry-construction oracle (oracle/construction.py) to what
geometry and mechanics fix: closed-form nearest surface points, brute-force
minimum distance over a dense surface grid, the normal condition of Eq.
(xtoxs), forces as minus the gradient of their potentials, the symmetric
fixed point, the optimal 2/4/6-point arrangements on a sphere and monotone
energy decrease of the damped (steepest-descent) scheme."""
import math

import numpy as np
import pytest

from oracle import construction as C


def _surface(ax, T, P):
    return np.stack([ax[0] * np.sin(T) * np.cos(P), ax[1] * np.sin(T) * np.sin(P), ax[2] * np.cos(T)], -1)


def _brute_min_distance(ax, p, n_t=400, n_p=800, n_ref=201):
    """Minimum distance from p to the surface over a (theta, phi) grid, then
    over a 100x finer grid around the best coarse point."""
    th = (np.arange(n_t) + 0.5) * math.pi / n_t
    ph = np.arange(n_p) * 2 * math.pi / n_p
    T, P = np.meshgrid(th, ph, indexing="ij")
    d = np.sqrt(((_surface(ax, T, P) - p) ** 2).sum(-1))
    i, j = np.unravel_index(np.argmin(d), d.shape)
    dt, dp = math.pi / n_t, 2 * math.pi / n_p
    T, P = np.meshgrid(th[i] + np.linspace(-2, 2, n_ref) * dt, ph[j] + np.linspace(-2, 2, n_ref) * dp, indexing="ij")
    return np.sqrt(((_surface(ax, T, P) - p) ** 2).sum(-1)).min()


def test_sphere_projection_is_radial():
    R = 2.5
    rng = np.random.default_rng(3)
    for _ in range(20):
        r = rng.normal(size=3) * rng.uniform(0.3, 2.0)
        rs, t = C.surface_point(r, [R, R, R])
        n = np.linalg.norm(r)
        assert np.allclose(rs, R * r / n, atol=1e-13)
        assert abs(t - R * (n - R)) < 1e-12


def test_axis_points_and_surface_points():
    ax = np.array([4.0, 2.0, 1.5])
    rs, t = C.surface_point([5.0, 0.0, 0.0], ax)        # outside, on the long axis
    assert np.allclose(rs, [4.0, 0.0, 0.0], atol=1e-14) and abs(t - 4.0 * (5.0 - 4.0)) < 1e-12
    rs, t = C.surface_point([0.0, 0.0, -3.0], ax)       # outside, on the short axis
    assert np.allclose(rs, [0.0, 0.0, -1.5], atol=1e-14) and abs(t - 1.5 * 1.5) < 1e-12
    rng = np.random.default_rng(4)
    for _ in range(20):                                  # points on the surface are their own
        u = rng.normal(size=3)
        p = ax * u / np.linalg.norm(u)
        p = p / math.sqrt(((p / ax) ** 2).sum())
        rs, t = C.surface_point(p, ax)
        assert np.allclose(rs, p, atol=1e-13) and abs(t) < 1e-12


@pytest.mark.parametrize("ax", [(4.0, 2.0, 1.5), (6.0, 2.0, 2.0), (1.5, 3.0, 3.0)])
def test_nearest_point_by_brute_force_and_normal_condition(ax):
    ax = np.array(ax)
    rng = np.random.default_rng(5)
    for _ in range(12):
        u = rng.normal(size=3)
        p = ax * u / np.linalg.norm(u)
        p = p / math.sqrt(((p / ax) ** 2).sum()) * rng.uniform(0.75, 1.3)   # inside and outside
        rs, t = C.surface_point(p, ax)
        assert abs(((rs / ax) ** 2).sum() - 1.0) < 1e-12                    # on the surface
        d = np.linalg.norm(p - rs)
        dmin = _brute_min_distance(ax, p)
        assert d <= dmin + 1e-12 and d >= dmin - 1e-6, (d, dmin)            # nearest, to grid resolution
        g = rs / ax ** 2                                                     # grad S / 2 at r_s
        assert np.linalg.norm(np.cross(p - rs, g)) < 1e-10 * max(1.0, d)     # r - r_s along the normal
        assert np.allclose(p, rs * (t / ax ** 2 + 1.0), atol=1e-12)          # Eq. (xtoxs)
        assert abs(C.bisection_function(t, p, ax)) < 1e-6                    # the paper's tolerance


def test_vectorised_forms_equal_the_per_bead_forms():
    ax = np.array([3.0, 2.0, 1.5])
    rng = np.random.default_rng(9)
    X = rng.normal(size=(30, 3)) * 1.5
    P = C.surface_points(X, ax)
    for i in range(len(X)):
        assert np.array_equal(P[i], C.surface_point(X[i], ax)[0])
    F = C.forces(X, ax, 1000.0, 1.4, 0.1)
    for i in range(len(X)):
        f = -2000.0 * (X[i] - P[i])
        for j in range(len(X)):
            if j != i:
                f = f + C.wca_force(X[i] - X[j], 1.4, 0.1)
        assert np.allclose(F[i], f, rtol=1e-13, atol=1e-13)


def test_printed_bisection_function_is_inconsistent():
    """Reading check: with the '+1' inside the squares, as printed, the exact
    nearest point's t does not solve the equation; without it, it does."""
    ax = np.array([3.0, 2.0, 1.0])
    p = np.array([3.5, 0.7, 0.2])
    rs, t = C.surface_point(p, ax)
    printed = sum((p[k] * ax[k] / (t + ax[k] ** 2) + 1.0) ** 2 for k in range(3)) - 1.0
    assert abs(printed) > 0.5 and abs(C.bisection_function(t, p, ax)) < 1e-12


def test_forces_are_minus_gradients():
    sig, eps, k = 1.4, 0.1, 1000.0
    rng = np.random.default_rng(6)
    h = 1e-6
    for _ in range(10):
        d = rng.normal(size=3)
        d *= rng.uniform(1.05, 1.5) / np.linalg.norm(d)
        F = C.wca_force(d, sig, eps)
        num = np.array([-(C.wca_energy(np.dot(d + h * e, d + h * e), sig, eps)
                          - C.wca_energy(np.dot(d - h * e, d - h * e), sig, eps)) / (2 * h) for e in np.eye(3)])
        assert np.allclose(F, num, rtol=1e-6, atol=1e-8)
    rc = C.WCA_CUT * sig
    assert abs(C.wca_energy(rc * rc * (1 - 1e-12), sig, eps)) < 1e-9
    assert not C.wca_force(np.array([rc, 0, 0]), sig, eps).any()
    ax = np.array([3.0, 2.0, 1.5])
    for _ in range(10):
        p = rng.normal(size=3) * 2.0
        rs, _ = C.surface_point(p, ax)
        U = lambda q: k * float(np.sum((q - C.surface_point(q, ax)[0]) ** 2))
        num = np.array([-(U(p + 1e-5 * e) - U(p - 1e-5 * e)) / 2e-5 for e in np.eye(3)])
        assert np.allclose(-2 * k * (p - rs), num, rtol=1e-5, atol=1e-6)


def test_symmetric_axis_configuration_stays_on_the_axes():
    ax = np.array([2.0, 1.2, 0.9])
    X0 = np.array([[ax[0], 0, 0], [-ax[0], 0, 0], [0, ax[1], 0], [0, -ax[1], 0], [0, 0, ax[2]], [0, 0, -ax[2]]])
    X = C.relax_shell(X0, ax, 200, dt=0.01, eta=100.0, project_final=False)
    for i in range(6):
        off = [q for q in range(3) if q != i // 2]
        assert np.all(np.abs(X[i, off]) < 1e-15)
        assert np.sign(X[i, i // 2]) == np.sign(X0[i, i // 2])
    assert np.allclose(X[0], -X[1], atol=1e-15) and np.allclose(X[2], -X[3], atol=1e-15)


@pytest.mark.parametrize("n,edge_over_R", [(2, 2.0), (4, math.sqrt(8.0 / 3.0)), (6, math.sqrt(2.0))])
def test_optimal_arrangements_on_a_small_sphere(n, edge_over_R):
    """All pairs within the WCA range on a sphere of radius 0.6: 2 beads end
    antipodal, 4 a regular tetrahedron, 6 a regular octahedron."""
    R = 0.6
    rng = np.random.default_rng(7 + n)
    u = rng.normal(size=(n, 3))
    X0 = R * u / np.linalg.norm(u, axis=1)[:, None]
    X = C.relax_shell(X0, [R, R, R], 4000, dt=0.01, eta=100.0)
    d = np.sqrt(((X[:, None] - X[None]) ** 2).sum(-1))
    nn = np.sort(d + np.eye(n) * 10, axis=1)[:, 0]
    assert np.allclose(nn, edge_over_R * R, atol=2e-6), nn
    assert np.allclose(np.linalg.norm(X, axis=1), R, atol=1e-13)
    if n == 6:
        assert np.allclose(np.sort(d, axis=1)[:, -1], 2 * R, atol=2e-6)


def test_damped_scheme_descends_the_energy():
    ax = np.array([3.0, 1.8, 1.8])
    rng = np.random.default_rng(8)
    u = rng.normal(size=(24, 3))
    X = ax * u / np.linalg.norm(u, axis=1)[:, None] * 1.05
    k, sig, eps = 1000.0, 1.4, 0.1
    E = [C.energy(X, ax, k, sig, eps)]
    for _ in range(15):
        X = C.relax_shell(X, ax, 4, k, sig, eps, dt=1e-3, eta=1000.0, project_final=False)
        E.append(C.energy(X, ax, k, sig, eps))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(E, E[1:])), E
    assert E[-1] < 0.5 * E[0]
