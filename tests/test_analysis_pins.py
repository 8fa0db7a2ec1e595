"""Pins of the trajectory-analysis oracle (Sec. 2.4-2.7 and the SI of
Ustach & Faller, arXiv:1604.01829) to closed forms: uniform translation,
steady rotation about each body axis, motion along a body axis while the
body turns, invariance under a rotation of the lab frame, and the
statistics of a synthetic random walk."""
import math

import numpy as np
import pytest

from oracle import analysis as A
from oracle import oracle as O


def _axis_quat(axis, angle):
    q = np.zeros(4)
    q[0] = math.cos(angle / 2)
    q[1 + axis] = math.sin(angle / 2)
    return q


def _random_unit_quat(rng):
    q = rng.normal(size=4)
    return q / np.linalg.norm(q)


def test_uniform_translation():
    """X_n = X_0 + n v at fixed orientation: lab MSD (l v_a)^2, body MSD
    (l (R^T v)_a)^2, no rotation."""
    rng = np.random.default_rng(1)
    q0 = _random_unit_quat(rng)
    v = np.array([0.3, -0.2, 0.05])
    n, L = 40, 12
    X = np.array([[1.0, 2.0, 3.0]]) + np.arange(n)[:, None] * v
    q = np.tile(q0, (n, 1))
    out = A.msd(X, q, L)
    lags = np.arange(1, L + 1)[:, None]
    vb = O.rotation(q0).T @ v
    assert np.allclose(out[:, 0:3], (lags * v) ** 2, rtol=1e-12, atol=1e-15)
    assert np.allclose(out[:, 3:6], (lags * vb) ** 2, rtol=1e-12, atol=1e-15)
    assert np.allclose(out[:, 6:10], 0.0, atol=1e-24)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_steady_rotation_about_a_body_axis(axis):
    """q_n = q_0 (x) exp(n theta/2 e_axis): the body-frame angle about that
    axis changes by theta per record (the projection method's sign makes it
    -theta), the other two not at all; a reference vector normal to the
    axis turns by l theta."""
    rng = np.random.default_rng(2 + axis)
    q0 = _random_unit_quat(rng)
    th, n, L = 0.07, 60, 20
    q = np.array([O.quat_mul(q0, _axis_quat(axis, k * th)) for k in range(n)])
    X = np.zeros((n, 3))
    p_ref = np.zeros(3)
    p_ref[(axis + 1) % 3] = 1.0
    out = A.msd(X, q, L, p_ref)
    lags = np.arange(1, L + 1)
    ang = A.body_frame_angles(q)
    assert np.allclose(np.diff(ang[:, axis]), -th, rtol=1e-12)
    others = [a for a in range(3) if a != axis]
    assert np.allclose(ang[:, others], 0.0, atol=1e-13)
    assert np.allclose(out[:, 7 + axis], (lags * th) ** 2, rtol=1e-10)
    assert np.allclose(out[:, 6], (lags * th) ** 2, rtol=1e-10)
    assert np.allclose(out[:, 0:6], 0.0, atol=1e-24)


def test_motion_along_a_body_axis_of_a_turning_body():
    """Each interval moves the body by s along its own x axis at the start of
    the interval while it turns about z: the lab path is a polygon, the
    body-frame trajectory a straight line, (n s, 0, 0)."""
    s, th, n, L = 0.4, 0.2, 50, 15
    q = np.array([_axis_quat(2, k * th) for k in range(n)])
    X = np.zeros((n, 3))
    for k in range(1, n):
        X[k] = X[k - 1] + O.rotation(q[k - 1]) @ np.array([s, 0.0, 0.0])
    Xb = A.body_frame_trajectory(X, q)
    assert np.allclose(Xb, np.arange(n)[:, None] * np.array([s, 0.0, 0.0]), atol=1e-12)
    out = A.msd(X, q, L)
    lags = np.arange(1, L + 1)
    assert np.allclose(out[:, 3], (lags * s) ** 2, rtol=1e-12)
    assert np.allclose(out[:, 4:6], 0.0, atol=1e-24)
    assert out[-1, 0:3].sum() < (L * s) ** 2 * 0.9           # the lab path is not straight


def test_invariance_under_a_rotation_of_the_lab_frame():
    """Rotating every centre and orientation by one lab rotation Q leaves
    the body-frame columns and the lab angle unchanged and the summed
    lab-frame MSD too."""
    rng = np.random.default_rng(9)
    n, L = 80, 25
    X = np.cumsum(rng.normal(scale=0.3, size=(n, 3)), axis=0)
    q = [_random_unit_quat(rng)]
    for _ in range(n - 1):
        dq = np.concatenate([[1.0], rng.normal(scale=0.05, size=3)])
        q.append(O.quat_mul(q[-1], dq / np.linalg.norm(dq)))
    q = np.array(q)
    Q = _random_unit_quat(rng)
    RQ = O.rotation(Q)
    X2 = X @ RQ.T
    q2 = np.array([O.quat_mul(Q, qq) for qq in q])
    a, b = A.msd(X, q, L, (0.3, 0.5, 0.8)), A.msd(X2, q2, L, (0.3, 0.5, 0.8))
    assert np.allclose(a[:, 3:10], b[:, 3:10], rtol=1e-10, atol=1e-14)
    assert np.allclose(a[:, 0:3].sum(1), b[:, 0:3].sum(1), rtol=1e-12)


def test_random_walk_statistics():
    """A Gaussian random walk of variance sigma^2 per axis and record, at
    fixed orientation: MSD per axis = l sigma^2 within sampling error, in
    the lab and in the body frame; and the paper's estimator gives
    D_t = sigma^2 / 2."""
    rng = np.random.default_rng(4)
    sig, n, L = 0.5, 20000, 5
    X = np.cumsum(rng.normal(scale=sig, size=(n, 3)), axis=0)
    q = np.tile(_random_unit_quat(rng), (n, 1))
    out = A.msd(X, q, L)
    lags = np.arange(1, L + 1)[:, None]
    assert np.allclose(out[:, 0:3] / (lags * sig ** 2), 1.0, atol=0.05)
    assert np.allclose(out[:, 3:6] / (lags * sig ** 2), 1.0, atol=0.05)
    D = A.diffusivities(out[0], 1.0)
    assert D["D_t"] == pytest.approx(sig ** 2 / 2, rel=0.05)


def test_lab_angle_equals_arccos_of_unit_vectors():
    """The atan2 form used for Eq. (delta_theta) is the printed arccosine of
    the dot product of the unit vectors."""
    rng = np.random.default_rng(5)
    for _ in range(50):
        a, b = rng.normal(size=3), rng.normal(size=3)
        ref = math.acos(np.dot(a, b) / np.linalg.norm(a) / np.linalg.norm(b))
        assert A.lab_angle(a, b) == pytest.approx(ref, rel=1e-12, abs=1e-12)


# ---------------------------------------------------------------- pore frame
SHAPE = (40, 40, 60)


def test_pore_frame_radial_motion():
    """Motion along a fixed radial direction: all of it is x^p (radial)."""
    phi, dr, n = 0.7, 0.05, 30
    r = 3.0 + dr * np.arange(n)
    X = np.stack([20 + r * np.cos(phi), 20 + r * np.sin(phi), np.full(n, 5.0)], axis=1)
    Xp, rr = A.pore_frame_trajectory(X, SHAPE, 2)
    assert np.allclose(Xp[:, 0], dr * np.arange(n), atol=1e-12)
    assert np.allclose(Xp[:, 1:], 0.0, atol=1e-12)
    assert np.allclose(rr, r, rtol=1e-12)


def test_pore_frame_circular_and_axial_motion():
    """Uniform circular motion at radius rho, dphi per record, plus a constant
    axial step: every interval adds (rho (cos dphi - 1), rho sin dphi, dz) in
    the frame of its start, so the MSD at lag l is l^2 times their squares."""
    rho, dphi, dz, n, L = 6.6, 0.05, 0.02, 200, 10
    k = np.arange(n)
    X = np.stack([20 + rho * np.cos(dphi * k), 20 + rho * np.sin(dphi * k), 30 + dz * k], axis=1)
    msd, cnt = A.pore_msd(X, SHAPE, 2, 12.0, 4, L)
    lags = np.arange(1, L + 1)[:, None]
    step = np.array([rho * (np.cos(dphi) - 1), rho * np.sin(dphi), dz])
    b = int(rho / 12.0 * 4)
    assert np.allclose(msd[b], (lags * step) ** 2, rtol=1e-10)
    assert np.array_equal(cnt[b], n - lags[:, 0])
    assert np.all(cnt[[i for i in range(4) if i != b]] == 0)


def test_pore_frame_bins_and_axes():
    """Binning by the radial coordinate at the start of each sub-trajectory:
    counts add up to the origins inside the pore; a pore along x uses (y, z)
    across it and x along it."""
    rng = np.random.default_rng(3)
    n, L, R = 400, 6, 15.0
    X = np.empty((n, 3))
    X[0] = [20.0, 20.0, 20.0]
    for k in range(1, n):
        X[k] = X[k - 1] + rng.normal(scale=0.4, size=3)
    r = np.hypot(X[:, 0] - 20, X[:, 1] - 20)
    msd, cnt = A.pore_msd(X, SHAPE, 2, R, 5, L)
    for lag in range(1, L + 1):
        assert cnt[:, lag - 1].sum() == np.sum(r[: n - lag] < R)
    # the same walk with the pore along x: swap the roles of the coordinates
    Xx = X[:, [2, 0, 1]]
    msd_x, cnt_x = A.pore_msd(Xx, (60, 40, 40), 0, R, 5, L)
    assert np.array_equal(cnt, cnt_x)
    assert np.allclose(msd, msd_x, rtol=1e-12, atol=1e-15)
