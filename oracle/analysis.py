"""Trajectory analysis of rigid raspberries, written from the paper's
definitions (test infrastructure only: only ``tests/`` imports this module;
no code shared with the CUDA library).

Ustach & Faller (arXiv:1604.01829) measure transport from recorded centres
X_n and orientation quaternions q_n:

* lab-frame translation: squared displacements of X, Eq. (dt_lab);
* body-frame translation (Sec. 2.6, SI "Body-frame translational
  displacement"): the displacement over one interval, Eq. (labdisp), is
  rotated into the body frame with the inverse quaternion, Eq. (quat), the
  rotated displacements are summed into a body-frame trajectory,
  Eq. (bodyframedisplacement), whose lagged differences, Eq.
  (bodyframetrajectory), enter Eq. (dt_body);
* lab-frame rotation (Sec. 2.5): the angle between a body-fixed reference
  vector at t and at t + tau, Eq. (delta_theta);
* body-frame rotation (Sec. 2.7, SI "Body-frame angular displacement"): the
  rotation over one interval about body axis x^b_i is the angle of the
  projection of a second body axis onto the plane normal to x^b_i(t-1),
  measured in the frame of the body at t-1; the angles are summed, Eq.
  (bodyframerotdisplacement), and lagged, Eq. (bodyframerottrajectory).

Readings (silent or ambiguous points): the quaternion of Eq. (quat) is the
orientation at the start of the interval; the arctangents of the SI are
taken as atan2 of the same two components (equal below 90 degrees per
interval); the arccosine of Eq. (delta_theta) is evaluated as
atan2(|p x p'|, p . p'), the same angle, well conditioned at small angles.
The quaternion products use the oracle's Hamilton product.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O

COLS = 10


def quat_conj(q):
    return np.array([q[0], -q[1], -q[2], -q[3]])


def quat_rotate(q, v):
    """q (0, v) q^-1 for a unit quaternion: a body vector into the lab frame,
    Eq. (bodyframeunitvectorcalc)."""
    return O.quat_mul(O.quat_mul(q, np.array([0.0, v[0], v[1], v[2]])), quat_conj(q))[1:]


def quat_unrotate(q, v):
    """q^-1 (0, v) q: a lab vector into the body frame, Eq. (quat)."""
    return O.quat_mul(O.quat_mul(quat_conj(q), np.array([0.0, v[0], v[1], v[2]])), q)[1:]


def body_frame_trajectory(X, q):
    """X^b_n for n = 0..nrec-1 (X^b_0 = 0), Eqs. (labdisp), (quat),
    (bodyframedisplacement)."""
    n = len(X)
    Xb = np.zeros((n, 3))
    for k in range(1, n):
        dX = X[k] - X[k - 1]
        Xb[k] = Xb[k - 1] + quat_unrotate(q[k - 1], dX)
    return Xb


def body_frame_angles(q):
    """Theta_{x^b}, Theta_{y^b}, Theta_{z^b} summed over the intervals (SI
    projection method, Eq. (bodyframerotdisplacement)); Theta(0) = 0."""
    e = np.eye(3)
    n = len(q)
    th = np.zeros((n, 3))
    for k in range(1, n):
        prev = [quat_rotate(q[k - 1], e[a]) for a in range(3)]     # i, j, k at t-1
        cur = [quat_rotate(q[k], e[a]) for a in range(3)]          # i, j, k at t
        A = np.array(prev)                                          # rows: body axes at t-1
        d = np.zeros(3)
        # about x^b: project k_t onto the plane normal to i_{t-1}, angle from (P2, P3)
        kP = A @ (cur[2] - prev[0] * np.dot(cur[2], prev[0]))
        d[0] = np.arctan2(kP[1], kP[2])
        # about y^b: project i_t onto the plane normal to j_{t-1}, angle from (P3, P1)
        iP = A @ (cur[0] - prev[1] * np.dot(cur[0], prev[1]))
        d[1] = np.arctan2(iP[2], iP[0])
        # about z^b: project j_t onto the plane normal to k_{t-1}, angle from (P1, P2)
        jP = A @ (cur[1] - prev[2] * np.dot(cur[1], prev[2]))
        d[2] = np.arctan2(jP[0], jP[1])
        th[k] = th[k - 1] + d
    return th


def lab_angle(p0, p1):
    """Angle between two vectors, Eq. (delta_theta) (read as atan2)."""
    return np.arctan2(np.linalg.norm(np.cross(p0, p1)), np.dot(p0, p1))


def msd(X, q, max_lag, p_ref=(1.0, 0.0, 0.0)):
    """[max_lag, 10] for one body: columns 0-2 lab-frame, 3-5 body-frame
    squared displacements per axis, 6 squared lab-frame angle of p_ref,
    7-9 squared body-frame angles, each averaged over the nrec - l time
    origins of lag l = 1..max_lag."""
    X = np.asarray(X, float)
    q = np.asarray(q, float)
    n = len(X)
    Xb = body_frame_trajectory(X, q)
    th = body_frame_angles(q)
    p_ref = np.asarray(p_ref, float) / np.linalg.norm(p_ref)
    p = np.array([quat_rotate(q[k], p_ref) for k in range(n)])
    out = np.zeros((max_lag, COLS))
    for lag in range(1, max_lag + 1):
        m = n - lag
        out[lag - 1, 0:3] = np.mean((X[lag:] - X[:m]) ** 2, axis=0)
        out[lag - 1, 3:6] = np.mean((Xb[lag:] - Xb[:m]) ** 2, axis=0)
        out[lag - 1, 6] = np.mean([lab_angle(p[t], p[t + lag]) ** 2 for t in range(m)])
        out[lag - 1, 7:10] = np.mean((th[lag:] - th[:m]) ** 2, axis=0)
    return out


def diffusivities(msd_row, tau):
    """The paper's estimators at lag time tau: D_t (Eq. (dt_lab): summed
    lab-frame MSD over 6 tau), D_t per body axis (Eq. (dt_body): 2 tau),
    D_r (Eq. (dr_lab): 6 tau) and D_r per body axis (Eq. (dr_body): with
    the (3/2) 2 tau denominator)."""
    return dict(D_t=msd_row[0:3].sum() / (6 * tau), D_t_body=msd_row[3:6] / (2 * tau),
                D_r=msd_row[6] / (6 * tau), D_r_body=msd_row[7:10] / (3 * tau))


# ------------------------------------------------------------ pore frame
def pore_frame_trajectory(X, shape, axis=2):
    """Sec. 2.8 and the SI "Pore-frame coordinate determination": centres
    relative to the pore axis (x^c, y^c across it, z along it), the angle
    theta = arctan(y^c / x^c) (read as atan2), one interval's displacement
    rotated by P(theta) = [[cos, sin, 0], [-sin, cos, 0], [0, 0, 1]] with
    theta at the start of the interval (x^p radial, y^p azimuthal, z^p
    axial), summed from the first record, Eq. (poreframedisplacement).
    Returns (X^p [n, 3], radial coordinate r [n])."""
    X = np.asarray(X, float)
    a1, a2 = (1, 2) if axis == 0 else ((0, 2) if axis == 1 else (0, 1))
    xc = X[:, a1] - 0.5 * shape[a1]
    yc = X[:, a2] - 0.5 * shape[a2]
    zc = X[:, axis]
    n = len(X)
    Xp = np.zeros((n, 3))
    for k in range(1, n):
        th = np.arctan2(yc[k - 1], xc[k - 1])
        P = np.array([[np.cos(th), np.sin(th), 0.0], [-np.sin(th), np.cos(th), 0.0], [0.0, 0.0, 1.0]])
        dXc = np.array([xc[k] - xc[k - 1], yc[k] - yc[k - 1], zc[k] - zc[k - 1]])
        Xp[k] = Xp[k - 1] + P @ dXc
    # r = sqrt(x^2 + y^2) in this order of operations: the bin decisions
    # below depend on its last bit
    return Xp, np.sqrt(xc * xc + yc * yc)


def pore_msd(X, shape, axis, R_pore, nbins, max_lag):
    """Binned pore-frame MSD (Sec. 2.8): each record t is binned by its
    radial coordinate, bin = floor(r(t) / R_pore * nbins) (records with
    r >= R_pore are left out), and the sub-trajectory starting there adds
    (X^p(t + l) - X^p(t))^2 per pore-frame axis to that bin, Eq.
    (poreframetrajectory). Returns (msd [nbins, max_lag, 3] averaged over
    the origins in each bin, counts [nbins, max_lag])."""
    Xp, r = pore_frame_trajectory(X, shape, axis)
    n = len(Xp)
    out = np.zeros((nbins, max_lag, 3))
    cnt = np.zeros((nbins, max_lag), np.int64)
    for lag in range(1, max_lag + 1):
        for t in range(n - lag):
            b = int(np.floor(r[t] / R_pore * nbins))      # same operations as the GPU
            if b < 0 or b >= nbins:
                continue
            out[b, lag - 1] += (Xp[t + lag] - Xp[t]) ** 2
            cnt[b, lag - 1] += 1
    nz = cnt > 0
    out[nz] /= cnt[nz][:, None]
    return out, cnt
