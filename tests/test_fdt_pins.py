"""Fluctuation-dissipation pin of the bead noise (Sec. 1.1, Eq.
(latticeboltzmannfriction): the random bead force f_s obeys the
fluctuation-dissipation theorem), on the oracle.

Free raspberries in a thermal fluid (fluctuating MRT, Sec. 1.1) exchange
momentum with it only through the bead friction; the bead noise has to put
back what the friction takes out. At equilibrium every body then carries
kT per degree of freedom: <M V_a^2> = kT (a = x, y, z) and, for a body that
can turn, <I_k w_k^2> = kT about each principal axis k (equipartition of
the coupled fluid + colloid system).

The bodies here are point-like (one bead, or six beads 0.6 apart), with
bead friction small against the fluid's own resistance to a point force
(about 25 eta a for trilinear coupling), so the bead noise supplies most of
a body's thermal forcing: a wrong amplitude moves the measured temperature
far from kT. Measured on this set-up with deliberately wrong amplitudes
(not kept): sqrt(kT gamma/dt) (factor 2 missing) gives 0.53 kT,
gamma sqrt(2 kT/dt) (gamma for sqrt(gamma)) 0.29 kT, sqrt(2 kT gamma)
with two MD substeps (1/dt missing) 0.54 kT.

Bound: 5 % of kT. The statistical error of each estimate (batch means
over 20 blocks) is 0.7-1.4 %, and the time discretisation of the coupling
(explicit drag, the fluid updated once per LB step while the bodies take
one or two MD substeps) leaves a bias of at most ~3 % in these runs.
Runs are seeded (Philox counter noise), so the numbers are reproducible.
"""
import numpy as np
import pytest

from oracle import oracle as O

THERMAL = dict(collision=1, gamma_shear=0.0, gamma_bulk=0.0, gamma_odd=0.0, gamma_even=0.0, kT=1e-4)
OCTAHEDRON = 0.6 * np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)


def equipartition(L, nbodies, beads, gamma, mass, inertia, nsub=1, steps=6000, burn=400, seed=7):
    """Runs nbodies free bodies at seeded positions in a thermal L^3 box and
    returns (T_trans, T_rot, sigma_trans, sigma_rot): <M V^2>/kT and
    <I w^2>/kT over bodies, components and steps after `burn`, with the
    standard errors of 20 batch means."""
    p = dict(THERMAL, seed=seed, gamma_bead=gamma, md_substeps=nsub)
    kT = p["kT"]
    o = O.OracleLB(L, L, L, **p)
    rng = np.random.default_rng(seed)
    for _ in range(nbodies):
        o.add_raspberry(beads, rng.uniform(0, L, 3), (1, 0, 0, 0), mass, (inertia,) * 3)
    o.step(burn)
    V2, W2 = [], []
    for _ in range(steps):
        o.step(1)
        V2.append(o._packed["V"] ** 2)
        W2.append(o._packed["w"] ** 2)
    nblk = 20

    def stat(a, m):
        a = np.asarray(a)[: steps // nblk * nblk] * m / kT
        blk = a.reshape(nblk, -1).mean(axis=1)
        return blk.mean(), blk.std(ddof=1) / np.sqrt(nblk)

    t, st = stat(V2, mass)
    r, sr = stat(W2, inertia)
    return t, r, st, sr


@pytest.mark.parametrize("nsub", [1, 2])
def test_point_colloids_take_the_fluid_temperature(nsub):
    """Six one-bead bodies (M = 1, gamma = 0.25) in a thermal 10^3 box: with
    one and with two MD substeps per LB step (the paper's ratio, noise
    variance 2 kT gamma / dt per substep)."""
    t, _, st, _ = equipartition(10, 6, np.zeros((1, 3)), 0.25, 1.0, 1.0, nsub=nsub)
    assert st < 0.0125, st
    assert abs(t - 1.0) < 0.05, (t, st)


def test_a_small_raspberry_takes_the_fluid_temperature_in_translation_and_rotation():
    """Four six-bead octahedral bodies (radius 0.6, gamma = 0.08, M = 2,
    I = 0.4): translation and rotation about every body axis at kT."""
    t, r, st, sr = equipartition(10, 4, OCTAHEDRON, 0.08, 2.0, 0.4)
    assert st < 0.015 and sr < 0.015, (st, sr)
    assert abs(t - 1.0) < 0.05, (t, st)
    assert abs(r - 1.0) < 0.05, (r, sr)


def test_the_temperature_does_not_depend_on_the_bead_friction():
    """Fluctuation-dissipation fixes the noise variance in proportion to the
    friction, so the colloid's temperature is kT for any gamma: a ten times
    smaller gamma = 0.025 (M = 0.25, so that the velocity still decorrelates
    within ~10 steps) gives kT as well. An amplitude with gamma in place of
    sqrt(gamma) would give about gamma kT here."""
    t, _, st, _ = equipartition(10, 6, np.zeros((1, 3)), 0.025, 0.25, 1.0)
    assert st < 0.015, st
    assert abs(t - 1.0) < 0.05, (t, st)
