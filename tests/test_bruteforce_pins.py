"""Brute-force pin of the oracle's whole coupled step on tiny lattices.

A 4^3 (and a 6x6x4 pore) lattice with one raspberry, stepped ten times by
the oracle and, side by side, by an independent evaluation written here from
the definitions alone, in forms the oracle does not use:

- D3Q19 weights solved from the isotropy conditions (sum w = 1,
  sum w c_x^2 = c_s^2, sum w c_x^2 c_y^2 = c_s^4), populations matched to the
  oracle's by their velocity vector;
- equilibrium and Guo source as Hermite reconstructions of their moments
  (Sec. 1.1 Maxwell-Boltzmann relaxation; density, momentum and second moment
  rho c_s^2 I + rho u u, resp. 0, F and u F + F u);
- the multiple-relaxation-time collision without a moment basis: the
  hydrodynamic part rebuilt from the relaxed momentum and stress (shear and
  bulk parts of the stress with their own rates), the kinetic (ghost) part
  of f - f_eq found as the residual of that projection and split by velocity
  parity into its odd and even modes, each scaled by its rate;
- trilinear interpolation weights from solving the 8x8 multilinear
  interpolation conditions at the cell's corners (Eq. (latticeboltzmannfriction):
  u interpolated between the nearest grid points);
- bead positions by the quaternion sandwich product q (0, s) q^-1 (Sec. 1.2);
- streaming as a pull from upstream nodes, with halfway bounce-back at
  wall nodes (Sec. 1.1, Sec. 2.3), where the oracle pushes.

A dropped term, a wrong sign or index, a transposed weight or a wrong rate
in any part of the oracle's step moves some population or force by far more
than the 1e-13 (relative to w_i rho0) allowed here for two FP64 evaluations
in different orders. The thermal noise is left out (kT = 0): its amplitudes
are pinned by equipartition in test_oracle_pins.py.
"""
import itertools

import numpy as np
import pytest

from oracle import oracle as O

CS2 = 1.0 / 3.0


# ------------------------------------------------------------------ lattice

def d3q19():
    """Velocities with |c|^2 <= 2, weights per shell from the isotropy
    conditions, the velocity-reversal map."""
    vel = np.array([c for c in itertools.product((-1, 0, 1), repeat=3) if sum(x * x for x in c) <= 2])
    shell = (vel * vel).sum(1)
    # unknowns w0, w1, w2 (per velocity of shell |c|^2 = 0, 1, 2)
    cond = np.zeros((3, 3))
    rhs = np.array([1.0, CS2, CS2 * CS2])
    for s in range(3):
        sel = vel[shell == s]
        cond[0, s] = len(sel)
        cond[1, s] = (sel[:, 0] ** 2).sum()
        cond[2, s] = (sel[:, 0] ** 2 * sel[:, 1] ** 2).sum()
    wshell = np.linalg.solve(cond, rhs)
    w = wshell[shell]
    rev = np.array([int(np.where((vel == -c).all(1))[0][0]) for c in vel])
    return vel, w, rev


C, W, REV = d3q19()
Q = len(C)
OC, OW, _ = O.lattice()
# oracle index k holds the velocity of our index PERM[k]
PERM = np.array([int(np.where((C == oc).all(1))[0][0]) for oc in OC])


def to_oracle(f):
    return f[PERM]


def from_oracle(fo):
    f = np.empty_like(fo)
    f[PERM] = fo
    return f


# ------------------------------------------------------- per-node collision

def hermite(rho, j, Pi):
    """Populations with density rho, momentum j and second moment Pi and no
    kinetic (ghost) content: w_i [rho + j.c/cs2 + (Pi - rho cs2 I):(c c - cs2 I)/(2 cs2^2)].
    rho: (N,), j: (N,3), Pi: (N,3,3); returns (Q,N)."""
    cc = np.einsum("ia,ib->iab", C, C) - CS2 * np.eye(3)[None]
    A = Pi - rho[:, None, None] * CS2 * np.eye(3)[None]
    return W[:, None] * (rho[None, :] + (j @ C.T).T / CS2
                         + np.einsum("iab,nab->in", cc, A) / (2 * CS2 * CS2))


def moments(f):
    rho = f.sum(0)
    j = (C.T @ f).T
    Pi = np.einsum("ia,ib,in->nab", C, C, f)
    return rho, j, Pi


def equilibrium(rho, u):
    return hermite(rho, rho[:, None] * u, rho[:, None, None] * (CS2 * np.eye(3)[None] + np.einsum("na,nb->nab", u, u)))


def split_trace(A):
    tr = np.trace(A, axis1=1, axis2=2)[:, None, None] / 3.0 * np.eye(3)[None]
    return A - tr, tr


def collide(f, F, p):
    """One collision of every node with Guo forcing; f (Q,N), F (N,3)."""
    rho, j, Pi = moments(f)
    u = (j + 0.5 * F) / rho[:, None]
    feq = equilibrium(rho, u)
    Psi = np.einsum("na,nb->nab", u, F) + np.einsum("na,nb->nab", F, u)
    if p["collision"] == 0:
        tau = p["tau"]
        S = hermite(np.zeros_like(rho), F, Psi)
        return f - (f - feq) / tau + (1.0 - 0.5 / tau) * S
    gs, gb, go, ge = p["gamma_shear"], p["gamma_bulk"], p["gamma_odd"], p["gamma_even"]
    Pi_eq = rho[:, None, None] * (CS2 * np.eye(3)[None] + np.einsum("na,nb->nab", u, u))
    neq_s, neq_b = split_trace(Pi - Pi_eq)
    Psi_s, Psi_b = split_trace(Psi)
    Pi_post = Pi_eq + gs * neq_s + gb * neq_b + 0.5 * (1 + gs) * Psi_s + 0.5 * (1 + gb) * Psi_b
    hydro = hermite(rho, j + F, Pi_post)
    d = f - feq
    ghost = d - hermite(*moments(d))
    g_odd = 0.5 * (ghost - ghost[REV])
    g_even = 0.5 * (ghost + ghost[REV])
    return hydro + go * g_odd + ge * g_even


# ----------------------------------------------------------------- geometry

def node_index(x, y, z, dims):
    nx, ny, nz = dims
    return (x % nx) + nx * ((y % ny) + ny * (z % nz))


def wall_mask(dims, R, axis):
    """Wall node: centre (integer + 1/2) at distance >= R from the axis
    through the box centre (Sec. 2.3)."""
    nx, ny, nz = dims
    m = np.zeros(nx * ny * nz, bool)
    others = [a for a in range(3) if a != axis]
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                r = np.array([x, y, z]) + 0.5
                d2 = sum((r[a] - dims[a] / 2.0) ** 2 for a in others)
                m[node_index(x, y, z, dims)] = d2 >= R * R
    return m


def stream_pull(fpost, dims, wall):
    nx, ny, nz = dims
    N = nx * ny * nz
    out = fpost.copy()
    for n in range(N):
        if wall is not None and wall[n]:
            continue
        x, y, z = n % nx, (n // nx) % ny, n // (nx * ny)
        for i in range(Q):
            up = node_index(x - C[i, 0], y - C[i, 1], z - C[i, 2], dims)
            if wall is not None and wall[up]:
                out[i, n] = fpost[REV[i], n]
            else:
                out[i, n] = fpost[i, up]
    return out


# ------------------------------------------------------------------- beads

def qmul(a, b):
    w1, v1 = a[0], np.asarray(a[1:])
    w2, v2 = b[0], np.asarray(b[1:])
    return np.concatenate([[w1 * w2 - v1 @ v2], w1 * v2 + w2 * v1 + np.cross(v1, v2)])


def rotate(q, s):
    qc = np.array([q[0], -q[1], -q[2], -q[3]])
    return qmul(qmul(q, np.concatenate([[0.0], s])), qc)[1:]


def corner_weights(r):
    """The 8 nodes around r (centres at integer + 1/2) and the weights that
    reproduce 1, x, y, z, xy, yz, zx, xyz at r exactly."""
    base = np.floor(r - 0.5).astype(int)
    corners = [base + np.array(o) for o in itertools.product((0, 1), repeat=3)]
    P = np.array([c + 0.5 for c in corners])

    def basis(p):
        x, y, z = p
        return [1.0, x, y, z, x * y, y * z, z * x, x * y * z]

    A = np.array([basis(p) for p in P]).T
    w = np.linalg.solve(A, np.array(basis(r)))
    return corners, w


class Brute:
    """The coupled step evaluated from the definitions above."""

    def __init__(self, dims, p, f, wall=None):
        self.dims, self.p, self.f, self.wall = dims, p, f.copy(), wall
        self.N = int(np.prod(dims))
        self.Fprev = np.zeros((self.N, 3))
        self.bodies = []

    def add_body(self, s, X, q, V, w, mass, F_ext, T_ext, fixed):
        self.bodies.append(dict(s=np.asarray(s, float).reshape(-1, 3), X=np.array(X, float),
                                q=np.array(q, float) / np.linalg.norm(q), V=np.array(V, float),
                                w=np.array(w, float), M=mass, F_ext=np.array(F_ext, float),
                                T_ext=np.array(T_ext, float), fixed=fixed, F_last=np.zeros(3)))

    def step(self):
        p, N = self.p, self.N
        fluid = np.ones(N, bool) if self.wall is None else ~self.wall
        g = np.array(p.get("body_force", (0, 0, 0)), float)
        if p.get("compensate_force", 0):
            for b in self.bodies:
                if b["fixed"] != 1:
                    g = g - b["F_ext"] / fluid.sum()
        for b in self.bodies:                          # first half kick and drift (translation only)
            if b["fixed"] == 2:
                b["V"] = b["V"] + 0.5 * b["F_last"] / b["M"]
                b["X"] = b["X"] + b["V"]
                b["w"] = np.zeros(3)
        rho, j, _ = moments(self.f)
        u = (j + 0.5 * (g[None, :] + self.Fprev)) / rho[:, None]
        Fnew = np.zeros((N, 3))
        self.bead_F = []
        for b in self.bodies:
            w_lab = rotate(b["q"], b["w"])
            Ft, Tt = b["F_ext"].copy(), b["T_ext"].copy()
            for s in b["s"]:
                rel = rotate(b["q"], s)
                r = b["X"] + rel
                v = b["V"] + np.cross(w_lab, rel)
                corners, wt = corner_weights(r)
                idx = [node_index(*c, self.dims) for c in corners]
                ub = sum(wk * (u[n] if fluid[n] else 0.0) for wk, n in zip(wt, idx))
                Fb = -p["gamma_bead"] * (v - ub)
                for wk, n in zip(wt, idx):
                    if fluid[n]:
                        Fnew[n] -= wk * Fb
                self.bead_F.append(Fb)
                Ft += Fb
                Tt += np.cross(rel, Fb)
            b["F"], b["T"] = Ft, Tt
        fpost = collide(self.f, g[None, :] + Fnew, p)
        if self.wall is not None:
            fpost[:, self.wall] = self.f[:, self.wall]
        self.f = stream_pull(fpost, self.dims, self.wall)
        self.Fprev = Fnew
        for b in self.bodies:                          # second half kick
            if b["fixed"] == 2:
                b["V"] = b["V"] + 0.5 * b["F"] / b["M"]
            b["F_last"] = b["F"]


def _start(dims, seed):
    """Seeded populations near equilibrium, in our own velocity order."""
    rng = np.random.default_rng(seed)
    N = int(np.prod(dims))
    rho = 1.0 + 0.05 * rng.standard_normal(N)
    u = 0.03 * rng.standard_normal((N, 3))
    f = equilibrium(rho, u) * (1 + 0.02 * rng.standard_normal((Q, N)))
    return f


def _run(dims, p, bodies, pore=None, steps=10, seed=0):
    f0 = _start(dims, seed)
    wall = None if pore is None else wall_mask(dims, *pore)
    brute = Brute(dims, p, f0, wall)
    orc = O.OracleLB(*dims, **{k: v for k, v in p.items()})
    if pore is not None:
        orc.set_pore(*pore)
        assert np.array_equal(orc.mask.astype(bool), wall)
    orc.set_populations(to_oracle(f0))
    for b in bodies:
        brute.add_body(**b)
        orc.add_raspberry(b["s"], b["X"], np.asarray(b["q"]) / np.linalg.norm(b["q"]), b["mass"], (1, 1, 1),
                          b["F_ext"], b["T_ext"], b["fixed"], V=b["V"], w=b["w"])
    fluid = np.ones(brute.N, bool) if wall is None else ~wall
    worst = 0.0
    for k in range(steps):
        brute.step()
        orc.step(1)
        fo = from_oracle(orc.populations())
        err = np.max(np.abs(fo[:, fluid] - brute.f[:, fluid]) / W[:, None])
        worst = max(worst, err)
        assert err <= 1e-13, (k, err)
        bead_o = np.concatenate([orc.bead_forces(i) for i in range(len(bodies))])
        bead_b = np.array(brute.bead_F)
        scale = np.abs(bead_b).max()
        assert scale > 1e-6                            # the coupling does act
        assert np.abs(bead_o - bead_b).max() <= 1e-12 * scale, k
        for i, b in enumerate(brute.bodies):
            ob = orc.body(i)
            assert np.abs(ob["F"] - b["F"]).max() <= 1e-12 * max(scale, np.abs(b["F"]).max())
            assert np.abs(ob["T"] - b["T"]).max() <= 1e-12 * max(scale, np.abs(b["T"]).max())
            assert np.abs(ob["X"] - b["X"]).max() <= 1e-13 and np.abs(ob["V"] - b["V"]).max() <= 1e-14
    return worst


BODY_FIXED = dict(s=[[0.0, 0.0, 0.0]], X=[2.13, 1.71, 2.46], q=[1, 0, 0, 0], V=[2e-3, -1e-3, 3e-3],
                  w=[0, 0, 0], mass=5.0, F_ext=[0, 0, 0], T_ext=[0, 0, 0], fixed=1)
# three beads off the centre of a rotating (held) body: v = V + w x r
BODY_SPIN = dict(s=[[0.6, -0.2, 0.3], [-0.4, 0.5, -0.1], [0.1, 0.2, -0.7]], X=[1.62, 2.37, 2.05],
                 q=[0.9, 0.2, -0.3, 0.25], V=[1e-3, 2e-3, -1e-3], w=[3e-3, -2e-3, 4e-3], mass=5.0,
                 F_ext=[1e-4, 0, -2e-4], T_ext=[0, 1e-4, 0], fixed=1)
# translating body (velocity Verlet), pulled with the compensating drive
BODY_FREE = dict(s=[[0.3, 0.2, -0.4], [-0.3, -0.1, 0.2]], X=[2.3, 1.9, 1.55], q=[0.7, -0.1, 0.6, 0.3],
                 V=[0, 1e-3, 0], w=[0, 0, 0], mass=3.0, F_ext=[2e-3, -1e-3, 1.5e-3], T_ext=[0, 0, 0], fixed=2)


def test_weights_solve_the_isotropy_conditions():
    assert Q == 19
    assert np.allclose(np.sort(W), np.sort(OW), rtol=0, atol=1e-15)
    assert np.allclose(W[PERM], OW, rtol=0, atol=1e-15)


@pytest.mark.parametrize("tau", [0.8, 1.3])
def test_bgk_step_with_one_bead(tau):
    p = dict(collision=0, tau=tau, gamma_bead=0.35, body_force=(1e-4, -2e-4, 5e-5))
    _run((4, 4, 4), p, [BODY_FIXED])


def test_mrt_step_with_a_spinning_body():
    p = dict(collision=1, gamma_shear=-0.45, gamma_bulk=0.15, gamma_odd=0.3, gamma_even=-0.25,
             gamma_bead=0.2, body_force=(0, 1e-4, 0))
    _run((4, 4, 4), p, [BODY_SPIN], seed=1)


def test_mrt_step_with_a_translating_body_and_compensation():
    p = dict(collision=1, gamma_shear=0.2, gamma_bulk=-0.6, gamma_odd=-0.4, gamma_even=0.5,
             gamma_bead=0.3, compensate_force=1)
    _run((4, 4, 4), p, [BODY_FREE], seed=2)


@pytest.mark.parametrize("axis", [2, 0])
def test_mrt_step_in_a_pore_with_a_bead_at_the_wall(axis):
    """Halfway bounce-back on the staircase wall of a narrow pore; the bead's
    corner nodes include wall nodes (u = 0 there, force dropped)."""
    dims = [6, 6, 6]
    dims[axis] = 4
    p = dict(collision=1, gamma_shear=-0.3, gamma_bulk=-0.1, gamma_odd=0.2, gamma_even=0.1,
             gamma_bead=0.25, body_force=tuple(1e-4 if a == axis else 0.0 for a in range(3)))
    X = [3.0, 3.0, 3.0]
    X[(axis + 1) % 3] = 4.6                            # next to the wall across the pore
    body = dict(BODY_FIXED, X=X)
    wall = wall_mask(tuple(dims), 2.3, axis)
    assert 0 < wall.sum() < wall.size
    corners, _ = corner_weights(np.array(X))
    assert any(wall[node_index(*c, tuple(dims))] for c in corners)
    _run(tuple(dims), p, [body], pore=(2.3, axis), seed=3)


def test_a_planted_mistake_is_caught():
    """The comparison fails if the brute force's own ghost rate is swapped:
    the two ghost families do act on the result at this tolerance."""
    p = dict(collision=1, gamma_shear=-0.45, gamma_bulk=0.15, gamma_odd=0.3, gamma_even=-0.25,
             gamma_bead=0.2)
    f0 = _start((4, 4, 4), 5)
    F = np.zeros((64, 3))
    good = collide(f0, F, p)
    bad = collide(f0, F, dict(p, gamma_odd=p["gamma_even"], gamma_even=p["gamma_odd"]))
    orc_post = np.array([from_oracle(O.collide_node(O.make_params(4, 4, 4, **{k: v for k, v in p.items()}),
                                                    to_oracle(f0[:, n]), F[n])[:, None])[:, 0]
                         for n in range(64)]).T
    assert np.max(np.abs(orc_post - good) / W[:, None]) <= 1e-14
    assert np.max(np.abs(orc_post - bad) / W[:, None]) > 1e-4
