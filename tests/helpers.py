"""Shared test helpers: build the same seeded case on the CUDA path and on the
oracle, and compare them."""
from __future__ import annotations

import os

import numpy as np

from oracle import oracle as O

W19 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)

ORACLE_KEYS = ("collision", "tau", "gamma_shear", "gamma_bulk", "gamma_odd", "gamma_even", "rho0",
               "kT", "gamma_bead", "seed", "instance", "body_force", "compensate_force", "md_substeps")


# Worst error observed per (test, quantity): parity tests report what they
# measured, so that the tolerances written in the tests can be compared with
# the errors actually seen. conftest.py writes the table to the file named
# by LB_PARITY_LOG at the end of the session.
OBSERVED: dict = {}


def observe(kind, value):
    test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    key = (test, kind)
    v = float(value)
    if key not in OBSERVED or v > OBSERVED[key]:
        OBSERVED[key] = v
    return value


def oracle_kw(params):
    return {k: params[k] for k in ORACLE_KEYS if k in params}


def perturbed_populations(n_nodes, rho0=1.0, amp=0.02, u_amp=0.02, seed=0):
    """f_i = f_eq(rho, u) (1 + amp xi) with seeded rho, u and xi per node."""
    rng = np.random.default_rng(seed)
    c = np.array(O.lattice()[0], dtype=np.float64)
    rho = rho0 * (1 + 0.05 * rng.standard_normal(n_nodes))
    u = u_amp * rng.standard_normal((n_nodes, 3))
    cu = u @ c.T
    uu = (u * u).sum(1)[:, None]
    feq = W19[None, :] * rho[:, None] * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu)
    f = feq * (1 + amp * rng.standard_normal(feq.shape))
    return np.ascontiguousarray(f.T)


class Pair:
    """The same case on the GPU (lb.LB) and in the oracle."""

    def __init__(self, nx, ny, nz, precision=64, pore=None, **params):
        from paper_1604_01829_gb300 import lb
        self.gpu = lb.LB(nx, ny, nz, precision=precision, **params)
        self.orc = O.OracleLB(nx, ny, nz, **oracle_kw(params))
        self.N = nx * ny * nz
        self.rho0 = params.get("rho0", 1.0)
        if pore is not None:
            self.gpu.lb_set_pore(*pore)
            self.orc.set_pore(*pore)
        self.fluid = np.ones(self.N, bool) if pore is None else self.orc.mask == 0
        self.nbodies = 0

    def set_populations(self, f):
        self.gpu.lb_set_populations(f)
        self.orc.set_populations(f)

    def add_body(self, beads, X, q=(1, 0, 0, 0), mass=1.0, inertia=(1, 1, 1), F_ext=(0, 0, 0),
                 T_ext=(0, 0, 0), fixed=False, V=(0, 0, 0), w=(0, 0, 0)):
        q = np.asarray(q, np.float64) / np.linalg.norm(q)
        b = self.gpu.lb_add_raspberry(beads, X, q, mass, inertia, F_ext, T_ext, fixed)
        self.gpu.lb_set_body_state(b, V=V, w=w)
        self.orc.add_raspberry(beads, X, q, mass, inertia, F_ext, T_ext, fixed, V=V, w=w)
        self.nbodies += 1
        return b

    def step(self, n):
        self.gpu.lb_step(n)
        self.orc.step(n)

    def pop_error(self):
        """max |f_gpu - f_oracle| / (w_i rho0) over fluid nodes."""
        fg = self.gpu.lb_get_populations()[:, self.fluid]
        fo = self.orc.populations()[:, self.fluid]
        return observe("pop", np.max(np.abs(fg - fo) / (W19[:, None] * self.rho0)))

    def body_errors(self, b):
        g = self.gpu.lb_get_body(b)
        o = self.orc.body(b)
        Fg, Tg, pbg = self.gpu.lb_forces(b, per_bead=True)
        pbo = self.orc.bead_forces(b)
        scaleF = max(np.abs(pbo).max(), 1e-300)
        e = dict(
            X=np.abs(g["X"] - o["X"]).max(), V=np.abs(g["V"] - o["V"]).max(),
            q=np.abs(g["q"] - o["q"]).max(), w=np.abs(g["w"] - o["w"]).max(),
            F=np.abs(Fg - o["F"]).max() / max(np.abs(o["F"]).max(), 1e-300),
            T=np.abs(Tg - o["T"]).max() / max(np.abs(o["T"]).max(), 1e-300),
            bead=np.abs(pbg - pbo).max() / scaleF)
        for k, v in e.items():
            observe(k, v)
        return e
