"""Python side of the FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module. It loads ``lb_oracle.c`` compiled with
plain ``gcc`` (no shared code with the CUDA library) and drives it with numpy
arrays. The step it runs is documented in ``lb_oracle.c``; every function
there cites the passage of Ustach & Faller (arXiv:1604.01829) it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

NQ = 19


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-std=c99", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("collision", C.c_int),
                ("tau", C.c_double),
                ("gamma_shear", C.c_double), ("gamma_bulk", C.c_double),
                ("gamma_odd", C.c_double), ("gamma_even", C.c_double),
                ("rho0", C.c_double), ("kT", C.c_double), ("gamma_bead", C.c_double),
                ("seed", C.c_uint64), ("instance", C.c_uint32),
                ("body_force", C.c_double * 3),
                ("compensate_force", C.c_int),
                ("wall_beads", C.c_int), ("wall_axis", C.c_int),
                ("wall_R", C.c_double), ("wall_spacing", C.c_double), ("wall_rp", C.c_double),
                ("wall_rr", C.c_double), ("wall_eps", C.c_double),
                ("ywalls", C.c_int), ("uw_lo", C.c_double * 3), ("uw_hi", C.c_double * 3),
                ("md_substeps", C.c_int)]


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class Bodies(C.Structure):
    _fields_ = [("nbodies", C.c_int), ("bead_start", _ip), ("s", _dp),
                ("X", _dp), ("V", _dp), ("q", _dp), ("w", _dp),
                ("F_last", _dp), ("T_last", _dp),
                ("mass", _dp), ("inertia", _dp), ("F_ext", _dp), ("T_ext", _dp),
                ("fixed", _ip), ("F_bead", _dp), ("F_tot", _dp), ("T_tot", _dp)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_step.argtypes = [C.POINTER(Params), _dp, C.c_void_p, _dp, C.c_void_p, C.c_int64]
            L.orc_step.restype = C.c_int
            L.orc_init.argtypes = [C.POINTER(Params), _dp]
            L.orc_wall_bead_force.argtypes = [C.POINTER(Params), _dp, _dp]
            L.orc_wall_bead_energy.argtypes = [C.POINTER(Params), _dp]
            L.orc_wall_bead_energy.restype = C.c_double
            L.orc_moments_sum.argtypes = [C.POINTER(Params), _dp, C.c_void_p, _dp]
            L.orc_node_velocity.argtypes = [C.POINTER(Params), _dp, C.c_void_p, _dp, _dp]
            L.orc_lattice.argtypes = [_ip, _dp, _ip]
            L.orc_mrt_tables.argtypes = [_dp, _dp, _dp]
            L.orc_philox.argtypes = [C.POINTER(C.c_uint32)] * 3
            L.orc_unit_uniform.argtypes = [C.c_uint32]
            L.orc_unit_uniform.restype = C.c_double
            L.orc_unit_uniform16.argtypes = [C.c_uint32]
            L.orc_unit_uniform16.restype = C.c_double
            L.orc_equilibrium.argtypes = [C.c_double, _dp, _dp]
            L.orc_collide_node.argtypes = [C.POINTER(Params), _dp, _dp, C.c_uint32, C.c_uint32, _dp]
            L.orc_rotation.argtypes = [_dp, _dp]
            L.orc_quat_mul.argtypes = [_dp, _dp, _dp]
            L.orc_pore_mask.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, C.c_void_p]
            L.orc_collide_node_adjoint.argtypes = [C.POINTER(Params), _dp, _dp, _dp, _dp, _dp]
            L.orc_adjoint_drag.argtypes = [C.POINTER(Params), _dp, C.c_void_p, _dp, C.c_void_p, C.c_int64,
                                           C.c_int, C.c_int, C.c_int, C.c_int, _dp, _dp, _dp]
            L.orc_adjoint_drag.restype = C.c_int
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


# ----------------------------------------------------------------- small helpers

def lattice():
    c = np.zeros((NQ, 3), np.int32)
    w = np.zeros(NQ)
    opp = np.zeros(NQ, np.int32)
    lib().orc_lattice(_i(c), _d(w), _i(opp))
    return c, w, opp


def mrt_tables():
    M = np.zeros((NQ, NQ))
    Minv = np.zeros((NQ, NQ))
    b = np.zeros(NQ)
    lib().orc_mrt_tables(_d(M), _d(Minv), _d(b))
    return M, Minv, b


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox(c, k, o)
    return [int(v) for v in o]


def unit_uniform(x):
    return lib().orc_unit_uniform(int(x) & 0xFFFFFFFF)


def unit_uniform16(h):
    return lib().orc_unit_uniform16(int(h) & 0xFFFF)


def equilibrium(rho, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    feq = np.zeros(NQ)
    lib().orc_equilibrium(float(rho), _d(u), _d(feq))
    return feq


def rotation(q):
    q = np.ascontiguousarray(q, dtype=np.float64)
    R = np.zeros(9)
    lib().orc_rotation(_d(q), _d(R))
    return R.reshape(3, 3)


def quat_mul(a, b):
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    o = np.zeros(4)
    lib().orc_quat_mul(_d(a), _d(b), _d(o))
    return o


def pore_mask(nx, ny, nz, R, axis=2):
    m = np.zeros(nx * ny * nz, np.uint8)
    lib().orc_pore_mask(nx, ny, nz, float(R), int(axis), m.ctypes.data_as(C.c_void_p))
    return m


def make_params(nx, ny, nz, collision=0, tau=1.0, gamma_shear=0.0, gamma_bulk=0.0,
                gamma_odd=0.0, gamma_even=0.0, rho0=1.0, kT=0.0, gamma_bead=0.0,
                seed=0, instance=0, body_force=(0.0, 0.0, 0.0), compensate_force=0, md_substeps=1):
    p = Params(nx, ny, nz, collision, tau, gamma_shear, gamma_bulk, gamma_odd, gamma_even,
               rho0, kT, gamma_bead, seed, instance, (C.c_double * 3)(*body_force),
               compensate_force)
    p.md_substeps = int(md_substeps)
    return p


def collide_node(p: Params, f, F, node_id=0, step=0):
    f = np.ascontiguousarray(f, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros(NQ)
    lib().orc_collide_node(C.byref(p), _d(f), _d(F), node_id, step, _d(out))
    return out


def collide_node_adjoint(p: Params, f, F, lam_out):
    f = np.ascontiguousarray(f, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    lo = np.ascontiguousarray(lam_out, dtype=np.float64)
    lf = np.zeros(NQ)
    lF = np.zeros(3)
    lib().orc_collide_node_adjoint(C.byref(p), _d(f), _d(F), _d(lo), _d(lf), _d(lF))
    return lf, lF


# ------------------------------------------------------------------ the stepper

class OracleLB:
    """State container around ``orc_step``: populations [19][N] in FP64,
    optional wall mask, the spread bead force of the last step, rigid bodies.

    Lattice units throughout (grid spacing 1, time step 1). Node (x, y, z)
    has linear index x + nx (y + ny z) and centre (x+1/2, y+1/2, z+1/2).
    """

    def __init__(self, nx, ny, nz, **kw):
        self.p = make_params(nx, ny, nz, **kw)
        self.N = nx * ny * nz
        self.f = np.zeros(NQ * self.N)
        lib().orc_init(C.byref(self.p), _d(self.f))
        self.mask = None
        self.Fnode = np.zeros(3 * self.N)
        self.step_index = 0
        self.bodies = []
        self._packed = None

    # geometry ---------------------------------------------------------------
    def set_pore(self, R, axis=2):
        self.mask = pore_mask(self.p.nx, self.p.ny, self.p.nz, R, axis)

    def set_channel_walls(self, u_lo, u_hi):
        """Moving walls at y = -1/2 and y = ny - 1/2 (see orc_params)."""
        self.p.ywalls = 1
        for a in range(3):
            self.p.uw_lo[a] = float(u_lo[a])
            self.p.uw_hi[a] = float(u_hi[a])

    def set_pore_beads(self, R, axis, spacing, r_pore_bead, r_bead, eps):
        """Repulsive pore-wall beads (see wall_bead_force in lb_oracle.c)."""
        self.p.wall_beads = 1
        self.p.wall_axis = int(axis)
        self.p.wall_R = float(R)
        self.p.wall_spacing = float(spacing)
        self.p.wall_rp = float(r_pore_bead)
        self.p.wall_rr = float(r_bead)
        self.p.wall_eps = float(eps)

    def wall_force(self, r):
        F = np.zeros(3)
        lib().orc_wall_bead_force(C.byref(self.p), _d(np.ascontiguousarray(r, np.float64)), _d(F))
        return F

    def wall_energy(self, r):
        return lib().orc_wall_bead_energy(C.byref(self.p), _d(np.ascontiguousarray(r, np.float64)))

    def set_mask(self, mask):
        self.mask = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)

    # bodies -----------------------------------------------------------------
    def add_raspberry(self, beads, X, q=(1, 0, 0, 0), mass=1.0, inertia=(1, 1, 1),
                      F_ext=(0, 0, 0), T_ext=(0, 0, 0), fixed=False, V=(0, 0, 0), w=(0, 0, 0)):
        self.bodies.append(dict(s=np.asarray(beads, np.float64).reshape(-1, 3),
                                X=np.array(X, np.float64), V=np.array(V, np.float64),
                                q=np.array(q, np.float64), w=np.array(w, np.float64),
                                mass=float(mass), inertia=np.array(inertia, np.float64),
                                F_ext=np.array(F_ext, np.float64), T_ext=np.array(T_ext, np.float64),
                                fixed=int(fixed)))
        self._packed = None
        return len(self.bodies) - 1

    def _pack(self):
        bl = self.bodies
        nb = len(bl)
        counts = [len(b["s"]) for b in bl]
        P = dict(
            bead_start=np.concatenate([[0], np.cumsum(counts)]).astype(np.int32),
            s=np.concatenate([b["s"].reshape(-1) for b in bl]),
            X=np.concatenate([b["X"] for b in bl]), V=np.concatenate([b["V"] for b in bl]),
            q=np.concatenate([b["q"] for b in bl]), w=np.concatenate([b["w"] for b in bl]),
            F_last=np.zeros(3 * nb), T_last=np.zeros(3 * nb),
            mass=np.array([b["mass"] for b in bl]),
            inertia=np.concatenate([b["inertia"] for b in bl]),
            F_ext=np.concatenate([b["F_ext"] for b in bl]),
            T_ext=np.concatenate([b["T_ext"] for b in bl]),
            fixed=np.array([b["fixed"] for b in bl], np.int32),
            F_bead=np.zeros(3 * sum(counts)), F_tot=np.zeros(3 * nb), T_tot=np.zeros(3 * nb))
        self._packed = P
        st = Bodies()
        st.nbodies = nb
        for k, v in P.items():
            setattr(st, k, _i(v) if v.dtype == np.int32 else _d(v))
        self._struct = st

    def set_external(self, body, F_ext=None, T_ext=None):
        if self._packed is None:
            b = self.bodies[body]
            if F_ext is not None:
                b["F_ext"] = np.array(F_ext, np.float64)
            if T_ext is not None:
                b["T_ext"] = np.array(T_ext, np.float64)
            return
        if F_ext is not None:
            self._packed["F_ext"][3 * body:3 * body + 3] = F_ext
        if T_ext is not None:
            self._packed["T_ext"][3 * body:3 * body + 3] = T_ext

    # stepping -----------------------------------------------------------------
    def step(self, n=1):
        if self.bodies and self._packed is None:
            self._pack()
        bptr = C.byref(self._struct) if self.bodies else None
        mptr = self.mask.ctypes.data_as(C.c_void_p) if self.mask is not None else None
        for _ in range(n):
            rc = lib().orc_step(C.byref(self.p), _d(self.f), mptr, _d(self.Fnode), bptr,
                                self.step_index)
            if rc != 0:
                raise ValueError("oracle step rejected its input")
            self.step_index += 1

    def adjoint_drag(self, nsteps, window, body=0, axis=2):
        """Runs nsteps steps (advancing the state like step()) and returns
        J = mean V_axis of `body` over the last `window` steps with dJ/dgamma
        and dJ/ds (3 per bead, all bodies), by the oracle's reverse pass."""
        if self.bodies and self._packed is None:
            self._pack()
        mptr = self.mask.ctypes.data_as(C.c_void_p) if self.mask is not None else None
        J = C.c_double()
        dg = C.c_double()
        ds = np.zeros(3 * int(self._packed["bead_start"][-1]))
        rc = lib().orc_adjoint_drag(C.byref(self.p), _d(self.f), mptr, _d(self.Fnode), C.byref(self._struct),
                                    self.step_index, int(nsteps), int(window), int(body), int(axis),
                                    C.byref(J), C.byref(dg), _d(ds))
        if rc != 0:
            raise ValueError(f"oracle adjoint rejected its input ({rc})")
        self.step_index += nsteps
        return J.value, dg.value, ds.reshape(-1, 3)

    def clone(self):
        """Deep copy of the whole state (for finite differences)."""
        import copy
        o = OracleLB.__new__(OracleLB)
        o.p = copy.copy(self.p)
        o.p.body_force = (C.c_double * 3)(*self.p.body_force)
        o.N = self.N
        o.f = self.f.copy()
        o.mask = None if self.mask is None else self.mask.copy()
        o.Fnode = self.Fnode.copy()
        o.step_index = self.step_index
        o.bodies = [{k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in b.items()} for b in self.bodies]
        o._packed = None
        if self._packed is not None:
            # carry the evolving body state
            P = self._packed
            for i, b in enumerate(o.bodies):
                for k, sz in (("X", 3), ("V", 3), ("q", 4), ("w", 3)):
                    b[k] = P[k][sz * i:sz * i + sz].copy()
            o._pack()
            for k in ("F_last", "T_last"):
                o._packed[k][:] = P[k]
        return o

    # state access -------------------------------------------------------------
    def populations(self):
        return self.f.reshape(NQ, self.N).copy()

    def set_populations(self, f):
        self.f[:] = np.asarray(f, np.float64).reshape(-1)

    def conservation(self):
        out = np.zeros(4)
        mptr = self.mask.ctypes.data_as(C.c_void_p) if self.mask is not None else None
        lib().orc_moments_sum(C.byref(self.p), _d(self.f), mptr, _d(out))
        return out[0], out[1:].copy()

    def node_velocity(self, with_force=True):
        rho = np.zeros(self.N)
        u = np.zeros(3 * self.N)
        lib().orc_node_velocity(C.byref(self.p), _d(self.f),
                                _d(self.Fnode) if with_force else None, _d(rho), _d(u))
        return rho, u.reshape(self.N, 3)

    def body(self, i):
        if self._packed is None:
            self._pack()
        P = self._packed
        return dict(X=P["X"][3 * i:3 * i + 3].copy(), V=P["V"][3 * i:3 * i + 3].copy(),
                    q=P["q"][4 * i:4 * i + 4].copy(), w=P["w"][3 * i:3 * i + 3].copy(),
                    F=P["F_tot"][3 * i:3 * i + 3].copy(), T=P["T_tot"][3 * i:3 * i + 3].copy(),
                    F_last=P["F_last"][3 * i:3 * i + 3].copy())

    def bead_forces(self, i):
        P = self._packed
        a, b = P["bead_start"][i], P["bead_start"][i + 1]
        return P["F_bead"][3 * a:3 * b].reshape(-1, 3).copy()
