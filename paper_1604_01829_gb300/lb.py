"""Python binding of the C ABI in include/lb.h (argument marshalling only).

Every step of the LB + coupling path runs in the CUDA library
``_lib/liblbrasp.so``; this module only converts numpy arrays to pointers and
lb_status codes to exceptions. There is no fallback: if the library has not
been built (``paper_1604_01829_gb300.build.build()``) or no GPU is present,
calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LB_CHECKED=1 selects the index-checked build (build.build(checked=True))
LIB_PATH = os.path.join(_HERE, "_lib", "liblbrasp_checked.so" if os.environ.get("LB_CHECKED") == "1"
                        else "liblbrasp.so")

LB_OK, LB_ERR_ARG, LB_ERR_OOM, LB_ERR_CUDA, LB_ERR_UNSTABLE, LB_ERR_TIMEOUT, LB_ERR_STATE = range(7)

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_llp = C.POINTER(C.c_longlong)


class lb_params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("precision", C.c_int), ("collision", C.c_int),
                ("tau", C.c_double),
                ("gamma_shear", C.c_double), ("gamma_bulk", C.c_double),
                ("gamma_odd", C.c_double), ("gamma_even", C.c_double),
                ("rho0", C.c_double), ("kT", C.c_double), ("gamma_bead", C.c_double),
                ("seed", C.c_ulonglong), ("instance", C.c_uint),
                ("body_force", C.c_double * 3),
                ("compensate_force", C.c_int), ("md_substeps", C.c_int)]


LB_ADJ_TWO_LEVEL = 0
LB_ADJ_BINOMIAL = 1


class lb_adjoint_opts(C.Structure):
    _fields_ = [("schedule", C.c_int), ("snapshots", C.c_int)]


class lb_adjoint_stats(C.Structure):
    _fields_ = [("alloc_ms", C.c_double), ("forward_ms", C.c_double), ("recompute_ms", C.c_double),
                ("reverse_ms", C.c_double), ("forward_steps", C.c_longlong), ("recompute_steps", C.c_longlong),
                ("reversed_steps", C.c_longlong), ("workspace_bytes", C.c_double)]


class lb_info_t(C.Structure):
    _fields_ = [("nodes", C.c_longlong), ("fluid_nodes", C.c_longlong), ("step", C.c_longlong),
                ("nbodies", C.c_int), ("nbeads", C.c_int), ("precision", C.c_int),
                ("device_bytes", C.c_size_t)]


_lock = threading.Lock()
_lib = None

# name -> (argtypes)
_SIGS = {
    "lb_create": [C.POINTER(lb_params), C.c_void_p, C.POINTER(C.c_void_p)],
    "lb_destroy": [C.c_void_p],
    "lb_set_pore": [C.c_void_p, C.c_double, C.c_int],
    "lb_set_pore_beads": [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double],
    "lb_set_channel_walls": [C.c_void_p, _dp, _dp],
    "lb_add_raspberry": [C.c_void_p, _dp, C.c_int, _dp, _dp, C.c_double, _dp, _dp, _dp, C.c_int, _ip],
    "lb_set_body_state": [C.c_void_p, C.c_int, _dp, _dp, _dp, _dp],
    "lb_set_external_forces": [C.c_void_p, C.c_int, _dp, _dp],
    "lb_step": [C.c_void_p, C.c_int],
    "lb_forces": [C.c_void_p, C.c_int, _dp, _dp, _dp],
    "lb_forces_all": [C.c_void_p, C.c_int, _dp, _dp],
    # raw addresses (ints): the per-step call of a host control loop
    "lb_step_io": [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "lb_get_body": [C.c_void_p, C.c_int, _dp, _dp, _dp, _dp],
    "lb_get_populations": [C.c_void_p, _dp, C.c_size_t],
    "lb_set_populations": [C.c_void_p, _dp, C.c_size_t],
    "lb_sample_populations": [C.c_void_p, _llp, C.c_int, _dp],
    "lb_get_node_force": [C.c_void_p, _dp, C.c_size_t],
    "lb_conservation": [C.c_void_p, _dp, _dp],
    "lb_info": [C.c_void_p, C.POINTER(lb_info_t)],
    "lb_set_timing": [C.c_void_p, C.c_int],
    "lb_set_kernel_variant": [C.c_void_p, C.c_int, C.c_int, C.c_int],
    "lb_set_wait_limit": [C.c_void_p, C.c_longlong],
    "lb_checkpoint_size": [C.c_void_p, C.POINTER(C.c_size_t)],
    "lb_checkpoint_save": [C.c_void_p, C.c_void_p, C.c_size_t],
    "lb_checkpoint_load": [C.c_void_p, C.c_void_p, C.c_size_t],
    "lb_adjoint_drag": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _dp, _dp, _dp],
    "lb_adjoint_drag_ex": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, _dp, _dp, _dp,
                           C.c_void_p],
    "lb_kernel_time": [C.c_void_p, _dp, _llp],
    "lb_record_bodies": [C.c_void_p, C.c_int, C.c_int],
    "lb_get_trajectory": [C.c_void_p, C.c_int, C.c_int, _llp, _dp, _dp, _ip],
}

_BSIGS = {
    "lb_batch_create": [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_void_p)],
    "lb_batch_destroy": [C.c_void_p],
    "lb_batch_set_pore": [C.c_void_p, C.c_int, C.c_double, C.c_int],
    "lb_batch_set_pore_beads": [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double],
    "lb_batch_add_raspberry": [C.c_void_p, C.c_int, _dp, C.c_int, _dp, _dp, C.c_double, _dp, _dp, _dp, C.c_int, _ip],
    "lb_batch_step": [C.c_void_p, C.c_int],
    "lb_batch_forces": [C.c_void_p, C.c_int, C.c_int, _dp, _dp],
    "lb_batch_get_body": [C.c_void_p, C.c_int, C.c_int, _dp, _dp, _dp, _dp],
    "lb_batch_get_populations": [C.c_void_p, C.c_int, _dp, C.c_size_t],
    "lb_batch_set_populations": [C.c_void_p, C.c_int, _dp, C.c_size_t],
    "lb_batch_set_schedule": [C.c_void_p, C.c_int, C.c_int, C.c_int],
    "lb_batch_autotune": [C.c_void_p, C.c_int, _ip, _dp],
    "lb_batch_info": [C.c_void_p, _llp, _llp, _ip],
    "lb_batch_set_timing": [C.c_void_p, C.c_int],
    "lb_batch_kernel_time": [C.c_void_p, _dp, _llp],
    "lb_batch_checkpoint_size": [C.c_void_p, C.POINTER(C.c_size_t)],
    "lb_batch_checkpoint_save": [C.c_void_p, C.c_void_p, C.c_size_t],
    "lb_batch_checkpoint_load": [C.c_void_p, C.c_void_p, C.c_size_t],
    "lb_batch_record_bodies": [C.c_void_p, C.c_int, C.c_int],
    "lb_batch_get_trajectory": [C.c_void_p, C.c_int, C.c_int, C.c_int, _llp, _dp, _dp, _ip],
}

# every symbol include/lb.h declares
EXPORTS = sorted(list(_SIGS) + list(_BSIGS) + ["lb_last_error", "lb_status_string", "lb_lattice",
                                                "lb_moments_noalloc", "lb_batch_last_error",
                                                "lb_msd_trajectory", "lb_pore_msd", "lb_relax_shells"])


def load():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"CUDA library {LIB_PATH} is missing: build it with "
                    "paper_1604_01829_gb300.build.build() (nvcc, sm_103a)")
            L = C.CDLL(LIB_PATH)
            for name, args in list(_SIGS.items()) + list(_BSIGS.items()):
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = C.c_int
            L.lb_batch_last_error.argtypes = [C.c_void_p]
            L.lb_batch_last_error.restype = C.c_char_p
            L.lb_last_error.argtypes = [C.c_void_p]
            L.lb_last_error.restype = C.c_char_p
            L.lb_status_string.argtypes = [C.c_int]
            L.lb_status_string.restype = C.c_char_p
            L.lb_lattice.argtypes = [_ip, _dp, _ip]
            L.lb_lattice.restype = C.c_int
            L.lb_moments_noalloc.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                             C.c_double, C.c_double, C.c_int, C.c_void_p, C.c_void_p,
                                             C.c_char_p, C.c_size_t]
            L.lb_moments_noalloc.restype = C.c_int
            L.lb_msd_trajectory.argtypes = [_dp, _dp, C.c_int, C.c_int, C.c_int, _dp, _dp, C.c_void_p,
                                            C.c_char_p, C.c_size_t]
            L.lb_msd_trajectory.restype = C.c_int
            L.lb_pore_msd.argtypes = [_dp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int,
                                      C.c_int, _dp, _llp, C.c_void_p, C.c_char_p, C.c_size_t]
            L.lb_pore_msd.restype = C.c_int
            L.lb_relax_shells.argtypes = [C.c_int, _dp, _ip, _dp, C.POINTER(lb_shell_params), C.c_void_p,
                                          C.c_char_p, C.c_size_t]
            L.lb_relax_shells.restype = C.c_int
            _lib = L
    return _lib


class LBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def _check(h, status):
    if status != LB_OK:
        L = load()
        msg = L.lb_last_error(h).decode() if L.lb_last_error(h) else ""
        raise LBError(status, msg or L.lb_status_string(status).decode())


def _d(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _vec(v, n):
    if v is None:
        return None
    a = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
    if a.size != n:
        raise ValueError(f"expected {n} values")
    return a


def lb_lattice():
    c = np.zeros(57, np.int32)
    w = np.zeros(19)
    opp = np.zeros(19, np.int32)
    load().lb_lattice(c.ctypes.data_as(_ip), _d(w), opp.ctypes.data_as(_ip))
    return c.reshape(19, 3), w, opp


def lb_moments_noalloc(d_populations, precision, nx, ny, nz, odd_parity, rho0, d_out,
                       pore_radius=0.0, pore_axis=2, stream=None):
    """Allocation-free mass/momentum sums of a device population array into
    the 4 doubles at device address d_out (see include/lb.h). Raises LBError
    with the library's message on failure."""
    err = C.create_string_buffer(256)
    st = load().lb_moments_noalloc(C.c_void_p(d_populations), int(precision), int(nx), int(ny), int(nz),
                                   int(odd_parity), float(rho0), float(pore_radius), int(pore_axis),
                                   C.c_void_p(d_out), C.c_void_p(stream) if stream else None, err, 256)
    if st != LB_OK:
        raise LBError(st, err.value.decode())


MSD_COLS = 10
MSD_COLUMNS = ("lab_x", "lab_y", "lab_z", "body_x", "body_y", "body_z", "rot_lab",
               "rot_body_x", "rot_body_y", "rot_body_z")


def lb_msd_trajectory(X, q, max_lag, p_ref=(1.0, 0.0, 0.0), stream=None):
    """Mean squared displacements of recorded trajectories on the GPU (see
    include/lb.h). X: [nbodies, nrec, 3], q: [nbodies, nrec, 4] (or one body
    without the leading axis). Returns [nbodies, max_lag, MSD_COLS]."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    if X.ndim == 2:
        X, q = X[None], q[None]
    nb, nrec = X.shape[0], X.shape[1]
    if X.shape != (nb, nrec, 3) or q.shape != (nb, nrec, 4):
        raise ValueError("X must be [nbodies, nrec, 3] and q [nbodies, nrec, 4]")
    out = np.zeros((nb, int(max_lag), MSD_COLS))
    err = C.create_string_buffer(256)
    st = load().lb_msd_trajectory(_d(X), _d(q), nrec, nb, int(max_lag), _d(_vec(p_ref, 3)), _d(out),
                                  C.c_void_p(stream) if stream else None, err, 256)
    if st != LB_OK:
        raise LBError(st, err.value.decode())
    return out


def lb_pore_msd(X, shape, axis, R_pore, nbins, max_lag, stream=None):
    """Binned pore-frame MSD of one trajectory on the GPU (see include/lb.h):
    returns (msd [nbins, max_lag, 3], counts [nbins, max_lag])."""
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((int(nbins), int(max_lag), 3))
    cnt = np.zeros((int(nbins), int(max_lag)), np.int64)
    err = C.create_string_buffer(256)
    st = load().lb_pore_msd(_d(X), len(X), int(shape[0]), int(shape[1]), int(shape[2]), int(axis),
                            float(R_pore), int(nbins), int(max_lag), _d(out), cnt.ctypes.data_as(_llp),
                            C.c_void_p(stream) if stream else None, err, 256)
    if st != LB_OK:
        raise LBError(st, err.value.decode())
    return out, cnt


class lb_shell_params(C.Structure):
    _fields_ = [("k_surface", C.c_double), ("sigma", C.c_double), ("epsilon", C.c_double),
                ("dt", C.c_double), ("eta", C.c_double), ("steps", C.c_longlong),
                ("precision", C.c_int), ("project_final", C.c_int), ("pair_search", C.c_int)]


SHELL_MAX_BEADS = 4096


def lb_relax_shells(axes, xyz, steps, k_surface=1000.0, sigma=1.4, epsilon=0.1, dt=1e-3, eta=1000.0,
                    precision=32, project_final=True, pair_search=0, stream=None):
    """Relax raspberry shells on the GPU (see include/lb.h). axes: [nshells, 3]
    semi-axes; xyz: a list of [n_s, 3] initial positions, one per shell.
    Returns the relaxed positions as a list of [n_s, 3] arrays."""
    axes = np.ascontiguousarray(axes, dtype=np.float64).reshape(-1, 3)
    shells = [np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3) for x in xyz]
    if len(shells) != len(axes):
        raise ValueError("one position array per shell")
    counts = np.array([len(x) for x in shells], np.int32)
    flat = np.ascontiguousarray(np.concatenate(shells).reshape(-1))
    p = lb_shell_params(float(k_surface), float(sigma), float(epsilon), float(dt), float(eta), int(steps),
                        int(precision), int(bool(project_final)), int(pair_search))
    err = C.create_string_buffer(256)
    st = load().lb_relax_shells(len(shells), _d(axes), counts.ctypes.data_as(_ip), _d(flat), C.byref(p),
                                C.c_void_p(stream) if stream else None, err, 256)
    if st != LB_OK:
        raise LBError(st, err.value.decode())
    out = flat.reshape(-1, 3)
    return np.split(out, np.cumsum(counts)[:-1])


def make_params(nx, ny, nz, precision=64, collision=0, tau=1.0, gamma_shear=0.0, gamma_bulk=0.0,
                gamma_odd=0.0, gamma_even=0.0, rho0=1.0, kT=0.0, gamma_bead=0.0, seed=0,
                instance=0, body_force=(0.0, 0.0, 0.0), compensate_force=0, md_substeps=1):
    return lb_params(nx, ny, nz, precision, collision, tau, gamma_shear, gamma_bulk, gamma_odd,
                     gamma_even, rho0, kT, gamma_bead, seed, instance,
                     (C.c_double * 3)(*body_force), compensate_force, md_substeps)


class LB:
    """One lattice (handle) of the CUDA library; method names follow lb.h."""

    def __init__(self, nx, ny, nz, stream=None, **kw):
        L = load()
        self.p = make_params(nx, ny, nz, **kw)
        self.N = nx * ny * nz
        h = C.c_void_p()
        st = L.lb_create(C.byref(self.p), C.c_void_p(stream) if stream else None, C.byref(h))
        if st != LB_OK:
            raise LBError(st, L.lb_last_error(None).decode())
        self.h = h
        self.bead_counts = []

    def close(self):
        if getattr(self, "h", None):
            load().lb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # set-up --------------------------------------------------------------
    def lb_set_pore(self, radius, axis=2):
        _check(self.h, load().lb_set_pore(self.h, float(radius), int(axis)))

    def lb_set_channel_walls(self, u_lo, u_hi):
        _check(self.h, load().lb_set_channel_walls(self.h, _d(_vec(u_lo, 3)), _d(_vec(u_hi, 3))))

    def lb_set_pore_beads(self, spacing, r_pore_bead, r_bead, epsilon):
        _check(self.h, load().lb_set_pore_beads(self.h, float(spacing), float(r_pore_bead), float(r_bead),
                                                float(epsilon)))

    def lb_add_raspberry(self, beads, X, q=(1, 0, 0, 0), mass=1.0, inertia=(1, 1, 1),
                         F_ext=None, T_ext=None, fixed=False):
        b = np.ascontiguousarray(beads, dtype=np.float64).reshape(-1)
        bid = C.c_int(-1)
        _check(self.h, load().lb_add_raspberry(
            self.h, _d(b), b.size // 3, _d(_vec(X, 3)), _d(_vec(q, 4)), float(mass),
            _d(_vec(inertia, 3)), _d(_vec(F_ext, 3)), _d(_vec(T_ext, 3)), int(fixed),
            C.byref(bid)))
        self.bead_counts.append(b.size // 3)
        return bid.value

    def lb_set_body_state(self, body, X=None, V=None, q=None, w=None):
        _check(self.h, load().lb_set_body_state(self.h, int(body), _d(_vec(X, 3)), _d(_vec(V, 3)),
                                                _d(_vec(q, 4)), _d(_vec(w, 3))))

    def lb_set_external_forces(self, F_ext, T_ext=None):
        F = np.ascontiguousarray(F_ext, dtype=np.float64).reshape(-1)
        T = None if T_ext is None else np.ascontiguousarray(T_ext, dtype=np.float64).reshape(-1)
        _check(self.h, load().lb_set_external_forces(self.h, F.size // 3, _d(F), _d(T)))

    # stepping ------------------------------------------------------------
    def lb_step(self, n=1):
        _check(self.h, load().lb_step(self.h, int(n)))

    # results -------------------------------------------------------------
    def lb_forces(self, body, per_bead=False):
        F = np.zeros(3)
        T = np.zeros(3)
        pb = np.zeros(3 * self.bead_counts[body]) if per_bead else None
        _check(self.h, load().lb_forces(self.h, int(body), _d(F), _d(T), _d(pb)))
        return (F, T, pb.reshape(-1, 3)) if per_bead else (F, T)

    def lb_step_io(self, F_ext, T_ext, F_out, T_out, n=1):
        """Sets the external forces and torques, takes n steps and reads every
        body's force and torque back into F_out / T_out, in one library call.
        Every array is float64, C-contiguous, 3 * nbodies long (F_ext None:
        keep the forces; F_out and T_out None: no read-back)."""
        nb = len(self.bead_counts)

        def addr(a, out):
            if a is None:
                return None
            if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous
                    and a.size == 3 * nb and (not out or a.flags.writeable)):
                raise ValueError("lb_step_io: float64 C-contiguous arrays of 3 * nbodies values")
            return a.ctypes.data

        _check(self.h, load().lb_step_io(self.h, int(n), nb, addr(F_ext, False), addr(T_ext, False),
                                         addr(F_out, True), addr(T_out, True)))

    def lb_forces_all(self, F=None, T=None):
        n = len(self.bead_counts)
        F = np.zeros(3 * n) if F is None else F
        T = np.zeros(3 * n) if T is None else T
        _check(self.h, load().lb_forces_all(self.h, n, _d(F), _d(T)))
        return F, T

    def lb_get_body(self, body):
        X, V, q, w = np.zeros(3), np.zeros(3), np.zeros(4), np.zeros(3)
        _check(self.h, load().lb_get_body(self.h, int(body), _d(X), _d(V), _d(q), _d(w)))
        return dict(X=X, V=V, q=q, w=w)

    def lb_get_populations(self):
        out = np.zeros(19 * self.N)
        _check(self.h, load().lb_get_populations(self.h, _d(out), out.size))
        return out.reshape(19, self.N)

    def lb_set_populations(self, f):
        a = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        _check(self.h, load().lb_set_populations(self.h, _d(a), a.size))

    def lb_sample_populations(self, nodes):
        nd = np.ascontiguousarray(nodes, dtype=np.int64).reshape(-1)
        out = np.zeros(19 * nd.size)
        _check(self.h, load().lb_sample_populations(self.h, nd.ctypes.data_as(_llp), nd.size, _d(out)))
        return out.reshape(-1, 19)

    def lb_get_node_force(self):
        out = np.zeros(3 * self.N)
        _check(self.h, load().lb_get_node_force(self.h, _d(out), out.size))
        return out.reshape(3, self.N)

    def lb_conservation(self):
        m = C.c_double()
        p = np.zeros(3)
        _check(self.h, load().lb_conservation(self.h, C.byref(m), _d(p)))
        return m.value, p

    def lb_info(self):
        i = lb_info_t()
        _check(self.h, load().lb_info(self.h, C.byref(i)))
        return {k: getattr(i, k) for k, _ in lb_info_t._fields_}

    def lb_set_kernel_variant(self, variant=0, stages=0, ctas_per_sm=0):
        _check(self.h, load().lb_set_kernel_variant(self.h, int(variant), int(stages), int(ctas_per_sm)))

    def lb_checkpoint_save(self):
        """The handle's full state as bytes (see lb_checkpoint_* in include/lb.h)."""
        n = C.c_size_t()
        _check(self.h, load().lb_checkpoint_size(self.h, C.byref(n)))
        buf = (C.c_char * n.value)()
        _check(self.h, load().lb_checkpoint_save(self.h, buf, n.value))
        return bytes(buf)

    def lb_checkpoint_load(self, data):
        buf = C.create_string_buffer(bytes(data), len(data))
        _check(self.h, load().lb_checkpoint_load(self.h, buf, len(data)))

    def lb_set_wait_limit(self, cycles=0):
        _check(self.h, load().lb_set_wait_limit(self.h, int(cycles)))

    def lb_set_timing(self, on=True):
        _check(self.h, load().lb_set_timing(self.h, int(bool(on))))

    def lb_adjoint_drag(self, nsteps, window, body=0, axis=2, checkpoints=0):
        """(J, dJ/dgamma, dJ/ds[nbeads, 3]) from the hand-written adjoint."""
        J, dg = C.c_double(), C.c_double()
        ds = np.zeros(3 * sum(self.bead_counts))
        _check(self.h, load().lb_adjoint_drag(self.h, int(nsteps), int(window), int(body), int(axis),
                                              int(checkpoints), C.byref(J), C.byref(dg), _d(ds)))
        return J.value, dg.value, ds.reshape(-1, 3)

    def lb_adjoint_drag_ex(self, nsteps, window, body=0, axis=2, schedule=LB_ADJ_TWO_LEVEL, snapshots=0,
                           with_stats=False):
        """(J, dJ/dgamma, dJ/ds[nbeads, 3], stats dict or None) with a chosen
        checkpointing schedule (LB_ADJ_TWO_LEVEL or LB_ADJ_BINOMIAL)."""
        J, dg = C.c_double(), C.c_double()
        ds = np.zeros(3 * sum(self.bead_counts))
        o = lb_adjoint_opts(int(schedule), int(snapshots))
        st = lb_adjoint_stats()
        _check(self.h, load().lb_adjoint_drag_ex(self.h, int(nsteps), int(window), int(body), int(axis),
                                                 C.byref(o), C.byref(J), C.byref(dg), _d(ds),
                                                 C.byref(st) if with_stats else None))
        stats = {k: getattr(st, k) for k, _ in lb_adjoint_stats._fields_} if with_stats else None
        return J.value, dg.value, ds.reshape(-1, 3), stats

    def lb_kernel_time(self):
        ms = C.c_double()
        n = C.c_longlong()
        _check(self.h, load().lb_kernel_time(self.h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def lb_record_bodies(self, every, capacity=4096):
        _check(self.h, load().lb_record_bodies(self.h, int(every), int(capacity)))
        self._rec_cap = int(capacity)

    def lb_get_trajectory(self, body=0, max_records=None):
        """(steps, X [n, 3], q [n, 4]) of the records still in the ring."""
        m = int(max_records if max_records is not None else getattr(self, "_rec_cap", 0))
        steps, X, q = np.zeros(m, np.int64), np.zeros((m, 3)), np.zeros((m, 4))
        n = C.c_int()
        _check(self.h, load().lb_get_trajectory(self.h, int(body), m, steps.ctypes.data_as(_llp), _d(X), _d(q),
                                                C.byref(n)))
        k = n.value
        return steps[:k], X[:k], q[:k]


def from_workload(w, stream=None, precision=None):
    """Create an LB handle holding a workloads.Workload (pore and bodies)."""
    kw = dict(w.params)
    if precision is not None:
        kw["precision"] = precision
    lb = LB(w.nx, w.ny, w.nz, stream=stream, **kw)
    if w.pore is not None:
        lb.lb_set_pore(*w.pore)
    for b in w.bodies:
        lb.lb_add_raspberry(b.beads, b.X, b.q, b.mass, b.inertia, b.F_ext, b.T_ext, b.fixed)
    return lb


def _bcheck(h, status):
    if status != LB_OK:
        msg = load().lb_batch_last_error(h)
        raise LBError(status, msg.decode() if msg else load().lb_status_string(status).decode())


class LBBatch:
    """A batch of independent lattices (lb_batch_* of include/lb.h)."""

    def __init__(self, param_dicts, stream=None):
        L = load()
        arr = (lb_params * len(param_dicts))(*[make_params(**d) for d in param_dicts])
        self.sizes = [d["nx"] * d["ny"] * d["nz"] for d in param_dicts]
        h = C.c_void_p()
        st = L.lb_batch_create(arr, len(param_dicts), C.c_void_p(stream) if stream else None, C.byref(h))
        if st != LB_OK:
            raise LBError(st, L.lb_batch_last_error(None).decode())
        self.h = h
        self.n = len(param_dicts)

    def close(self):
        if getattr(self, "h", None):
            load().lb_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def lb_batch_set_pore(self, inst, radius, axis=2):
        _bcheck(self.h, load().lb_batch_set_pore(self.h, int(inst), float(radius), int(axis)))

    def lb_batch_set_pore_beads(self, inst, spacing, r_pore_bead, r_bead, epsilon):
        _bcheck(self.h, load().lb_batch_set_pore_beads(self.h, int(inst), float(spacing), float(r_pore_bead),
                                                       float(r_bead), float(epsilon)))

    def lb_batch_add_raspberry(self, inst, beads, X, q=(1, 0, 0, 0), mass=1.0, inertia=(1, 1, 1),
                               F_ext=None, T_ext=None, fixed=False):
        b = np.ascontiguousarray(beads, dtype=np.float64).reshape(-1)
        bid = C.c_int(-1)
        _bcheck(self.h, load().lb_batch_add_raspberry(
            self.h, int(inst), _d(b), b.size // 3, _d(_vec(X, 3)), _d(_vec(q, 4)), float(mass),
            _d(_vec(inertia, 3)), _d(_vec(F_ext, 3)), _d(_vec(T_ext, 3)), int(fixed), C.byref(bid)))
        return bid.value

    def lb_batch_step(self, n=1):
        _bcheck(self.h, load().lb_batch_step(self.h, int(n)))

    def lb_batch_forces(self, inst, body=0):
        F, T = np.zeros(3), np.zeros(3)
        _bcheck(self.h, load().lb_batch_forces(self.h, int(inst), int(body), _d(F), _d(T)))
        return F, T

    def lb_batch_get_body(self, inst, body=0):
        X, V, q, w = np.zeros(3), np.zeros(3), np.zeros(4), np.zeros(3)
        _bcheck(self.h, load().lb_batch_get_body(self.h, int(inst), int(body), _d(X), _d(V), _d(q), _d(w)))
        return dict(X=X, V=V, q=q, w=w)

    def lb_batch_get_populations(self, inst):
        out = np.zeros(19 * self.sizes[inst])
        _bcheck(self.h, load().lb_batch_get_populations(self.h, int(inst), _d(out), out.size))
        return out.reshape(19, -1)

    def lb_batch_set_populations(self, inst, f):
        a = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        _bcheck(self.h, load().lb_batch_set_populations(self.h, int(inst), _d(a), a.size))

    def lb_batch_set_schedule(self, tile_nodes=128, blocks_per_sm=8, order=0):
        _bcheck(self.h, load().lb_batch_set_schedule(self.h, int(tile_nodes), int(blocks_per_sm), int(order)))

    def lb_batch_autotune(self, trial_steps=10):
        ch = (C.c_int * 3)()
        ms = C.c_double()
        _bcheck(self.h, load().lb_batch_autotune(self.h, int(trial_steps), ch, C.byref(ms)))
        return list(ch), ms.value

    def lb_batch_info(self):
        n, st = C.c_longlong(), C.c_longlong()
        sch = (C.c_int * 3)()
        _bcheck(self.h, load().lb_batch_info(self.h, C.byref(n), C.byref(st), sch))
        return dict(total_nodes=n.value, step=st.value, schedule=list(sch))

    def lb_batch_set_timing(self, on=True):
        _bcheck(self.h, load().lb_batch_set_timing(self.h, int(bool(on))))

    def lb_batch_checkpoint_save(self):
        """The whole batch's state as bytes (see lb_batch_checkpoint_* in include/lb.h)."""
        n = C.c_size_t()
        _bcheck(self.h, load().lb_batch_checkpoint_size(self.h, C.byref(n)))
        buf = (C.c_char * n.value)()
        _bcheck(self.h, load().lb_batch_checkpoint_save(self.h, buf, n.value))
        return bytes(buf)

    def lb_batch_checkpoint_load(self, data):
        buf = C.create_string_buffer(bytes(data), len(data))
        _bcheck(self.h, load().lb_batch_checkpoint_load(self.h, buf, len(data)))

    def lb_batch_kernel_time(self):
        ms, n = C.c_double(), C.c_longlong()
        _bcheck(self.h, load().lb_batch_kernel_time(self.h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def lb_batch_record_bodies(self, every, capacity=4096):
        _bcheck(self.h, load().lb_batch_record_bodies(self.h, int(every), int(capacity)))
        self._rec_cap = int(capacity)

    def lb_batch_get_trajectory(self, inst, body=0, max_records=None):
        m = int(max_records if max_records is not None else getattr(self, "_rec_cap", 0))
        steps, X, q = np.zeros(m, np.int64), np.zeros((m, 3)), np.zeros((m, 4))
        n = C.c_int()
        _bcheck(self.h, load().lb_batch_get_trajectory(self.h, int(inst), int(body), m,
                                                       steps.ctypes.data_as(_llp), _d(X), _d(q), C.byref(n)))
        k = n.value
        return steps[:k], X[:k], q[:k]


def batch_from_workloads(workloads, stream=None, precision=None):
    """An LBBatch holding a list of workloads.Workload instances."""
    dicts = []
    for w in workloads:
        d = dict(w.params)
        if precision is not None:
            d["precision"] = precision
        d.update(nx=w.nx, ny=w.ny, nz=w.nz)
        dicts.append(d)
    B = LBBatch(dicts, stream=stream)
    for k, w in enumerate(workloads):
        if w.pore is not None:
            B.lb_batch_set_pore(k, *w.pore)
        for b in w.bodies:
            B.lb_batch_add_raspberry(k, b.beads, b.X, b.q, b.mass, b.inertia, b.F_ext, b.T_ext, b.fixed)
    return B
