"""Parity at the full sizes of the measured workloads, built as bench.py
builds them (workloads.py, lb.from_workload / lb.batch_from_workloads, the
default launch shape; eager steps as in the timed region, graph replay as in
lb_step):

- 256^3 periodic, FP32 deviations, MRT with fluctuations, 64 ellipsoidal
  raspberries (23,360 beads): two steps (both AA parities) against the oracle
  running the same two steps on the whole lattice, every population and every
  body and bead force compared; the same lattice with FP64 populations, one
  step. The oracle takes ~13 s per step at this size.
- the 48x48x96 pore with pore-wall beads, FP32 and FP64, 20 steps;
- the 32^3 FP64 BGK sphere, the 200 steps the bench times;
- the 256-instance batch: every instance steps on the GPU, the oracle runs a
  sample of instances (the largest box, the largest pore, four seeded ones)
  one by one;
- the 96^3 adjoint workload (3000 steps): its dJ/dgamma in FP64 against a
  central difference of two FP64 forward runs, a property at any size (the
  oracle's reverse pass stores every state, too much for 3000 steps at 96^3).

Tolerances as in test_gpu_parity.py: populations 1e-12 (FP64) / 1e-5 (FP32)
of w_i rho0; bead forces 1e-11 / 1e-5 relative; body force and torque the
same relative to the magnitudes of the bead terms they sum."""
import numpy as np
import pytest

from helpers import W19, observe, oracle_kw
from oracle import oracle as O
from paper_1604_01829_gb300 import workloads as Wl

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 1e-5}
TOL_F = {64: 1e-11, 32: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1604_01829_gb300 import build
    build.build()


def _pair(w, precision):
    """The workload on the GPU (as lb.from_workload builds it) and in the oracle."""
    from paper_1604_01829_gb300 import lb
    g = lb.from_workload(w, precision=precision)
    o = O.OracleLB(w.nx, w.ny, w.nz, **oracle_kw(w.params))
    if w.pore is not None:
        o.set_pore(*w.pore)
    for b in w.bodies:
        q = np.asarray(b.q, np.float64)
        o.add_raspberry(b.beads, b.X, q / np.linalg.norm(q), b.mass, b.inertia, b.F_ext, b.T_ext, b.fixed)
    return g, o


def _pop_error(fg, o):
    fo = o.f.reshape(19, -1)
    fl = slice(None) if o.mask is None else (o.mask == 0)
    err = 0.0
    for i in range(19):                                  # plane by plane: bounded host memory
        err = max(err, float(np.max(np.abs(fg[i][fl] - fo[i][fl]))) / W19[i])
    return observe("pop", err)


def _body_errors(g, o, bodies):
    """Worst errors over the bodies. Body force and torque are sums over the
    beads that nearly cancel once the drag balances the external force, so
    their errors are scaled by the sum of the magnitudes summed (the
    condition of the sum), not by the small result."""
    worst = dict(F=0.0, T=0.0, bead=0.0, X=0.0, q=0.0)
    for b, body in enumerate(bodies):
        Fg, Tg, pbg = g.lb_forces(b, per_bead=True)
        ob = o.body(b)
        pbo = o.bead_forces(b)
        gb = g.lb_get_body(b)
        summed = np.abs(pbo).sum(0).max()
        rmax = np.sqrt((np.asarray(body.beads) ** 2).sum(1)).max()
        sF = max(np.abs(ob["F"]).max(), summed, 1e-300)
        sT = max(np.abs(ob["T"]).max(), rmax * summed, 1e-300)
        worst["F"] = max(worst["F"], np.abs(Fg - ob["F"]).max() / sF)
        worst["T"] = max(worst["T"], np.abs(Tg - ob["T"]).max() / sT)
        worst["bead"] = max(worst["bead"], np.abs(pbg - pbo).max() / max(np.abs(pbo).max(), 1e-300))
        worst["X"] = max(worst["X"], np.abs(gb["X"] - ob["X"]).max())
        worst["q"] = max(worst["q"], np.abs(gb["q"] - ob["q"]).max())
    for k, v in worst.items():
        observe(k, v)
    return worst


@pytest.mark.parametrize("precision,steps", [(32, 2), (64, 1)])
def test_headline_256_workload_matches_oracle_on_the_whole_lattice(precision, steps):
    w = Wl.ellipsoids_256(n_bodies=64, kT=1e-4, precision=precision)
    assert (w.nx, w.ny, w.nz, len(w.bodies), w.nbeads) == (256, 256, 256, 64, 23360)
    g, o = _pair(w, precision)
    for k in range(steps):
        g.lb_set_timing(k == 0)            # the first step eager, as in the timed region; then a graph
        g.lb_step(1)
        o.step(1)
        assert _pop_error(g.lb_get_populations(), o) <= TOL[precision], k
        e = _body_errors(g, o, w.bodies)
        tb = TOL_F[precision]
        assert e["bead"] <= tb and e["F"] <= tb and e["T"] <= tb, (k, e)
        assert e["X"] <= tb and e["q"] <= tb, (k, e)
    g.lb_set_timing(False)
    m, _ = g.lb_conservation()
    mo, _ = o.conservation()
    assert abs(m - mo) <= (1e-12 if precision == 64 else 1e-8) * mo


@pytest.mark.parametrize("precision", [32, 64])
def test_pore_workload_with_wall_beads_matches_oracle(precision):
    w = Wl.pore_48(offset_frac=0.4, precision=precision)
    g, o = _pair(w, precision)
    kT = w.params["kT"]
    g.lb_set_pore_beads(5.0, 6.25, 0.5, kT)
    o.set_pore_beads(w.pore[0], w.pore[1], 5.0, 6.25, 0.5, kT)
    g.lb_record_bodies(200, 64)
    for n in (1, 19):                      # eager single step, then graph replays and an odd step
        g.lb_step(n)
        o.step(n)
        assert _pop_error(g.lb_get_populations(), o) <= TOL[precision]
        e = _body_errors(g, o, w.bodies)
        assert e["bead"] <= TOL_F[precision] and e["F"] <= TOL_F[precision], e


def test_sphere_32_workload_matches_oracle_over_the_timed_steps():
    w = Wl.sphere_32()
    precision = w.params.get("precision", 64)
    assert precision == 64
    g, o = _pair(w, precision)
    g.lb_step(200)
    o.step(200)
    assert _pop_error(g.lb_get_populations(), o) <= TOL[64]
    e = _body_errors(g, o, w.bodies)
    assert e["bead"] <= TOL_F[64] and e["F"] <= TOL_F[64] and e["X"] <= TOL_F[64], e


def test_batched_256_instances_match_oracle_on_sampled_instances():
    from paper_1604_01829_gb300 import lb
    ws = Wl.batched_instances(256)
    B = lb.batch_from_workloads(ws)
    B.lb_batch_set_schedule(256, 4, 0)
    cubic = [k for k, w in enumerate(ws) if w.pore is None]
    pores = [k for k, w in enumerate(ws) if w.pore is not None]
    pick = {max(cubic, key=lambda k: ws[k].nodes), max(pores, key=lambda k: ws[k].nodes)}
    pick |= set(int(k) for k in np.random.default_rng(5).choice(len(ws), 4, replace=False))
    orcs = {}
    for k in sorted(pick):
        w = ws[k]
        o = O.OracleLB(w.nx, w.ny, w.nz, **oracle_kw(w.params))
        if w.pore is not None:
            o.set_pore(*w.pore)
        for b in w.bodies:
            o.add_raspberry(b.beads, b.X, np.asarray(b.q) / np.linalg.norm(b.q), b.mass, b.inertia, b.F_ext,
                            b.T_ext, b.fixed)
        orcs[k] = o
    for n in (1, 4):                       # an eager step, then two graph-replayed pairs
        B.lb_batch_step(n)
        for o in orcs.values():
            o.step(n)
        for k, o in orcs.items():
            assert _pop_error(B.lb_batch_get_populations(k), o) <= TOL[32], k
            F, _ = B.lb_batch_forces(k, 0)
            Fo = o.body(0)["F"]
            assert np.abs(F - Fo).max() <= TOL_F[32] * max(np.abs(Fo).max(), 1e-30), k


def test_adjoint_96_workload_gradient_matches_central_difference():
    from paper_1604_01829_gb300 import lb
    T, Wn = 3000, 200
    w = Wl.ellipsoid_adjoint_96(precision=64)
    assert (w.nx, w.ny, w.nz) == (96, 96, 96)
    L = lb.from_workload(w)
    J, dJdg, _ = L.lb_adjoint_drag(T, Wn, body=0, axis=0)
    L.close()

    def forward(gamma):
        wg = Wl.ellipsoid_adjoint_96(precision=64)
        wg.params["gamma_bead"] = gamma
        Lg = lb.from_workload(wg)
        Lg.lb_step(T - Wn)
        vs = []
        for _ in range(Wn):
            Lg.lb_step(1)
            vs.append(Lg.lb_get_body(0)["V"][0])
        Lg.close()
        return float(np.mean(vs))

    g0 = w.params["gamma_bead"]
    h = 1e-4 * g0
    assert abs(forward(g0) - J) <= 1e-10 * abs(J)
    fd = (forward(g0 + h) - forward(g0 - h)) / (2 * h)
    assert abs(dJdg - fd) <= 1e-4 * abs(fd), (dJdg, fd)
