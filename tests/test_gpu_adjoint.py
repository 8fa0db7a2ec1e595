"""Hand-written adjoint of the deterministic step (lb_adjoint_drag) against
the oracle's reverse pass (itself pinned to finite differences on the CPU),
in FP64 and FP32, periodic and pore, BGK and MRT, several checkpoint
schedules; and the autograd wrapper.

Tolerances: FP64 J to 1e-12 and gradients to 1e-8 relative (the two reverse
passes differ in formulation and summation order, accumulated over tens of
steps); FP32 storage: J and gradients to 1e-5 relative (the FP32 forward
state and adjoint fields round to 6e-8 relative per operation; the worst
errors these tests have shown on GB300 are 8.5e-8 for J and 1.2e-7 for the
gradients)."""
import numpy as np
import pytest

from helpers import observe, oracle_kw
from oracle import oracle as O
from paper_1604_01829_gb300 import workloads as Wl

pytestmark = pytest.mark.gpu

MRT = dict(collision=1, gamma_shear=-0.3, gamma_bulk=-0.3, gamma_odd=0.1, gamma_even=0.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1604_01829_gb300 import build
    build.build()


def _pair(precision, params, pore=None, gamma=0.1, n=12):
    from paper_1604_01829_gb300 import lb
    params = dict(params, gamma_bead=gamma, compensate_force=0 if pore else 1)
    g = lb.LB(n, n, n, precision=precision, **params)
    o = O.OracleLB(n, n, n, **oracle_kw(params))
    if pore:
        g.lb_set_pore(*pore)
        o.set_pore(*pore)
    sph = Wl.sphere_raspberry(2.0)
    for tgt in (g, o):
        tgt_add = tgt.lb_add_raspberry if hasattr(tgt, "lb_add_raspberry") else tgt.add_raspberry
        tgt_add(sph, [6.3, 5.9, 6.1], [1, 0, 0, 0], 40.0, (60, 60, 60), (0, 0, 2e-3), (0, 0, 0), 2)
    g.lb_step(5)
    o.step(5)
    return g, o


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("case", ["mrt", "bgk", "pore"])
@pytest.mark.parametrize("checkpoints", [0, 3, 30])
def test_adjoint_matches_oracle(precision, case, checkpoints):
    params = dict(collision=0, tau=0.9) if case == "bgk" else dict(MRT)
    pore = (5.5, 2) if case == "pore" else None
    g, o = _pair(precision, params, pore)
    Jg, dgg, dsg = g.lb_adjoint_drag(30, 10, body=0, axis=2, checkpoints=checkpoints)
    Jo, dgo, dso = o.adjoint_drag(30, 10, body=0, axis=2)
    observe("J", abs(Jg - Jo) / abs(Jo))
    observe("dJ_dgamma", abs(dgg - dgo) / abs(dgo))
    observe("dJ_ds", np.abs(dsg - dso).max() / np.abs(dso).max())
    if precision == 64:
        assert abs(Jg - Jo) <= 1e-9 * abs(Jo)
        assert abs(dgg - dgo) <= 1e-8 * abs(dgo)
        assert np.abs(dsg - dso).max() <= 1e-8 * np.abs(dso).max()
    else:
        assert abs(Jg - Jo) <= 1e-5 * abs(Jo)
        assert abs(dgg - dgo) <= 1e-5 * abs(dgo)
        assert np.abs(dsg - dso).max() <= 1e-5 * np.abs(dso).max()
    # the handle ends where plain steps would leave it
    assert observe("pop", np.abs(g.lb_get_populations() - o.populations()).max()) <= (1e-12 if precision == 64 else 1e-5)


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("case", ["mrt", "pore"])
@pytest.mark.parametrize("snapshots", [1, 2, 4, 16])
def test_binomial_schedule_matches_oracle(precision, case, snapshots):
    """Binomial (revolve) checkpointing with 1-16 kept states: each reversed
    step re-runs only its prologue and coupling from a restored state. Same
    results as the oracle's stored-every-state reverse pass, and the handle
    ends where plain steps would leave it."""
    from paper_1604_01829_gb300 import lb
    params = dict(MRT)
    pore = (5.5, 2) if case == "pore" else None
    g, o = _pair(precision, params, pore)
    Jg, dgg, dsg, st = g.lb_adjoint_drag_ex(30, 10, body=0, axis=2, schedule=lb.LB_ADJ_BINOMIAL,
                                            snapshots=snapshots, with_stats=True)
    Jo, dgo, dso = o.adjoint_drag(30, 10, body=0, axis=2)
    observe("J", abs(Jg - Jo) / abs(Jo))
    observe("dJ_dgamma", abs(dgg - dgo) / abs(dgo))
    observe("dJ_ds", np.abs(dsg - dso).max() / np.abs(dso).max())
    if precision == 64:
        assert abs(Jg - Jo) <= 1e-9 * abs(Jo)
        assert abs(dgg - dgo) <= 1e-8 * abs(dgo)
        assert np.abs(dsg - dso).max() <= 1e-8 * np.abs(dso).max()
    else:
        assert abs(Jg - Jo) <= 1e-5 * abs(Jo)
        assert abs(dgg - dgo) <= 1e-5 * abs(dgo)
        assert np.abs(dsg - dso).max() <= 1e-5 * np.abs(dso).max()
    assert observe("pop", np.abs(g.lb_get_populations() - o.populations()).max()) <= \
        (1e-12 if precision == 64 else 1e-5)
    # no step runs more often than the binomial bound allows
    from math import comb
    r = 0
    S = min(snapshots, 30)
    while comb(S + r, S) < 30:
        r += 1
    assert st["forward_steps"] == 30 and st["reversed_steps"] == 30
    assert 0 < st["recompute_steps"] <= r * 30, (st, r)


def test_schedules_agree_and_the_workspace_is_reused():
    """Two-level with every state kept (one step per segment), two-level
    with sqrt(T) slots and binomial with 3 states: the same gradients to
    the summation order of the re-run steps' atomics (FP64, 1e-12); a second
    call of the same size reuses the workspace (no allocation), and the time
    split adds up."""
    from paper_1604_01829_gb300 import lb
    out = []
    for sched, snaps in ((lb.LB_ADJ_TWO_LEVEL, 40), (lb.LB_ADJ_TWO_LEVEL, 0), (lb.LB_ADJ_BINOMIAL, 3)):
        g, _ = _pair(64, dict(MRT))
        r1 = g.lb_adjoint_drag_ex(40, 10, schedule=sched, snapshots=snaps, with_stats=True)
        r2 = g.lb_adjoint_drag_ex(40, 10, schedule=sched, snapshots=snaps, with_stats=True)
        assert r1[3]["alloc_ms"] > 0 and r2[3]["alloc_ms"] == 0.0
        assert r2[3]["workspace_bytes"] == r1[3]["workspace_bytes"]
        for st in (r1[3], r2[3]):
            assert st["forward_ms"] > 0 and st["reverse_ms"] > 0 and st["recompute_ms"] >= 0
        out.append(r1[:3])
        g.close()
    J0, dg0, ds0 = out[0]
    for J, dg, ds in out[1:]:
        assert abs(J - J0) <= 1e-12 * abs(J0)
        assert abs(dg - dg0) <= 1e-12 * abs(dg0)
        assert np.abs(ds - ds0).max() <= 1e-12 * np.abs(ds0).max()


def test_fp32_drag_against_the_fp64_oracle():
    """The drag error of FP32 deviation storage against the FP64 oracle, on
    a reduced form of the adjoint workload (the same physics: MRT at the
    paper's nu = 0.016, kT = 0, the paper's bead friction, a 1:3 prolate
    raspberry pulled along its long axis with the compensating force on the
    fluid): 24^3 box, semi-axes 6 x 2 x 2, 400 steps, J = mean velocity over
    the last 50. FP64 on the GPU gives the oracle's J to 1e-9 relative (the
    two differ in summation order and FMA contraction, O(1e-16) per operation
    accumulated over 400 steps; measured on GB300: 5.5e-11); FP32 within
    1e-4 (measured on GB300: 2.7e-6; the 96^3 / 3000-step bench workload
    gives 2.2e-5 between the FP32 and FP64 GPU runs)."""
    import math
    from paper_1604_01829_gb300 import lb
    beads = Wl.ellipsoid_raspberry(6.0, 2.0, 2.0, seed=1609)
    mass = 4.0 / 3.0 * math.pi * 6 * 4
    inertia = tuple(Wl.solid_ellipsoid_inertia(mass, 6, 2, 2))
    params = dict(collision=1, rho0=1.0, kT=0.0, gamma_bead=Wl.paper_gamma_to_lattice(20.0), compensate_force=1,
                  **Wl.mrt_rates(Wl.NU_PAPER))
    T, W = 400, 50
    X = [12.0, 12.0, 12.0]

    def run_gpu(precision):
        h = lb.LB(24, 24, 24, precision=precision, **params)
        h.lb_add_raspberry(beads, X, (1, 0, 0, 0), mass, inertia, (1e-3, 0, 0), None, 2)
        h.lb_step(T - W)
        v = []
        for _ in range(W):
            h.lb_step(1)
            v.append(h.lb_get_body(0)["V"][0])
        h.close()
        return float(np.mean(v))

    o = O.OracleLB(24, 24, 24, **oracle_kw(params))
    o.add_raspberry(beads, X, (1, 0, 0, 0), mass, inertia, (1e-3, 0, 0), (0, 0, 0), 2)
    o.step(T - W)
    vo = []
    for _ in range(W):
        o.step(1)
        vo.append(o.body(0)["V"][0])
    Jo = float(np.mean(vo))
    J64, J32 = run_gpu(64), run_gpu(32)
    e32 = observe("drag_fp32_vs_oracle", abs(J32 / Jo - 1))
    assert observe("drag_fp64_vs_oracle", abs(J64 / Jo - 1)) <= 1e-9
    assert e32 <= 1e-4, e32


def test_adjoint_rejects_noise_and_free_rotation():
    from paper_1604_01829_gb300 import lb
    g = lb.LB(8, 8, 8, precision=64, kT=1e-4, gamma_bead=0.1, **MRT)
    g.lb_add_raspberry(Wl.sphere_raspberry(1.5), [4, 4, 4], fixed=2)
    with pytest.raises(lb.LBError):
        g.lb_adjoint_drag(4, 2)
    h = lb.LB(8, 8, 8, precision=64, gamma_bead=0.1, **MRT)
    h.lb_add_raspberry(Wl.sphere_raspberry(1.5), [4, 4, 4], fixed=0)
    with pytest.raises(lb.LBError):
        h.lb_adjoint_drag(4, 2)


def test_autograd_function_chains_the_adjoint():
    import torch
    from paper_1604_01829_gb300 import adjoint, lb
    sph = Wl.sphere_raspberry(2.0)

    def make(gamma, beads):
        L = lb.LB(12, 12, 12, precision=64, gamma_bead=gamma, compensate_force=1, **MRT)
        L.lb_add_raspberry(beads, [6.3, 5.9, 6.1], mass=40.0, inertia=(60, 60, 60), F_ext=(0, 0, 2e-3), fixed=2)
        return L

    gamma = torch.tensor(0.1, dtype=torch.float64, requires_grad=True)
    beads = torch.tensor(sph, dtype=torch.float64, requires_grad=True)
    J = adjoint.terminal_velocity(gamma, beads, make, 30, 10)
    xi = 2e-3 / J                    # drag of the pulled colloid
    xi.backward()
    o = O.OracleLB(12, 12, 12, gamma_bead=0.1, compensate_force=1, **MRT)
    o.add_raspberry(sph, [6.3, 5.9, 6.1], mass=40.0, inertia=(60, 60, 60), F_ext=(0, 0, 2e-3), fixed=2)
    Jo, dgo, dso = o.adjoint_drag(30, 10)
    assert abs(J.item() - Jo) <= 1e-9 * abs(Jo)
    assert abs(gamma.grad.item() - (-2e-3 / Jo ** 2) * dgo) <= 1e-8 * abs((2e-3 / Jo ** 2) * dgo)
    assert np.abs(beads.grad.numpy() - (-2e-3 / Jo ** 2) * dso).max() <= 1e-8 * np.abs((2e-3 / Jo ** 2) * dso).max()


@pytest.mark.parametrize("param,p_true,p0", [("gamma", 0.15, 0.08), ("scale", 1.1, 1.0)])
def test_calibration_recovers_the_parameter_of_a_target_drag(param, p_true, p0):
    """Calibration with the adjoint: the drag of the pulled raspberry for a
    known bead friction (or size) is the target; Newton iterations with the
    adjoint's derivative from another starting value recover that friction
    (or size)."""
    from paper_1604_01829_gb300 import adjoint, lb
    sph = Wl.sphere_raspberry(2.0)
    F = 2e-3

    def make(gamma, beads):
        L = lb.LB(12, 12, 12, precision=64, gamma_bead=gamma, compensate_force=1, **MRT)
        L.lb_add_raspberry(beads, [6.3, 5.9, 6.1], mass=40.0, inertia=(60, 60, 60), F_ext=(0, 0, F), fixed=2)
        return L

    g_fix = 0.12
    if param == "gamma":
        L = make(p_true, sph)
    else:
        L = make(g_fix, p_true * np.asarray(sph))
    J, _, _ = L.lb_adjoint_drag(40, 10)
    L.close()
    target = F / J
    p, xi, hist = adjoint.calibrate(target, F, make, sph, p0 if param == "gamma" else g_fix, 40, 10, param=param)
    if param == "scale":
        assert abs(hist[0][0] - 1.0) < 1e-15
    assert abs(p / p_true - 1) < 1e-6, hist
    assert abs(xi / target - 1) < 1e-6
    assert len(hist) <= 8
