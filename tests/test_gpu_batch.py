"""Batched lattices (lb_batch_*): every instance of a batch of uneven
periodic and pore lattices, with and without raspberries, against the FP64
oracle run on that instance alone; schedule and autotuner leave results
unchanged; a batch checkpoint resumes every instance. Tolerances as in
test_gpu_parity.py."""
import numpy as np
import pytest

from helpers import W19, observe, oracle_kw, perturbed_populations
from oracle import oracle as O
from paper_1604_01829_gb300 import workloads as Wl

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 1e-5}
MRT = dict(collision=1, gamma_shear=-0.45, gamma_bulk=-0.2, gamma_odd=0.3, gamma_even=-0.1)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1604_01829_gb300 import build
    build.build()


def _cases(noise):
    """(params, pore, bodies) of six uneven instances (pores along z, x and y)."""
    kT = dict(kT=1e-4) if noise else {}
    g = Wl.paper_gamma_to_lattice(50.0)
    sph = Wl.sphere_raspberry(2.0)
    ell = Wl.ellipsoid_raspberry(3.0, 1.5, 1.5, seed=4)
    return [
        (dict(nx=20, ny=11, nz=9, seed=1, body_force=(1e-5, 0, 0), **MRT, **kT), None, []),
        (dict(nx=18, ny=18, nz=7, seed=2, gamma_bead=g, **MRT, **kT), (7.2, 2),
         [dict(beads=sph, X=[9.4, 8.7, 3.3], mass=34.0, inertia=(50, 50, 50), F_ext=(0, 0, 1e-3))]),
        (dict(nx=13, ny=16, nz=17, seed=3, gamma_bead=g, compensate_force=1, instance=7, **MRT, **kT), None,
         [dict(beads=ell, X=[6.2, 8.1, 8.9], q=[0.9, 0.1, 0.3, -0.2], mass=40.0, inertia=(20, 50, 50),
               F_ext=(5e-4, 0, 0))]),
        (dict(nx=9, ny=14, nz=14, seed=4, **MRT, **kT), (5.5, 0), []),
        (dict(nx=24, ny=8, nz=12, seed=5, gamma_bead=g, **MRT, **kT), None,
         [dict(beads=sph, X=[5.1, 4.3, 6.2], fixed=True, V=(0, 0, 0)),
          dict(beads=sph, X=[17.3, 4.1, 5.8], mass=34.0, inertia=(50, 50, 50), F_ext=(0, 1e-3, 0))]),
        (dict(nx=15, ny=11, nz=13, seed=6, gamma_bead=g, **MRT, **kT), (5.6, 1),
         [dict(beads=sph, X=[7.6, 5.2, 6.9], mass=34.0, inertia=(50, 50, 50), F_ext=(0, 1e-3, 0))]),
    ]


def _build(cases, precision):
    from paper_1604_01829_gb300 import lb
    B = lb.LBBatch([dict(c[0], precision=precision) for c in cases])
    orcs = []
    for k, (p, pore, bodies) in enumerate(cases):
        o = O.OracleLB(p["nx"], p["ny"], p["nz"], **oracle_kw(p))
        if pore is not None:
            B.lb_batch_set_pore(k, *pore)
            o.set_pore(*pore)
        f = perturbed_populations(p["nx"] * p["ny"] * p["nz"], seed=30 + k)
        B.lb_batch_set_populations(k, f)
        o.set_populations(f)
        for b in bodies:
            q = b.get("q", [1, 0, 0, 0])
            B.lb_batch_add_raspberry(k, b["beads"], b["X"], q, b.get("mass", 1.0), b.get("inertia", (1, 1, 1)),
                                     b.get("F_ext"), None, b.get("fixed", False))
            o.add_raspberry(b["beads"], b["X"], np.asarray(q) / np.linalg.norm(q), b.get("mass", 1.0),
                            b.get("inertia", (1, 1, 1)), b.get("F_ext", (0, 0, 0)), (0, 0, 0),
                            b.get("fixed", False))
        orcs.append(o)
    return B, orcs


def _errors(B, orcs, cases):
    out = []
    for k, o in enumerate(orcs):
        fg = B.lb_batch_get_populations(k)
        fo = o.populations()
        fl = np.ones(fg.shape[1], bool) if o.mask is None else o.mask == 0
        out.append(observe("pop", np.max(np.abs(fg[:, fl] - fo[:, fl]) / W19[:, None])))
        for j in range(len(cases[k][2])):
            F, _ = B.lb_batch_forces(k, j)
            Fo = o.body(j)["F"]
            out.append(observe("F", np.abs(F - Fo).max() / max(np.abs(Fo).max(), 1e-30)) * 1e-1)
    return out


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("noise", [False, True])
def test_batch_matches_oracle_per_instance(precision, noise):
    cases = _cases(noise)
    B, orcs = _build(cases, precision)
    for n in (1, 2, 5):          # odd counts mix eager steps with the two-step graph
        B.lb_batch_step(n)
        for o in orcs:
            o.step(n)
        errs = _errors(B, orcs, cases)
        assert max(errs) <= TOL[precision], errs


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("nsub", [2, 3])
def test_batch_md_substeps_match_oracle(precision, nsub):
    """MD substeps in a batch (every instance the same count): bodies move by
    1/n between the couplings of one LB step, with per-substep bead noise."""
    cases = [(dict(c[0], md_substeps=nsub), c[1], c[2]) for c in _cases(noise=True)]
    B, orcs = _build(cases, precision)
    for n in (1, 2, 3):
        B.lb_batch_step(n)
        for o in orcs:
            o.step(n)
        errs = _errors(B, orcs, cases)
        assert max(errs) <= TOL[precision], errs


@pytest.mark.parametrize("schedule", [(64, 4, 0), (128, 8, 1), (256, 4, 0), (256, 2, 1), (128, 2, 2)])
def test_batch_schedule_does_not_change_results(schedule):
    cases = _cases(True)
    B, orcs = _build(cases, 32)
    B.lb_batch_set_schedule(*schedule)
    B.lb_batch_step(4)
    for o in orcs:
        o.step(4)
    assert max(_errors(B, orcs, cases)) <= TOL[32]


def test_autotune_restores_state_and_picks_a_valid_schedule():
    cases = _cases(False)
    B, orcs = _build(cases, 64)
    B.lb_batch_step(3)
    for o in orcs:
        o.step(3)
    before = [B.lb_batch_get_populations(k) for k in range(len(cases))]
    chosen, ms = B.lb_batch_autotune(4)
    assert chosen[0] in (64, 128, 256) and chosen[1] >= 1 and chosen[2] in (0, 1, 2) and ms > 0
    info = B.lb_batch_info()
    assert info["step"] == 3 and info["schedule"] == chosen
    for k in range(len(cases)):
        assert np.array_equal(B.lb_batch_get_populations(k), before[k])
    B.lb_batch_step(3)
    for o in orcs:
        o.step(3)
    assert max(_errors(B, orcs, cases)) <= TOL[64]


def test_batch_instance_equals_single_handle():
    from paper_1604_01829_gb300 import lb
    cases = _cases(True)
    B, _ = _build(cases, 64)
    k = 2
    p, pore, bodies = cases[k]
    kw = {key: v for key, v in p.items() if key not in ("nx", "ny", "nz")}
    S = lb.LB(p["nx"], p["ny"], p["nz"], precision=64, **kw)
    S.lb_set_populations(perturbed_populations(p["nx"] * p["ny"] * p["nz"], seed=30 + k))
    b = bodies[0]
    S.lb_add_raspberry(b["beads"], b["X"], b["q"], b["mass"], b["inertia"], b["F_ext"])
    B.lb_batch_step(6)
    S.lb_step(6)
    assert np.abs(B.lb_batch_get_populations(k) - S.lb_get_populations()).max() <= 1e-13
    assert np.abs(B.lb_batch_get_body(k)["X"] - S.lb_get_body(0)["X"]).max() <= 1e-13


def test_pore_wall_beads_in_a_batch():
    """Two pore instances with wall beads (one along z, one along x) and a
    periodic one; each equals the oracle run on that instance alone."""
    from paper_1604_01829_gb300 import lb
    g = Wl.paper_gamma_to_lattice(50.0)
    sph = Wl.sphere_raspberry(2.0)
    cases = [(dict(nx=20, ny=20, nz=14, seed=1, gamma_bead=g, kT=1e-4, **MRT), (7.5, 2), (10 + 4.9, 10.3, 6.1),
              (2e-3, 0, 0)),
             (dict(nx=12, ny=10, nz=9, seed=2, kT=1e-4, **MRT), None, None, None),
             (dict(nx=14, ny=18, nz=18, seed=3, gamma_bead=g, kT=1e-4, **MRT), (7.0, 0), (7.2, 9.1, 9 - 4.4),
              (0, 0, -2e-3))]
    B = lb.LBBatch([dict(c[0], precision=64) for c in cases])
    orcs = []
    for k, (p, pore, X, F) in enumerate(cases):
        o = O.OracleLB(p["nx"], p["ny"], p["nz"], **oracle_kw(p))
        if pore is not None:
            B.lb_batch_set_pore(k, *pore)
            o.set_pore(*pore)
            B.lb_batch_set_pore_beads(k, 2.0, 2.5, 0.5, 2e-3)
            o.set_pore_beads(pore[0], pore[1], 2.0, 2.5, 0.5, 2e-3)
            B.lb_batch_add_raspberry(k, sph, X, [1, 0, 0, 0], 34.0, (50, 50, 50), F, None, False)
            o.add_raspberry(sph, X, (1, 0, 0, 0), 34.0, (50, 50, 50), F, (0, 0, 0), False)
        orcs.append(o)
    for _ in range(3):
        B.lb_batch_step(3)
        for o in orcs:
            o.step(3)
        for k in (0, 2):
            F, T = B.lb_batch_forces(k, 0)
            Fo, To = orcs[k].body(0)["F"], orcs[k].body(0)["T"]
            assert np.abs(F - Fo).max() <= 1e-11 * np.abs(Fo).max(), (k, F, Fo)
            assert np.abs(T - To).max() <= 1e-11 * np.abs(To).max(), (k, T, To)
            Xg = B.lb_batch_get_body(k, 0)["X"]
            assert np.abs(Xg - orcs[k].body(0)["X"]).max() <= 1e-11


@pytest.mark.parametrize("precision", [64, 32])
def test_batch_checkpoint_resume(precision):
    """A checkpoint of the whole batch taken at an odd step count and loaded
    into a fresh batch built the same way resumes every instance (up to the
    order of the bead-force atomics); a batch with other instances refuses it."""
    from paper_1604_01829_gb300 import lb
    cases = _cases(noise=True)
    A, _ = _build(cases, precision)
    A.lb_batch_step(5)
    ck = A.lb_batch_checkpoint_save()
    A.lb_batch_step(6)
    B, _ = _build(cases, precision)
    B.lb_batch_step(2)                     # some other state first: the load replaces all of it
    B.lb_batch_checkpoint_load(ck)
    B.lb_batch_step(6)
    assert A.lb_batch_info()["step"] == B.lb_batch_info()["step"] == 11
    for k in range(len(cases)):
        fa, fb = A.lb_batch_get_populations(k), B.lb_batch_get_populations(k)
        d = float((np.abs(fa - fb).max(axis=1) / W19).max())
        assert d <= (1e-13 if precision == 64 else 1e-6), (k, d)
        for j in range(len(cases[k][2])):
            Fa, _ = A.lb_batch_forces(k, j)
            Fb, _ = B.lb_batch_forces(k, j)
            assert np.abs(Fa - Fb).max() <= (1e-12 if precision == 64 else 1e-6) * max(np.abs(Fa).max(), 1e-30)
    other_cases = [(dict(c[0], nx=c[0]["nx"] + (k == 3)), c[1], c[2]) for k, c in enumerate(cases)]
    C2, _ = _build(other_cases, precision)
    with pytest.raises(lb.LBError) as e:
        C2.lb_batch_checkpoint_load(ck)
    assert e.value.status == lb.LB_ERR_STATE
    with pytest.raises(lb.LBError) as e:
        C2.lb_batch_checkpoint_load(ck[:50])
    assert e.value.status == lb.LB_ERR_ARG


def test_pore_cross_section_beyond_the_compact_limit_is_refused():
    """A batched pore instance stores its fluid nodes only from the first step
    on, indexing a cross-section's fluid positions in 16 bits: a pore of
    radius 150 (about 70,700 fluid positions across the axis) is refused at
    the first step with LB_ERR_ARG and a message naming the limit, and a
    pore just inside it steps."""
    from paper_1604_01829_gb300 import lb
    big = lb.LBBatch([dict(nx=304, ny=304, nz=2, **MRT)])
    big.lb_batch_set_pore(0, 150.0, 2)
    with pytest.raises(lb.LBError) as ei:
        big.lb_batch_step(1)
    assert ei.value.status == lb.LB_ERR_ARG and "65534" in str(ei.value)
    big.close()
    ok = lb.LBBatch([dict(nx=290, ny=290, nz=2, **MRT)])
    ok.lb_batch_set_pore(0, 144.0, 2)                      # about 65,100 fluid positions
    ok.lb_batch_step(2)
    f = ok.lb_batch_get_populations(0)
    assert np.isfinite(f).all()
    ok.close()
