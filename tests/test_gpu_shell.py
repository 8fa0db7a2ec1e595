"""Raspberry shell construction on the GPU (lb_relax_shells, through the C ABI)
against the construction oracle (oracle/construction.py): element-wise
parity of the nearest surface points and of whole relaxations in FP64 and
FP32, sampled one-step parity at the largest shell sizes, the optimal
2/4/6-point arrangements, many shells in one launch equal to each shell
alone, the cell-list pair search against the all-pairs one and its fallback
for beads outside its box, and argument errors.

Tolerances: FP64 differs from the oracle by contraction (FMA) and division
rounding only, O(1e-15) per operation, and the damped scheme does not amplify
it over the short runs compared: 1e-9 absolute on positions of order 1-10.
FP32 rounds positions to 2^-21 ~ 5e-7 at |x| < 8 and forces to ~1e-6
relative each step, and the damped, contracting scheme does not amplify
it: over the 150-200 steps compared the errors stay below 1e-5 absolute
(worst seen on GB300: 4.0e-6; the FP32 kernel sums in a fixed order, so the
figure repeats run to run)."""
import math

import numpy as np
import pytest

from helpers import observe
from oracle import construction as C

pytestmark = pytest.mark.gpu

SHAPES = [(3.0, 3.0, 3.0), (6.0, 2.5, 2.5), (2.0, 4.0, 4.0), (4.0, 3.0, 2.0)]


def _random_starts(n_per, spread, seed=11):
    from paper_1604_01829_gb300 import workloads as W
    return [W.random_shell_start(*ax, n_per, seed=seed + i, spread=spread) for i, ax in enumerate(SHAPES)]


def _spread_starts(density=0.8, jitter=0.05, seed=21):
    """Evenly spread starts, about `density` beads per unit area (at 0.5 no
    pair starts closer than ~1, so steps of dt^2 = 1e-4 stay stable; at 0.8
    pairs start from ~0.65 and need the paper's dt^2 = 1e-6)."""
    from paper_1604_01829_gb300 import workloads as W
    return [W.spread_shell_start(*ax, max(4, int(density * W.ellipsoid_area(*ax))), seed=seed + i, jitter=jitter)
            for i, ax in enumerate(SHAPES)]


@pytest.mark.parametrize("precision,tol", [(64, 1e-12), (32, 2e-6)])
def test_nearest_surface_points_match_oracle(precision, tol):
    from paper_1604_01829_gb300 import lb
    starts = _random_starts(64, spread=0.4)
    out = lb.lb_relax_shells(SHAPES, starts, steps=0, precision=precision, project_final=True)
    for ax, X0, X in zip(SHAPES, starts, out):
        ref = np.array([C.surface_point(p, ax)[0] for p in X0])
        scale = max(ax)
        assert np.abs(X - ref).max() <= tol * scale, (precision, ax, np.abs(X - ref).max())
        assert np.abs(((X / np.array(ax)) ** 2).sum(1) - 1).max() < (1e-12 if precision == 64 else 2e-6)


@pytest.mark.parametrize("precision,tol", [(64, 1e-9), (32, 1e-5)])
@pytest.mark.parametrize("project", [False, True])
@pytest.mark.parametrize("search", [1, 2])
def test_relaxation_matches_oracle(precision, tol, project, search):
    from paper_1604_01829_gb300 import lb
    starts = _spread_starts(density=0.5)
    steps = 150
    out = lb.lb_relax_shells(SHAPES, starts, steps=steps, dt=0.01, eta=100.0, precision=precision,
                             project_final=project, pair_search=search)
    for ax, X0, X in zip(SHAPES, starts, out):
        ref = C.relax_shell(X0, ax, steps, dt=0.01, eta=100.0, project_final=project)
        err = observe("X", np.abs(X - ref).max())
        assert err <= tol, (precision, ax, err)
        assert np.abs(X - X0).max() > 100 * tol          # the beads did move


def test_paper_time_step_matches_oracle():
    """The paper's own dt = 0.001, eta = 1000 (eta dt = 1) from a start at
    0.8 beads per unit area, FP64 and FP32."""
    from paper_1604_01829_gb300 import lb
    starts = _spread_starts()
    for precision, tol, search in ((64, 1e-9, 1), (64, 1e-9, 2), (32, 1e-5, 2)):
        out = lb.lb_relax_shells(SHAPES, starts, steps=200, precision=precision, project_final=False,
                                 pair_search=search)
        for ax, X0, X in zip(SHAPES, starts, out):
            ref = C.relax_shell(X0, ax, 200, project_final=False)
            assert observe(f"X{precision}", np.abs(X - ref).max()) <= tol, (precision, ax, np.abs(X - ref).max())
            assert np.abs(X - X0).max() > 100 * tol


@pytest.mark.parametrize("n", [1000, 1500, 3000, 4096])
@pytest.mark.parametrize("search", [1, 2])
def test_one_step_at_full_shell_sizes_on_sampled_beads(n, search):
    """From rest, one step moves bead i by dt^2 F_i; the oracle computes F_i
    of sampled beads one by one (all n - 1 partners) at every beads-per-thread
    layout (1, 2 and 4 beads per thread)."""
    from paper_1604_01829_gb300 import lb, workloads as W
    a = math.sqrt(n / (4 * math.pi))          # sphere with one bead per unit area
    ax = (1.3 * a, a, 0.8 * a)
    X0 = W.spread_shell_start(*ax, n, seed=n, jitter=0.02)
    dt = 0.001
    p64 = 32 if (search == 2 and n == 4096) else 64          # an FP64 cell list of 4096 beads does not fit
    (X,) = lb.lb_relax_shells([ax], [X0], steps=1, dt=dt, eta=1000.0, precision=p64, project_final=False,
                              pair_search=search)
    rng = np.random.default_rng(3)
    for i in rng.choice(n, 12, replace=False):
        rs, _ = C.surface_point(X0[i], ax)
        F = -2.0 * 1000.0 * (X0[i] - rs)
        d = X0[i] - X0
        r2 = (d * d).sum(1)
        for j in np.nonzero(r2 < (C.WCA_CUT * 1.4) ** 2)[0]:
            if j != i:
                F = F + C.wca_force(d[j], 1.4, 0.1)
        assert np.allclose(X[i], X0[i] + dt * dt * F, rtol=0, atol=1e-10 if p64 == 64 else 1e-5), i
    (X32,) = lb.lb_relax_shells([ax], [X0], steps=1, dt=dt, eta=1000.0, precision=32, project_final=False,
                                pair_search=search)
    assert observe("X32_vs_64", np.abs(X32 - X).max()) < 1e-4


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("n,edge_over_R", [(2, 2.0), (4, math.sqrt(8.0 / 3.0)), (6, math.sqrt(2.0))])
def test_optimal_arrangements_on_a_small_sphere(precision, n, edge_over_R):
    from paper_1604_01829_gb300 import lb
    R = 0.6
    rng = np.random.default_rng(7 + n)
    u = rng.normal(size=(n, 3))
    X0 = R * u / np.linalg.norm(u, axis=1)[:, None]
    (X,) = lb.lb_relax_shells([(R, R, R)], [X0], steps=4000, dt=0.01, eta=100.0, precision=precision)
    d = np.sqrt(((X[:, None] - X[None]) ** 2).sum(-1))
    nn = np.sort(d + np.eye(n) * 10, axis=1)[:, 0]
    tol = 2e-6 if precision == 64 else 2e-5
    assert np.allclose(nn, edge_over_R * R, atol=tol), nn


def test_many_shells_in_one_launch_equal_each_alone():
    from paper_1604_01829_gb300 import lb, workloads as W
    rng = np.random.default_rng(5)
    axes, starts = [], []
    for s in range(40):
        ax = tuple(rng.uniform(1.5, 6.0, 3))
        n = int(rng.integers(5, 300))
        axes.append(ax)
        starts.append(W.spread_shell_start(*ax, n, seed=100 + s, jitter=0.05))
    for search in (1, 2):
        together = lb.lb_relax_shells(axes, starts, steps=60, precision=32, pair_search=search)
        for s in (0, 7, 23, 39):
            (alone,) = lb.lb_relax_shells([axes[s]], [starts[s]], steps=60, precision=32, pair_search=search)
            assert np.array_equal(alone, together[s])


def test_cell_list_falls_back_when_beads_leave_its_box():
    """Beads started far outside the surface lie outside the cell grid's box
    (1.25 a + 1): those steps test all pairs; the result matches the oracle."""
    from paper_1604_01829_gb300 import lb, workloads as W
    ax = (4.0, 3.0, 2.5)
    X0 = W.spread_shell_start(*ax, 60, seed=3, jitter=0.02)
    X0[:5] *= 1.9                                              # beyond 1.25 a + 1 on every axis
    out = lb.lb_relax_shells([ax], [X0], steps=120, precision=64, project_final=False, pair_search=2)
    ref = C.relax_shell(X0, ax, 120, project_final=False)
    assert np.abs(out[0] - ref).max() <= 1e-9


def test_long_relaxation_spreads_beads_evenly():
    """A raspberry's outer shell (one bead per unit area) after 2e5 steps:
    every bead on the surface and nearest-neighbour distances close to the
    hexagonal spacing (2/sqrt3)^(1/2) = 1.075 at unit density, more evenly
    than the farthest-point start."""
    from paper_1604_01829_gb300 import raspberry, workloads as W
    (beads,) = raspberry.build_raspberries([(8.0, 4.0, 4.0)], steps=200000, seed=1, fill=False,
                                           inner_offset=0.0)
    start = W.spread_shell_start(8.0, 4.0, 4.0, len(beads), seed=1 * 1000003)
    nn0 = C.nearest_neighbour_distances(start)
    ax = np.array([8.0, 4.0, 4.0])
    assert np.abs(((beads / ax) ** 2).sum(1) - 1).max() < 2e-6
    nn = C.nearest_neighbour_distances(beads)
    assert nn.min() > 0.8 and abs(np.median(nn) - 1.075) < 0.1, (nn.min(), np.median(nn))
    assert nn.std() / nn.mean() < 0.5 * nn0.std() / nn0.mean(), (nn.std() / nn.mean(), nn0.std() / nn0.mean())


def test_argument_errors():
    from paper_1604_01829_gb300 import lb
    X0 = np.zeros((5, 3)) + 1.0
    with pytest.raises(lb.LBError) as e:
        lb.lb_relax_shells([(1, 1, 1)], [np.ones((4097, 3))], steps=1)
    assert e.value.status == lb.LB_ERR_ARG
    with pytest.raises(lb.LBError) as e:
        lb.lb_relax_shells([(1, 1, -1)], [X0], steps=1)
    assert e.value.status == lb.LB_ERR_ARG
    with pytest.raises(lb.LBError) as e:
        lb.lb_relax_shells([(1, 1, 1)], [X0], steps=1, dt=0.1, eta=100.0)     # eta dt > 2
    assert e.value.status == lb.LB_ERR_ARG
    with pytest.raises(lb.LBError) as e:
        lb.lb_relax_shells([(1, 1, 1)], [X0], steps=1, precision=16)
    assert e.value.status == lb.LB_ERR_ARG
    with pytest.raises(lb.LBError) as e:
        lb.lb_relax_shells([(1, 1, 1)], [X0], steps=1, pair_search=3)
    assert e.value.status == lb.LB_ERR_ARG
    with pytest.raises(lb.LBError) as e:                     # FP64 cell list of 4096 beads: no room
        lb.lb_relax_shells([(20, 20, 20)], [np.ones((4096, 3))], steps=1, precision=64, pair_search=2)
    assert e.value.status == lb.LB_ERR_ARG
