"""Edge cases of the CUDA path against the oracle (through the C ABI):

- the smallest lattices the library accepts (2 nodes along an axis: both
  neighbours of a node along that axis are the same node), with MRT noise and
  a body force, FP64 and FP32, odd and even step counts;
- a raspberry whose beads straddle every periodic face of the box;
- zero bead friction (the beads exert nothing: the fluid evolves as without
  bodies, and the bodies move under their external forces alone);
- a body of one bead at its own centre (no lever arm, no torque);
- no-op calls: zero steps, forces before the first step; non-finite body
  inputs rejected with LB_ERR_ARG, leaving the handle usable;
- the largest lattice the library accepts (1260 x 1260 x 1259 = 1.9988e9
  nodes, 152 GB of FP32 deviations): both AA parities checked on sampled
  nodes, which the oracle computes one by one from the sampled upstream
  populations (the corner nodes, the last nodes of the array and seeded ones,
  so that 32-bit node indices and Philox counters near 2^31 are exercised).

Tolerances as in test_gpu_parity.py."""
import numpy as np
import pytest

from helpers import Pair, W19, oracle_kw, perturbed_populations
from oracle import oracle as O
from paper_1604_01829_gb300 import workloads as Wl

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 1e-5}
MRT = dict(collision=1, gamma_shear=-0.45, gamma_bulk=-0.2, gamma_odd=0.3, gamma_even=-0.1)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1604_01829_gb300 import build
    build.build()


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("dims", [(2, 2, 2), (2, 9, 5), (7, 2, 3), (3, 4, 2)])
def test_smallest_lattices_match_oracle(precision, dims):
    P = Pair(*dims, precision=precision, kT=1e-4, seed=77, body_force=(2e-5, -1e-5, 3e-5), **MRT)
    P.set_populations(perturbed_populations(P.N, seed=8))
    for n in (1, 2, 5):
        P.step(n)
        assert P.pop_error() <= TOL[precision], n


@pytest.mark.parametrize("precision", [64, 32])
def test_raspberry_straddling_every_periodic_face(precision):
    params = dict(MRT, kT=1e-4, seed=5, gamma_bead=Wl.paper_gamma_to_lattice(50.0))
    P = Pair(12, 10, 14, precision=precision, **params)
    P.set_populations(perturbed_populations(P.N, seed=4))
    beads = Wl.ellipsoid_raspberry(3.0, 2.0, 2.0, seed=9)
    b = P.add_body(beads, [0.3, 9.8, 13.9], [0.7, 0.3, -0.5, 0.4], mass=60.0, inertia=(30, 70, 70),
                   F_ext=(1e-3, -5e-4, 2e-4), V=(1e-3, 0, -1e-3), w=(0, 1e-3, 0))
    tb = 1e-11 if precision == 64 else 1e-5
    for n in (1, 4, 3):
        P.step(n)
        assert P.pop_error() <= TOL[precision]
        e = P.body_errors(b)
        assert e["bead"] <= tb and e["F"] <= tb and e["T"] <= tb and e["X"] <= tb, e


@pytest.mark.parametrize("precision", [64, 32])
def test_zero_bead_friction_decouples_bodies_and_fluid(precision):
    params = dict(MRT, kT=1e-4, seed=3, gamma_bead=0.0)
    P = Pair(10, 9, 11, precision=precision, **params)
    f0 = perturbed_populations(P.N, seed=2)
    P.set_populations(f0)
    b = P.add_body(Wl.sphere_raspberry(2.0), [5.2, 4.1, 6.3], mass=34.0, inertia=(50, 50, 50),
                   F_ext=(1e-3, 0, -2e-3), T_ext=(0, 0, 1e-3))
    P.step(6)
    assert P.pop_error() <= TOL[precision]
    # the fluid is that of the same lattice without the body
    from paper_1604_01829_gb300 import lb
    ref = lb.LB(10, 9, 11, precision=precision, **params)
    ref.lb_set_populations(f0)
    ref.lb_step(6)
    assert np.abs(P.gpu.lb_get_populations() - ref.lb_get_populations()).max() == 0.0
    # no bead force; the body accelerates under its external force alone:
    # velocity Verlet from rest, whose first half kick uses the force known
    # before the first step (none), gives V = 5.5 F / M after six steps
    F, T, pb = P.gpu.lb_forces(b, per_bead=True)
    assert np.all(pb == 0.0)
    assert np.allclose(F, [1e-3, 0, -2e-3], rtol=0, atol=1e-15)
    V = P.gpu.lb_get_body(b)["V"]
    assert np.allclose(V, 5.5 * np.array([1e-3, 0, -2e-3]) / 34.0, rtol=1e-12, atol=0)
    e = P.body_errors(b)
    assert e["X"] <= 1e-13 and e["V"] <= 1e-15 and e["w"] <= 1e-15, e


@pytest.mark.parametrize("precision", [64, 32])
def test_single_bead_body_at_its_centre(precision):
    params = dict(collision=0, tau=0.9, gamma_bead=0.2)
    P = Pair(9, 8, 10, precision=precision, **params)
    P.set_populations(perturbed_populations(P.N, seed=12))
    b = P.add_body(np.zeros((1, 3)), [4.3, 3.7, 5.1], q=[0.8, 0.2, 0.3, -0.1], mass=3.0, inertia=(1, 2, 3),
                   F_ext=(2e-4, 1e-4, 0), w=(1e-3, -2e-3, 5e-4))
    tb = 1e-11 if precision == 64 else 1e-5
    for n in (1, 2, 4):
        P.step(n)
        assert P.pop_error() <= TOL[precision]
        e = P.body_errors(b)
        assert e["bead"] <= tb and e["F"] <= tb and e["X"] <= tb, e
        _, T, _ = P.gpu.lb_forces(b, per_bead=True)
        assert np.all(T == 0.0)


def test_no_op_calls():
    from paper_1604_01829_gb300 import lb
    g = lb.LB(6, 5, 7, precision=32, **MRT)
    f = perturbed_populations(6 * 5 * 7, seed=1)
    g.lb_set_populations(f)
    b = g.lb_add_raspberry(Wl.sphere_raspberry(1.5), [3, 2.5, 3.5], [1, 0, 0, 0], 10.0, (4, 4, 4), (1e-3, 0, 0),
                           (0, 0, 0), False)
    F, T, pb = g.lb_forces(b, per_bead=True)            # before the first step: nothing applied yet
    assert np.all(F == 0) and np.all(T == 0) and np.all(pb == 0)
    before = g.lb_get_populations()
    g.lb_step(0)
    assert np.array_equal(g.lb_get_populations(), before)
    assert g.lb_info()["step"] == 0


def test_non_finite_body_inputs_are_rejected():
    from paper_1604_01829_gb300 import lb
    nan, inf = float("nan"), float("inf")
    sph = Wl.sphere_raspberry(1.5)
    good = dict(X=[3, 3, 3], q=[1, 0, 0, 0], mass=10.0, inertia=(4, 4, 4), F_ext=(1e-3, 0, 0), T_ext=(0, 0, 0))
    bad = [dict(X=[3, nan, 3]), dict(mass=inf), dict(inertia=(4, inf, 4)), dict(F_ext=(0, 0, nan)),
           dict(T_ext=(inf, 0, 0)), dict(q=[nan, 0, 0, 1])]
    for b in bad:
        kw = dict(good, **b)
        g = lb.LB(8, 8, 8, precision=32)
        with pytest.raises(lb.LBError) as e:
            g.lb_add_raspberry(sph, **kw)
        assert e.value.status == lb.LB_ERR_ARG, b
        B = lb.LBBatch([dict(nx=8, ny=8, nz=8, precision=32)])
        with pytest.raises(lb.LBError) as e:
            B.lb_batch_add_raspberry(0, sph, **kw)
        assert e.value.status == lb.LB_ERR_ARG, b
    g = lb.LB(8, 8, 8, precision=32)
    bid = g.lb_add_raspberry(sph[:1], **good)
    for kw in (dict(V=(nan, 0, 0)), dict(w=(0, inf, 0)), dict(X=(nan, 1, 1))):
        with pytest.raises(lb.LBError) as e:
            g.lb_set_body_state(bid, **kw)
        assert e.value.status == lb.LB_ERR_ARG, kw
    with pytest.raises(lb.LBError) as e:
        g.lb_set_external_forces([[0, nan, 0]])
    assert e.value.status == lb.LB_ERR_ARG
    g.lb_step(2)                                         # the rejected calls left the handle usable
    m, _ = g.lb_conservation()
    assert abs(m - 512) <= 1e-4


def _upstream(nodes, dims):
    """Linear ids of x - c_i (periodic) for each node, [n, 19]."""
    nx, ny, nz = dims
    c = np.array(O.lattice()[0], dtype=np.int64).reshape(19, 3)
    x = nodes % nx
    y = (nodes // nx) % ny
    z = nodes // (nx * ny)
    ux = (x[:, None] - c[None, :, 0]) % nx
    uy = (y[:, None] - c[None, :, 1]) % ny
    uz = (z[:, None] - c[None, :, 2]) % nz
    return ux + nx * (uy + ny * uz)


@pytest.mark.parametrize("precision", [64, 32])
def test_long_calls_on_large_lattices_equal_single_steps(precision):
    """From 2^20 nodes on, lb_step calls of four or more steps launch every
    step eagerly instead of replaying captured graphs; shorter calls replay
    one-step graphs. A 128 x 128 x 64 lattice (2^20 nodes) with two
    raspberries and thermal noise, stepped once by lb_step(7) and once by
    seven lb_step(1), ends in the same state to the rounding of the atomics
    that spread bead forces in no fixed order (FP64 1e-11, FP32 1e-5 of
    w_i rho0; bodies to the same relative bound)."""
    from paper_1604_01829_gb300 import lb
    params = dict(collision=1, gamma_shear=-0.45, gamma_bulk=-0.2, gamma_odd=0.3, gamma_even=-0.1, kT=1e-4,
                  seed=9, gamma_bead=Wl.paper_gamma_to_lattice(50.0), compensate_force=1)
    sph = Wl.sphere_raspberry(3.0)
    ell = Wl.ellipsoid_raspberry(6.0, 2.5, 2.5, seed=4)
    hs = []
    for _ in range(2):
        h = lb.LB(128, 128, 64, precision=precision, **params)
        h.lb_add_raspberry(sph, [30.2, 60.7, 20.1], mass=113.0, inertia=(400, 400, 400), F_ext=(1e-3, 0, 0))
        h.lb_add_raspberry(ell, [90.6, 40.3, 44.9], [0.9, 0.1, -0.2, 0.3], 160.0, (500, 1500, 1500))
        hs.append(h)
    A, B = hs
    A.lb_step(7)
    for _ in range(7):
        B.lb_step(1)
    tol = 1e-11 if precision == 64 else 1e-5
    d = float((np.abs(A.lb_get_populations() - B.lb_get_populations()).max(axis=1) / W19).max())
    assert d <= tol, d
    for b in range(2):
        sa, sb = A.lb_get_body(b), B.lb_get_body(b)
        for k in ("X", "V", "q"):
            assert np.abs(sa[k] - sb[k]).max() <= tol * max(np.abs(sa[k]).max(), 1e-3), (b, k)
    A.close()
    B.close()


def test_largest_lattice_on_sampled_nodes():
    import torch
    from paper_1604_01829_gb300 import lb
    dims = (1260, 1260, 1259)
    N = dims[0] * dims[1] * dims[2]
    assert 1.99e9 < N <= 2.0e9
    free, _ = torch.cuda.mem_get_info()
    if free < 19 * 4 * N + (4 << 30):
        pytest.skip(f"needs {19 * 4 * N / 1e9:.0f} GB of free device memory, {free / 1e9:.0f} GB free")
    params = dict(MRT, kT=1e-4, seed=0x5EED1604, body_force=(1e-6, -2e-6, 3e-6))
    g = lb.LB(*dims, precision=32, **params)
    p = O.make_params(*dims, **oracle_kw(params))
    nx, ny, nz = dims
    rng = np.random.default_rng(17)
    corners = [x + nx * (y + ny * z) for x in (0, nx - 1) for y in (0, ny - 1) for z in (0, nz - 1)]
    nodes = np.unique(np.concatenate([corners, N - 1 - np.arange(8), rng.integers(0, N, 48)]).astype(np.int64))
    up = _upstream(nodes, dims)
    g.lb_step(1)
    for step in (1, 2):                                 # an odd and an even step
        ids, inv = np.unique(up.reshape(-1), return_inverse=True)
        pre = g.lb_sample_populations(ids)[inv].reshape(len(nodes), 19, 19)   # [node, link, population]
        g.lb_step(1)
        post = g.lb_sample_populations(nodes)
        for s in range(len(nodes)):
            for i in range(19):
                fs = O.collide_node(p, pre[s, i], params["body_force"], node_id=int(up[s, i]), step=step)
                assert abs(post[s, i] - fs[i]) <= TOL[32] * W19[i], (int(nodes[s]), i, step)
    m, _ = g.lb_conservation()
    assert abs(m - N) <= 1e-8 * N
    g.close()
