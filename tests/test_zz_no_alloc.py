"""The allocation-free reduction lb_moments_noalloc, called through the C ABI,
against the allocating lb_conservation of a handle holding the same
populations, on two calls in a row.

lb_moments_noalloc serves callers that cannot call cudaMalloc: callers whose
device memory is already held by another allocator, or that must not let an
allocation synchronise the device while a simulation runs. Its scratch is a
static device array shared by every call. This file is collected last so
that a run stopping at its first failure has already run every other test;
it also passes alone in a fresh process (the first call on the device looks
up the array's address)."""
import numpy as np
import pytest

from helpers import W19, perturbed_populations
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1604_01829_gb300 import build
    build.build()


def _device_layout(f, precision, rho0):
    import torch
    if precision == 64:
        return torch.tensor(np.ascontiguousarray(f), dtype=torch.float64, device="cuda")
    return torch.tensor(np.ascontiguousarray(f - W19[:, None] * rho0), dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("pore", [None, (7.5, 2), (6.0, 0)])
def test_noalloc_matches_lb_conservation(precision, pore):
    import torch
    from paper_1604_01829_gb300 import lb
    nx, ny, nz = 19, 17, 23
    rho0 = 1.0
    g = lb.LB(nx, ny, nz, precision=precision, collision=0, tau=1.0, rho0=rho0)
    if pore is not None:
        g.lb_set_pore(*pore)
    f = perturbed_populations(nx * ny * nz, rho0=rho0, seed=21)
    g.lb_set_populations(f)
    m_ref, p_ref = g.lb_conservation()
    # the handle's populations as the library stores them after 0 steps
    dev = _device_layout(g.lb_get_populations(), precision, rho0)
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out.fill_(float("nan"))
        lb.lb_moments_noalloc(dev.data_ptr(), precision, nx, ny, nz, 0, rho0, out.data_ptr(),
                              pore_radius=pore[0] if pore else 0.0, pore_axis=pore[1] if pore else 2,
                              stream=stream)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        tol = 1e-12 if precision == 64 else 1e-8
        assert abs(o[0] - m_ref) <= tol * m_ref
        assert np.abs(o[1:] - p_ref).max() <= tol * m_ref
    g.close()


def _odd_layout(f, nx, ny, nz, mask):
    """The in-place (AA) storage after an odd number of steps, built in numpy
    from the logical pre-collision populations f [19][N]: population i of
    node n sits in slot opp(i) of its upstream neighbour n - c_i, or in its
    own slot i when that neighbour is a wall node (halfway bounce-back)."""
    c, _, opp = O.lattice()
    N = nx * ny * nz
    n = np.arange(N)
    x, y, z = n % nx, (n // nx) % ny, n // (nx * ny)
    fluid = np.ones(N, bool) if mask is None else mask == 0
    A = np.zeros_like(f)
    A[0] = f[0]
    for i in range(1, 19):
        s = ((x - c[i, 0]) % nx) + nx * (((y - c[i, 1]) % ny) + ny * ((z - c[i, 2]) % nz))
        up_fluid = fluid[s]
        sel = fluid & up_fluid
        A[opp[i], s[sel]] = f[i, sel]
        sel = fluid & ~up_fluid
        A[i, sel] = f[i, sel]
    return A


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("pore", [None, (7.5, 2), (6.0, 0)])
@pytest.mark.parametrize("steps", [3, 4])
def test_noalloc_after_odd_and_even_step_counts(precision, pore, steps):
    """A thermal MRT handle stepped an odd (3) or even (4) number of times:
    its populations laid out as the library stores them at that parity
    (odd_parity = steps % 2), reduced twice in a row, equal lb_conservation
    of the handle."""
    import torch
    from paper_1604_01829_gb300 import lb
    nx, ny, nz = 19, 17, 23
    rho0 = 1.0
    g = lb.LB(nx, ny, nz, precision=precision, collision=1, gamma_shear=-0.45, gamma_bulk=-0.2,
              gamma_odd=0.3, gamma_even=-0.1, kT=1e-4, seed=33, rho0=rho0)
    mask = None
    if pore is not None:
        g.lb_set_pore(*pore)
        mask = O.pore_mask(nx, ny, nz, *pore)
    g.lb_set_populations(perturbed_populations(nx * ny * nz, rho0=rho0, seed=22))
    g.lb_step(steps)
    m_ref, p_ref = g.lb_conservation()
    f = g.lb_get_populations()
    A = _odd_layout(f, nx, ny, nz, mask) if steps % 2 else f
    dev = _device_layout(A, precision, rho0)
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    tol = 1e-12 if precision == 64 else 1e-8
    for _ in range(2):
        out.fill_(float("nan"))
        lb.lb_moments_noalloc(dev.data_ptr(), precision, nx, ny, nz, steps % 2, rho0, out.data_ptr(),
                              pore_radius=pore[0] if pore else 0.0, pore_axis=pore[1] if pore else 2,
                              stream=stream)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert abs(o[0] - m_ref) <= tol * m_ref
        assert np.abs(o[1:] - p_ref).max() <= tol * m_ref
    g.close()


def test_noalloc_rejects_lattices_beyond_its_scratch():
    import torch
    from paper_1604_01829_gb300 import lb
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(lb.LBError) as ei:
        lb.lb_moments_noalloc(buf.data_ptr(), 64, 400, 400, 400, 0, 1.0, buf.data_ptr())
    assert ei.value.status == lb.LB_ERR_ARG
    assert "limit" in str(ei.value)
