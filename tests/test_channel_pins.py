"""Pins of the oracle's moving channel walls (the Stokes-flow set-up of
Sec. 2.3 of Ustach & Faller, arXiv:1604.01829: boundary nodes along the +y
and -y faces with an imposed velocity): plane Couette flow is the exact
linear profile for halfway bounce-back, equal wall velocities give plug
flow, mass stays exact, and a bead next to a wall interpolates the wall's
velocity."""
import numpy as np
import pytest

from helpers import perturbed_populations
from oracle import oracle as O

MRT = dict(collision=1, gamma_shear=-0.45, gamma_bulk=-0.2, gamma_odd=0.3, gamma_even=-0.1)


def _profile(o, nx, ny, nz, comp):
    rho, u = o.node_velocity()
    return u[:, comp].reshape(nz, ny, nx)


@pytest.mark.parametrize("params,tol", [(dict(collision=0, tau=0.8), 1e-12), (dict(collision=0, tau=1.7), 1e-12),
                                        (MRT, 1e-8)])
def test_couette_flow_is_the_exact_linear_profile(params, tol):
    """Walls at y = -1/2 and ny - 1/2 moving at -U and +U along x: the
    steady velocity at node centre y + 1/2 is -U + 2U (y + 1/2) / ny, exact
    for BGK at any tau; with MRT rates whose odd (ghost) modes relax at a
    different rate a boundary layer of relative size ~1e-9 remains."""
    U, nx, ny, nz = 1e-3, 4, 8, 4
    o = O.OracleLB(nx, ny, nz, **params)
    o.set_channel_walls((-U, 0, 0), (U, 0, 0))
    o.step(6000)
    ux = _profile(o, nx, ny, nz, 0)
    y = np.arange(ny)
    exact = -U + 2 * U * (y + 0.5) / ny
    assert np.abs(ux - exact[None, :, None]).max() <= tol * U
    assert np.abs(_profile(o, nx, ny, nz, 1)).max() <= 1e-11 * U


def test_equal_wall_velocities_give_plug_flow():
    U, nx, ny, nz = 2e-3, 4, 6, 4
    o = O.OracleLB(nx, ny, nz, **MRT)
    o.set_channel_walls((0, 0, U), (0, 0, U))
    o.step(8000)
    uz = _profile(o, nx, ny, nz, 2)
    assert np.abs(uz - U).max() <= 1e-10 * U


def test_mass_is_exact_with_moving_walls_and_noise():
    nx, ny, nz = 6, 7, 5
    o = O.OracleLB(nx, ny, nz, **MRT, kT=1e-4, seed=3)
    o.set_channel_walls((1e-3, 0, -2e-3), (-3e-3, 0, 1e-3))
    o.set_populations(perturbed_populations(nx * ny * nz, seed=4))
    m0 = o.conservation()[0]
    o.step(300)
    assert abs(o.conservation()[0] - m0) <= 1e-13 * m0


def test_bead_next_to_a_wall_interpolates_the_wall_velocity():
    """In steady Couette flow a fixed single bead with negligible friction
    reads u = F_b / gamma. Between the last node row and the node beyond the
    wall, that node carries the wall's velocity (the reading that wall nodes
    carry their wall's velocity): at y_b = 0.2 the weights are 0.3 on the
    wall node (-U) and 0.7 on the first row (-U + U/ny); at y_b = 7.6, 0.9 on
    the last row (U - U/ny) and 0.1 on the wall node (+U)."""
    U, nx, ny, nz, gam = 1e-3, 4, 8, 4, 1e-7
    for yb, exact in ((0.2, 0.3 * -U + 0.7 * (-U + U / ny)), (7.6, 0.9 * (U - U / ny) + 0.1 * U)):
        o2 = O.OracleLB(nx, ny, nz, collision=0, tau=0.8, gamma_bead=gam)
        o2.set_channel_walls((-U, 0, 0), (U, 0, 0))
        o2.add_raspberry(np.zeros((1, 3)), [1.3, yb, 2.1], fixed=True)
        o2.step(6000)
        u = o2.bead_forces(0)[0] / gam
        assert abs(u[0] - exact) <= 1e-6 * U, (yb, u, exact)
