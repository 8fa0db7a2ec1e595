"""Physics of the CUDA path itself (beyond parity): the Hasimoto finite-size
law for the drag of a fixed raspberry (Sec. 2.4, Eq. (hasimoto)), measured
through the C ABI with the protocol of the oracle pin."""
import math

import numpy as np
import pytest

from paper_1604_01829_gb300 import workloads as Wl

pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1604_01829_gb300 import build
    build.build()


def _drag_cuda(L, g=1e-6):
    from paper_1604_01829_gb300 import lb
    h = lb.LB(L, L, L, precision=64, collision=0, tau=1.0, gamma_bead=0.3, body_force=(g, 0, 0))
    h.lb_add_raspberry(Wl.sphere_raspberry(2.0), [L / 2 + 0.13, L / 2 - 0.21, L / 2 + 0.07], fixed=1)
    h.lb_step(int(1.5 * L * L))
    us = []
    for k in range(3):
        m, p = h.lb_conservation()
        us.append(p[0] / m)
        if k < 2:
            h.lb_step(int(0.6 * L * L))
    h.close()
    U1, U2, U3 = us
    return g * L ** 3 / ((U1 * U3 - U2 * U2) / (U1 + U3 - 2 * U2))


def test_hasimoto_slope_on_the_cuda_path():
    """FP64 CUDA path, L = 16-40, raspberry R = 2: same protocol and bound
    as the oracle pin (mean momentum sampled after the viscous transient,
    steady mean flow by Aitken extrapolation, 1/L coefficient fitted with the
    L^-3 term free)."""
    Ls = np.array([16, 20, 24, 32, 40], float)
    xi = np.array([_drag_cuda(int(L)) for L in Ls])
    x = 1.0 / Ls
    A = np.stack([np.ones_like(x), x, x ** 3], axis=1)
    b = np.linalg.lstsq(A, 1.0 / xi, rcond=None)[0][1]
    eta = 0.5 / 3.0
    assert abs(b / (-2.837 / (6 * math.pi * eta)) - 1) < 0.02, (xi, b)
    assert np.all(np.diff(xi) < 0)
