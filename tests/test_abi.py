"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/lb.h declares; its host-side tables agree with the
oracle's independently written ones (CPU only, no compute calls)."""
import os
import re

import numpy as np
import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1604_01829_gb300 import build, lb
    build.build()
    return lb.load()


def header_functions():
    src = open(os.path.join(ROOT, "include", "lb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = header_functions()
    assert "lb_create" in names and "lb_step" in names and "lb_forces" in names
    for n in names:
        assert hasattr(lib, n), n
    from paper_1604_01829_gb300 import lb
    assert sorted(lb.EXPORTS) == names


def test_lattice_tables_match_oracle(lib):
    from paper_1604_01829_gb300 import lb
    c, w, opp = lb.lb_lattice()
    c2, w2, opp2 = O.lattice()
    assert np.array_equal(c, c2)
    assert np.array_equal(w, w2)
    assert np.array_equal(opp, opp2)


def test_status_strings(lib):
    from paper_1604_01829_gb300 import lb
    for s in range(7):
        assert lib.lb_status_string(s)
    assert lib.lb_last_error(None) is not None


def test_create_fails_loudly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1604_01829_gb300 import lb
    with pytest.raises(lb.LBError) as ei:
        lb.LB(8, 8, 8)
    assert ei.value.status == lb.LB_ERR_CUDA


@pytest.mark.parametrize("bad", [
    dict(nx=1), dict(nz=0), dict(nx=1300, ny=1300, nz=1300),          # below 2 per axis; beyond 2e9 nodes
    dict(precision=16), dict(collision=2), dict(collision=0, tau=0.5),
    dict(collision=1, gamma_shear=1.0), dict(collision=1, gamma_odd=-1.0), dict(rho0=0.0),
    dict(kT=-1e-4), dict(collision=0, kT=1e-4), dict(gamma_bead=-0.1), dict(md_substeps=5),
    dict(body_force=(float("nan"), 0.0, 0.0)), dict(rho0=float("inf")), dict(kT=float("inf"), collision=1),
    dict(gamma_bead=float("inf"))])
def test_create_rejects_bad_arguments_before_any_device_call(lib, bad):
    """lb_create and lb_batch_create check every argument before they look
    for a device, so these run (and fail with LB_ERR_ARG) without a GPU."""
    from paper_1604_01829_gb300 import lb
    args = dict(nx=8, ny=8, nz=8, precision=32)
    args.update(bad)
    nx, ny, nz = args.pop("nx"), args.pop("ny"), args.pop("nz")
    with pytest.raises(lb.LBError) as e:
        lb.LB(nx, ny, nz, **args)
    assert e.value.status == lb.LB_ERR_ARG, bad
    with pytest.raises(lb.LBError) as e:
        lb.LBBatch([dict(nx=8, ny=8, nz=8, precision=32), dict(nx=nx, ny=ny, nz=nz, **args)])
    assert e.value.status == lb.LB_ERR_ARG, bad


def test_batch_rejects_mixed_precision_and_noise_without_a_device(lib):
    from paper_1604_01829_gb300 import lb
    for second in (dict(precision=64), dict(collision=1, kT=1e-4), dict(md_substeps=2)):
        with pytest.raises(lb.LBError) as e:
            lb.LBBatch([dict(nx=8, ny=8, nz=8, precision=32, collision=1),
                        dict(dict(nx=8, ny=8, nz=8, precision=32, collision=1), **second)])
        assert e.value.status == lb.LB_ERR_ARG
