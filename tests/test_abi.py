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
