"""The C-ABI library loads and exports every entry point of include/ac.h; argument
checks that need no GPU reject bad input with AC_ERR_ARG.  (CPU only: no compute.)"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ac():
    import __graft_entry__
    __graft_entry__.build()
    import paper_cs_0502039_gb300 as ac
    return ac


def _declared():
    text = open(os.path.join(ROOT, "include", "ac.h")).read()
    return sorted(set(re.findall(r"^\s*(?:ac_status|void|const char\*)\s+(ac_\w+)\s*\(", text, re.M)))


def test_library_exports_every_declared_symbol(ac):
    names = _declared()
    assert len(names) >= 18
    lib = ctypes.CDLL(ac.ac.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(ac.ac.EXPORTS)


def test_threshold_table_equals_oracle(ac):
    for beta, J, h in [(0.44, 1.0, 0.0), (0.3, 1.0, 0.0), (0.4407, 1.0, 0.0), (0.6, 1.0, 0.0),
                       (1.0, 1.0, 0.05), (0.25, -0.7, 0.3), (0.0, 1.0, 0.0), (40.0, 1.0, 0.0)]:
        assert np.array_equal(ac.ac_thresholds(beta, J, h), oracle.thresholds(beta, J, h))


@pytest.mark.parametrize("rows,cols,init,beta,J,h", [
    (1, 4, 0, 0.4, 1.0, 0.0), (4, 1, 0, 0.4, 1.0, 0.0), (65536, 65536, 0, 0.4, 1.0, 0.0),
    (4, 4, 3, 0.4, 1.0, 0.0), (4, 4, 0, -0.1, 1.0, 0.0), (4, 4, 0, float("nan"), 1.0, 0.0),
    (4, 4, 0, 0.4, float("inf"), 0.0)])
def test_create_rejects_bad_arguments(ac, rows, cols, init, beta, J, h):
    with pytest.raises(ac.ACError) as ei:
        ac.ac_create(rows, cols, init, beta, J, h, 1)
    assert ei.value.status == ac.ac.AC_ERR_ARG


def test_null_handles_are_rejected(ac):
    for fn, args in [(ac.ac_run_until, (0, 1.0)), (ac.ac_configure, (0, 1, 64, 1, 8)),
                     (ac.ac_reset, (0, 1, 0)), (ac.ac_set_option, (0, 1, 10**9))]:
        with pytest.raises(ac.ACError) as ei:
            fn(*args)
        assert ei.value.status == ac.ac.AC_ERR_ARG
    ac.ac_destroy(0)
