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


def test_model_and_frame_entry_points_reject_bad_arguments(ac):
    """Argument checks of the model, frame, rate, class and time-model calls (all run
    before any device work)."""
    ERR = ac.ac.AC_ERR_ARG
    bad_calls = [
        (ac.ac_create_q, (16, 16, 0, 0.4, 1.0, 0.0, 1, 1)),          # q = 1 is ac_create
        (ac.ac_create_q, (16, 16, 0, 0.4, 1.0, 0.0, 4, 1)),          # q above 3
        (ac.ac_create_q, (7, 8, 0, 0.4, 1.0, 0.0, 2, 1)),            # rows < 4q
        (ac.ac_create_q, (16, 16, 0, -1.0, 1.0, 0.0, 2, 1)),         # beta < 0
        (ac.ac_create_life, (3, 10, 0, 0, 8, 12, 1)),                # rows < 4
        (ac.ac_create_life, (10, 10, 0, 0, 1 << 9, 12, 1)),          # 10-bit birth mask
        (ac.ac_time_model, (0, 64, ac.AC_LAW_EXP, 1, 10, 4)),        # dims 0
        (ac.ac_time_model, (4, 64, ac.AC_LAW_EXP, 1, 10, 4)),        # dims 4
        (ac.ac_time_model, (1, 1, ac.AC_LAW_EXP, 1, 10, 4)),         # n < 2
        (ac.ac_time_model, (1, 64, 3, 1, 10, 4)),                    # unknown law
        (ac.ac_time_model, (1, 64, ac.AC_LAW_EXP, 1, -1, 4)),        # t_end < 0
        (ac.ac_time_model, (3, 1 << 11, ac.AC_LAW_EXP, 1, 10, 4)),   # n^3 >= 2^32 cells
        (ac.ac_frames_configure, (0, 1 << 32, 0, 4)),                # null handle
        (ac.ac_frames_status, (0,)),
        (ac.ac_set_rates, (0, None)),
        (ac.ac_class_counts, (0,)),
        (ac.ac_run_until_ticks, (0, 1)),
        (ac.ac_read_state, (0, None, None, None)),
        (ac.ac_batch_create, ([], [], [], [], [])),                  # empty batch
    ]
    for fn, args in bad_calls:
        with pytest.raises(ac.ACError) as ei:
            fn(*args)
        assert ei.value.status == ERR, (fn.__name__, args)
    with pytest.raises(ac.ACError) as ei:
        ac.ac_time_model(1, 64, ac.AC_LAW_EXP, 1, 10, 4, q=9)        # radius above 8
    assert ei.value.status == ERR
