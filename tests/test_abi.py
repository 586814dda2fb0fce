"""The C-ABI library builds, loads without a GPU and exports every function include/mpr.h declares.

No compute call is made here; only argument validation that returns before any device work.
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    txt = open(os.path.join(ROOT, "include", "mpr.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"\b(mpr_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1910_08448_gb300 as mpr

    return mpr.load()


def test_exports_every_declared_function(lib):
    import paper_1910_08448_gb300 as mpr

    declared = _declared_functions()
    assert len(declared) >= 19
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(mpr.exported_symbols()) == declared


def test_library_is_sm103a_build():
    from paper_1910_08448_gb300 import _build

    assert "arch=compute_103a,code=sm_103a" in _build.ARCH


def test_mufu_probe_is_built(lib):
    # the special-function throughput probe that bench.py runs for its roofline
    from paper_1910_08448_gb300 import _build

    assert os.path.isfile(_build.PROBE) and os.access(_build.PROBE, os.X_OK)


def test_status_strings(lib):
    import paper_1910_08448_gb300 as mpr

    for st in range(9):
        assert mpr.mpr_status_string(st) not in ("", "unknown status")
    assert mpr.mpr_status_string(99) == "unknown status"


def test_host_validation_before_device_work(lib):
    import paper_1910_08448_gb300 as mpr

    h = ctypes.c_void_p()
    z = np.zeros(8)
    m = np.ones(8, np.uint8)
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    assert lib.mpr_create(1, 8, vp(z), vp(m), ctypes.byref(h)) == mpr.MPR_ERR_INVALID_ARG
    assert h.value is None
    assert lib.mpr_create(4, 2, None, vp(m), ctypes.byref(h)) == mpr.MPR_ERR_INVALID_ARG
    assert lib.mpr_create(70000, 70000, vp(z), vp(m), ctypes.byref(h)) == mpr.MPR_ERR_INVALID_ARG
    assert "2^31" in mpr.mpr_last_error()
    assert lib.mpr_run(None, 1, 1) == mpr.MPR_ERR_INVALID_ARG
    assert lib.mpr_philox4x32_10_dev(None, None, -1, 0, None) == mpr.MPR_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        mpr.make_options("XYZ")
    # the options of the hot path refuse a missing handle or bad arguments before any CUDA call
    d = ctypes.c_double()
    T = np.array([0.1, 0.2])
    assert lib.mpr_set_proposal(None, 1.0, 0.4) == mpr.MPR_ERR_INVALID_ARG
    assert lib.mpr_get_proposal(None, ctypes.byref(d)) == mpr.MPR_ERR_INVALID_ARG
    assert lib.mpr_tune_heating(None, 1.5, ctypes.byref(d)) == mpr.MPR_ERR_INVALID_ARG
    assert lib.mpr_tune_from_curve(None, vp(T), vp(T), 2, ctypes.byref(d)) == mpr.MPR_ERR_INVALID_ARG
    assert lib.mpr_energy_curve(8, 8, None, None, vp(T), 0, vp(T)) == mpr.MPR_ERR_INVALID_ARG
    bad = np.array([0.1, -1.0])
    assert lib.mpr_energy_curve(8, 8, None, None, vp(bad), 2, vp(T)) == mpr.MPR_ERR_INVALID_ARG
    assert lib.mpr_run_auto(None, 10, 100, 10, None) == mpr.MPR_ERR_INVALID_ARG
    assert lib.mpr_set_sweep_kernel(None, 0) == mpr.MPR_ERR_INVALID_ARG
    assert lib.mpr_trim_memory() == mpr.MPR_OK   # no pool created yet: nothing to return
