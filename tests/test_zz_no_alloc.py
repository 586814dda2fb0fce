"""mpr_bond_energy_noalloc: the allocation-free bond-energy entry point, for callers that cannot
call cudaMalloc (e.g. while a CUDA graph is being captured, or under a device-memory budget owned
by another allocator).

It is checked against the library's handle-based energy (mpr_energy on a handle whose state holds
the same angles), within the tolerance the other energy tests use, on two calls in a row that
share the fixed scratch array. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import mpr_inputs

pytestmark = pytest.mark.gpu

TOL = 1e-13


@pytest.fixture(scope="module")
def mpr():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1910_08448_gb300 as m

    m.load()
    return m


def _state_and_reference(mpr, Lx, Ly, p, seed):
    """A full state on a DDD handle and the handle's own FP64 bond energy of it."""
    pr = mpr_inputs.make_problem(Lx, Ly, p, field_seed=seed, mask_seed=seed + 1)
    rng = np.random.default_rng(seed)
    h = mpr.mpr_create(pr.z, pr.mask)
    try:
        mpr.mpr_set_options(h, "DDD", seed=seed)
        mpr.mpr_set_state(h, rng.random((Ly, Lx)) * 2 * np.pi, 0)
        angles, _ = mpr.mpr_get_state(h)
        e_ref, _ = mpr.mpr_energy(h)
    finally:
        mpr.mpr_destroy(h)
    return angles, e_ref


def test_noalloc_bond_energy_matches_handle_energy_twice(mpr):
    import torch

    a1, e1 = _state_and_reference(mpr, 257, 129, 0.66, 3)
    a2, e2 = _state_and_reference(mpr, 64, 48, 0.33, 4)
    lib = mpr.load()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    t1 = torch.from_numpy(a1).cuda()
    t2 = torch.from_numpy(a2).cuda()
    # two calls in a row through the C ABI, on different grids, sharing the scratch
    st = lib.mpr_bond_energy_noalloc(257, 129, ctypes.c_void_p(t1.data_ptr()), 0.5,
                                     ctypes.c_void_p(out.data_ptr()), None)
    assert st == mpr.MPR_OK, mpr.mpr_last_error()
    st = lib.mpr_bond_energy_noalloc(64, 48, ctypes.c_void_p(t2.data_ptr()), 0.5,
                                     ctypes.c_void_p(out.data_ptr() + 8), None)
    assert st == mpr.MPR_OK, mpr.mpr_last_error()
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert abs(got[0] - e1) <= TOL, (got[0], e1)
    assert abs(got[1] - e2) <= TOL, (got[1], e2)
    # the first grid again: same result after the scratch held the second call's partials
    again = mpr.mpr_bond_energy_noalloc(t1, 0.5, torch.zeros(1, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    assert float(again.item()) == got[0]


def test_noalloc_rejects_grids_beyond_its_scratch(mpr):
    import torch

    lib = mpr.load()
    buf = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    st = lib.mpr_bond_energy_noalloc(16385, 16384, p, 0.5, p, None)
    assert st == mpr.MPR_ERR_INVALID_ARG
    assert "2^28" in mpr.mpr_last_error()
    assert lib.mpr_bond_energy_noalloc(1, 16, p, 0.5, p, None) == mpr.MPR_ERR_INVALID_ARG
    assert lib.mpr_bond_energy_noalloc(4, 4, None, 0.5, p, None) == mpr.MPR_ERR_INVALID_ARG
    assert float(buf.sum().item()) == 0.0     # nothing was written
