"""mpr_bond_energy_noalloc: the bond-energy entry point that allocates no device memory, for
callers that cannot call cudaMalloc (their device memory is owned by another allocator or a fixed
budget, or they run in a loop that must not take the allocator's locks or wait for the device).

Each result is checked against the FP64 oracle's bond energy of the same angles (plain C, summed
in row-major order) and against the library's handle-based energy (mpr_energy on a handle whose
state holds the same angles), on two calls in a row that share the fixed scratch array, and once
at the largest grid the scratch covers (2^28 sites). This file is collected last on purpose.
"""
import ctypes
import math

import numpy as np
import pytest

import mpr_inputs

pytestmark = pytest.mark.gpu

# The handle energy and this entry point sum FP64 terms in fixed tree orders, the oracle one by
# one. Summed in two orders, n_b terms of magnitude <= 1 (a sum of magnitude <= n_b) differ by
# about sqrt(n_b) random rounding errors of relative size 2^-53, i.e. about sqrt(n_b) * 2^-53 in
# the per-bond energy; allowed: 8 times that, and at least 1e-13.
def _tol(n_bonds):
    return max(1e-13, 8.0 * math.sqrt(n_bonds) * 2.0**-53)


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


def test_noalloc_bond_energy_matches_oracle_and_handle_twice(mpr, orc):
    import torch

    a1, e1 = _state_and_reference(mpr, 257, 129, 0.66, 3)
    a2, e2 = _state_and_reference(mpr, 64, 48, 0.33, 4)
    o1 = orc.Oracle(257, 129).energy_bond(a1)
    o2 = orc.Oracle(64, 48).energy_bond(a2)
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
    nb1 = 257 * 128 + 129 * 256
    nb2 = 64 * 47 + 48 * 63
    assert abs(got[0] - o1) <= _tol(nb1), (got[0], o1)
    assert abs(got[1] - o2) <= _tol(nb2), (got[1], o2)
    assert abs(got[0] - e1) <= _tol(nb1), (got[0], e1)
    assert abs(got[1] - e2) <= _tol(nb2), (got[1], e2)
    # the first grid again: same result after the scratch held the second call's partials
    again = mpr.mpr_bond_energy_noalloc(t1, 0.5, torch.zeros(1, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    assert float(again.item()) == got[0]


def test_noalloc_at_its_largest_grid(mpr, orc):
    # 16384 x 16384 = 2^28 sites: every one of the 4096 scratch slots is used
    import torch

    L = 16384
    rng = np.random.default_rng(11)
    a = rng.random((L, L)) * (2 * np.pi)
    exp = orc.Oracle(L, L).energy_bond(a)
    t = torch.from_numpy(a).cuda()
    del a
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    got = float(mpr.mpr_bond_energy_noalloc(t, 0.5, out).item())
    assert abs(got - exp) <= _tol(2 * L * (L - 1)), (got, exp)


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
