"""Alternative temperature tunings through the C ABI against the oracle: heating until the bond
energy crosses the sample's, the energy curve of the unconditional lattice, and tuning by
inverting a tabulated curve (readings of Sec. 2, which leaves the tuning procedure open)."""
import numpy as np
import pytest

import mpr_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpr():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1910_08448_gb300 as m

    m.load()
    return m


def test_heating_matches_oracle_ddd(mpr, orc):
    # the same chain on both sides: identical probes, temperature and sweep count
    pr = mpr_inputs.make_problem(48, 40, 0.33, field_seed=27, mask_seed=28)
    kw = dict(n_eq=40, n_meas=20)
    h = mpr.mpr_create(pr.z, pr.mask)
    try:
        mpr.mpr_set_options(h, "DDD", seed=8)
        mpr.mpr_set_tuning(h, **kw)
        T_gpu, st = mpr.mpr_tune_heating(h, 1.7)
        info = mpr.mpr_get_info(h)
    finally:
        mpr.mpr_destroy(h)
    o = orc.Oracle(48, 40, seed=8)
    phi, _, _ = o.map(pr.z, pr.mask)
    phi = o.init(phi, pr.mask)
    e_s, _ = o.energy_sample(phi, pr.mask)
    st_o, T_o, _, sw, trace = o.tune_heating(phi, pr.mask, e_s, 0, factor=1.7, **kw)
    assert st == st_o == 0
    assert len(trace) > 3   # heating steps and bisection both ran
    assert info["n_probes"] == len(trace) and info["sweep"] == sw
    assert abs(T_gpu / T_o - 1.0) < 1e-9


def test_energy_curve_matches_oracle_ddd(mpr, orc):
    # The same chain on both sides, but a lattice without frozen sites is chaotic: a rounding
    # difference (the GPU contracts a*b + c into one FMA, the oracle does not) grows about tenfold
    # every two to three sweeps (energies 1e-15 apart after 5 sweeps, 1e-13 after 10, 1e-4 after
    # 30 at T = 2). So the run is kept short here; longer curves compare statistically below.
    Ts = [2.0, 0.5, 0.2, 0.08]
    e_gpu = mpr.mpr_energy_curve(40, 32, Ts, setup="DDD", seed=12, n_eq=2, n_meas=1)
    e_orc = orc.Oracle(40, 32, seed=12).energy_curve(Ts, n_eq=2, n_meas=1)
    assert np.allclose(e_gpu, e_orc, rtol=1e-9, atol=0.0), (e_gpu, e_orc)
    # a long DDD curve: an independent-looking chain, the same equilibrium energies
    e_gpu = mpr.mpr_energy_curve(64, 64, Ts, setup="DDD", seed=12, n_eq=400, n_meas=400)
    e_orc = orc.Oracle(64, 64, seed=12).energy_curve(Ts, n_eq=400, n_meas=400)
    assert np.all(np.abs(e_gpu - e_orc) < 3e-3), (e_gpu, e_orc)


@pytest.mark.parametrize("setup", ["SDS", "HDS"])
def test_energy_curve_fp32_matches_oracle(mpr, orc, setup):
    # FP32 functions: a different chain, the same equilibrium curve
    Ts = [1.0, 0.4, 0.15, 0.06]
    e_gpu = mpr.mpr_energy_curve(64, 64, Ts, setup=setup, seed=13, n_eq=400, n_meas=400)
    e_orc = orc.Oracle(64, 64, seed=13).energy_curve(Ts, n_eq=400, n_meas=400)
    assert np.all(np.abs(e_gpu - e_orc) < 3e-3), (e_gpu, e_orc)
    assert np.all(np.diff(e_gpu) < 0)


def test_tune_from_curve_matches_oracle(mpr, orc):
    pr = mpr_inputs.make_problem(64, 64, 0.5, field_seed=29, mask_seed=30)
    h = mpr.mpr_create(pr.z, pr.mask)
    try:
        _, e_s = mpr.mpr_energy(h)
        T = np.geomspace(0.02, 3.0, 9)
        e = mpr.mpr_energy_curve(128, 128, T, setup="SDS", seed=1, n_eq=200, n_meas=100)
        T_gpu, st = mpr.mpr_tune_from_curve(h, T, e)
        st_o, T_o = orc.invert_curve(T, e, e_s)
        assert st == st_o == 0 and abs(T_gpu / T_o - 1.0) < 1e-14
        assert mpr.mpr_get_info(h)["T"] == T_gpu
        # above the curve's top: the last temperature and "no convergence"
        T2, st2 = mpr.mpr_tune_from_curve(h, T[:2], np.array([-1.0, e_s - 0.1]))
        assert st2 == mpr.MPR_ERR_TUNE_NO_CONVERGE and T2 == T[1]
        for bad_T, bad_e in [([0.1], [-0.9]), ([0.2, 0.1], [-0.9, -0.8]), ([0.1, 0.2], [-0.9, np.nan])]:
            with pytest.raises(mpr.MPRError) as ei:
                mpr.mpr_tune_from_curve(h, bad_T, bad_e)
            assert ei.value.status == mpr.MPR_ERR_INVALID_ARG
        with pytest.raises(mpr.MPRError) as ei:
            mpr.mpr_tune_heating(h, 1.0)
        assert ei.value.status == mpr.MPR_ERR_INVALID_ARG
    finally:
        mpr.mpr_destroy(h)


def test_bisection_and_heating_agree(mpr):
    # both solve e_b(T) = e_s on the same conditional lattice (FP16 spins, FP32 functions)
    pr = mpr_inputs.make_problem(256, 256, 0.66, field_seed=31, mask_seed=32)
    Ts = {}
    for method in ("bisect", "heat"):
        h = mpr.mpr_create(pr.z, pr.mask)
        try:
            mpr.mpr_set_options(h, "HDS", seed=5)
            T, st = (mpr.mpr_tune_temperature(h) if method == "bisect"
                     else mpr.mpr_tune_heating(h, 1.5))
            assert st == 0
            Ts[method] = T
        finally:
            mpr.mpr_destroy(h)
    assert abs(Ts["heat"] / Ts["bisect"] - 1.0) < 0.1, Ts
