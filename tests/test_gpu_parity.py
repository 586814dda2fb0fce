"""GPU-vs-oracle parity through the C ABI (Sec. 2: conditional hybrid MC on Eq. 2).

Rules (the method is a stochastic iteration driven by counter-based random numbers, so the GPU
and the oracle can be compared sweep by sweep from an identical state and Philox stream):
  - integer work (Philox words, mask bits, counts) is bit-exact;
  - FP64 (DDD) states agree to 1e-9 except at sites whose Metropolis margin |u - exp(-dE/T)| or
    over-relaxation domain margin is below 1e-11 (a decision rounding can flip), and at the
    black neighbours of such red sites;
  - FP32 function setups use the oracle's 23-bit uniforms and agree to 1e-4 rad outside margins
    of 1e-4; 16-bit storage setups start from states rounded to the storage type and agree to a
    few storage ulps, with margins scaled by the storage ulp.
"""
import math

import numpy as np
import pytest

import mpr_inputs

pytestmark = pytest.mark.gpu

TWO_PI = 2.0 * math.pi
SETUPS_ALL = ["DDD", "SDS", "SSS", "SDD", "DDS", "HDS", "BDS", "HSS", "HDH"]


@pytest.fixture(scope="module")
def mpr():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1910_08448_gb300 as m

    m.load()
    return m


def _round_store(a, setup):
    s = setup[0]
    if s == "D":
        return np.asarray(a, np.float64)
    if s == "S":
        return np.asarray(a, np.float32).astype(np.float64)
    if s == "H":
        return np.asarray(a, np.float16).astype(np.float64)
    import torch

    return torch.tensor(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _ulp_store(setup):
    # spacing of the storage type in [4, 8), where angles near 2*pi live
    return {"D": 2.0**-50, "S": 2.0**-21, "H": 2.0**-8, "B": 2.0**-5}[setup[0]]


def _oracle(orc, Lx, Ly, seed, setup):
    return orc.Oracle(Lx, Ly, seed=seed, ubits=32 if setup[2] == "D" else 23)


def _neighbours(mask_bool):
    out = np.zeros_like(mask_bool)
    out[:, 1:] |= mask_bool[:, :-1]
    out[:, :-1] |= mask_bool[:, 1:]
    out[1:, :] |= mask_bool[:-1, :]
    out[:-1, :] |= mask_bool[1:, :]
    return out


def _colour(Lx, Ly):
    return (np.arange(Ly)[:, None] + np.arange(Lx)[None, :]) % 2


# --- random numbers ------------------------------------------------------------------------

def test_philox_bit_exact(mpr, orc):
    import torch

    # 1e6 random counters plus the edge counters (all zero, all ones), every word compared
    rng = np.random.default_rng(0)
    n = 1_000_000
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    seed = (0xDEADBEEF << 32) | 0x12345678
    t = torch.from_numpy(ctr.astype(np.uint32).view(np.int32)).cuda()
    out = mpr.mpr_philox4x32_10_dev(t, seed).cpu().numpy().view(np.uint32)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    exp = orc.philox_many(32, 10, ctr, key)
    bad = np.nonzero(np.any(out.astype(np.uint64) != exp, axis=1))[0]
    assert bad.size == 0, bad[:10]


# --- mapping, initial state, sample energy -------------------------------------------------

SHAPES = [(64, 64, 0.33), (131, 37, 0.9), (3, 5, 0.4), (2, 7, 0.3), (257, 129, 0.66)]


@pytest.mark.parametrize("Lx,Ly,p", SHAPES)
@pytest.mark.parametrize("setup", ["DDD", "SDS", "HDS", "BDS"])
def test_initial_state_matches_oracle(mpr, orc, Lx, Ly, p, setup):
    pr = mpr_inputs.make_problem(Lx, Ly, p, field_seed=Lx, mask_seed=Ly)
    h = mpr.mpr_create(pr.z, pr.mask)
    try:
        mpr.mpr_set_options(h, setup, seed=123)
        got, sweep = mpr.mpr_get_state(h)
        info = mpr.mpr_get_info(h)
    finally:
        mpr.mpr_destroy(h)
    o = _oracle(orc, Lx, Ly, 123, setup)
    phi, zmin, zmax = o.map(pr.z, pr.mask)
    exp = _round_store(o.init(phi, pr.mask), setup)
    assert sweep == 0
    assert (info["zmin"], info["zmax"]) == (zmin, zmax)
    assert info["n_pred"] == int((pr.mask == 0).sum())
    if setup[0] == "B":
        assert np.max(np.abs(got - exp)) <= 2.0**-5
    else:
        assert np.array_equal(got, exp)


@pytest.mark.parametrize("Lx,Ly,p", SHAPES)
def test_sample_energy_matches_oracle(mpr, orc, Lx, Ly, p):
    pr = mpr_inputs.make_problem(Lx, Ly, p, field_seed=2 * Lx, mask_seed=3 * Ly)
    o = orc.Oracle(Lx, Ly)
    phi, _, _ = o.map(pr.z, pr.mask)
    try:
        e_s, n = o.energy_sample(phi, pr.mask)
    except ValueError:
        with pytest.raises(mpr.MPRError) as ei:
            mpr.mpr_create(pr.z, pr.mask)
        assert ei.value.status == mpr.MPR_ERR_NO_PAIRS
        return
    h = mpr.mpr_create(pr.z, pr.mask)
    try:
        _, e_gpu = mpr.mpr_energy(h)
        info = mpr.mpr_get_info(h)
    finally:
        mpr.mpr_destroy(h)
    assert info["n_sample_pairs"] == n
    assert abs(e_gpu - e_s) <= 1e-13 * abs(e_s) + 1e-15


# --- one sweep from an identical state -----------------------------------------------------

def _start_state(orc, pr, setup, seed):
    o = _oracle(orc, pr.Lx, pr.Ly, seed, setup)
    phi, _, _ = o.map(pr.z, pr.mask)
    rng = np.random.default_rng(seed)
    state = np.where(pr.mask == 1, phi, rng.random(pr.z.shape) * TWO_PI)
    return o, _round_store(state, setup)


def _gpu_sweeps(mpr, pr, setup, seed, state, sweep, T, equil, samples=0):
    h = mpr.mpr_create(pr.z, pr.mask)
    try:
        mpr.mpr_set_options(h, setup, seed=seed)
        mpr.mpr_set_state(h, state, sweep)
        mpr.mpr_set_temperature(h, T)
        mpr.mpr_run(h, equil, samples)
        got, sw = mpr.mpr_get_state(h)
        info = mpr.mpr_get_info(h)
        zhat = mpr.mpr_predict(h) if samples else None
        eb, _ = mpr.mpr_energy(h)
    finally:
        mpr.mpr_destroy(h)
    return got, sw, info, zhat, eb


@pytest.mark.parametrize("Lx,Ly,p", SHAPES)
@pytest.mark.parametrize("T", [0.08, 1.0])
def test_single_sweep_ddd(mpr, orc, excusal_log, Lx, Ly, p, T):
    pr = mpr_inputs.make_problem(Lx, Ly, p, field_seed=5, mask_seed=6)
    o, state = _start_state(orc, pr, "DDD", 99)
    got, sw, info, _, _ = _gpu_sweeps(mpr, pr, "DDD", 99, state, 17, T, 1)
    exp, mm, om = o.sweep(state, pr.mask, T, 17, margins=True)
    assert sw == 18 and info["site_updates"] == info["n_pred"]
    bad = (mm < 1e-11) | (om < 1e-11)
    excused = bad | (_neighbours(bad & (_colour(Lx, Ly) == 0)) & (_colour(Lx, Ly) == 1))
    d = np.abs(got - exp)
    assert np.all(d[~excused] <= 1e-9), d[~excused].max()
    # FP64 margins below 1e-11 are rare (< 1e-5 of the sites)
    excusal_log("DDD", excused.sum(), Lx * Ly, 1e-5 * Lx * Ly)
    assert excused.sum() <= 1e-5 * Lx * Ly
    m = pr.mask == 1
    assert np.array_equal(got[m].view(np.uint64), state[m].view(np.uint64))


# Lattices with Lx > 256 run the TMA-fed kernel (300 x 45: ragged tile column and row; 2100 x 1300:
# several tiles per block); the others the one-tile-per-block kernel.
@pytest.mark.parametrize("Lx,Ly,p", [(64, 64, 0.33), (131, 37, 0.9), (257, 129, 0.66),
                                     (300, 45, 0.66), (2100, 1300, 0.9)])
@pytest.mark.parametrize("setup", ["SDS", "SSS", "SDD", "DDS"])
def test_single_sweep_fp32_functions(mpr, orc, excusal_log, Lx, Ly, p, setup):
    T = 0.3
    pr = mpr_inputs.make_problem(Lx, Ly, p, field_seed=7, mask_seed=8)
    o, state = _start_state(orc, pr, setup, 5)
    got, _, _, _, _ = _gpu_sweeps(mpr, pr, setup, 5, state, 3, T, 1)
    exp, mm, om = o.sweep(state, pr.mask, T, 3, margins=True)
    thr = 1e-4 if (setup[2] == "S" or setup[0] != "D") else 1e-11
    tol = 1e-4 if setup[2] == "S" or setup[0] == "S" else 1e-9
    bad = (mm < thr) | (om < thr)
    excused = bad | (_neighbours(bad & (_colour(Lx, Ly) == 0)) & (_colour(Lx, Ly) == 1))
    d = np.abs(got - exp)
    assert np.all(d[~excused] <= tol + 2 * _ulp_store(setup)), d[~excused].max()
    # the excused set comes from the oracle's margins alone (inputs fixed by the seeds); measured
    # 4.6e-4 of the sites at 2100 x 1300, 1.9e-3 at 131 x 37: the bound is about 3x that
    bound = max(10, 1.5e-3 * Lx * Ly)
    excusal_log(setup, excused.sum(), Lx * Ly, bound)
    assert excused.sum() <= bound


@pytest.mark.parametrize("Lx,Ly,p", [(64, 64, 0.33), (131, 37, 0.9), (300, 45, 0.66),
                                     (2100, 1300, 0.9)])
@pytest.mark.parametrize("setup", ["HDS", "BDS", "HSS"])
def test_single_sweep_16bit_storage(mpr, orc, excusal_log, Lx, Ly, p, setup):
    # Red phase: identical inputs; the GPU result is its FP32 update rounded to the storage type.
    # Black phase: against the oracle's black update on the oracle's own red result rounded to the
    # storage type. Both sides round FP32/FP64 red results to the same 16-bit value except near a
    # rounding boundary; black sites next to a red site where the two roundings differ are
    # excused, like those next to a red decision within the margin.
    T = 0.5
    pr = mpr_inputs.make_problem(Lx, Ly, p, field_seed=9, mask_seed=10)
    o, state = _start_state(orc, pr, setup, 8)
    got, _, _, _, _ = _gpu_sweeps(mpr, pr, setup, 8, state, 40, T, 1)
    red, mm_r, om_r = o.half_sweep(state, pr.mask, T, 40, 0)
    red_r = _round_store(red, setup)
    col = _colour(Lx, Ly)
    ulp = _ulp_store(setup)
    bad_r = (mm_r < 1e-4) | (om_r < 1e-4)
    sel = (col == 0) & ~bad_r
    d = np.abs(got - red_r)
    assert np.all(d[sel] <= ulp + 1e-4), d[sel].max()
    differs = (col == 0) & (bad_r | (got != red_r))
    assert differs.sum() <= (0.01 if setup[0] == "H" else 0.0025) * (col == 0).sum()
    blk, mm_b, om_b = o.half_sweep(red_r, pr.mask, T, 40, 1)
    bad_b = (mm_b < 1e-4) | (om_b < 1e-4)
    excused = bad_b | (_neighbours(differs) & (col == 1))
    sel = (col == 1) & ~excused
    d = np.abs(got - _round_store(blk, setup))
    assert np.all(d[sel] <= ulp + 1e-4), d[sel].max()
    # red sites whose stored result differs from the oracle's rounded one (a 16-bit rounding that
    # went the other way, or a decision within the margin) and the black sites they excuse:
    # measured up to 3.8e-3 / 1.5e-2 of the sites (FP16), 9e-4 / 3.4e-3 (BF16); bounds about 3x
    red_b, black_b = (0.01, 0.045) if setup[0] == "H" else (0.0025, 0.01)
    excusal_log(setup + " red", differs.sum(), (col == 0).sum(), red_b * (col == 0).sum())
    excusal_log(setup + " black", excused[col == 1].sum(), (col == 1).sum(),
                black_b * (col == 1).sum())
    assert excused[col == 1].mean() < black_b


# FP16 functions (HDH): as HDS, except that the doubled field angle of the over-relaxation is
# FP16 arithmetic. Its error is at most 3.4e-3 rad (2.4e-3 from the FP16 polynomial and result,
# 1e-3 from the FP16 rounding of the FP32 field components, which turns the field by at most
# 2^-11 rad whatever |h|), so an over-relaxed angle phi' = 2 r moves by up to 6.8e-3 rad; with
# both sides rounded to FP16 the results agree within 2^-8 + 6.8e-3. Sites whose over-relaxation
# decision lies within 4e-3 of the domain boundary (or whose Metropolis decision lies within 1e-4)
# are excused; the black pass starts from the GPU's red result on both sides.
HDH_TOL = 2.0**-8 + 6.8e-3
HDH_OR_MARGIN = 4e-3


@pytest.mark.parametrize("Lx,Ly,p", [(64, 64, 0.33), (131, 37, 0.9), (300, 45, 0.66),
                                     (2100, 1300, 0.9)])
def test_single_sweep_fp16_functions(mpr, orc, excusal_log, Lx, Ly, p):
    T = 0.5
    pr = mpr_inputs.make_problem(Lx, Ly, p, field_seed=19, mask_seed=20)
    o, state = _start_state(orc, pr, "HDH", 8)
    got, _, info, _, _ = _gpu_sweeps(mpr, pr, "HDH", 8, state, 40, T, 1)
    assert info["sweep_kernel"] == 0
    red, mm_r, om_r = o.half_sweep(state, pr.mask, T, 40, 0)
    red_r = _round_store(red, "HDH")
    col = _colour(Lx, Ly)
    bad_r = (mm_r < 1e-4) | (om_r < HDH_OR_MARGIN)
    sel = (col == 0) & ~bad_r
    d = np.abs(got - red_r)
    assert np.all(d[sel] <= HDH_TOL), d[sel].max()
    # black pass: the oracle's black update from the GPU's own red result (red values that differ
    # within the tolerance would otherwise move the black fields)
    start_b = np.where(col == 0, got, state)
    blk, mm_b, om_b = o.half_sweep(start_b, pr.mask, T, 40, 1)
    bad_b = (col == 1) & ((mm_b < 1e-4) | (om_b < HDH_OR_MARGIN))
    sel = (col == 1) & ~bad_b
    d = np.abs(got - _round_store(blk, "HDH"))
    assert np.all(d[sel] <= HDH_TOL), d[sel].max()
    bad_r = (col == 0) & bad_r
    excusal_log("HDH red", bad_r.sum(), (col == 0).sum(), 0.05 * (col == 0).sum())
    excusal_log("HDH black", bad_b.sum(), (col == 1).sum(), 0.05 * (col == 1).sum())
    assert bad_r.sum() <= 0.05 * (col == 0).sum() and bad_b.sum() <= 0.05 * (col == 1).sum()
    m = pr.mask == 1
    assert np.array_equal(got[m], state[m])


def test_fp16_functions_option_errors(mpr):
    pr = mpr_inputs.make_problem(64, 48, 0.5, field_seed=1, mask_seed=2)
    h = mpr.mpr_create(pr.z, pr.mask)
    try:
        for bad in ("SDH", "BDH", "DDH"):   # FP16 functions need FP16 spins
            with pytest.raises(mpr.MPRError) as e:
                mpr.mpr_set_options(h, bad)
            assert e.value.status == mpr.MPR_ERR_INVALID_ARG
        mpr.mpr_set_options(h, "HDH")
        with pytest.raises(mpr.MPRError) as e:   # uniform proposals only
            mpr.mpr_set_proposal(h, 0.5, 0.4)
        assert e.value.status == mpr.MPR_ERR_INVALID_ARG
        with pytest.raises(mpr.MPRError):        # no TMA kernel for FP16 functions
            mpr.mpr_set_sweep_kernel(h, 1)
    finally:
        mpr.mpr_destroy(h)


# --- energies, trajectories, predictions ---------------------------------------------------

@pytest.mark.parametrize("setup", ["DDD", "SDS", "HDS"])
def test_bond_energy_of_state(mpr, orc, setup):
    pr = mpr_inputs.make_problem(131, 37, 0.66, field_seed=11, mask_seed=12)
    o, state = _start_state(orc, pr, setup, 3)
    h = mpr.mpr_create(pr.z, pr.mask)
    try:
        mpr.mpr_set_options(h, setup)
        mpr.mpr_set_state(h, state, 0)
        eb, _ = mpr.mpr_energy(h)
    finally:
        mpr.mpr_destroy(h)
    assert abs(eb - o.energy_bond(state)) < 1e-13


def test_ddd_trajectory_prediction_and_energy(mpr, orc):
    pr = mpr_inputs.make_problem(64, 64, 0.33, field_seed=13, mask_seed=14)
    o, state = _start_state(orc, pr, "DDD", 21)
    T, equil, ns = 0.25, 60, 20
    got, sw, info, zhat, _ = _gpu_sweeps(mpr, pr, "DDD", 21, state, 0, T, equil, ns)
    phi, zmin, zmax = o.map(pr.z, pr.mask)
    st, _, _ = o.run(state, pr.mask, T, 0, equil)
    st, acc, e = o.run(st, pr.mask, T, equil, ns, acc=np.zeros_like(st), energies=True)
    exp_z = o.predict(acc, ns, pr.z, pr.mask, zmin, zmax)
    pred = pr.mask == 0
    close = np.abs(got - st) < 1e-9
    assert close.mean() > 0.999
    assert np.array_equal(zhat[~pred], pr.z[~pred])
    assert np.mean(np.abs(zhat - exp_z)[pred] < 1e-7) > 0.999
    if close.all():
        assert abs(info["e_bond_mean"] - e.mean()) < 1e-12
    assert sw == equil + ns and info["n_samples"] == ns


@pytest.mark.parametrize("setup", SETUPS_ALL)
@pytest.mark.parametrize("acc", ["f64", "kahan"])
def test_frozen_sites_bit_exact_and_predictions_in_range(mpr, setup, acc):
    pr = mpr_inputs.make_problem(131, 37, 0.66, field_seed=15, mask_seed=16)
    h = mpr.mpr_create(pr.z, pr.mask)
    try:
        mpr.mpr_set_options(h, setup, seed=4, acc=acc)
        before, _ = mpr.mpr_get_state(h)
        mpr.mpr_set_temperature(h, 0.2)
        mpr.mpr_run(h, 30, 10)
        after, _ = mpr.mpr_get_state(h)
        zhat = mpr.mpr_predict(h)
        info = mpr.mpr_get_info(h)
    finally:
        mpr.mpr_destroy(h)
    m = pr.mask == 1
    assert np.array_equal(after[m].view(np.uint64), before[m].view(np.uint64))
    # angles stay in [0, 2*pi] as rounded to the storage type (FP32 rounds 2*pi up)
    assert np.all((after >= 0) & (after <= _round_store(np.float32(TWO_PI), setup).max()))
    assert np.array_equal(zhat[m], pr.z[m])
    assert np.all((zhat >= info["zmin"] - 1e-9) & (zhat <= info["zmax"] + 1e-9))
    assert np.isfinite(info["e_bond_mean"])


def test_tuning_matches_oracle_ddd(mpr, orc):
    pr = mpr_inputs.make_problem(48, 40, 0.33, field_seed=17, mask_seed=18)
    kw = dict(n_eq=40, n_meas=20)
    h = mpr.mpr_create(pr.z, pr.mask)
    try:
        mpr.mpr_set_options(h, "DDD", seed=6)
        mpr.mpr_set_tuning(h, **kw)
        T_gpu, st = mpr.mpr_tune_temperature(h)
        info = mpr.mpr_get_info(h)
    finally:
        mpr.mpr_destroy(h)
    o = orc.Oracle(48, 40, seed=6)
    phi, _, _ = o.map(pr.z, pr.mask)
    phi = o.init(phi, pr.mask)
    e_s, _ = o.energy_sample(phi, pr.mask)
    st_o, T_o, _, sw, trace = o.tune(phi, pr.mask, e_s, 0, **kw)
    assert st == st_o == 0
    assert info["n_probes"] == len(trace) and info["sweep"] == sw
    assert abs(T_gpu / T_o - 1.0) < 1e-9


# --- edge cases ----------------------------------------------------------------------------

def test_edge_cases(mpr):
    z = np.arange(12, dtype=np.float64).reshape(3, 4)
    with pytest.raises(mpr.MPRError) as e:
        mpr.mpr_create(np.full((3, 4), 2.0), np.ones((3, 4)))
    assert e.value.status == mpr.MPR_ERR_DEGENERATE
    m = np.zeros((3, 4), np.uint8)
    m[0, 0] = 1
    with pytest.raises(mpr.MPRError) as e:
        mpr.mpr_create(z, m)
    assert e.value.status == mpr.MPR_ERR_DEGENERATE
    m[2, 3] = 1
    with pytest.raises(mpr.MPRError) as e:
        mpr.mpr_create(z, m)
    assert e.value.status == mpr.MPR_ERR_NO_PAIRS
    bad = z.copy()
    bad[0, 0] = np.nan
    with pytest.raises(mpr.MPRError) as e:
        mpr.mpr_create(bad, np.ones((3, 4)))
    assert e.value.status == mpr.MPR_ERR_INVALID_ARG
    # NaN at a prediction site is ignored
    m2 = np.ones((3, 4), np.uint8)
    m2[1, 1] = 0
    h = mpr.mpr_create(np.where(m2 == 1, z, np.nan), m2)
    try:
        with pytest.raises(mpr.MPRError) as e:
            mpr.mpr_run(h, 1, 1)
        assert e.value.status == mpr.MPR_ERR_STATE
        with pytest.raises(mpr.MPRError) as e:
            mpr.mpr_predict(h)
        assert e.value.status == mpr.MPR_ERR_STATE
        mpr.mpr_set_temperature(h, 0.5)
        mpr.mpr_run(h, 3, 2)
        zh = mpr.mpr_predict(h)
        assert np.isfinite(zh).all()
    finally:
        mpr.mpr_destroy(h)
    # every site measured: nothing to update, prediction = data
    h = mpr.mpr_create(z, np.ones((3, 4)))
    try:
        mpr.mpr_set_temperature(h, 0.5)
        mpr.mpr_run(h, 2, 2)
        assert np.array_equal(mpr.mpr_predict(h), z)
        assert mpr.mpr_get_info(h)["site_updates"] == 0
    finally:
        mpr.mpr_destroy(h)


def test_device_entry_points(mpr):
    import torch

    pr = mpr_inputs.make_problem(96, 80, 0.66, field_seed=19, mask_seed=20)
    s = torch.cuda.Stream()
    zt = torch.from_numpy(pr.z).cuda()
    mt = torch.from_numpy(pr.mask).cuda()
    h1 = mpr.mpr_create_dev(zt, mt, stream=s)
    h2 = mpr.mpr_create(pr.z, pr.mask)
    try:
        for h in (h1, h2):
            mpr.mpr_set_options(h, "SDS", seed=3)
            mpr.mpr_set_temperature(h, 0.3)
            mpr.mpr_run(h, 20, 5)
        out = torch.empty_like(zt)
        mpr.mpr_predict_dev(h1, out)
        assert np.array_equal(out.cpu().numpy(), mpr.mpr_predict(h2))
    finally:
        mpr.mpr_destroy(h1)
        mpr.mpr_destroy(h2)


def test_problem_class_equals_the_c_calls(mpr):
    # the convenience class (host and device inputs) runs the same chain as the plain calls
    import torch

    pr = mpr_inputs.make_problem(120, 90, 0.66, field_seed=21, mask_seed=22)
    h = mpr.mpr_create(pr.z, pr.mask)
    try:
        mpr.mpr_set_options(h, "HDS", seed=4)
        T, _ = mpr.mpr_tune_temperature(h)
        mpr.mpr_run(h, 30, 10)
        ref = mpr.mpr_predict(h)
    finally:
        mpr.mpr_destroy(h)
    with mpr.Problem(pr.z, pr.mask, setup="HDS", seed=4) as p:
        assert p.tune() == T
        p.run(30, 10)
        assert np.array_equal(p.predict(), ref)
    zt = torch.from_numpy(pr.z).cuda()
    mt = torch.from_numpy(pr.mask).cuda()
    with mpr.GapFiller(zt, mt, setup="HDS", seed=4) as p:
        assert np.array_equal(p.fill(30, 10), ref) and p.T == T
        out = p.predict(torch.empty_like(zt))
        assert np.array_equal(out.cpu().numpy(), ref)


def test_handles_reuse_pooled_memory(mpr):
    # handles of one size in a row draw their device memory from the library's pool: every run
    # starts from its own initialisation (nothing leaks from the previous handle's blocks), and
    # trimming the pool leaves later handles working
    pr = mpr_inputs.make_problem(600, 300, 0.9, field_seed=23, mask_seed=24)
    out = []
    for k in range(4):
        h = mpr.mpr_create(pr.z, pr.mask)
        try:
            mpr.mpr_set_options(h, "HDS", seed=3)
            mpr.mpr_set_temperature(h, 0.2)
            mpr.mpr_run(h, 20, 5)
            out.append((mpr.mpr_get_state(h)[0], mpr.mpr_predict(h)))
        finally:
            mpr.mpr_destroy(h)
        if k == 1:
            mpr.mpr_trim_memory()
    for st, zh in out[1:]:
        assert np.array_equal(st, out[0][0]) and np.array_equal(zh, out[0][1])


# --- checkpoint / resume and other q -------------------------------------------------------

@pytest.mark.parametrize("setup", ["DDD", "SDS", "HDS"])
def test_checkpoint_resume_is_bit_exact(mpr, setup):
    # counter-based random numbers: run(2n) == run(n); save; restore into a new handle; run(n)
    pr = mpr_inputs.make_problem(131, 37, 0.66, field_seed=21, mask_seed=22)
    T, n = 0.3, 25
    h1 = mpr.mpr_create(pr.z, pr.mask)
    h2 = mpr.mpr_create(pr.z, pr.mask)
    h3 = mpr.mpr_create(pr.z, pr.mask)
    try:
        for h in (h1, h2, h3):
            mpr.mpr_set_options(h, setup, seed=11)
            mpr.mpr_set_temperature(h, T)
        mpr.mpr_run(h1, 2 * n, 0)
        full, sw_full = mpr.mpr_get_state(h1)
        mpr.mpr_run(h2, n, 0)
        half, sw_half = mpr.mpr_get_state(h2)
        mpr.mpr_set_state(h3, half, sw_half)
        mpr.mpr_run(h3, n, 0)
        resumed, sw_res = mpr.mpr_get_state(h3)
    finally:
        for h in (h1, h2, h3):
            mpr.mpr_destroy(h)
    assert sw_full == sw_res == 2 * n
    assert np.array_equal(full.view(np.uint64), resumed.view(np.uint64))


@pytest.mark.parametrize("q", [0.3, 1.0])
@pytest.mark.parametrize("setup", ["DDD", "SDS"])
def test_single_sweep_other_q(mpr, orc, excusal_log, setup, q):
    # the general over-relaxation (any q in (0, 1]; q = 1 is the planar rotator of Eq. 1)
    T = 0.4
    pr = mpr_inputs.make_problem(131, 37, 0.66, field_seed=23, mask_seed=24)
    o = orc.Oracle(131, 37, seed=12, q=q, ubits=32 if setup[2] == "D" else 23)
    phi, _, _ = o.map(pr.z, pr.mask)
    rng = np.random.default_rng(12)
    state = _round_store(np.where(pr.mask == 1, phi, rng.random(pr.z.shape) * TWO_PI), setup)
    h = mpr.mpr_create(pr.z, pr.mask)
    try:
        mpr.mpr_set_options(h, setup, seed=12, q=q)
        mpr.mpr_set_state(h, state, 5)
        mpr.mpr_set_temperature(h, T)
        mpr.mpr_run(h, 1, 0)
        got, _ = mpr.mpr_get_state(h)
        e_gpu, e_s = mpr.mpr_energy(h)
    finally:
        mpr.mpr_destroy(h)
    exp, mm, om = o.sweep(state, pr.mask, T, 5, margins=True)
    thr = 1e-11 if setup == "DDD" else 1e-4
    tol = 1e-9 if setup == "DDD" else 1e-4
    bad = (mm < thr) | (om < thr)
    col = _colour(131, 37)
    excused = bad | (_neighbours(bad & (col == 0)) & (col == 1))
    d = np.abs(got - exp)
    assert np.all(d[~excused] <= tol + 2 * _ulp_store(setup)), d[~excused].max()
    bound = 1e-5 * excused.size if setup == "DDD" else max(10, 1.5e-3 * excused.size)
    excusal_log(f"{setup} q={q}", excused.sum(), excused.size, bound)
    assert excused.sum() <= bound
    assert abs(e_s - o.energy_sample(phi, pr.mask)[0]) < 1e-12


def test_tall_thin_grid_beyond_grid_limits(mpr, orc):
    # more rows than a 2-D launch grid has in y (65535): init, sweeps, energy and prediction
    Lx, Ly = 3, 70001
    pr = mpr_inputs.make_problem(Lx, Ly, 0.5, field_seed=31, mask_seed=32, periodic=True)
    for setup in ("DDD", "SDS"):
        o, state = _start_state(orc, pr, setup, 2)
        h = mpr.mpr_create(pr.z, pr.mask)
        try:
            mpr.mpr_set_options(h, setup, seed=2)
            init, _ = mpr.mpr_get_state(h)
            exp0 = _round_store(o.init(o.map(pr.z, pr.mask)[0], pr.mask), setup)
            assert np.array_equal(init, exp0)
            mpr.mpr_set_state(h, state, 0)
            mpr.mpr_set_temperature(h, 0.5)
            mpr.mpr_run(h, 0, 1)   # one sweep, sampled
            got, _ = mpr.mpr_get_state(h)
            zhat = mpr.mpr_predict(h)
        finally:
            mpr.mpr_destroy(h)
        exp, mm, om = o.sweep(state, pr.mask, 0.5, 0, margins=True)
        thr = 1e-11 if setup == "DDD" else 1e-4
        bad = (mm < thr) | (om < thr)
        col = _colour(Lx, Ly)
        excused = bad | (_neighbours(bad & (col == 0)) & (col == 1))
        assert np.all(np.abs(got - exp)[~excused] <= (1e-9 if setup == "DDD" else 1e-4))
        assert np.array_equal(zhat[pr.mask == 1], pr.z[pr.mask == 1])


# --- the two FP32 sweep kernels ------------------------------------------------------------

def _kernel_run(mpr, pr, setup, state, kind, equil, samples, T=0.3):
    h = mpr.mpr_create(pr.z, pr.mask)
    try:
        mpr.mpr_set_options(h, setup, seed=31)
        mpr.mpr_set_sweep_kernel(h, kind)
        mpr.mpr_set_state(h, state, 5)
        mpr.mpr_set_temperature(h, T)
        mpr.mpr_run(h, equil, samples)
        got, sw = mpr.mpr_get_state(h)
        info = mpr.mpr_get_info(h)
        zhat = mpr.mpr_predict(h) if samples else None
    finally:
        mpr.mpr_destroy(h)
    return got, sw, info, zhat


@pytest.mark.parametrize("Lx,Ly,p", [(300, 45, 0.66), (2100, 1300, 0.9), (517, 34, 0.33)])
@pytest.mark.parametrize("setup", ["HDS", "SDS", "DDS", "BDS"])
def test_tma_kernel_equals_tile_kernel(mpr, orc, Lx, Ly, p, setup):
    # The TMA-fed persistent kernel (kind 1: 128 x 32 tiles, several per block at 2100 x 1300,
    # ragged last tile column and row) and the one-tile-per-block kernel (kind 0) apply the same
    # per-site arithmetic: states after plain sweeps, and predictions and energies after sampling
    # sweeps (whose energy passes always run kind 0), agree bit for bit.
    pr = mpr_inputs.make_problem(Lx, Ly, p, field_seed=41, mask_seed=42)
    _, state = _start_state(orc, pr, setup, 31)
    g0, s0, i0, z0 = _kernel_run(mpr, pr, setup, state, 0, 6, 3)
    g1, s1, i1, z1 = _kernel_run(mpr, pr, setup, state, 1, 6, 3)
    assert i0["sweep_kernel"] == 0 and i1["sweep_kernel"] == 1
    assert s0 == s1 == 14
    assert np.array_equal(g0, g1)
    assert np.array_equal(z0, z1)
    assert i0["e_bond_mean"] == i1["e_bond_mean"]


@pytest.mark.parametrize("Lx,Ly,setup", [(4096, 2048, "HDS"), (2100, 1301, "SDS"), (4096, 4096, "HDS"),
                                          (2048, 1024, "SDS"), (2100, 2200, "HDS"),
                                          (4096, 1200, "SDS"), (8192, 4096, "HDS")])
def test_tma_kernel_equals_tile_kernel_over_many_sweeps(mpr, orc, Lx, Ly, setup):
    # The two FP32 sweep kernels over 200 sweeps with several waves of tiles (and an odd Ly, whose
    # last Philox group of rows has one row): identical chains, bit for bit. On a 152-SM GPU, at
    # 4096^2 both kernels run the last 224 tiles of a plain pass as half-height tiles, the tile
    # kernel at 2048 x 1024 all of them (one partial wave). The persistent TMA kernel (4 blocks per
    # SM with 16-bit spins, 3 with FP32) also splits at 2100 x 2200 (621 tiles, the last 13 split,
    # ragged last tile column and row) and at 4096 x 1200 (608 tiles on 456 blocks: the last 152
    # split, the lower halves of the last tile row lie wholly below the lattice). The FP16 lattices
    # up to 4096^2 fit the L2 and run the tile kernel's plain pass that loads each own row at its
    # update; 8192 x 4096 (67 MB) runs the one that loads them all before the staging.
    pr = mpr_inputs.make_problem(Lx, Ly, 0.9, field_seed=43, mask_seed=44)
    _, state = _start_state(orc, pr, setup, 33)
    g0, s0, i0, _ = _kernel_run(mpr, pr, setup, state, 0, 200, 0, T=0.07)
    g1, s1, i1, _ = _kernel_run(mpr, pr, setup, state, 1, 200, 0, T=0.07)
    assert i0["sweep_kernel"] == 0 and i1["sweep_kernel"] == 1 and s0 == s1 == 205
    assert np.array_equal(g0, g1)


def test_sweep_kernel_choice(mpr, orc):
    pr = mpr_inputs.make_problem(700, 300, 0.9, field_seed=43, mask_seed=44)
    _, state = _start_state(orc, pr, "HDS", 31)
    # automatic: the first run of >= 12 plain sweeps times both kernels inside the chain
    ga, _, ia, _ = _kernel_run(mpr, pr, "HDS", state, -1, 20, 0)
    g0, _, _, _ = _kernel_run(mpr, pr, "HDS", state, 0, 20, 0)
    assert ia["sweep_kernel"] in (0, 1)
    assert np.array_equal(ga, g0)
    # not chosen yet after a short run
    _, _, ib, _ = _kernel_run(mpr, pr, "HDS", state, -1, 3, 0)
    assert ib["sweep_kernel"] == -1
    # kind 1 needs FP32 functions and a lattice wider than one tile with >= 34 rows
    for shape, setup in [((256, 300), "HDS"), ((700, 33), "SDS"), ((700, 300), "DDD")]:
        q = mpr_inputs.make_problem(*shape, 0.5, field_seed=45, mask_seed=46)
        h = mpr.mpr_create(q.z, q.mask)
        try:
            mpr.mpr_set_options(h, setup, seed=1)
            with pytest.raises(mpr.MPRError) as e:
                mpr.mpr_set_sweep_kernel(h, 1)
            assert e.value.status == mpr.MPR_ERR_INVALID_ARG
            mpr.mpr_set_sweep_kernel(h, 0)
            assert mpr.mpr_get_info(h)["sweep_kernel"] == (-1 if setup == "DDD" else 0)
        finally:
            mpr.mpr_destroy(h)
    h = mpr.mpr_create(pr.z, pr.mask)
    try:
        for bad in (-2, 2):
            with pytest.raises(mpr.MPRError):
                mpr.mpr_set_sweep_kernel(h, bad)
    finally:
        mpr.mpr_destroy(h)


def test_tma_wait_timeout_is_reported(mpr, orc):
    # The TMA kernel's mbarrier wait is bounded: with the copies of block 0's first tile left out
    # (host-side injection), the wait runs out, the block records the error and returns, the
    # launch ends normally and the next synchronising call reports MPR_ERR_DEVICE_TIMEOUT. The
    # handle stays usable afterwards.
    pr = mpr_inputs.make_problem(700, 300, 0.9, field_seed=47, mask_seed=48)
    h = mpr.mpr_create(pr.z, pr.mask)
    try:
        mpr.mpr_set_options(h, "HDS", seed=2)
        mpr.mpr_set_sweep_kernel(h, 1)
        mpr.mpr_set_temperature(h, 0.3)
        mpr.mpr_run(h, 2, 0)
        mpr.mpr_inject_tma_stall(h, 0.05)
        with pytest.raises(mpr.MPRError) as e:
            mpr.mpr_run(h, 2, 0)
        assert e.value.status == mpr.MPR_ERR_DEVICE_TIMEOUT
        mpr.mpr_run(h, 2, 0)   # the error was reported once; the handle keeps working
        st, sw = mpr.mpr_get_state(h)
        assert sw == 6 and np.all(np.isfinite(st))
    finally:
        mpr.mpr_destroy(h)
    q = mpr_inputs.make_problem(64, 64, 0.5, field_seed=49, mask_seed=50)
    h = mpr.mpr_create(q.z, q.mask)
    try:
        with pytest.raises(mpr.MPRError):
            mpr.mpr_inject_tma_stall(h, 0.05)   # no TMA kernel for a lattice this narrow
    finally:
        mpr.mpr_destroy(h)


# --- the bench's workloads at full size, sampled --------------------------------------------

@pytest.mark.parametrize("L,setup", [(4096, "HDS"), (8192, "HDS"), (16384, "SDS")])
def test_full_size_sweep_sampled_sites(mpr, orc, excusal_log, L, setup):
    # The workloads bench.py times (4096^2 and 16384^2, p = 0.9) through the C ABI in its launch
    # configuration (the tile kernel, which the automatic choice keeps at these sizes), and 8192^2
    # with FP16 spins, whose 134 MB state takes the plain pass that loads all own rows before the
    # staging (at 4096^2 the state fits the L2 and each own row is loaded at its update): one sweep
    # from an identical state; 2000 sampled sites of each colour are recomputed one by one by the
    # oracle -- red sites from the initial state, black sites from the GPU's red neighbours -- and
    # must agree within the FP32 tolerance outside near-threshold decisions. Frozen sites are
    # compared in full, bit for bit.
    import torch

    dev = torch.device("cuda", 0)
    pr = mpr_inputs.make_problem(L, L, 0.9, field_seed=1, mask_seed=101, periodic=L > 4096,
                                 device=dev)
    o = _oracle(orc, L, L, 7, setup)
    phi, _, _ = o.map(pr.z, pr.mask)
    rng = np.random.default_rng(3)
    state = np.where(pr.mask == 1, phi.reshape(L, L), rng.random((L, L)) * TWO_PI)
    state = np.ascontiguousarray(_round_store(state, setup))
    T, sweep = 0.07, 11
    got, sw, info, _, _ = _gpu_sweeps(mpr, pr, setup, 7, state, sweep, T, 1)
    # one sweep is too short for the automatic choice (-1: not chosen yet), which runs kind 0
    assert sw == sweep + 1 and info["sweep_kernel"] in (-1, 0)
    frozen = pr.mask == 1
    assert np.array_equal(got[frozen].view(np.uint64), state[frozen].view(np.uint64))
    col = _colour(L, L)
    tol = 1e-4 + 2 * _ulp_store(setup)
    work = state.copy()
    mask8 = np.ascontiguousarray(pr.mask, dtype=np.uint8)   # passed to the oracle without a copy
    for c in (0, 1):
        ys, xs = np.nonzero((col == c) & ~frozen)
        pick = rng.choice(ys.size, 2000, replace=False)
        bad = excused = 0
        for k in pick:
            y, x = int(ys[k]), int(xs[k])
            nbr = [(yy, xx) for yy, xx in ((y, x - 1), (y, x + 1), (y - 1, x), (y + 1, x))
                   if 0 <= yy < L and 0 <= xx < L]
            if c == 1:   # black: the GPU's red neighbours as inputs
                for yy, xx in nbr:
                    work[yy, xx] = got[yy, xx]
            f, mm, om = o.update_site(work, mask8, x, y, T, sweep)
            if c == 1:
                for yy, xx in nbr:
                    work[yy, xx] = state[yy, xx]
            if mm < 1e-4 or om < 1e-4:
                excused += 1
                continue
            if abs(got[y, x] - _round_store(np.array([f]), setup)[0]) > tol:
                bad += 1
        assert bad == 0, (c, bad)
        # about 1 of 2000 expected (margins below 1e-4 on ~5e-4 of the sites); measured 0
        excusal_log(f"{setup} c{c}", excused, 2000, 10)
        assert excused <= 10, (c, excused)


@pytest.mark.slow
def test_maximum_lattice_size(mpr, orc):
    # The largest lattice the ABI accepts (N < 2^31 sites: 65536 x 32767 = 2 147 418 112), HDS,
    # inputs on the device: every element offset beyond 2^31 bytes (FP64 inputs, accumulators,
    # state transfer) and the last rows and columns go through the same one-sweep check as the
    # full-size test, with the sampled sites weighted toward the end of the arrays; frozen sites
    # bit for bit.
    import torch

    Lx, Ly = 65536, 32767
    dev = torch.device("cuda", 0)
    # one row more is 2^31 sites: refused before the buffers are read
    import ctypes

    small = np.zeros(4)
    hh = ctypes.c_void_p()
    st = mpr.load().mpr_create(Lx, Ly + 1, small.ctypes.data_as(ctypes.c_void_p),
                               small.ctypes.data_as(ctypes.c_void_p), ctypes.byref(hh))
    assert st == mpr.MPR_ERR_INVALID_ARG and not hh.value
    ys = torch.arange(Ly, device=dev, dtype=torch.float64)[:, None]
    xs = torch.arange(Lx, device=dev, dtype=torch.float64)[None, :]
    z = 50.0 + 10.0 * torch.sin(xs / 61.0) * torch.cos(ys / 47.0)
    del xs, ys
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    mask = (torch.rand((Ly, Lx), generator=g, device=dev) >= 0.9).to(torch.uint8)
    T, seed = 0.07, 7
    h = mpr.mpr_create_dev(z, mask)
    try:
        mpr.mpr_set_options(h, "HDS", seed=seed)
        state, sw0 = mpr.mpr_get_state(h)
        mpr.mpr_set_temperature(h, T)
        mpr.mpr_run(h, 1, 0)
        got, sw = mpr.mpr_get_state(h)
        info = mpr.mpr_get_info(h)
    finally:
        mpr.mpr_destroy(h)
    del z
    mask8 = mask.cpu().numpy()
    del mask
    torch.cuda.empty_cache()
    assert sw == sw0 + 1 and info["n_sites"] == Lx * Ly
    frozen = mask8 == 1
    assert np.array_equal(got[frozen].view(np.uint64), state[frozen].view(np.uint64))
    del frozen
    o = _oracle(orc, Lx, Ly, seed, "HDS")
    tol = 1e-4 + 2 * _ulp_store("HDS")
    rng = np.random.default_rng(11)
    # sampled rows: uniform, plus the last 16 rows; columns uniform plus the last 16
    rows = np.concatenate([rng.integers(0, Ly, 300), Ly - 1 - rng.integers(0, 16, 300)])
    cols = np.concatenate([rng.integers(0, Lx, 300), Lx - 1 - rng.integers(0, 16, 300)])
    rng.shuffle(cols)
    checked = {0: 0, 1: 0}
    for c in (0, 1):
        bad = excused = 0
        for y, x in zip(rows, cols):
            y, x = int(y), int(x)
            if (x + y) % 2 != c:   # move to the neighbouring column: a site of colour c
                x = x - 1 if x > 0 else x + 1
            if mask8[y, x]:
                continue
            nbr = [(yy, xx) for yy, xx in ((y, x - 1), (y, x + 1), (y - 1, x), (y + 1, x))
                   if 0 <= yy < Ly and 0 <= xx < Lx]
            saved = [state[yy, xx] for yy, xx in nbr]
            if c == 1:   # black: the GPU's red neighbours as inputs
                for yy, xx in nbr:
                    state[yy, xx] = got[yy, xx]
            f, mm, om = o.update_site(state, mask8, x, y, T, sw0)
            for (yy, xx), v in zip(nbr, saved):
                state[yy, xx] = v
            checked[c] += 1
            if mm < 1e-4 or om < 1e-4:
                excused += 1
                continue
            if abs(got[y, x] - _round_store(np.array([f]), "HDS")[0]) > tol:
                bad += 1
        assert bad == 0, (c, bad)
        assert excused < 20, (c, excused)
    assert min(checked.values()) > 400, checked


# --- energy-slope equilibration ----------------------------------------------------------------

def test_run_auto_matches_oracle_ddd(mpr, orc):
    # mpr_run_auto against the oracle's mpro_equilibrate (same stopping rule): in FP64 the two
    # chains and their energy series agree to rounding, so they stop after the same number of
    # sweeps and end in the same state; then the samples as mpr_run.
    pr = mpr_inputs.make_problem(64, 64, 0.33, field_seed=51, mask_seed=52)
    o, state = _start_state(orc, pr, "DDD", 23)
    T, chunk, ns = 0.05, 10, 5
    h = mpr.mpr_create(pr.z, pr.mask)
    try:
        mpr.mpr_set_options(h, "DDD", seed=23)
        mpr.mpr_set_state(h, state, 0)
        mpr.mpr_set_temperature(h, T)
        n = mpr.mpr_run_auto(h, chunk, 5000, ns)
        got, sw = mpr.mpr_get_state(h)
        info = mpr.mpr_get_info(h)
    finally:
        mpr.mpr_destroy(h)
    p, n_o, sw_o = o.equilibrate(state, pr.mask, T, 0, chunk, 5000)
    assert n == n_o and 2 * chunk <= n < 5000
    p, _, e = o.run(p, pr.mask, T, sw_o, ns, energies=True)
    assert sw == n + ns and info["n_samples"] == ns
    assert np.mean(np.abs(got - p) < 1e-9) > 0.999


@pytest.mark.parametrize("setup", ["HDS", "SDS"])
def test_run_auto_reaches_the_long_run_energy(mpr, setup):
    # FP32 functions: the stop comes after the relaxation, at the energy of a long plain run.
    pr = mpr_inputs.make_problem(512, 512, 0.9, field_seed=53, mask_seed=54)
    T = 0.06
    h = mpr.mpr_create(pr.z, pr.mask)
    try:
        mpr.mpr_set_options(h, setup, seed=5)
        mpr.mpr_set_temperature(h, T)
        n = mpr.mpr_run_auto(h, 20, 20000, 50)
        e_stop = mpr.mpr_get_info(h)["e_bond_mean"]
        mpr.mpr_run(h, 2000, 200)
        e_long = mpr.mpr_get_info(h)["e_bond_mean"]
        with pytest.raises(mpr.MPRError):
            mpr.mpr_run_auto(h, 1, 100, 0)
    finally:
        mpr.mpr_destroy(h)
    assert 40 <= n < 20000
    assert abs(e_stop - e_long) < 2e-3, (n, e_stop, e_long)
