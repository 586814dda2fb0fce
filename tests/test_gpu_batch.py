"""Batched persistent path: many problems of uneven size in one cooperative launch.

Checks: problem i of a batch follows the chain of the oracle with Philox problem id i (single
sweep from the initial state); problem 0 follows the single-handle GPU path bit for bit; results
do not depend on the launch shape or on the graph launch; tuning in the batch matches the
single-handle tuning; a grid-barrier wait that cannot complete ends the launch with
MPR_ERR_DEVICE_TIMEOUT (fault injected on the host side; the wait is bounded, nothing hangs).
"""
import math

import numpy as np
import pytest

import mpr_inputs

pytestmark = pytest.mark.gpu

TWO_PI = 2.0 * math.pi
SHAPES = [(64, 64, 0.33), (131, 37, 0.9), (3, 5, 0.4), (200, 90, 0.66), (57, 301, 0.9), (2, 9, 0.3)]


@pytest.fixture(scope="module")
def mpr():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1910_08448_gb300 as m

    m.load()
    return m


def _problems(shapes=SHAPES, base=0):
    return [mpr_inputs.make_problem(Lx, Ly, p, field_seed=base + 11 * i + 1, mask_seed=base + 11 * i + 2)
            for i, (Lx, Ly, p) in enumerate(shapes)]


def _neighbours(b):
    out = np.zeros_like(b)
    out[:, 1:] |= b[:, :-1]
    out[:, :-1] |= b[:, 1:]
    out[1:, :] |= b[:-1, :]
    out[:-1, :] |= b[1:, :]
    return out


@pytest.mark.parametrize("setup", ["SDS", "HDS", "SSS"])
def test_batch_single_sweep_matches_oracle_per_problem(mpr, orc, excusal_log, setup):
    probs = _problems()
    b = mpr.mpr_batch_create([p.z for p in probs], [p.mask for p in probs], setup, seed=17)
    try:
        T = np.full(len(probs), 0.4)
        mpr.mpr_batch_fill(b, 1, 0, T=T)
        for i, pr in enumerate(probs):
            got, sw = mpr.mpr_batch_get_state(b, i)
            assert sw == 1
            o = orc.Oracle(pr.Lx, pr.Ly, seed=17, problem=i, ubits=23)
            dt = np.float16 if setup[0] == "H" else np.float32
            rnd = lambda a: a.astype(dt).astype(np.float64)   # storage rounding, test side
            ulp = 2.0**-8 if setup[0] == "H" else 2.0**-21
            phi, _, _ = o.map(pr.z, pr.mask)
            start = rnd(o.init(phi, pr.mask))
            # red pass on identical inputs; black pass on the oracle's own red result rounded to
            # the storage type (the GPU stores every result in that type)
            red, mm_r, om_r = o.half_sweep(start, pr.mask, 0.4, 0, 0)
            red_r = rnd(red)
            blk, mm_b, om_b = o.half_sweep(red_r, pr.mask, 0.4, 0, 1)
            col = (np.arange(pr.Ly)[:, None] + np.arange(pr.Lx)[None, :]) % 2
            bad_r = (col == 0) & ((mm_r < 1e-4) | (om_r < 1e-4))
            sel = (col == 0) & ~bad_r
            assert np.all(np.abs(got - red_r)[sel] <= ulp + 1e-4), i
            # red sites whose stored result differs from the oracle's by more than FP32 error (a
            # 16-bit rounding that went the other way): their black neighbours see other inputs
            differs = bad_r | ((col == 0) & (np.abs(got - red_r) > 1e-4))
            # bounds about 3x the measured rates (as in the single-handle 16-bit test)
            red_b, black_b = (0.01, 0.045) if setup[0] == "H" else (0.0025, 0.01)
            assert differs.sum() <= max(2, red_b * (col == 0).sum())
            excused = ((col == 1) & ((mm_b < 1e-4) | (om_b < 1e-4))) | (_neighbours(differs) & (col == 1))
            sel = (col == 1) & ~excused
            d = np.abs(got - rnd(blk))
            assert np.all(d[sel] <= ulp + 1e-4), (i, d[sel].max())
            excusal_log(f"{setup} p{i} red", differs.sum(), (col == 0).sum(),
                        max(2, red_b * (col == 0).sum()))
            excusal_log(f"{setup} p{i} blk", excused[col == 1].sum(), (col == 1).sum(),
                        max(8, black_b * (col == 1).sum()))
            assert excused[col == 1].sum() <= max(8, black_b * (col == 1).sum())
            m = pr.mask == 1
            assert np.array_equal(got[m], start[m])
    finally:
        mpr.mpr_batch_destroy(b)


def test_batch_problem0_equals_single_handle(mpr):
    probs = _problems()
    b = mpr.mpr_batch_create([p.z for p in probs], [p.mask for p in probs], "SDS", seed=5)
    h = mpr.mpr_create(probs[0].z, probs[0].mask)
    try:
        mpr.mpr_set_options(h, "SDS", seed=5)
        mpr.mpr_set_temperature(h, 0.3)
        mpr.mpr_run(h, 40, 10)
        single, _ = mpr.mpr_get_state(h)
        zs = mpr.mpr_predict(h)
        mpr.mpr_batch_fill(b, 40, 10, T=np.full(len(probs), 0.3))
        got, sw = mpr.mpr_batch_get_state(b, 0)
        zb = mpr.mpr_batch_predict(b, 0)
        assert sw == 50
        assert np.array_equal(got, single)
        assert np.array_equal(zb, zs)
        ib, ih = mpr.mpr_batch_get_info(b, 0), mpr.mpr_get_info(h)
        assert ib["site_updates"] == ih["site_updates"]
        assert abs(ib["e_bond_mean"] - ih["e_bond_mean"]) < 1e-12
    finally:
        mpr.mpr_batch_destroy(b)
        mpr.mpr_destroy(h)


@pytest.mark.parametrize("setup", ["SDS", "HDS"])
def test_batch_equals_tma_single_handle(mpr, setup):
    # Lattices wider than one tile run the single-handle sweeps through the TMA-fed persistent
    # kernel (2100 x 1300: 738 tiles, more than one tile per block on 152 SMs); the batch stages
    # with plain loads. Both apply the same per-site arithmetic, so problem 0's state, prediction
    # and mean energy agree bit for bit.
    probs = _problems([(2100, 1300, 0.9), (700, 45, 0.66), (64, 64, 0.33)], base=300)
    b = mpr.mpr_batch_create([p.z for p in probs], [p.mask for p in probs], setup, seed=21)
    h = mpr.mpr_create(probs[0].z, probs[0].mask)
    try:
        mpr.mpr_batch_fill(b, 12, 4, T=np.full(len(probs), 0.2))
        mpr.mpr_set_options(h, setup, seed=21)
        mpr.mpr_set_temperature(h, 0.2)
        mpr.mpr_run(h, 12, 4)
        single, _ = mpr.mpr_get_state(h)
        got, sw = mpr.mpr_batch_get_state(b, 0)
        assert sw == 16
        assert np.array_equal(got, single)
        assert np.array_equal(mpr.mpr_batch_predict(b, 0), mpr.mpr_predict(h))
        assert mpr.mpr_batch_get_info(b, 0)["e_bond_mean"] == mpr.mpr_get_info(h)["e_bond_mean"]
    finally:
        mpr.mpr_batch_destroy(b)
        mpr.mpr_destroy(h)


def test_batch_tuning_matches_single_handle(mpr):
    probs = _problems()
    b = mpr.mpr_batch_create([p.z for p in probs], [p.mask for p in probs], "SDS", seed=9)
    h = mpr.mpr_create(probs[0].z, probs[0].mask)
    try:
        kw = dict(n_eq=30, n_meas=10)
        mpr.mpr_batch_set_tuning(b, **kw)
        Tb, st = mpr.mpr_batch_fill(b, 20, 5)
        mpr.mpr_set_options(h, "SDS", seed=9)
        mpr.mpr_set_tuning(h, **kw)
        Th, sth = mpr.mpr_tune_temperature(h)
        mpr.mpr_run(h, 20, 5)
        assert st[0] == sth
        assert abs(Tb[0] / Th - 1.0) < 1e-12
        info = mpr.mpr_batch_get_info(b, 0)
        assert info["n_probes"] == mpr.mpr_get_info(h)["n_probes"]
        got, _ = mpr.mpr_batch_get_state(b, 0)
        single, _ = mpr.mpr_get_state(h)
        assert np.mean(got == single) > 0.999
        for i in range(len(probs)):
            inf = mpr.mpr_batch_get_info(b, i)
            assert 1e-3 <= Tb[i] <= 10.0 and inf["n_samples"] == 5 and np.isfinite(inf["e_bond_mean"])
    finally:
        mpr.mpr_batch_destroy(b)
        mpr.mpr_destroy(h)


def test_batch_launch_shape_and_graph_do_not_change_results(mpr):
    probs = _problems(base=100)
    states = []
    shapes = [(8, 128, 1, 0), (16, 128, 0, 2), (32, 128, 2, 1), (16, 128, 1, 0), (32, 128, 0, 2),
              (8, 128, 0, 2), (16, 64, 0, 2), (32, 64, 1, 0), (32, 64, 0, 2), (16, 64, 2, 1)]
    for rows, cols, bps, mode in shapes:
        b = mpr.mpr_batch_create([p.z for p in probs], [p.mask for p in probs], "HDS", seed=3,
                                 acc="kahan")
        try:
            mpr.mpr_batch_set_launch(b, rows, cols, bps, mode)
            mpr.mpr_batch_fill(b, 15, 5, T=np.linspace(0.1, 1.0, len(probs)))
            states.append([mpr.mpr_batch_get_state(b, i)[0] for i in range(len(probs))]
                          + [mpr.mpr_batch_predict(b, i) for i in range(len(probs))])
        finally:
            mpr.mpr_batch_destroy(b)
    for s in states[1:]:
        for a, c in zip(states[0], s):
            assert np.array_equal(a, c)


def test_batch_autotune_keeps_state(mpr):
    probs = _problems(base=200)
    b = mpr.mpr_batch_create([p.z for p in probs], [p.mask for p in probs], "SDS", seed=1)
    try:
        before = [mpr.mpr_batch_get_state(b, i) for i in range(len(probs))]
        rows, cols, bps, mode = mpr.mpr_batch_autotune(b, 5)
        assert (rows, cols) in ((8, 128), (16, 128), (32, 128), (16, 64), (32, 64))
        assert mode in (0, 2) and (bps >= 1 or mode == 2)
        after = [mpr.mpr_batch_get_state(b, i) for i in range(len(probs))]
        for (a, sa), (c, sc) in zip(before, after):
            assert np.array_equal(a, c) and sa == sc
        mpr.mpr_batch_fill(b, 5, 2, T=np.full(len(probs), 0.5))
        assert mpr.mpr_batch_get_info(b, 0)["sweep"] == 7
    finally:
        mpr.mpr_batch_destroy(b)


def test_batch_barrier_timeout_is_reported(mpr):
    probs = _problems()[:3]
    b = mpr.mpr_batch_create([p.z for p in probs], [p.mask for p in probs], "SDS")
    try:
        mpr.mpr_batch_set_launch(b, 16, 128, 0, 0)   # the persistent kernel is the one with barriers
        mpr.mpr_batch_inject_barrier_fault(b, 1, 0.05)
        with pytest.raises(mpr.MPRError) as e:
            mpr.mpr_batch_fill(b, 3, 1, T=np.full(3, 0.5))
        assert e.value.status == mpr.MPR_ERR_DEVICE_TIMEOUT
        with pytest.raises(mpr.MPRError) as e:
            mpr.mpr_batch_fill(b, 3, 1, T=np.full(3, 0.5))
        assert e.value.status == mpr.MPR_ERR_STATE
    finally:
        mpr.mpr_batch_destroy(b)
    # the context is still usable
    b = mpr.mpr_batch_create([p.z for p in probs], [p.mask for p in probs], "SDS")
    try:
        mpr.mpr_batch_fill(b, 3, 1, T=np.full(3, 0.5))
        assert mpr.mpr_batch_get_info(b, 2)["n_samples"] == 1
    finally:
        mpr.mpr_batch_destroy(b)


def test_batch_errors_name_the_problem(mpr):
    probs = _problems()[:3]
    zs = [p.z for p in probs]
    ms = [p.mask for p in probs]
    zs[1] = np.full_like(zs[1], 3.0)
    with pytest.raises(mpr.MPRError) as e:
        mpr.mpr_batch_create(zs, ms, "SDS")
    assert e.value.status == mpr.MPR_ERR_DEGENERATE and "problem 1" in str(e.value)
    with pytest.raises(mpr.MPRError) as e:
        mpr.mpr_batch_create([p.z for p in probs], ms, "SDD")
    assert e.value.status == mpr.MPR_ERR_INVALID_ARG


def test_fixed_point_sample_sums_equal_fp64_sums(mpr):
    # With FP16 spins and FP64 sums both paths add samples as exact int32 partials (units of
    # 2^-24): the single handle folds them into the FP64 sums every 16 samples and before a
    # prediction (a separate kernel), the batch after every 16th sample and the last sample of a
    # fill (each tile folds its own sites). Every add is exact, so predictions agree bit for bit
    # with those of FP64 sums -- across folds (40 samples in one fill: folds after 16, 32, 40),
    # with a prediction taken in between (after 21), and over two fills (21 + 19 samples).
    probs = _problems([(300, 200, 0.9), (64, 64, 0.33)], base=500)
    b = mpr.mpr_batch_create([p.z for p in probs], [p.mask for p in probs], "HDS", seed=13)
    b2 = mpr.mpr_batch_create([p.z for p in probs], [p.mask for p in probs], "HDS", seed=13)
    h = mpr.mpr_create(probs[0].z, probs[0].mask)
    try:
        mpr.mpr_batch_fill(b, 10, 40, T=np.full(len(probs), 0.25))
        mpr.mpr_batch_fill(b2, 10, 21, T=np.full(len(probs), 0.25))
        mpr.mpr_batch_fill(b2, 0, 19, T=np.full(len(probs), 0.25))
        mpr.mpr_set_options(h, "HDS", seed=13)
        mpr.mpr_set_temperature(h, 0.25)
        mpr.mpr_run(h, 10, 21)
        mid = mpr.mpr_predict(h)
        mpr.mpr_run(h, 0, 19)
        zh = mpr.mpr_predict(h)
        assert np.array_equal(zh, mpr.mpr_batch_predict(b, 0))
        assert np.array_equal(zh, mpr.mpr_batch_predict(b2, 0))
        for i in range(len(probs)):
            assert np.array_equal(mpr.mpr_batch_predict(b, i), mpr.mpr_batch_predict(b2, i))
        assert np.all(np.isfinite(mid))
        assert mpr.mpr_get_info(h)["n_samples"] == 40
        assert mpr.mpr_batch_get_info(b2, 0)["n_samples"] == 40
        # the mean bond energy is over the latest run (fill) that sampled, as a handle reports it
        assert mpr.mpr_batch_get_info(b2, 0)["e_bond_mean"] == mpr.mpr_get_info(h)["e_bond_mean"]
    finally:
        mpr.mpr_batch_destroy(b)
        mpr.mpr_batch_destroy(b2)
        mpr.mpr_destroy(h)
