"""Statistical parity over seeds (Sec. 3: AAE of Eq. 4 over prediction sites, mean over samples).

Config 1 of the workload: 64 x 64 Gaussian fields (m = 50, sigma = 10, exponential covariance,
kappa = 0.2), 33 % removed, temperature tuning, 1000 equilibration and 100 sampling sweeps; 10
seeds. The FP64 oracle runs the same jobs. For every precision setup the seed-averaged MAE, RMSE
and equilibrium bond energy must lie within 1 % of the oracle's.

The larger configs compare reduced precision against the GPU FP64 (DDD) path on the same
problems and Monte Carlo seeds (the oracle would take hours there): config 2 (1024 x 1024, 66 %
removed, tuning + 2000 + 200, SDS) and config 3 (4096 x 4096, 90 % removed, the bench's job:
tuning + 2000 + 200; HDS, BDS, HDS with Kahan sums) over 10 seeds each, config 5 (16384 x 16384,
SDS, 500 + 100 sweeps at one tuned temperature) on one. Every measured gap is printed at the end
of the session (and written to $MPR_GAPS_JSON when set).
"""
import numpy as np
import pytest

import mpr_inputs

pytestmark = pytest.mark.gpu

SEEDS = range(10)


@pytest.fixture(scope="module")
def mpr():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1910_08448_gb300 as m

    m.load()
    return m


def _metrics(zhat, pr):
    pred = pr.mask == 0
    err = (zhat - pr.z)[pred]
    return float(np.mean(np.abs(err))), float(np.sqrt(np.mean(err ** 2)))


def _gpu_job(mpr, pr, setup, seed, equil, samples, acc="f64", T=None):
    h = mpr.mpr_create(pr.z, pr.mask)
    try:
        mpr.mpr_set_options(h, setup, seed=seed, acc=acc)
        if T is None:
            T, _ = mpr.mpr_tune_temperature(h)
        else:
            mpr.mpr_set_temperature(h, T)
        mpr.mpr_run(h, equil, samples)
        zhat = mpr.mpr_predict(h)
        info = mpr.mpr_get_info(h)
    finally:
        mpr.mpr_destroy(h)
    return zhat, info["e_bond_mean"], T


@pytest.fixture(scope="module")
def oracle_config1(orc):
    out = []
    for s in SEEDS:
        pr = mpr_inputs.make_problem(64, 64, 0.33, field_seed=s, mask_seed=100 + s)
        o = orc.Oracle(64, 64, seed=s)
        r = o.gap_fill(pr.z, pr.mask, 1000, 100)
        mae, rmse = _metrics(r["zhat"], pr)
        out.append((pr, mae, rmse, float(np.mean(r["e_samples"])), r["T"]))
    return out


@pytest.mark.parametrize("setup,acc", [("DDD", "f64"), ("SDS", "f64"), ("SSS", "f64"),
                                       ("HDS", "f64"), ("BDS", "f64"), ("SDS", "kahan"),
                                       ("HSS", "kahan"), ("HDH", "f64")])
def test_config1_within_one_percent_of_oracle(mpr, orc, oracle_config1, gap_log, setup, acc):
    g_mae, g_rmse, g_e, o_mae, o_rmse, o_e = [], [], [], [], [], []
    for s, (pr, mae, rmse, e, T) in zip(SEEDS, oracle_config1):
        zhat, eb, Tg = _gpu_job(mpr, pr, setup, s, 1000, 100, acc)
        m, r = _metrics(zhat, pr)
        g_mae.append(m), g_rmse.append(r), g_e.append(eb)
        o_mae.append(mae), o_rmse.append(rmse), o_e.append(e)
    gaps = {k: np.mean(a) / np.mean(b) - 1.0
            for k, a, b in (("mae", g_mae, o_mae), ("rmse", g_rmse, o_rmse), ("e_bond", g_e, o_e))}
    for k, v in gaps.items():
        gap_log(f"config 1 {setup}/{acc} vs oracle, 10 seeds", k, v, 0.01)
    for k, v in gaps.items():
        assert abs(v) < 0.01, (k, v)


def _dev_problem(L, p, field_seed, mask_seed):
    import torch

    return mpr_inputs.make_problem(L, L, p, field_seed=field_seed, mask_seed=mask_seed,
                                   periodic=L > 4096, device=torch.device("cuda", 0))


def _seed_gaps(rows):
    """Relative gaps of seed-averaged MAE, RMSE and e_b: rows of (mae, rmse, e_b, mae_ref,
    rmse_ref, e_b_ref)."""
    a = np.array(rows)
    return {"mae": a[:, 0].mean() / a[:, 3].mean() - 1.0,
            "rmse": a[:, 1].mean() / a[:, 4].mean() - 1.0,
            "e_bond": a[:, 2].mean() / a[:, 5].mean() - 1.0}


def test_config2_fp32_vs_fp64_gpu_ten_seeds(mpr, gap_log):
    # Config 2: 1024 x 1024, 66 % removed, tuning + 2000 + 200 sweeps, 10 seeds; FP32 intrinsics
    # with FP64 energy (SDS) against the FP64 path (DDD) on the same problems and Monte Carlo seeds
    rows = []
    for s in SEEDS:
        pr = _dev_problem(1024, 0.66, 10 + s, 20 + s)
        zd, ed, _ = _gpu_job(mpr, pr, "DDD", s, 2000, 200)
        zs, es, _ = _gpu_job(mpr, pr, "SDS", s, 2000, 200)
        rows.append((*_metrics(zs, pr), es, *_metrics(zd, pr), ed))
    g = _seed_gaps(rows)
    for k, v in g.items():
        gap_log("config 2 SDS vs DDD, 10 seeds", k, v, 0.01)
    assert all(abs(v) < 0.01 for v in g.values()), g


@pytest.fixture(scope="module")
def config3_fp64(mpr):
    # Config 3 as bench.py runs it: 4096 x 4096, 90 % removed, tuning + 2000 + 200 sweeps; the
    # FP64 (DDD) job of every seed, shared by the 16-bit setups below
    out = []
    for s in SEEDS:
        pr = _dev_problem(4096, 0.9, 1 + s, 101 + s)
        zd, ed, Td = _gpu_job(mpr, pr, "DDD", 7 + s, 2000, 200)
        out.append((pr, *_metrics(zd, pr), ed))
    return out


@pytest.mark.parametrize("setup,acc", [("HDS", "f64"), ("BDS", "f64"), ("HDS", "kahan"),
                                       ("HDH", "f64")])
def test_config3_16bit_storage_vs_fp64_gpu_ten_seeds(mpr, config3_fp64, gap_log, setup, acc):
    rows = []
    for s, (pr, md, rd, ed) in zip(SEEDS, config3_fp64):
        zh, eh, _ = _gpu_job(mpr, pr, setup, 7 + s, 2000, 200, acc=acc)
        rows.append((*_metrics(zh, pr), eh, md, rd, ed))
    g = _seed_gaps(rows)
    for k, v in g.items():
        gap_log(f"config 3 {setup}/{acc} vs DDD, 10 seeds", k, v, 0.01)
    assert all(abs(v) < 0.01 for v in g.values()), g


def test_config5_fp32_vs_fp64_gpu_16384(mpr, gap_log):
    # Config 5: 16384 x 16384, 90 % removed; one tuning (SDS), then SDS and DDD jobs of
    # 500 + 100 sweeps at that temperature, same Monte Carlo seed
    pr = _dev_problem(16384, 0.9, 1, 101)
    h = mpr.mpr_create(pr.z, pr.mask)
    try:
        mpr.mpr_set_options(h, "SDS", seed=7)
        T, _ = mpr.mpr_tune_temperature(h)
    finally:
        mpr.mpr_destroy(h)
    zd, ed, _ = _gpu_job(mpr, pr, "DDD", 7, 500, 100, T=T)
    zs, es, _ = _gpu_job(mpr, pr, "SDS", 7, 500, 100, T=T)
    g = _seed_gaps([(*_metrics(zs, pr), es, *_metrics(zd, pr), ed)])
    for k, v in g.items():
        gap_log("config 5 SDS vs DDD (16384^2)", k, v, 0.01)
    assert all(abs(v) < 0.01 for v in g.values()), g


def _job_from(mpr, pr, setup, seed, T, equil, samples, start=None, proposal=None):
    h = mpr.mpr_create(pr.z, pr.mask)
    try:
        mpr.mpr_set_options(h, setup, seed=seed)
        if start is not None:
            mpr.mpr_set_state(h, start, 0)
        if proposal is not None:
            mpr.mpr_set_proposal(h, *proposal)
        mpr.mpr_set_temperature(h, T)
        mpr.mpr_run(h, equil, samples)
        zhat = mpr.mpr_predict(h)
        info = mpr.mpr_get_info(h)
    finally:
        mpr.mpr_destroy(h)
    return zhat, info["e_bond_mean"]


def _tuned_T(mpr, pr, setup, seed):
    h = mpr.mpr_create(pr.z, pr.mask)
    try:
        mpr.mpr_set_options(h, setup, seed=seed)
        T, _ = mpr.mpr_tune_temperature(h)
    finally:
        mpr.mpr_destroy(h)
    return T


def test_equilibrium_does_not_depend_on_the_start(mpr):
    # Sec. 2 averages equilibrium configurations: a hot start (uniform angles) and a cold start
    # (every prediction site at the mean measured angle) give the same predictions and energy
    gaps = []
    for s in range(3):
        pr = mpr_inputs.make_problem(256, 256, 0.66, field_seed=40 + s, mask_seed=50 + s)
        T = _tuned_T(mpr, pr, "SDS", s)
        h = mpr.mpr_create(pr.z, pr.mask)
        try:
            hot, _ = mpr.mpr_get_state(h)
        finally:
            mpr.mpr_destroy(h)
        cold = np.where(pr.mask == 1, hot, hot[pr.mask == 1].mean())
        zh, eh = _job_from(mpr, pr, "SDS", s, T, 2000, 200)
        zc, ec = _job_from(mpr, pr, "SDS", s, T, 2000, 200, start=cold)
        gaps.append((_metrics(zc, pr)[0] / _metrics(zh, pr)[0] - 1.0, ec / eh - 1.0))
    g = np.mean(np.array(gaps), axis=0)
    print(f"\ncold vs hot start: MAE gap {g[0]:.2e}, e_bond gap {g[1]:.2e}")
    assert abs(g[0]) < 0.01 and abs(g[1]) < 0.01


@pytest.mark.parametrize("setup", ["SDS", "HDS"])
def test_bounded_proposals_give_the_same_predictions(mpr, setup):
    # the adapted-width proposal samples the same conditional measure as the uniform one
    gaps = []
    for s in range(3):
        pr = mpr_inputs.make_problem(256, 256, 0.9, field_seed=60 + s, mask_seed=70 + s)
        T = _tuned_T(mpr, pr, setup, s)
        zu, eu = _job_from(mpr, pr, setup, s, T, 1500, 200)
        zb, eb = _job_from(mpr, pr, setup, s, T, 1500, 200, proposal=(2.0 * np.pi, 0.4))
        gaps.append((_metrics(zb, pr)[0] / _metrics(zu, pr)[0] - 1.0, eb / eu - 1.0))
    g = np.mean(np.array(gaps), axis=0)
    print(f"\n{setup} bounded vs uniform proposals: MAE gap {g[0]:.2e}, e_bond gap {g[1]:.2e}")
    assert abs(g[0]) < 0.01 and abs(g[1]) < 0.01
