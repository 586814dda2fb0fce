"""Pins of the alternative temperature tunings (readings: Sec. 2 says only that the reduced
temperature is inferred from the incomplete data): heating from T_lo until the bond energy
crosses the sample's, the energy curve of the unconditional lattice, and its inversion.

The curve is pinned by two limits of Eq. 2 that the oracle does not encode: equipartition at low T
(harmonic bonds -cos(q d) ~ -1 + q^2 d^2 / 2 give each of the N - 1 non-uniform modes T/2, so
e_b ~ -1 + (N - 1) T / (2 N_b)) and the infinite-temperature mean -4/pi^2.
"""
import math

import numpy as np
import pytest

import mpr_inputs


def test_energy_curve_low_temperature_equipartition(orc):
    L = 16
    N, Nb = L * L, 2 * L * (L - 1)
    o = orc.Oracle(L, L, seed=3)
    Ts = [1.0, 0.5, 0.3, 0.2, 0.1, 0.05, 0.03, 0.02, 0.01]   # cooling: each T starts equilibrated
    e = o.energy_curve(Ts, n_eq=1000, n_meas=2000)
    slope = (e[-1] + 1.0) / Ts[-1]
    assert abs(slope / ((N - 1) / (2.0 * Nb)) - 1.0) < 0.03, slope
    assert np.all(np.diff(e) < 0)   # e_b increases with T (read in cooling order: decreases)


def test_energy_curve_infinite_temperature(orc):
    o = orc.Oracle(24, 24, seed=4)
    e = o.energy_curve([1e4], n_eq=50, n_meas=400)
    # per-sweep fluctuation of e_b at T = inf: var(cos(q d)) = 1/2 - 16/pi^4 per bond, bonds nearly
    # independent; 400 sweeps of 1104 bonds, each sweep a fresh uniform draw
    se = math.sqrt((0.5 - 16 / math.pi**4) / (2 * 24 * 23) / 400)
    assert abs(e[0] + 4 / math.pi**2) < 5 * se, (e[0], se)


def test_invert_curve(orc):
    T = np.array([0.01, 0.1, 1.0, 10.0])
    e = np.array([-0.99, -0.9, -0.6, -0.45])
    for Ti, ei in zip(T, e):                     # exact at the nodes
        st, t = orc.invert_curve(T, e, ei)
        assert st == 0 and abs(t / Ti - 1) < 1e-14
    st, t = orc.invert_curve(T, e, -0.75)        # linear in log T: halfway in e -> geometric mean
    assert st == 0 and abs(t - math.sqrt(0.1 * 1.0)) < 1e-14
    assert orc.invert_curve(T, e, -1.5) == (0, 0.01)
    assert orc.invert_curve(T, e, -0.1) == (4, 10.0)
    # a non-monotone (noisy) curve: the first crossing counts
    st, t = orc.invert_curve(T, np.array([-0.99, -0.7, -0.8, -0.45]), -0.75)
    assert st == 0 and 0.01 < t < 0.1


def _equilibrium_sample(orc, L, T0, seed):
    o = orc.Oracle(L, L, seed=seed)
    m0 = np.zeros((L, L), np.uint8)
    p = o.init(np.zeros((L, L)), m0)
    sweep = 0
    for T in np.geomspace(1.0, T0, 10):
        p, _, _ = o.run(p, m0, float(T), sweep, 200)
        sweep += 200
    p, _, _ = o.run(p, m0, T0, sweep, 1000)
    return p


def test_heating_recovers_temperature_like_bisection(orc):
    # an equilibrium configuration of Eq. 2 at T0, half of it kept as data: heating finds the same
    # temperature as bisection (both solve e_b(T) = e_s), close to T0
    T0, L = 0.35, 64
    p = _equilibrium_sample(orc, L, T0, 31)
    mask = mpr_inputs.removal_mask(L, L, 0.5, seed=9)
    o = orc.Oracle(L, L, seed=77)
    e_s, _ = o.energy_sample(p, mask)
    start = o.init(np.where(mask == 1, p, 0.0), mask)
    st_h, T_h, _, _, tr_h = o.tune_heating(start, mask, e_s, 0, factor=2.0, n_eq=150, n_meas=50)
    st_b, T_b, _, _, _ = o.tune(start, mask, e_s, 0, n_eq=150, n_meas=50)
    assert st_h == 0 and st_b == 0
    assert abs(T_h / T0 - 1.0) < 0.25 and abs(T_h / T_b - 1.0) < 0.1, (T_h, T_b)
    # the heating phase multiplies T by the factor until the energy passes e_s; the refinement
    # probes lie inside the last bracket
    Ts = np.array([t for t, _ in tr_h])
    Es = np.array([e for _, e in tr_h])
    k = int(np.argmax(Es > e_s))                 # first probe above e_s ends the heating
    assert k >= 1 and np.allclose(Ts[1:k + 1] / Ts[:k], 2.0)
    assert np.all(Es[:k] < e_s)
    assert np.all((Ts[k + 1:] > Ts[k - 1]) & (Ts[k + 1:] < Ts[k]))


def test_curve_inversion_recovers_temperature(orc):
    # unconditional model: the energy of an equilibrium sample at T0 inverted through the model's
    # own curve gives back T0
    T0, L = 0.3, 48
    p = _equilibrium_sample(orc, L, T0, 41)
    o = orc.Oracle(L, L, seed=5)
    e_s = o.energy_bond(p)
    Ts = np.geomspace(0.05, 2.0, 14)
    e = o.energy_curve(Ts, n_eq=300, n_meas=300)
    st, T = orc.invert_curve(Ts, e, e_s)
    assert st == 0 and abs(T / T0 - 1.0) < 0.1, (T, e_s, e)


def test_heating_edge_cases(orc):
    pr = mpr_inputs.make_problem(16, 16, 0.5, field_seed=5, mask_seed=6)
    o = orc.Oracle(16, 16, seed=2)
    phi, _, _ = o.map(pr.z, pr.mask)
    phi = o.init(phi, pr.mask)
    # below what T_lo reaches: T_lo after one probe
    st, T, _, sw, tr = o.tune_heating(phi, pr.mask, -1.5, 0, n_eq=20, n_meas=10)
    assert st == 0 and T == 1e-3 and len(tr) == 1 and sw == 30
    # above what T_hi reaches: every heating step up to T_hi (clamped), then "no convergence"
    st, T, _, sw, tr = o.tune_heating(phi, pr.mask, 0.5, 0, factor=10.0, n_eq=20, n_meas=10)
    assert st == 4 and T == 10.0
    assert [t for t, _ in tr] == pytest.approx([1e-3, 1e-2, 1e-1, 1.0, 10.0])
    assert sw == 30 * len(tr)
    # the probe budget ends the heating too
    st, T, _, _, tr = o.tune_heating(phi, pr.mask, 0.5, 0, factor=1.1, n_eq=5, n_meas=5,
                                     max_probes=6)
    assert st == 4 and len(tr) == 6 and T == pytest.approx(1e-3 * 1.1**5)
