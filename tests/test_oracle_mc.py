"""Pins of the oracle's Monte Carlo moves (Sec. 2: conditional hybrid algorithm on Eq. 2).

The hybrid chain must sample the conditional Gibbs measure exp(-H/T) of Eq. 2 with the measured
spins frozen. These tests check it against: exact properties of the over-relaxation move, the
planar-rotator reflection it reduces to at q = 1, brute-force quadrature of the Gibbs measure on
tiny lattices, the closed-form T -> infinity energies, and the T -> 0 ground state.
"""
import math

import numpy as np
import pytest

TWO_PI = 2.0 * math.pi


def _H(phi, Lx, Ly, q=0.5):
    """Eq. 2 with J = 1, open boundaries, written independently of the oracle (vectorised over
    leading axes): phi has shape (..., Ly, Lx)."""
    h = -np.cos(q * (phi[..., :, :-1] - phi[..., :, 1:])).sum(axis=(-1, -2))
    v = -np.cos(q * (phi[..., :-1, :] - phi[..., 1:, :])).sum(axis=(-1, -2))
    return h + v


# --- over-relaxation ---------------------------------------------------------------------------

def test_overrelax_conserves_energy_and_is_involution(orc):
    rng = np.random.default_rng(0)
    q = 0.5
    n_moved = 0
    for _ in range(20000):
        hx, hy = rng.normal(size=2) * 2.0
        f = rng.random() * TWO_PI
        g, _ = orc.overrelax(q, hx, hy, f)
        e0 = -(hx * math.cos(q * f) + hy * math.sin(q * f))
        e1 = -(hx * math.cos(q * g) + hy * math.sin(q * g))
        assert abs(e1 - e0) <= 1e-12
        assert 0.0 <= g <= TWO_PI
        back, _ = orc.overrelax(q, hx, hy, g)
        assert abs(back - f) <= 1e-12
        n_moved += g != f
    assert n_moved > 5000       # the reflection is admissible a good part of the time


def test_overrelax_q1_is_planar_rotator_reflection(orc):
    # Eq. 1 (q = 1): the textbook over-relaxation phi' = 2*theta - phi (mod 2*pi), theta = arg h
    rng = np.random.default_rng(1)
    for _ in range(5000):
        hx, hy = rng.normal(size=2)
        f = rng.random() * TWO_PI
        g, _ = orc.overrelax(1.0, hx, hy, f)
        ref = (2.0 * math.atan2(hy, hx) - f) % TWO_PI
        d = abs(g - ref)
        assert min(d, TWO_PI - d) < 1e-12


def test_overrelax_preserves_uniform_measure(orc):
    # a measure-preserving involution maps uniform angles to uniform angles
    from scipy import stats

    rng = np.random.default_rng(2)
    hx, hy = 1.3, -0.7
    f = rng.random(20000) * TWO_PI
    g = np.array([orc.overrelax(0.5, hx, hy, v)[0] for v in f])
    assert stats.kstest(g / TWO_PI, "uniform").pvalue > 1e-3


def test_overrelax_zero_field_keeps_angle(orc):
    assert orc.overrelax(0.5, 0.0, 0.0, 1.234)[0] == 1.234


# --- frozen sites ------------------------------------------------------------------------------

def test_frozen_sites_bit_exact(orc):
    rng = np.random.default_rng(4)
    Lx, Ly = 17, 13
    mask = (rng.random((Ly, Lx)) < 0.4).astype(np.uint8)
    phi = rng.random((Ly, Lx)) * TWO_PI
    o = orc.Oracle(Lx, Ly, seed=11)
    out, _, _ = o.run(phi, mask, 0.7, 0, 60)
    m = mask.astype(bool)
    assert np.array_equal(out[m].view(np.uint64), phi[m].view(np.uint64))
    assert np.all(out[~m] != phi[~m])


# --- brute-force Gibbs measure on tiny lattices -------------------------------------------------

def _exact_moments(Lx, Ly, frozen, T, n=48):
    """<e_b> and <phi_s> of the conditional Gibbs measure by tensor Gauss-Legendre quadrature
    over the free angles on [0, 2*pi]^k. frozen: dict site -> angle, every other site free."""
    free = [s for s in range(Lx * Ly) if s not in frozen]
    k = len(free)
    x, w = np.polynomial.legendre.leggauss(n)
    x = (x + 1.0) * math.pi
    w = w * math.pi
    grids = np.meshgrid(*([x] * k), indexing="ij")
    wts = np.ones_like(grids[0])
    for g in np.meshgrid(*([w] * k), indexing="ij"):
        wts = wts * g
    phi = np.zeros(grids[0].shape + (Ly * Lx,))
    for s, a in frozen.items():
        phi[..., s] = a
    for i, s in enumerate(free):
        phi[..., s] = grids[i]
    phi = phi.reshape(grids[0].shape + (Ly, Lx))
    H = _H(phi, Lx, Ly)
    nb = Lx * (Ly - 1) + Ly * (Lx - 1)
    b = np.exp(-(H - H.min()) / T) * wts
    Z = b.sum()
    e = float((b * H).sum() / Z / nb)
    means = {s: float((b * grids[i]).sum() / Z) for i, s in enumerate(free)}
    return e, means


def _mc_moments(orc, Lx, Ly, frozen, T, chains=16, equil=500, nsweeps=12000, width=0.0, ubits=32):
    mask = np.zeros((Ly, Lx), np.uint8)
    phi = np.zeros((Ly, Lx))
    for s, a in frozen.items():
        mask.flat[s] = 1
        phi.flat[s] = a
    es, ms = [], []
    for c in range(chains):
        o = orc.Oracle(Lx, Ly, seed=1000 + c, width=width, ubits=ubits)
        p = o.init(phi, mask)
        p, _, _ = o.run(p, mask, T, 0, equil)
        p, acc, e = o.run(p, mask, T, equil, nsweeps, acc=np.zeros_like(p), energies=True)
        es.append(e.mean())
        ms.append(acc / nsweeps)
    es = np.array(es)
    ms = np.array(ms)
    return es.mean(), es.std(ddof=1) / math.sqrt(chains), ms.mean(0), ms.std(0, ddof=1) / math.sqrt(chains)


CASES = [
    # (Lx, Ly, frozen {site: angle}, T)
    (3, 3, {0: 0.3, 1: 2.0, 2: 4.0, 3: 5.5, 5: 1.0, 6: 3.0, 7: 6.0, 8: 0.1}, 0.4),   # one free site
    (3, 3, {0: 0.3, 1: 2.0, 2: 4.0, 3: 5.5, 5: 1.0, 6: 3.0, 7: 6.0, 8: 0.1}, 3.0),
    (2, 2, {0: 1.0, 3: 4.0}, 0.5),                                                   # two free
    (2, 2, {0: 5.0}, 0.8),                                                           # three free
    (3, 3, {0: 0.5, 2: 5.0, 4: 3.0, 6: 1.5, 8: 6.0, 1: 2.5}, 0.6),                   # three free
]


# ubits = 23: the FP32 setting's 23-bit uniforms, three Philox calls per group of eight sites
# (on 3 x 3 lattices both rows of a group occur, so both the first-row and the byte-assembled
# second-row acceptance uniforms drive the chain)
@pytest.mark.parametrize("ubits", [32, 23])
@pytest.mark.parametrize("Lx,Ly,frozen,T", CASES)
def test_mc_matches_brute_force_gibbs(orc, Lx, Ly, frozen, T, ubits):
    e_ex, m_ex = _exact_moments(Lx, Ly, frozen, T)
    e_ex2, _ = _exact_moments(Lx, Ly, frozen, T, n=64 if len(frozen) < Lx * Ly - 1 else 128)
    assert abs(e_ex - e_ex2) < 1e-9           # quadrature converged
    e_mc, e_se, m_mc, m_se = _mc_moments(orc, Lx, Ly, frozen, T, ubits=ubits)
    assert abs(e_mc - e_ex) < 4.5 * e_se + 1e-4, (e_mc, e_ex, e_se)
    for s, v in m_ex.items():
        y, x = divmod(s, Lx)
        assert abs(m_mc[y, x] - v) < 4.5 * m_se[y, x] + 1e-3, (s, m_mc[y, x], v, m_se[y, x])


# --- T -> infinity and T -> 0 limits ----------------------------------------------------------

def test_high_temperature_closed_form(orc):
    # At T -> inf every prediction angle is uniform on [0, 2*pi] and independent:
    #   pred-pred bond  E cos((a-b)/2) = (E sin(a/2))^2 = (2/pi)^2,
    #   pred-frozen bond with frozen angle a: (2/pi) sin(a/2), frozen-frozen bond: fixed.
    rng = np.random.default_rng(7)
    Lx, Ly = 10, 8
    mask = (rng.random((Ly, Lx)) < 0.5).astype(np.uint8)
    phi = np.where(mask == 1, rng.random((Ly, Lx)) * TWO_PI, 0.0)
    s = 0.0
    nb = 0
    for y in range(Ly):
        for x in range(Lx):
            for yy, xx in ((y, x + 1), (y + 1, x)):
                if yy >= Ly or xx >= Lx:
                    continue
                nb += 1
                a, b = mask[y, x], mask[yy, xx]
                if a and b:
                    s += math.cos(0.5 * (phi[y, x] - phi[yy, xx]))
                elif a:
                    s += (2 / math.pi) * math.sin(0.5 * phi[y, x])
                elif b:
                    s += (2 / math.pi) * math.sin(0.5 * phi[yy, xx])
                else:
                    s += 4 / math.pi**2
    e_inf = -s / nb
    o = orc.Oracle(Lx, Ly, seed=3)
    p = o.init(phi, mask)
    _, _, e = o.run(p, mask, 1e8, 0, 40000, energies=True)
    se = e.std() / math.sqrt(e.size)
    assert abs(e.mean() - e_inf) < 4 * se, (e.mean(), e_inf, se)
    # unconditional limit -4/pi^2
    o2 = orc.Oracle(12, 12, seed=4)
    m0 = np.zeros((12, 12), np.uint8)
    p2 = o2.init(np.zeros((12, 12)), m0)
    _, _, e2 = o2.run(p2, m0, 1e8, 0, 20000, energies=True)
    assert abs(e2.mean() + 4 / math.pi**2) < 4 * e2.std() / math.sqrt(e2.size)


def _anneal(orc, o, phi, mask, T_end, stages=40, per=400):
    sweep = 0
    for T in np.geomspace(1.0, T_end, stages):
        phi, _, _ = o.run(phi, mask, float(T), sweep, per)
        sweep += per
    return phi, sweep


def test_low_temperature_chain_is_linear_interpolation(orc):
    # T -> 0: a 1 x n chain with frozen ends a, b minimises H with equal steps
    Lx, Ly = 10, 1
    a, b = 0.5, 5.0
    mask = np.zeros((1, Lx), np.uint8)
    mask[0, 0] = mask[0, -1] = 1
    phi = np.zeros((1, Lx))
    phi[0, 0], phi[0, -1] = a, b
    o = orc.Oracle(Lx, Ly, seed=21)
    phi = o.init(phi, mask)
    T = 1e-4
    phi, sweep = _anneal(orc, o, phi, mask, T)
    _, acc, _ = o.run(phi, mask, T, sweep, 4000, acc=np.zeros_like(phi))
    mean = acc[0] / 4000
    lin = a + (b - a) * np.arange(Lx) / (Lx - 1)
    assert np.max(np.abs(mean[1:-1] - lin[1:-1])) < 0.01, mean - lin


def test_low_temperature_unconditional_energy(orc):
    # T -> 0 without frozen sites: all angles align and e_b -> -1
    o = orc.Oracle(8, 8, seed=5)
    m0 = np.zeros((8, 8), np.uint8)
    p = o.init(np.zeros((8, 8)), m0)
    p, sweep = _anneal(orc, o, p, m0, 1e-4, stages=40, per=300)
    _, _, e = o.run(p, m0, 1e-4, sweep, 200, energies=True)
    assert e.mean() < -1.0 + 2e-3


# --- temperature dependence and tuning ---------------------------------------------------------

def test_bond_energy_increases_with_temperature(orc):
    import mpr_inputs

    pr = mpr_inputs.make_problem(24, 24, 0.5, field_seed=1, mask_seed=2)
    o = orc.Oracle(24, 24, seed=8)
    phi, _, _ = o.map(pr.z, pr.mask)
    phi = o.init(phi, pr.mask)
    es = []
    sweep = 0
    for T in (0.02, 0.1, 0.5, 2.5, 12.5):
        phi, _, _ = o.run(phi, pr.mask, T, sweep, 300)
        phi, _, e = o.run(phi, pr.mask, T, sweep + 300, 300, energies=True)
        sweep += 600
        es.append(e.mean())
    assert all(b > a for a, b in zip(es, es[1:])), es


def test_tuning_recovers_temperature(orc):
    # Draw an equilibrium configuration of Eq. 2 at T0 with no frozen site, keep half of it as
    # measured data, and tune: the equilibrium bond energy at the tuned T must match the sample's
    # and T must come back close to T0.
    T0 = 0.35
    L = 64
    o = orc.Oracle(L, L, seed=31)
    m0 = np.zeros((L, L), np.uint8)
    p = o.init(np.zeros((L, L)), m0)
    p, sweep = _anneal(orc, o, p, m0, T0, stages=10, per=200)
    p, _, _ = o.run(p, m0, T0, sweep, 1000)
    import mpr_inputs

    mask = mpr_inputs.removal_mask(L, L, 0.5, seed=9)
    o2 = orc.Oracle(L, L, seed=77)
    e_s, _ = o2.energy_sample(p, mask)
    start = o2.init(np.where(mask == 1, p, 0.0), mask)
    st, T, _, _, trace = o2.tune(start, mask, e_s, 0, n_eq=150, n_meas=50)
    assert st == 0
    assert abs(T / T0 - 1.0) < 0.25, (T, trace)
    # monotone bracket: the probe energies straddle e_s around the returned T
    Ts = np.array([t for t, _ in trace])
    Es = np.array([e for _, e in trace])
    assert np.all(Es[Ts < 0.5 * T] < e_s) and np.all(Es[Ts > 2.0 * T] > e_s)


def test_tuning_edge_cases(orc):
    # a sample energy below what T_lo reaches returns T_lo; above T_hi's returns "no convergence"
    import mpr_inputs

    pr = mpr_inputs.make_problem(16, 16, 0.5, field_seed=5, mask_seed=6)
    o = orc.Oracle(16, 16, seed=2)
    phi, _, _ = o.map(pr.z, pr.mask)
    phi = o.init(phi, pr.mask)
    st, T, _, sw, tr = o.tune(phi, pr.mask, -1.5, 0, n_eq=20, n_meas=10)
    assert st == 0 and T == 1e-3 and len(tr) == 1 and sw == 30
    st, T, _, sw, tr = o.tune(phi, pr.mask, 0.5, 0, n_eq=20, n_meas=10)
    assert st == 4 and T == 10.0 and len(tr) == 2 and sw == 60


# --- energy-slope equilibration ----------------------------------------------------------------

def _relaxing_problem(orc):
    import mpr_inputs

    pr = mpr_inputs.make_problem(32, 32, 0.66, field_seed=3, mask_seed=4)
    o = orc.Oracle(32, 32, seed=12)
    phi, _, _ = o.map(pr.z, pr.mask)
    return pr, o, o.init(phi, pr.mask)   # a hot (uniform random) start


def test_equilibrate_control_flow(orc):
    pr, o, phi = _relaxing_problem(orc)
    # an infinite tolerance accepts the first comparison: exactly two chunks
    _, n, sw = o.equilibrate(phi, pr.mask, 0.1, 0, 25, 10000, z=math.inf)
    assert n == 50 and sw == 50
    # a zero tolerance never accepts (the chunk means of a continuous chain never tie): the cap
    _, n, sw = o.equilibrate(phi, pr.mask, 0.1, 7, 25, 260, z=0.0)
    assert n == 250 and sw == 257
    # one chunk fits below the cap: nothing to compare, one chunk run; chunks below 2 run nothing
    _, n, _ = o.equilibrate(phi, pr.mask, 0.1, 0, 25, 49)
    assert n == 25
    _, n, _ = o.equilibrate(phi, pr.mask, 0.1, 0, 1, 100)
    assert n == 0
    # the sweeps are the chain's ordinary sweeps: same state as a plain run of that length
    p_eq, n, _ = o.equilibrate(phi, pr.mask, 0.1, 0, 25, 10000, z=math.inf)
    p_run, _, _ = o.run(phi, pr.mask, 0.1, 0, n)
    assert np.array_equal(p_eq, p_run)


def test_equilibrate_stops_when_the_energy_has_relaxed(orc):
    # From a hot start at low T the bond energy falls over the first tens of sweeps: the rule must
    # not stop during the fall, and where it stops the energy must already sit at its long-run
    # level.
    pr, o, phi = _relaxing_problem(orc)
    T, chunk = 0.05, 10
    p_eq, n, sw = o.equilibrate(phi, pr.mask, T, 0, chunk, 20000)
    assert 2 * chunk < n < 20000
    _, _, e_before = o.run(phi, pr.mask, T, 0, n, energies=True)
    _, _, e_after = o.run(p_eq, pr.mask, T, sw, 2000, energies=True)
    drop = e_before[:chunk].mean() - e_after.mean()
    assert drop > 0.05   # the relaxation was real: the first chunk lies far above the long run
    assert abs(e_before[-chunk:].mean() - e_after.mean()) < 0.1 * drop


# --- bounded Metropolis proposals with an adapted width ----------------------------------------

@pytest.mark.parametrize("case", [0, 2, 3])
@pytest.mark.parametrize("width", [0.4, 2.5])
def test_bounded_proposal_samples_the_same_gibbs_measure(orc, case, width):
    # A symmetric proposal on the segment of half-width w around the angle, rejected outside
    # [0, 2 pi): the chain must sample the same conditional Gibbs measure as with the uniform one.
    Lx, Ly, frozen, T = CASES[case]
    e_ex, m_ex = _exact_moments(Lx, Ly, frozen, T)
    e_mc, e_se, m_mc, m_se = _mc_moments(orc, Lx, Ly, frozen, T, width=width)
    assert abs(e_mc - e_ex) < 4.5 * e_se + 1e-4, (e_mc, e_ex, e_se)
    for s, v in m_ex.items():
        y, x = divmod(s, Lx)
        assert abs(m_mc[y, x] - v) < 4.5 * m_se[y, x] + 1e-3, (s, m_mc[y, x], v, m_se[y, x])


def test_width_adaptation_reaches_target_acceptance(orc):
    import mpr_inputs

    pr = mpr_inputs.make_problem(48, 48, 0.66, field_seed=7, mask_seed=8)
    T, target = 0.05, 0.5
    o = orc.Oracle(48, 48, seed=4, width=2.0 * math.pi)
    phi, _, _ = o.map(pr.z, pr.mask)
    phi = o.init(phi, pr.mask)
    n_pred = int((pr.mask == 0).sum())
    # the uniform-like start accepts few proposals at this temperature
    a0 = o.accepted(phi, pr.mask, T, 0) / n_pred
    phi, widths = o.run_adapt(phi, pr.mask, T, 0, 400, target)
    assert widths[0] == 2.0 * math.pi and widths[-1] < 0.5 * widths[0]
    # widths follow the rule: w_{k+1} = w_k exp(a_k - target), within [1e-3, 2 pi]
    assert np.all((widths > 1e-3 - 1e-15) & (widths <= 2.0 * math.pi))
    # with the adapted width held fixed, the acceptance sits near the target
    acc = [o.accepted(phi, pr.mask, T, 400 + k) / n_pred for k in range(20)]
    assert a0 < 0.3 and abs(np.mean(acc) - target) < 0.1, (a0, np.mean(acc), o.cfg.width)


def _gauss_seidel_ground_state(phi, mask, q=0.5, sweeps=20000, tol=1e-13):
    # Independent FP64 minimiser of Eq. 2: each free angle in turn moves to the exact minimiser of
    # its site energy -|h| cos(q phi - theta) over phi in [0, 2 pi] (q phi = theta when that lies
    # in [0, 2 pi q], else the nearer end of the segment in angle), until nothing moves.
    phi = phi.copy()
    Ly, Lx = phi.shape
    free = [(y, x) for y in range(Ly) for x in range(Lx) if mask[y, x] == 0]
    for _ in range(sweeps):
        moved = 0.0
        for y, x in free:
            hx = hy = 0.0
            for yy, xx in ((y, x - 1), (y, x + 1), (y - 1, x), (y + 1, x)):
                if 0 <= yy < Ly and 0 <= xx < Lx:
                    hx += math.cos(q * phi[yy, xx])
                    hy += math.sin(q * phi[yy, xx])
            th = math.atan2(hy, hx) % (2.0 * math.pi)
            if th <= 2.0 * math.pi * q:
                new = th / q
            else:
                # distance in angle from theta to the two ends 0 and 2 pi q of the segment
                d0 = min(th, 2.0 * math.pi - th)
                d1 = abs(th - 2.0 * math.pi * q)
                new = 0.0 if d0 < d1 else 2.0 * math.pi
            moved = max(moved, abs(new - phi[y, x]))
            phi[y, x] = new
        if moved < tol:
            break
    return phi


def _energy_eq2(phi, q=0.5):
    return -(np.cos(q * (phi[:, 1:] - phi[:, :-1])).sum() + np.cos(q * (phi[1:, :] - phi[:-1, :])).sum())


def test_low_temperature_2d_matches_gauss_seidel_minimiser(orc):
    # T -> 0 on a 2-D conditional lattice: the annealed chain's mean configuration is the ground
    # state an independent coordinate-wise minimiser finds (Sec. 2, Eq. 2 at vanishing T)
    import mpr_inputs

    pr = mpr_inputs.make_problem(12, 12, 0.5, field_seed=31, mask_seed=32)
    o = orc.Oracle(12, 12, seed=33)
    phi, _, _ = o.map(pr.z, pr.mask)
    phi = o.init(phi, pr.mask)
    T = 1e-4
    phi, sweep = _anneal(orc, o, phi, pr.mask, T, stages=30, per=300)
    n = 2000
    _, acc, _ = o.run(phi, pr.mask, T, sweep, n, acc=np.zeros_like(phi))
    mean = np.where(pr.mask == 1, phi, acc / n)
    start = np.where(pr.mask == 1, phi, math.pi)
    gs = _gauss_seidel_ground_state(start, pr.mask)
    gs_from_mean = _gauss_seidel_ground_state(mean, pr.mask)
    # the chain's mean sits at a minimum (the minimiser barely moves it) ...
    assert np.max(np.abs(gs_from_mean - mean)) < 0.02
    # ... and no higher than the one the minimiser reaches from its own start
    assert _energy_eq2(gs_from_mean) <= _energy_eq2(gs) + 1e-9
    assert np.max(np.abs(gs_from_mean - gs)) < 1e-6 or _energy_eq2(gs_from_mean) < _energy_eq2(gs) - 1e-9
