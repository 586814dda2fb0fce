"""The synthetic inputs stand in for the paper's data (Sec. 3): Gaussian fields with mean 50,
standard deviation 10 and the exponential covariance of Eq. 3, sigma^2 exp(-kappa |h|) with
kappa = 0.2, and a fraction p of the sites removed at random. These tests check the generator
against those definitions (moments and covariance at several lags, averaged over seeds), the
exact removal count, and the batch shape ranges."""
import math

import numpy as np
import pytest

import mpr_inputs


def _moments(z):
    m = z.mean()
    d = z - m
    cov = [float(d.var())]
    for h in (1, 2, 5, 10):
        cov.append(0.5 * (float((d[:, :-h] * d[:, h:]).mean()) + float((d[:-h, :] * d[h:, :]).mean())))
    return m, np.array(cov)


@pytest.mark.parametrize("periodic", [False, True])
def test_field_has_the_exponential_covariance(periodic):
    # 8 fields of 256^2; per field the estimates scatter by ~2 (~4 on the small torus), so the
    # seed means sit within a few units of sigma^2 exp(-kappa h)
    ms, cs = [], []
    for s in range(8):
        m, c = _moments(mpr_inputs.gaussian_field(256, 256, s, periodic=periodic))
        ms.append(m)
        cs.append(c)
    target = np.array([100.0] + [100.0 * math.exp(-0.2 * h) for h in (1, 2, 5, 10)])
    tol = 3.0 if not periodic else 5.5
    assert abs(np.mean(ms) - 50.0) < 1.0
    assert np.all(np.abs(np.mean(cs, axis=0) - target) < tol), (np.mean(cs, axis=0), target)


def test_field_is_seeded_and_kappa_sets_the_range():
    a = mpr_inputs.gaussian_field(64, 48, 3)
    b = mpr_inputs.gaussian_field(64, 48, 3)
    assert a.shape == (48, 64) and np.array_equal(a, b)
    assert not np.array_equal(a, mpr_inputs.gaussian_field(64, 48, 4))
    # the neighbour correlation follows exp(-kappa) (0.95 at kappa = 0.05, 0.61 at 0.5)
    for kappa in (0.05, 0.5):
        rho = np.mean([c[1] / c[0] for c in (_moments(mpr_inputs.gaussian_field(
            128, 128, s, kappa=kappa))[1] for s in range(4))])
        assert abs(rho - math.exp(-kappa)) < 0.03, (kappa, rho)


@pytest.mark.parametrize("Lx,Ly,p", [(64, 64, 0.33), (131, 37, 0.9), (5, 3, 0.5), (4096, 1, 0.66)])
def test_removal_mask_removes_exactly_round_pN(Lx, Ly, p):
    m = mpr_inputs.removal_mask(Lx, Ly, p, seed=7)
    assert m.shape == (Ly, Lx) and m.dtype == np.uint8
    assert int((m == 0).sum()) == int(round(p * Lx * Ly))
    assert np.array_equal(m, mpr_inputs.removal_mask(Lx, Ly, p, seed=7))


def test_batch_shapes_ranges():
    shapes = mpr_inputs.batch_shapes(256, seed=1)
    assert len(shapes) == 256
    for Lx, Ly, p, kappa in shapes:
        L = math.sqrt(Lx * Ly)
        assert 64 * 0.99 <= L <= 1024 * 1.01
        assert 1 / 4.05 <= Lx / Ly <= 4.05
        assert p in (0.33, 0.66, 0.9) and 0.05 <= kappa <= 0.5
    assert len({p for _, _, p, _ in shapes}) == 3
