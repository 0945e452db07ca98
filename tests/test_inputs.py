"""The seeded input recipes as stated: the generators are deterministic per
seed, and the fields have the statistics and structure the recipes give
(unit-variance Gaussian random field with a 5-cell Gaussian correlation, a
mean-one log-normal factor, the dust fraction and settling formula, the
batched workload's shape mix).  CPU only."""
import math

import numpy as np
import pytest

from paper_2506_10812_gb300 import inputs


def test_recipes_are_deterministic_per_seed():
    a, b = inputs.lognormal_gas(64, 128), inputs.lognormal_gas(64, 128)
    assert np.array_equal(a.sigma_g, b.sigma_g)
    c = inputs.lognormal_gas(64, 128, offset=7)
    assert not np.array_equal(a.sigma_g, c.sigma_g)
    s1, s2 = inputs.spiral_bifluid(St=1.0), inputs.spiral_bifluid(St=1.0)
    assert np.array_equal(s1.sigma_d, s2.sigma_d)


def test_grid_centres():
    """Cell centres r_i = r_in exp((i + 1/2) du) and phi_j = (j + 1/2) 2 pi / nphi."""
    r, phi = inputs._centres(8, 16, 0.1, 5.0)
    du = math.log(50.0) / 8
    assert np.allclose(r, 0.1 * np.exp((np.arange(8) + 0.5) * du), rtol=1e-15, atol=0)
    assert np.allclose(phi, (np.arange(16) + 0.5) * 2 * math.pi / 16, rtol=1e-15, atol=0)
    assert r[0] > 0.1 and r[-1] < 5.0


def test_gaussian_random_field_statistics():
    """Unit variance and the Gaussian autocorrelation exp(-l^2 / (2 c^2)) of
    the filtered white noise (c = 5 cells: 0.61 at l = 5, 0.14 at l = 10),
    measured along phi (periodic) on 512 x 1024."""
    rng = inputs._rng(99)
    g = inputs.gaussian_random_field(rng, 512, 1024, 5.0)
    assert g.shape == (512, 1024)
    assert abs(g.std() - 1.0) < 1e-12
    assert abs(g.mean()) < 0.05
    f = np.fft.rfft(g - g.mean(), axis=1)
    acf = np.fft.irfft(np.abs(f) ** 2, n=1024, axis=1).mean(axis=0)
    acf /= acf[0]
    for lag in (2, 5, 10):
        assert abs(acf[lag] - math.exp(-lag * lag / 50.0)) < 0.03, (lag, acf[lag])


def test_lognormal_disc_structure():
    """Sigma r = exp(0.3 G - 0.045) x (1 + spiral terms): the log-normal factor
    has mean one (E exp(s G - s^2 / 2) = 1), and the m = 2, 3, 4 spiral terms
    of amplitude 0.05 each leave the azimuthal mean at one."""
    d = inputs.lognormal_gas(256, 512)
    r, _ = inputs._centres(d.nr, d.nphi, d.r_in, d.r_out)
    x = d.sigma_g * r[:, None]
    assert (x > 0).all()
    assert abs(x.mean() - 1.0) < 0.03
    assert abs(np.log(x).std() - 0.3) < 0.03
    assert d.h_g == 0.05 and d.sigma_d is None and (d.r_in, d.r_out) == (0.1, 5.0)


def test_spiral_bifluid_recipe():
    """Sigma_d = 0.01 Sigma_g (1 + 0.01 U'), H_d / H_g = sqrt(alpha / (alpha + St)),
    alpha = 1e-3 (St = 1: h_d = 1.58e-3), and the m = 2 spiral of amplitude 0.1."""
    for St in (0.01, 0.1, 1.0):
        d = inputs.spiral_bifluid(St=St)
        ratio = d.sigma_d / d.sigma_g
        assert np.all(np.abs(ratio - 0.01) <= 0.01 * 0.01 + 1e-15)
        assert d.h_d == pytest.approx(0.05 * math.sqrt(1e-3 / (1e-3 + St)), rel=1e-14)
    assert inputs.spiral_bifluid(St=1.0).h_d == pytest.approx(1.5803e-3, rel=1e-4)
    d = inputs.spiral_bifluid(St=0.1)
    r, _ = inputs._centres(d.nr, d.nphi, d.r_in, d.r_out)
    amp = np.abs(np.fft.rfft(d.sigma_g * r[:, None], axis=1)) / (d.nphi / 2)
    assert np.all(np.abs(amp[:, 2] - 0.1) < 0.005)
    assert np.all(amp[:, 3] < 0.005)


def test_batch_workload_mix():
    """64 gas + dust discs, seed offset 10: 13 / 15 / 18 / 18 discs of the four
    sizes (49.6 M cells), h_g in [0.03, 0.1], St from {0.01, 0.1, 1}, each with
    a 1 % dust fraction."""
    discs = inputs.batch_discs()
    assert len(discs) == 64
    counts = {}
    for d in discs:
        counts[(d.nr, d.nphi)] = counts.get((d.nr, d.nphi), 0) + 1
        assert 0.03 <= d.h_g <= 0.1
        St = 1e-3 * ((d.h_g / d.h_d) ** 2 - 1.0)
        assert min(abs(St - s) / s for s in (0.01, 0.1, 1.0)) < 1e-9
        assert np.all(np.abs(d.sigma_d / d.sigma_g - 0.01) <= 1e-4 + 1e-15)
    assert counts == {(128, 256): 13, (256, 512): 15, (512, 1024): 18, (1024, 2048): 18}
    assert sum(d.cells for d in discs) == 49577984
