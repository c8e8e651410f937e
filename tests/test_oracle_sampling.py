"""Monte Carlo initialisation by the density (Sec. 4.1), oracle side.

Pins: rho = 1 keeps every candidate in order; the kept fraction equals
int rho / (4 pi rho_max) (closed form for X3, a zonal Gauss-Legendre
integral for the tanh cap) within 5 binomial standard deviations; a moment
of the kept points matches its closed form for X3."""
import math

import numpy as np

import oracle
from paper_1709_06924_gb300 import inputs as I
from tests.spherical_refs import zonal_integral


def test_uniform_density_keeps_every_candidate_in_order():
    cand, u = I.mc_candidates(5000, 3)
    z = oracle.sample_density(I.density_uniform(), cand, u, 4000)
    assert z.shape == (4000, 3) and np.array_equal(z, cand[:4000])


def _kept_fraction(dens, m=200000, seed=5):
    cand, u = I.mc_candidates(m, seed)
    z = oracle.sample_density(dens, cand, u, m)
    return len(z) / m, z


def test_x3_kept_fraction_and_moment():
    g = I.density_x3().gamma
    frac, z = _kept_fraction(I.density_x3())
    p = (1 - g) / 5 + g  # mean of (1 - gamma) z^4 + gamma over S^2, rho_max = 1
    assert abs(frac - p) <= 5 * math.sqrt(p * (1 - p) / 200000)
    # E[z^2 | kept] = int z^2 rho / int rho = ((1 - g)/7 + g/3) / ((1 - g)/5 + g)
    e2 = ((1 - g) / 7 + g / 3) / p
    sd = math.sqrt(np.var(z[:, 2] ** 2) / len(z))
    assert abs(np.mean(z[:, 2] ** 2) - e2) <= 5 * sd


def test_tanh_cap_kept_fraction():
    d = I.density_tanh((1 / 4) ** 4, 0.15, math.pi / 6, I.latlon_to_xyz(30, 0))

    def rho_of_cos(t):
        th = np.arccos(np.clip(t, -1, 1))
        return (1 - d.gamma) / (1 + np.exp(-2 * (d.beta - th) / d.alpha)) + d.gamma

    rmax = (1 - d.gamma) / (1 + math.exp(-2 * d.beta / d.alpha)) + d.gamma
    p = zonal_integral(rho_of_cos) / (4 * math.pi * rmax)
    frac, _ = _kept_fraction(d)
    assert abs(frac - p) <= 5 * math.sqrt(p * (1 - p) / 200000)


def test_square_root_sampling_kept_fraction():
    # e = 1/2: kept with probability sqrt(rho / rho_max); for X3 that is the
    # mean of sqrt((1 - g) z^4 + g), a zonal integral
    d = I.density_x3()
    cand, u = I.mc_candidates(200000, 8)
    z = oracle.sample_density(d, cand, u, 200000, exponent=0.5)
    p = zonal_integral(lambda t: np.sqrt((1 - d.gamma) * t ** 4 + d.gamma)) / (4 * math.pi)
    frac = len(z) / 200000
    assert abs(frac - p) <= 5 * math.sqrt(p * (1 - p) / 200000)
