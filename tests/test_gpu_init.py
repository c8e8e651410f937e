"""Initialisation and mesh-quality entries against the oracle (needs a GPU):
Monte Carlo sampling by the density, bisection refinement, cellQ / triQ."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
from paper_1709_06924_gb300 import inputs as I
from paper_1709_06924_gb300.engine import Engine, sample_density


@pytest.mark.parametrize("dens", [I.density_uniform(), I.density_x3(), I.density_x64(),
                                  I.Density(I.RHO_TANH_CAP_POW4, 0.25, 0.15, math.pi / 6, I.latlon_to_xyz(30, 0))])
@pytest.mark.parametrize("exponent", [1.0, 0.5])
def test_monte_carlo_sampling_keeps_the_oracle_candidates(dens, exponent):
    cand, u = I.mc_candidates(300001, 12)
    g = sample_density(dens, cand, u, 20000, exponent)
    o = oracle.sample_density(dens, cand, u, 20000, exponent)
    assert g.shape == o.shape
    assert np.array_equal(g, o)  # kept candidates are copied, so the sets are bit-identical


def test_sampling_when_candidates_run_out():
    cand, u = I.mc_candidates(1000, 13)
    g = sample_density(I.density_x64(), cand, u, 10**6)
    o = oracle.sample_density(I.density_x64(), cand, u, 10**6)
    assert 0 < len(g) == len(o) < 1000 and np.array_equal(g, o)


@pytest.mark.parametrize("n,seed", [(12, -1), (642, 1), (10001, 2)])
def test_bisection_matches_the_oracle_bitwise(n, seed):
    z = I.icosahedral_grid(0) if seed < 0 else I.uniform_sphere(n, seed)
    with Engine(len(z), I.density_uniform()) as e:
        zb = e.bisect(torch.from_numpy(z).cuda()).cpu().numpy()
    zo = oracle.bisect(z)
    assert zb.shape == zo.shape == (4 * len(z) - 6, 3)
    assert np.array_equal(zb, zo)


@pytest.mark.parametrize("n,seed", [(12, -1), (2562, 3), (40962, 4)])
def test_mesh_quality_matches_the_oracle(n, seed):
    z = I.icosahedral_grid(0) if seed < 0 else I.uniform_sphere(n, seed)
    with Engine(len(z), I.density_uniform()) as e:
        cq, tq = e.mesh_quality(torch.from_numpy(z).cuda())
    cqo, tqo = oracle.mesh_quality(z)
    assert len(tq) == len(tqo) == 2 * len(z) - 4
    assert np.abs(cq.cpu().numpy() - cqo).max() <= 1e-10
    assert np.abs(tq.cpu().numpy() - tqo).max() <= 1e-10
