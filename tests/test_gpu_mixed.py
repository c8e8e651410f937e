"""Mixed-precision form (precision = 1) against the FP64 oracle (needs a GPU).

The topology is the FP64 mode's (same kernels, certified), so neighbour
cycles must still be identical.  Corners and the quadrature run in FP32 on
offsets from z_i and are summed in FP64.  Error bounds, derived from the
arithmetic: every FP32 quantity carries a few units of 6e-8 relative to the
cell scale; the signed sub-triangles of a cell can cancel by up to ~20x on
irregular cells, so m_i, c_i and h_i are held to 1e-5 relative and F_i (a
second moment) to 2e-5.  The gradient is formed from the FP64 sum of the
offsets p - z_i and is held to 1e-6 of |c_i|; totals (F, ||g||) sum many
independent cell errors, 2e-6.  Measured worst cells on these inputs:
m 1.3e-6, c 1.2e-6, F_i 3.3e-6, g 3.4e-8 |c|, F 3.0e-7, ||g|| 1.6e-7.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
from paper_1709_06924_gb300 import inputs as I
from paper_1709_06924_gb300.engine import Engine
from tests.parity import assert_mixed_within_bounds, assert_topology_equal


def mixed_eval(z, dens, decomposition=0):
    with Engine(len(z), dens, precision=1, decomposition=decomposition) as e:
        zt = torch.from_numpy(z).cuda()
        out = e.evaluate(zt)
        deg, nbr = e.voronoi(zt, max_deg=64)
        res = {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in out.items()}
        res["deg"], res["nbr"] = deg.cpu().numpy(), nbr.cpu().numpy()
    return res


@pytest.mark.parametrize("n,seed,dens,fan", [
    (2562, 0, I.density_uniform(), 0),
    (5001, 1, I.density_x3(), 0),
    (40962, 2, I.density_x64(), 0),
    (163842, 3, I.WORKLOADS["tanh-2621442"].density, 0),
    (40962, 4, I.WORKLOADS["tanh-163842"].density, 1),
])
def test_mixed_precision_error_against_oracle(n, seed, dens, fan):
    z = I.uniform_sphere(n, seed)
    r = mixed_eval(z, dens, fan)
    o = oracle.energy_grad(z, dens, fan=bool(fan))
    _, nbr_o, _ = oracle.voronoi(z)
    assert_topology_equal(r["deg"], r["nbr"], nbr_o)
    assert_mixed_within_bounds(r, o)
    cn = np.linalg.norm(o["c"], axis=1)
    # the gradient stays tangential
    gz = np.abs((r["grad"] * z).sum(axis=1))
    assert (gz <= 1e-12 * cn).all()


def test_mixed_solver_decreases_energy_like_fp64():
    z = I.uniform_sphere(20000, 5)
    dens = I.WORKLOADS["tanh-163842"].density
    reps = {}
    for prec in (0, 1):
        with Engine(len(z), dens, precision=prec) as e:
            zt = torch.from_numpy(z).cuda()
            reps[prec] = e.lbfgs_solve(zt, max_iter=30, grad_tol=0.0)
    assert reps[1]["iters"] == 30
    # both forms follow the same minimisation: energies agree to the mixed bound
    assert abs(reps[1]["energy"] / reps[0]["energy"] - 1) < 1e-3
    assert reps[1]["grad_norm"] < 0.5 * oracle.energy_grad(z, dens)["gnorm"]
