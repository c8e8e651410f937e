"""Every cell of the 2,621,442-generator workload against the FP64 oracle
(needs a GPU).

Workload: N = 2,621,442 seeded uniform generators, tanh cap gamma = (1/8)^4,
alpha = 0.10, beta = pi/9, x_c at 45N 270E (LBFGS memory 7).  Checked on all
cells, not a sample:

* the cold start (no radius hints) in the FP64 form, the plain FP64 form
  and the mixed form (against its stated per-quantity bounds);
* the state the benchmark times: five LBFGS iterations on the GPU (radius
  hints carried from evaluation to evaluation), then the tuning the
  autotuner picks at that iterate and a fixed tuning with 16 topology lanes
  per cell and four concurrent cell pipelines; both tunings must give the
  same bits, and those must match the oracle at the GPU's iterate;
* the mixed form's warm state at N = 163,842.

Topology: neighbour cycles identical (vectorised comparison).  Geometry:
m_i, c_i, F_i, g_i, h_i within 1e-12 relative (tests/parity.py gives the
scales) in the FP64 forms; the mixed form within MIXED_BOUNDS."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
from paper_1709_06924_gb300 import inputs as I
from paper_1709_06924_gb300.engine import Engine
from tests.parity import RTOL, assert_geometry_close, assert_mixed_within_bounds, assert_topology_equal_all

W = I.WORKLOADS["tanh-2621442"]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def evaluate(e, zt):
    out = e.evaluate(zt)
    deg, nbr = e.voronoi(zt, max_deg=32)
    res = {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in out.items()}
    res["deg"] = deg.cpu().numpy()
    res["nbr"] = nbr.cpu().numpy()
    res["stats"] = e.stats()
    return res


def reference(z, dens):
    o = oracle.energy_grad(z, dens)
    o["topo"] = oracle.voronoi_flat(z)
    return o


def check_fp64(g, o):
    deg_o, off_o, flat_o = o["topo"]
    assert g["stats"]["ambiguous"] == 0
    assert_topology_equal_all(g["deg"], g["nbr"], deg_o, off_o, flat_o)
    errs = assert_geometry_close(g, o)
    assert abs(g["energy"] - o["F"]) <= RTOL * o["F"]
    assert abs(g["grad_norm"] - o["gnorm"]) <= 1e-10 * o["gnorm"]
    assert int(g["deg"].sum()) == 6 * len(g["deg"]) - 12
    return errs


@pytest.fixture(scope="module")
def cold():
    z = I.uniform_sphere(W.n, 0)
    return z, reference(z, W.density)


@pytest.mark.parametrize("precision", [0, 2])
def test_every_cell_cold_start(cold, precision):
    z, o = cold
    with Engine(W.n, W.density, lbfgs_m=W.lbfgs_m, precision=precision) as e:
        g = evaluate(e, dev(z))
    errs = check_fp64(g, o)
    print("precision %d, worst relative errors over %d cells: %s" % (precision, W.n, errs))


def test_every_cell_cold_start_mixed(cold):
    z, o = cold
    with Engine(W.n, W.density, lbfgs_m=W.lbfgs_m, precision=1) as e:
        g = evaluate(e, dev(z))
    deg_o, off_o, flat_o = o["topo"]
    assert_topology_equal_all(g["deg"], g["nbr"], deg_o, off_o, flat_o)
    err = assert_mixed_within_bounds(g, o)
    print("mixed form, worst per-cell errors over %d cells: %s" % (W.n, err))


def test_every_cell_in_the_benchmarked_warm_state():
    z0 = I.uniform_sphere(W.n, 0)
    with Engine(W.n, W.density, lbfgs_m=W.lbfgs_m, precision=0) as e:
        zt = dev(z0)
        rep = e.lbfgs_solve(zt, max_iter=5, grad_tol=0.0)
        assert rep["iters"] == 5
        tuned = e.tune(zt)
        a = evaluate(e, zt)
        e.set_tuning(topo_cell_lanes=16, chunks=4)
        b = evaluate(e, zt)
        z = zt.cpu().numpy()
    for k in ("grad", "mass", "moment", "cell_energy", "precond", "deg", "nbr"):
        assert np.array_equal(a[k], b[k]), k
    assert a["energy"] == b["energy"]
    o = reference(z, W.density)
    errs = check_fp64(a, o)
    print("warm state after 5 iterations, tuning %s: worst relative errors %s" % (tuned, errs))


def test_mixed_warm_state_163842():
    w = I.WORKLOADS["tanh-163842"]
    z0 = I.uniform_sphere(w.n, 1)
    with Engine(w.n, w.density, lbfgs_m=w.lbfgs_m, precision=1) as e:
        zt = dev(z0)
        e.lbfgs_solve(zt, max_iter=5, grad_tol=0.0)
        e.tune(zt)
        g = evaluate(e, zt)
        z = zt.cpu().numpy()
    o = reference(z, w.density)
    deg_o, off_o, flat_o = o["topo"]
    assert_topology_equal_all(g["deg"], g["nbr"], deg_o, off_o, flat_o)
    err = assert_mixed_within_bounds(g, o)
    print("mixed form, warm state at N = 163,842: %s" % err)
