"""CUDA path vs the FP64 oracle through the C ABI (needs a GPU).

Topology: Voronoi neighbour cycles must be identical (bit-exact ids and
order) on generic inputs.  Geometry: m_i, c_i, F_i, g_i, h_i and F within
1e-12 relative (tests/parity.py explains the scales).  Sizes span several
thread blocks with ragged tails; the full 2,621,442-generator workload is
checked on every cell in tests/test_gpu_fullsize.py."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
from paper_1709_06924_gb300 import inputs as I
from paper_1709_06924_gb300.engine import Engine
from tests.parity import assert_geometry_close, assert_topology_equal, canon, RTOL

DENS = {
    "uniform": I.density_uniform(),
    "x3": I.density_x3(),
    "tanh163842": I.WORKLOADS["tanh-163842"].density,
    "tanh2621442": I.WORKLOADS["tanh-2621442"].density,
    "x64": I.density_x64(),
    "pow4": I.Density(I.RHO_TANH_CAP_POW4, (1 / 4), 0.15, math.pi / 6, I.latlon_to_xyz(30, 0)),
}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_eval(z, dens, **kw):
    with Engine(len(z), dens, **kw) as e:
        out = e.evaluate(dev(z))
        deg, nbr = e.voronoi(dev(z), max_deg=64)
        res = {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in out.items()}
        res["deg"] = deg.cpu().numpy()
        res["nbr"] = nbr.cpu().numpy()
        res["stats"] = e.stats()
    return res


def valid_small(n, seed):
    from tests.test_oracle_hull import valid_small as vs
    return vs(n, seed)


CASES = [
    # (n, seed, density): several blocks of 128 threads with ragged tails
    (2562, 0, "uniform"),
    (2562, 1, "x3"),
    (1000, 2, "tanh163842"),
    (4097, 3, "x64"),
    (5001, 4, "pow4"),
    (40962, 5, "tanh2621442"),
    (163842, 0, "tanh163842"),
]


@pytest.mark.parametrize("n,seed,dname", CASES)
def test_topology_and_geometry_match_oracle(n, seed, dname):
    z = I.uniform_sphere(n, seed)
    dens = DENS[dname]
    g = gpu_eval(z, dens)
    o = oracle.energy_grad(z, dens)
    _, nbr_o, _ = oracle.voronoi(z)
    assert g["stats"]["ambiguous"] == 0
    assert_topology_equal(g["deg"], g["nbr"], nbr_o)
    assert_geometry_close(g, o)
    assert abs(g["energy"] - o["F"]) <= RTOL * o["F"]
    assert abs(g["grad_norm"] - o["gnorm"]) <= 1e-10 * o["gnorm"]


@pytest.mark.parametrize("n,seed,dname", [c for c in CASES if c[0] <= 40962])
def test_plain_fp64_form_matches_oracle(n, seed, dname):
    # precision 2: corners and rule points in FP64 arithmetic
    z = I.uniform_sphere(n, seed)
    dens = DENS[dname]
    g = gpu_eval(z, dens, precision=2)
    o = oracle.energy_grad(z, dens)
    _, nbr_o, _ = oracle.voronoi(z)
    assert_topology_equal(g["deg"], g["nbr"], nbr_o)
    assert_geometry_close(g, o)
    assert abs(g["energy"] - o["F"]) <= RTOL * o["F"]


@pytest.mark.parametrize("n", [4, 5, 6, 7, 10, 12, 33, 100, 129])
def test_small_and_platonic_sets(n):
    z = I.platonic(n) if n in (4, 6, 12) else valid_small(n, 40 + n)
    for dens in (DENS["uniform"], DENS["x64"]):
        g = gpu_eval(z, dens)
        o = oracle.energy_grad(z, dens)
        _, nbr_o, _ = oracle.voronoi(z)
        assert_topology_equal(g["deg"], g["nbr"], nbr_o)
        assert_geometry_close(g, o)


@pytest.mark.parametrize("n", [8, 20])
def test_degenerate_platonic_geometry(n):
    # cube / dodecahedron: four or five generators per Voronoi vertex; the
    # Delaunay triangulation is not unique, the cells are
    # (the evaluation succeeding shows the cells agreed on every vertex: the
    # edge list did not overflow its 6N capacity)
    z = I.platonic(n)
    g = gpu_eval(z, DENS["uniform"])
    o = oracle.energy_grad(z, DENS["uniform"])
    assert int(g["deg"].sum()) <= 6 * n
    assert np.allclose(g["mass"], 4 * math.pi / n, rtol=1e-13, atol=0)
    assert_geometry_close(g, o, rtol=1e-12)


def test_icosahedral_grid_is_a_critical_point():
    z = I.icosahedral_grid(3)  # 642 points, icosahedral symmetry
    g = gpu_eval(z, DENS["uniform"])
    assert abs(g["mass"].sum() / (4 * math.pi) - 1) < 1e-13
    o = oracle.energy_grad(z, DENS["uniform"])
    assert_geometry_close(g, o)


def test_lloyd_step_matches_oracle():
    z = I.uniform_sphere(10242, 7)
    dens = DENS["tanh163842"]
    with Engine(len(z), dens) as e:
        zl = e.lloyd_step(dev(z)).cpu().numpy()
        zl_host = e.lloyd_step(z)  # host arrays are staged through the device
    ref = oracle.lloyd_step(z, dens)
    assert np.abs(zl - ref).max() <= 1e-13
    assert np.array_equal(zl, zl_host)


# 1 .. 8 pairs take the gathered passes (the products s_a.y_b formed first
# for the external history), 0 and 9+ the step-by-step passes
@pytest.mark.parametrize("count", [0, 1, 2, 3, 7, 8, 9, 12])
def test_two_loop_matches_oracle(count):
    n = 3001
    rng = np.random.default_rng(100 + count)
    g = rng.standard_normal((n, 3))
    h = rng.uniform(0.5, 2.0, n)
    S, Y = [], []
    for _ in range(count):
        s = rng.standard_normal((n, 3))
        S.append(s)
        Y.append(s * rng.uniform(0.5, 1.5, (n, 3)))  # y.s > 0
    ref = oracle.two_loop(g, h, S, Y)
    with Engine(n, DENS["uniform"]) as e:
        St = dev(np.stack(S)) if count else None
        Yt = dev(np.stack(Y)) if count else None
        q = e.lbfgs_direction(dev(g), dev(h), St, Yt).cpu().numpy()
    assert np.abs(q - ref).max() <= 1e-12 * np.abs(ref).max()


def test_first_iteration_is_the_lloyd_step():
    z = I.uniform_sphere(2562, 8)
    dens = DENS["x3"]
    with Engine(len(z), dens, lbfgs_m=5) as e:
        zt = dev(z)
        rep = e.lbfgs_solve(zt, max_iter=1, grad_tol=0.0)
        zl = e.lloyd_step(dev(z)).cpu().numpy()
    assert rep["iters"] == 1
    if rep["fevals"] == 2:  # unit step accepted at the first trial
        assert np.abs(zt.cpu().numpy() - zl).max() <= 1e-15


@pytest.mark.parametrize("iters", [1, 5])
def test_solver_lockstep_with_oracle(iters):
    z = I.uniform_sphere(2562, 9)
    dens = DENS["uniform"]
    zo, rep_o, tr = oracle.lbfgs_solve(z, dens, lbfgs_m=5, max_iter=iters, grad_tol=0.0)
    with Engine(len(z), dens, lbfgs_m=5) as e:
        zt = dev(z)
        rep = e.lbfgs_solve(zt, max_iter=iters, grad_tol=0.0)
    assert rep["iters"] == rep_o["iters"] == iters
    assert rep["fevals"] == rep_o["fevals"]
    assert abs(rep["energy"] - rep_o["energy"]) <= 1e-12 * rep_o["energy"]
    assert np.abs(zt.cpu().numpy() - zo).max() <= 1e-11


def test_solver_lockstep_with_oracle_through_a_full_memory():
    # m = 7 over 12 iterations: the history ring fills, drops its oldest pair
    # and reuses slots, so the products s_a.y_b kept by slot are reused across
    # directions
    z = I.uniform_sphere(2562, 29)
    dens = DENS["x3"]
    zo, rep_o, tr = oracle.lbfgs_solve(z, dens, lbfgs_m=7, max_iter=12, grad_tol=0.0)
    with Engine(len(z), dens, lbfgs_m=7) as e:
        zt = dev(z)
        rep = e.lbfgs_solve(zt, max_iter=12, grad_tol=0.0)
    assert rep["iters"] == rep_o["iters"] == 12
    assert rep["fevals"] == rep_o["fevals"]
    assert rep["skipped"] == rep_o["skipped"] and rep["resets"] == rep_o["resets"]
    assert abs(rep["energy"] - rep_o["energy"]) <= 1e-12 * rep_o["energy"]
    assert np.abs(zt.cpu().numpy() - zo).max() <= 1e-10


def test_solver_reaches_tolerance_uniform_2562():
    z = I.uniform_sphere(2562, 0)
    dens = DENS["uniform"]
    with Engine(len(z), dens, lbfgs_m=5) as e:
        zt = dev(z)
        rep = e.lbfgs_solve(zt, max_iter=200, grad_tol=1e-8)
    assert rep["status"] in (0, 6)
    assert rep["grad_norm"] < 1e-5
    pred = 5 / (18 * math.sqrt(3)) * (4 * math.pi) ** 2 / 2562
    assert 0.95 <= rep["energy"] / pred <= 1.03
    zf = zt.cpu().numpy()
    assert np.allclose(np.linalg.norm(zf, axis=1), 1.0, atol=1e-15)


def test_warm_start_continues_the_same_trajectory():
    z = I.uniform_sphere(5000, 10)
    dens = DENS["tanh163842"]
    with Engine(len(z), dens, lbfgs_m=7) as e:
        a = dev(z)
        e.lbfgs_solve(a, max_iter=6, grad_tol=0.0)
        b = dev(z)
        e.lbfgs_solve(b, max_iter=3, grad_tol=0.0)
        e.lbfgs_solve(b, max_iter=3, grad_tol=0.0, warm_start=True)
    assert torch.equal(a, b)


def test_evaluation_is_deterministic_and_order_independent():
    n = 20000
    z = I.uniform_sphere(n, 11)
    dens = DENS["tanh2621442"]
    perm = np.random.default_rng(12).permutation(n)
    with Engine(n, dens) as e:
        a = e.evaluate(dev(z))
        b = e.evaluate(dev(z))
        c = e.evaluate(dev(z[perm]))
    for k in ("grad", "mass", "moment", "cell_energy", "precond"):
        assert torch.equal(a[k], b[k]), k
        assert torch.equal(a[k][perm], c[k]), k
    assert a["energy"] == b["energy"]


def test_host_and_device_pointers_agree():
    z = I.uniform_sphere(3000, 13)
    with Engine(len(z), DENS["x3"]) as e:
        F1, g1, m1, c1 = e.energy_grad(dev(z))
        F2, g2, m2, c2 = e.energy_grad(z)
    assert F1 == F2 and torch.equal(g1, g2) and torch.equal(m1, m2)


def _status_of(fn):
    from paper_1709_06924_gb300.capi import ScvtError
    with pytest.raises(ScvtError) as ei:
        fn()
    return ei.value.status


def test_invalid_and_degenerate_inputs_are_reported():
    from paper_1709_06924_gb300 import capi
    n = 500
    z = I.uniform_sphere(n, 14)
    with Engine(n, DENS["uniform"]) as e:
        bad = z.copy(); bad[7] *= 1.001
        assert _status_of(lambda: e.energy_grad(dev(bad))) == capi.ERR_INVALID
        nan = z.copy(); nan[3, 1] = np.nan
        assert _status_of(lambda: e.energy_grad(dev(nan))) == capi.ERR_INVALID
        dup = z.copy(); dup[9] = dup[2]
        assert _status_of(lambda: e.energy_grad(dev(dup))) == capi.ERR_INVALID
        hemi = z.copy(); hemi[:, 2] = np.abs(hemi[:, 2]) + 0.05
        hemi /= np.linalg.norm(hemi, axis=1)[:, None]
        assert _status_of(lambda: e.energy_grad(dev(hemi))) == capi.ERR_DEGENERATE
        # the handle stays usable after errors
        F, *_ = e.energy_grad(dev(z))
        assert abs(F - oracle.energy_grad(z, DENS["uniform"])["F"]) <= RTOL * F


@pytest.mark.parametrize("kind", [I.RHO_TANH_CAP, I.RHO_TANH_CAP_POW4])
def test_density_series_and_its_fallback_match_oracle(kind):
    # a narrow cap (alpha = 0.05) centred on a generator, at a size where cells
    # are wide against alpha: most edges take the density table's series, the
    # cells at the cap centre and the widest edges fall back to the direct formula
    n = 5000
    z = I.uniform_sphere(n, 77)
    dens = I.Density(kind, (1 / 16) ** 4, 0.05, math.pi / 12, tuple(z[123]))
    g = gpu_eval(z, dens)
    o = oracle.energy_grad(z, dens)
    st = g["stats"]
    per_eval = st["series_edges"] / st["evaluations"]
    assert 0 < per_eval < 6 * n - 12
    assert 3 <= st["series_terms"] / st["series_edges"] <= 23
    assert_geometry_close(g, o)
    assert abs(g["energy"] - o["F"]) <= RTOL * o["F"]


@pytest.mark.parametrize("method", ["lbfgs", "lloyd"])
@pytest.mark.parametrize("iters", [1, 5])
def test_other_methods_lockstep_with_oracle(method, iters):
    z = I.uniform_sphere(2562, 19)
    dens = DENS["x3"]
    zo, rep_o, tr = oracle.lbfgs_solve(z, dens, lbfgs_m=5, max_iter=iters, grad_tol=0.0, method=method)
    with Engine(len(z), dens, lbfgs_m=5) as e:
        zt = dev(z)
        rep = e.lbfgs_solve(zt, max_iter=iters, grad_tol=0.0, method=method)
    assert rep["iters"] == rep_o["iters"] == iters
    assert rep["fevals"] == rep_o["fevals"]
    assert rep["skipped"] == rep_o["skipped"] and rep["resets"] == rep_o["resets"]
    assert abs(rep["energy"] - rep_o["energy"]) <= 1e-12 * rep_o["energy"]
    assert np.abs(zt.cpu().numpy() - zo).max() <= 1e-11


def test_lloyd_mode_matches_the_lloyd_step_entry():
    z = I.uniform_sphere(4001, 21)
    dens = DENS["tanh163842"]
    with Engine(len(z), dens, lbfgs_m=5) as e:
        zt = dev(z)
        rep = e.lbfgs_solve(zt, max_iter=1, grad_tol=0.0, method="lloyd")
        zl = e.lloyd_step(dev(z)).cpu().numpy()
    assert rep["iters"] == 1 and rep["fevals"] == 2
    assert np.abs(zt.cpu().numpy() - zl).max() <= 1e-14


def test_cells_wider_than_the_neighbour_search_match_oracle():
    # a narrow cap sampled by rho^(1/2) at small N: most generators inside the
    # cap, a few hundred outside with cells reaching ~60 degrees; those cells
    # need the last pass's clip by every generator within the security radius
    dens = I.density_x64()
    cand, u = I.mc_candidates(400000, 2024)
    z = oracle.sample_density(dens, cand, u, 2562, 0.5)
    g = gpu_eval(z, dens)
    o = oracle.energy_grad(z, dens)
    _, nbr_o, _ = oracle.voronoi(z)
    assert_topology_equal(g["deg"], g["nbr"], nbr_o)
    assert_geometry_close(g, o)


@pytest.mark.parametrize("n,seed,dname", [(2562, 30, "uniform"), (5001, 31, "x3"), (40962, 32, "tanh2621442"),
                                          (12, None, "uniform")])
def test_fan_decomposition_matches_oracle(n, seed, dname):
    z = I.platonic(12) if seed is None else I.uniform_sphere(n, seed)
    dens = DENS[dname]
    g = gpu_eval(z, dens, decomposition=1)
    o = oracle.energy_grad(z, dens, fan=True)
    assert_geometry_close(g, o)
    assert abs(g["energy"] - o["F"]) <= RTOL * o["F"]
