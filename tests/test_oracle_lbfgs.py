"""Pins for the oracle's Lloyd map, two-loop recursion, line search and solver.

* Lloyd map = radial projection of the mass centroid (Sec. 2.1 / 2.2.1) and it
  never increases F (Sec. 2.2.1);
* with empty memory the preconditioned direction is the Lloyd direction and
  the unit step lands exactly on the Lloyd iterate (Sec. 3.1);
* the two-loop result equals the dense BFGS update applied to the same pairs
  with H0 = diag(h) (Sec. 2.2.2 product form, in its textbook form), and the
  newest pair satisfies the secant equation;
* the line search returns strong-Wolfe points on analytic 1D functions;
* the solver reaches a small gradient and the asymptotic CVT energy law
  F ~ G (int sqrt(rho))^2 / N (G = 5/(18 sqrt 3)); the X3 run lands in the
  band of the paper's Table 1 (tests/golden/paper_tables.txt).
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1709_06924_gb300 import inputs as I
from tests.spherical_refs import HEX_G, zonal_integral

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.txt")


def paper_rows():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, n, it, fe, F, g = line.split()
        rows[(name, int(n))] = dict(iters=int(it), fevals=int(fe), F=float(F), gnorm=float(g))
    return rows


def test_lloyd_step_is_projected_centroid():
    z = I.uniform_sphere(1000, 1)
    dens = I.density_x3()
    r = oracle.energy_grad(z, dens)
    zl = oracle.lloyd_step(z, dens)
    ref = r["c"] / np.linalg.norm(r["c"], axis=1)[:, None]
    assert np.abs(zl - ref).max() < 1e-15


def test_lloyd_decreases_energy():
    z = I.uniform_sphere(642, 2)
    dens = I.density_x3()
    F = [oracle.energy_grad(z, dens)["F"]]
    for _ in range(8):
        z = oracle.lloyd_step(z, dens)
        F.append(oracle.energy_grad(z, dens)["F"])
    assert all(b < a for a, b in zip(F, F[1:]))


def test_empty_memory_direction_is_lloyd():
    z = I.uniform_sphere(500, 3)
    dens = I.WORKLOADS["tanh-163842"].density
    r = oracle.energy_grad(z, dens)
    q = oracle.two_loop(r["g"], r["h"], [], [])
    assert np.allclose(q, -r["h"][:, None] * r["g"], rtol=0, atol=1e-17)
    # q_i = c_i/(c_i.z_i) - z_i, so normalize(z + q) is the Lloyd iterate
    x = z + q
    x /= np.linalg.norm(x, axis=1)[:, None]
    assert np.abs(x - oracle.lloyd_step(z, dens)).max() < 1e-15


def dense_bfgs_inverse(hdiag3, S, Y):
    H = np.diag(hdiag3)
    n = len(hdiag3)
    for s, y in zip(S, Y):
        rho = 1.0 / (y @ s)
        V = np.eye(n) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    return H


@pytest.mark.parametrize("m", [1, 3, 5, 7])
def test_two_loop_equals_dense_bfgs(m):
    rng = np.random.default_rng(10 + m)
    n = 12
    L = 3 * n
    h = rng.uniform(0.5, 2.0, n)
    S, Y = [], []
    A = rng.standard_normal((L, L))
    A = A @ A.T + L * np.eye(L)   # an SPD model Hessian gives y.s > 0
    for _ in range(m):
        s = rng.standard_normal(L)
        S.append(s.reshape(n, 3))
        Y.append((A @ s).reshape(n, 3))
    g = rng.standard_normal((n, 3))
    q = oracle.two_loop(g, h, S, Y)
    H = dense_bfgs_inverse(np.repeat(h, 3), [s.ravel() for s in S], [y.ravel() for y in Y])
    ref = -(H @ g.ravel())
    assert np.abs(q.ravel() - ref).max() <= 1e-12 * np.abs(ref).max()
    # secant equation for the newest pair: H y = s  (q(-y) = H y)
    hy = oracle.two_loop(-Y[-1], h, S, Y)
    assert np.abs(hy - S[-1]).max() <= 1e-12 * np.abs(S[-1]).max()


def _wolfe_ok(res, f0, g0, ftol=1e-4, gtol=0.9):
    a, f, g = res["stp"], res["f"], res["g"]
    return f <= f0 + ftol * a * g0 and abs(g) <= gtol * abs(g0)


@pytest.mark.parametrize("a0", [1e-3, 1e-1, 1.0, 10.0, 1e3])
def test_line_search_strong_wolfe_on_analytic_functions(a0):
    beta = 2.0

    def phi1(a):  # -a/(a^2 + beta): minimiser sqrt(beta)
        return -a / (a * a + beta), (a * a - beta) / (a * a + beta) ** 2

    def phi2(a):  # (a - 3)^2 - 1
        return (a - 3.0) ** 2 - 1.0, 2.0 * (a - 3.0)

    def phi3(a):  # smooth with a wiggle: a^4 - 3 a + 0.1 sin(20 a)
        return a ** 4 - 3 * a + 0.1 * math.sin(20 * a), 4 * a ** 3 - 3 + 2 * math.cos(20 * a)

    for phi in (phi1, phi2, phi3):
        f0, g0 = phi(0.0)
        res = oracle.line_search(phi, f0, g0, stp0=a0, maxfev=40)
        assert res["info"] == 1, res
        assert _wolfe_ok(res, f0, g0)
        assert res["nfev"] == len(res["calls"]) <= 40
        # the returned values are those of the last evaluation
        assert res["calls"][-1] == (res["stp"], res["f"], res["g"])


def test_line_search_backs_off_invalid_trial_points():
    # (a - 3)^2 whose trial points beyond a = 2.5 are not valid: the search
    # halves toward the best step, never returns above the first invalid one
    def phi(a):
        return None if a > 2.5 else ((a - 3.0) ** 2, 2.0 * (a - 3.0))

    res = oracle.line_search(phi, 9.0, -6.0, stp0=10.0, maxfev=20)
    assert res["info"] == 1
    assert res["stp"] <= 2.5 and _wolfe_ok(res, 9.0, -6.0)
    bad = [a for a, f, g in res["calls"] if f is None]
    assert bad and all(a > 2.5 for a in bad)
    firstbad = bad[0]
    assert all(a < firstbad for a, f, g in res["calls"][res["calls"].index((firstbad, None, None)) + 1:])


def test_line_search_quadratic_unit_step_accepted():
    # phi(a) = (a - 1)^2: the unit step is the exact minimiser
    res = oracle.line_search(lambda a: ((a - 1) ** 2, 2 * (a - 1)), 1.0, -2.0, stp0=1.0)
    assert res["info"] == 1 and res["nfev"] == 1 and res["stp"] == 1.0


def test_solver_uniform_reaches_tolerance_and_energy_law():
    n = 642
    z = I.uniform_sphere(n, 4)
    zf, rep, tr = oracle.lbfgs_solve(z, I.density_uniform(), lbfgs_m=5, max_iter=400, grad_tol=1e-8)
    # ends by tolerance, iteration cap, or a line search stalled at F's
    # rounding floor (status 6) once ||g|| is tiny
    assert rep["status"] in (0, oracle.LINESEARCH)
    assert rep["grad_norm"] <= 1e-8 or rep["iters"] == 400 or rep["status"] == oracle.LINESEARCH
    assert rep["grad_norm"] < 1e-6
    assert np.allclose(np.linalg.norm(zf, axis=1), 1.0, atol=1e-15)
    # energy decreases monotonically along the accepted iterates
    assert (np.diff(tr["F"]) <= 0).all()
    pred = HEX_G * (4 * math.pi) ** 2 / n
    assert 0.95 <= rep["energy"] / pred <= 1.03
    # energies of the recomputed final state agree
    assert abs(oracle.energy_grad(zf, I.density_uniform())["F"] - rep["energy"]) <= 1e-14 * rep["energy"]


def _paper_stop(z, dens):
    # the paper's stopping rules (Sec. 4.1): ||g||/F <= 5e-4 or |dF|/F < 1e-7, 2000 iterations
    return oracle.lbfgs_solve(z, dens, lbfgs_m=7, max_iter=2000, grad_tol=0.0,
                              rel_grad_tol=5e-4, rel_df_tol=1e-7)


def test_solver_x64_lands_in_paper_table1_band():
    row = paper_rows()[("X64", 2562)]
    dens = I.density_x64()
    zf, rep, tr = _paper_stop(I.uniform_sphere(2562, 0), dens)
    assert rep["converged"] == 1
    # measured 1.04297e-4 against the printed 1.04699e-4 (-0.4%)
    assert abs(rep["energy"] / row["F"] - 1) < 1e-2

    def rho_of_cos(t):
        d = np.arccos(np.clip(t, -1, 1))
        return (1 - dens.gamma) / 2 * (np.tanh((dens.beta - d) / dens.alpha) + 1) + dens.gamma
    pred = HEX_G * zonal_integral(lambda t: np.sqrt(rho_of_cos(t))) ** 2 / 2562
    assert 0.95 <= rep["energy"] / pred <= 1.03


def test_solver_x3_energy_law_and_paper_value():
    row = paper_rows()[("X3", 2562)]
    dens = I.density_x3()
    zf, rep, tr = _paper_stop(I.uniform_sphere(2562, 0), dens)
    assert rep["converged"] == 1
    sqrt_rho = zonal_integral(lambda t: np.sqrt((1 - dens.gamma) * t ** 4 + dens.gamma))
    pred = HEX_G * sqrt_rho ** 2 / 2562
    # measured 1.0079 x the hexagonal-cell law; the printed X3 value sits at
    # 0.974 x the law, so the paper's own X3 run (4-point rule, Monte Carlo
    # start) is 3.4% below ours: a 5% band around the printed value
    assert 0.95 <= rep["energy"] / pred <= 1.03
    assert abs(rep["energy"] / row["F"] - 1) < 5e-2


@pytest.mark.parametrize("m", [0, 1, 4])
def test_plain_lbfgs_two_loop_equals_dense_bfgs_with_scaled_identity(m):
    # Sec. 2.2.2: H0 = gamma I with gamma = y.s / y.y of the newest pair
    rng = np.random.default_rng(40 + m)
    n = 10
    L = 3 * n
    A = rng.standard_normal((L, L))
    A = A @ A.T + L * np.eye(L)
    S, Y = [], []
    for _ in range(m):
        s = rng.standard_normal(L)
        S.append(s.reshape(n, 3))
        Y.append((A @ s).reshape(n, 3))
    gamma = float(S[-1].ravel() @ Y[-1].ravel() / (Y[-1].ravel() @ Y[-1].ravel())) if m else 1.0
    g = rng.standard_normal((n, 3))
    q = oracle.two_loop_scalar(g, gamma, S, Y)
    H = dense_bfgs_inverse(np.full(L, gamma), [s.ravel() for s in S], [y.ravel() for y in Y])
    ref = -(H @ g.ravel())
    assert np.abs(q.ravel() - ref).max() <= 1e-12 * np.abs(ref).max()


def test_lloyd_mode_is_the_iterated_lloyd_map():
    # the Lloyd mode steps to normalize(z - h g) = c / |c| without a line search
    z = I.uniform_sphere(162, 8)
    dens = I.density_x3()
    zl, rep, trace = oracle.lbfgs_solve(z, dens, method="lloyd", max_iter=6, grad_tol=0.0)
    assert rep["iters"] == 6 and rep["fevals"] == 7
    zr = z.copy()
    for _ in range(6):
        zr = oracle.lloyd_step(zr, dens)
    assert np.abs(zl - zr).max() <= 1e-12
    assert np.all(np.diff(trace["F"]) < 0)  # Lloyd decreases the energy


@pytest.mark.parametrize("method", ["lbfgs", "lloyd"])
def test_other_methods_decrease_energy_and_converge(method):
    z = I.uniform_sphere(642, 9)
    dens = I.density_uniform()
    F0 = oracle.energy_grad(z, dens)["F"]
    zf, rep, trace = oracle.lbfgs_solve(z, dens, method=method, max_iter=60, grad_tol=0.0, lbfgs_m=5)
    assert rep["status"] == oracle.OK and rep["iters"] == 60
    assert trace["F"][-1] < F0 and np.all(np.diff(trace["F"]) <= 1e-18)
    assert trace["gnorm"][-1] < 0.2 * oracle.energy_grad(z, dens)["gnorm"]
