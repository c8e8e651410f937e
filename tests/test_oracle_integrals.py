"""Pins for the oracle's cell integrals, energy and gradient.

References independent of the oracle's arithmetic:
* rho == 1: cell areas sum to 4 pi (Sec. 2.1 partition); Platonic sets have
  equal areas 4 pi / N and zero gradient by symmetry;
* rho == 1: closed-form first moment of a spherical polygon (Stokes) and
  F_i = 2 m_i - 2 z_i.c_i;
* a high-order conical Gauss rule with the exact radial-projection Jacobian
  (built from numpy's Gauss-Legendre nodes) as the near-exact integral;
* brute-force nearest-generator Monte Carlo (no Voronoi construction);
* central finite differences of F along tangent retractions (gradient
  formula of Sec. 2.2.1 / Sec. 3.1, which relies on dF/dV = 0);
* g_i . z_i = 0 (tangential gradient, Sec. 3.1).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1709_06924_gb300 import inputs as I
from tests.spherical_refs import conical_rule, polygon_area, polygon_first_moment

UNI = I.density_uniform()


@pytest.mark.parametrize("n,seed", [(12, None), (100, 1), (2562, 2), (40962, 3)])
def test_total_area_is_4pi(n, seed):
    z = I.platonic(12) if seed is None else I.uniform_sphere(n, seed)
    r = oracle.energy_grad(z, UNI)
    assert abs(r["m"].sum() / (4 * math.pi) - 1) < 1e-13


@pytest.mark.parametrize("n", [4, 6, 8, 12, 20])
def test_platonic_equal_areas_zero_gradient(n):
    z = I.platonic(n)
    r = oracle.energy_grad(z, UNI)
    assert np.allclose(r["m"], 4 * math.pi / n, rtol=1e-13, atol=0)
    assert np.abs(r["g"]).max() <= 1e-14 * r["m"].max()
    assert np.allclose(r["Fi"], r["Fi"][0], rtol=1e-12, atol=0)


def test_icosahedron_energy_closed_form():
    # rho == 1: F_i = 2 m_i - 2 z_i . c_i with c_i from Stokes' theorem
    z = I.platonic(12)
    r = oracle.energy_grad(z, UNI)
    deg, nbr, vx = oracle.voronoi(z)
    c0 = polygon_first_moment(vx[0])
    assert abs(polygon_area(z[0], vx[0]) - math.pi / 3) < 1e-14
    F0 = 2 * (math.pi / 3) - 2 * z[0] @ c0
    hi = oracle.energy_grad(z, UNI, rule=conical_rule(8), exact_jacobian=True)
    assert abs(hi["Fi"][0] - F0) / F0 < 1e-12
    assert np.abs(hi["c"][0] - c0).max() < 1e-13
    # the 7-point rule on cells ~37 degrees wide carries about 1% error
    assert abs(r["Fi"][0] - F0) / F0 < 2e-2


def test_gradient_is_tangential():
    z = I.uniform_sphere(3000, 4)
    for dens in (UNI, I.density_x3(), I.WORKLOADS["tanh-163842"].density):
        r = oracle.energy_grad(z, dens)
        gz = np.abs((r["g"] * z).sum(axis=1))
        assert (gz <= 1e-15 * np.linalg.norm(r["c"], axis=1) * 8).all()
        assert (r["h"] > 0).all()


def midpoint_polygon(z, i, nbr, vx):
    """Cell i with the Delaunay edge midpoints normalize(z_i + z_j) inserted
    between consecutive corners: the region the paper's sub-triangles cover
    (its edges meet the bisector great circles up to input rounding, and
    neighbouring cells share them, so the cells still tile the sphere)."""
    out = []
    d = len(nbr[i])
    for t in range(d):
        mu = z[i] + z[nbr[i][t]]
        out += [vx[i][t], mu / np.linalg.norm(mu)]
    return out


def _closed_form_errors(n, seed):
    z = I.uniform_sphere(n, seed)
    r = oracle.energy_grad(z, UNI)
    _, nbr, vx = oracle.voronoi(z)
    polys = [midpoint_polygon(z, i, nbr, vx) for i in range(n)]
    ce = np.array([polygon_first_moment(v) for v in polys])
    me = np.array([polygon_area(z[i], polys[i]) for i in range(n)])
    Fe = 2 * me - 2 * (z * ce).sum(axis=1)
    err_c = np.abs(r["c"] - ce).max(axis=1) / np.linalg.norm(ce, axis=1)
    err_F = np.abs(r["Fi"] - Fe) / Fe
    return r, me, ce, err_c.max(), err_F.max()


def test_first_moment_and_energy_closed_form_and_order():
    errs = []
    for n in (642, 2562, 10242):
        r, me, ce, ec, eF = _closed_form_errors(n, 5)
        assert np.allclose(r["m"], me, rtol=1e-12, atol=0)   # areas are exact
        errs.append((n, ec, eF))
    # quadrature error is small and shrinks under refinement (h ~ N^-1/2)
    for (n0, c0, f0), (n1, c1, f1) in zip(errs, errs[1:]):
        assert c1 < c0 and f1 < f0
    n0, c0, f0 = errs[0]
    n2, c2, f2 = errs[-1]
    order_c = math.log(c0 / c2) / math.log(math.sqrt(n2 / n0))
    # measured: worst-cell relative error of c_i 2.3e-6 and of F_i 1.0e-4 at
    # N = 10,242; observed order in h about 2.6 (c) and 1.6 (F)
    assert errs[-1][1] < 5e-6 and errs[-1][2] < 2e-4
    assert order_c > 2.0


def test_exact_jacobian_rule_reproduces_closed_form():
    # high-order rule + exact Jacobian integrates rho == 1 quantities to
    # rounding: pins the signed sub-triangle decomposition covering each cell
    z = I.uniform_sphere(1000, 6)
    rule = conical_rule(8)
    r = oracle.energy_grad(z, UNI, rule=rule, exact_jacobian=True)
    _, nbr, vx = oracle.voronoi(z)
    polys = [midpoint_polygon(z, i, nbr, vx) for i in range(1000)]
    ce = np.array([polygon_first_moment(v) for v in polys])
    me = np.array([polygon_area(z[i], polys[i]) for i in range(1000)])
    assert np.allclose(r["m"], me, rtol=1e-11, atol=0)
    assert np.abs(r["c"] - ce).max() <= 1e-11 * np.abs(ce).max()


def test_variable_density_rule_error_small_and_shrinking():
    dens = I.WORKLOADS["tanh-163842"].density
    rule = conical_rule(8)
    prev = None
    for n in (2562, 10242):
        z = I.uniform_sphere(n, 7)
        a = oracle.energy_grad(z, dens)
        b = oracle.energy_grad(z, dens, rule=rule, exact_jacobian=True)
        em = np.abs(a["m"] - b["m"]).max() / b["m"].max()
        eF = abs(a["F"] - b["F"]) / b["F"]
        # measured: 1.2e-5 / 1.4e-6 (max-normalised m error), F 1.1e-4 / 2.6e-5
        assert em < 3e-5 and eF < 3e-4
        if prev is not None:
            assert em < prev
        prev = em


def _valid_small(n, seed):
    from tests.test_oracle_hull import valid_small
    return valid_small(n, seed)


@pytest.mark.parametrize("dens_name", ["uniform", "x3"])
def test_monte_carlo_cell_membership(dens_name):
    n = 24
    z = _valid_small(n, 8)
    dens = UNI if dens_name == "uniform" else I.density_x3()
    r = oracle.energy_grad(z, dens)
    rng = np.random.default_rng(9)
    M = 2_000_000
    msum = np.zeros(n)
    csum = np.zeros((n, 3))
    m2 = np.zeros(n)
    for _ in range(M // 200_000):
        x = rng.standard_normal((200_000, 3))
        x /= np.linalg.norm(x, axis=1)[:, None]
        owner = np.argmax(x @ z.T, axis=1)                 # nearest generator
        w = np.ones(len(x)) if dens_name == "uniform" else (1 - dens.gamma) * x[:, 2] ** 4 + dens.gamma
        msum += np.bincount(owner, weights=w, minlength=n)
        m2 += np.bincount(owner, weights=w * w, minlength=n)
        for d in range(3):
            csum[:, d] += np.bincount(owner, weights=w * x[:, d], minlength=n)
    scale = 4 * math.pi / M
    m_mc = msum * scale
    sig = np.sqrt(np.maximum(m2 / M - (msum / M) ** 2, 0) / M) * 4 * math.pi
    assert (np.abs(r["m"] - m_mc) <= 5 * sig + 1e-12).all()
    c_mc = csum * scale
    assert (np.abs(r["c"] - c_mc).max(axis=1) <= 5 * sig + 1e-4 * r["m"]).all()


def test_density_closed_forms():
    x3 = I.density_x3()
    assert oracle.rho(x3, [0, 0, 1]) == pytest.approx(1.0, abs=1e-15)
    assert oracle.rho(x3, [1, 0, 0]) == pytest.approx(x3.gamma, rel=1e-15)
    d = I.WORKLOADS["tanh-2621442"].density
    xc = np.array(d.xc)
    top = (1 - d.gamma) / 2 * (math.tanh(d.beta / d.alpha) + 1) + d.gamma
    assert oracle.rho(d, xc) == pytest.approx(top, rel=1e-14)
    # on the circle at geodesic distance beta from x_c the tanh term vanishes
    e = np.cross(xc, [1.0, 0, 0]); e /= np.linalg.norm(e)
    p = math.cos(d.beta) * xc + math.sin(d.beta) * e
    assert oracle.rho(d, p) == pytest.approx((1 - d.gamma) / 2 + d.gamma, rel=1e-12)
    assert oracle.rho(d, -xc) == pytest.approx(d.gamma, rel=1e-6)


def _tangent_fd(z, dens, i, t, eps, rule):
    zp = z.copy(); zm = z.copy()
    zp[i] = (z[i] + eps * t) / np.linalg.norm(z[i] + eps * t)
    zm[i] = (z[i] - eps * t) / np.linalg.norm(z[i] - eps * t)
    kw = dict(rule=rule, exact_jacobian=True) if rule is not None else {}
    return (oracle.energy_grad(zp, dens, **kw)["F"] - oracle.energy_grad(zm, dens, **kw)["F"]) / (2 * eps)


def test_gradient_matches_finite_differences():
    z = I.uniform_sphere(162, 10)
    dens = I.density_x3()
    rule = conical_rule(8)
    r_hi = oracle.energy_grad(z, dens, rule=rule, exact_jacobian=True)
    r_7 = oracle.energy_grad(z, dens)
    rng = np.random.default_rng(11)
    h = math.sqrt(4 * math.pi / 162)
    worst_hi = worst_7 = 0.0
    for i in rng.choice(162, 8, replace=False):
        t = rng.standard_normal(3)
        t -= (t @ z[i]) * z[i]
        t /= np.linalg.norm(t)
        eps = 1e-4 * h
        fd_hi = _tangent_fd(z, dens, i, t, eps, rule)
        fd_7 = _tangent_fd(z, dens, i, t, eps, None)
        scale = np.linalg.norm(r_hi["c"][i])
        worst_hi = max(worst_hi, abs(fd_hi - r_hi["g"][i] @ t) / scale)
        worst_7 = max(worst_7, abs(fd_7 - r_7["g"][i] @ t) / scale)
    assert worst_hi < 1e-7
    assert worst_7 < 1e-3


# ---- the fan decomposition: one triangle (z_i, v_a, v_b) per Voronoi edge
@pytest.mark.parametrize("n,seed", [(12, None), (2562, 2)])
def test_fan_total_area_and_platonic_symmetry(n, seed):
    z = I.platonic(12) if seed is None else I.uniform_sphere(n, seed)
    r = oracle.energy_grad(z, UNI, fan=True)
    assert abs(r["m"].sum() / (4 * math.pi) - 1) < 1e-13
    if seed is None:
        assert np.allclose(r["m"], math.pi / 3, rtol=1e-13, atol=0)
        assert np.abs(r["g"]).max() <= 1e-14 * r["m"].max()


def test_fan_integrates_the_voronoi_cell_itself():
    # the fan covers exactly the Voronoi polygon: areas exact, first moments
    # and energies approach the Stokes closed form of the polygon
    errs = []
    for n in (642, 2562, 10242):
        z = I.uniform_sphere(n, 5)
        r = oracle.energy_grad(z, UNI, fan=True)
        _, nbr, vx = oracle.voronoi(z)
        me = np.array([polygon_area(z[i], vx[i]) for i in range(n)])
        ce = np.array([polygon_first_moment(vx[i]) for i in range(n)])
        assert np.allclose(r["m"], me, rtol=1e-12, atol=0)
        errs.append(np.max(np.abs(r["c"] - ce).max(axis=1) / np.linalg.norm(ce, axis=1)))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-5
    # and both decompositions approximate the same integrals
    z = I.uniform_sphere(10242, 5)
    a = oracle.energy_grad(z, I.density_x3(), fan=True)
    b = oracle.energy_grad(z, I.density_x3())
    assert abs(a["F"] - b["F"]) / b["F"] < 1e-4
