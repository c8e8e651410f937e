"""Numerical accuracy of the oracle's cell integrals on the most irregular
cells (CPU only).

The parity tests hold the CUDA path to 1e-12 relative per cell, so the
oracle's own rounding error must sit well below that, also in the smallest,
most irregular cells of a random point set, where FP64 unit vectors lose up
to ~1e-12 of a cell's energy.

* Pin (closed form): with rho = 1 the 7-point rule is exact for the mass, and
  with the fan decomposition (one triangle z_i, v_a, v_b per Voronoi edge)
  m_i is the area of the spherical Voronoi polygon, which Girard's theorem
  gives as (sum of interior angles) - (d - 2) pi; the angles are taken in
  40-digit arithmetic at the exact circumcentres of the Delaunay triangles.
  (The paper's sub-triangles through mu = normalize(z_i + z_j) add slivers
  of relative size up to ~1e-10 in such cells: with generators unit only to
  rounding, mu lies off the Voronoi edge's great circle by ~1e-16/|z_j - z_i|.
  That is part of the definition both sides evaluate, so the next check
  covers the paper's decomposition.)
* Accuracy check: for the tanh-cap density, F_i and m_i against a 40-digit
  evaluation of the same quadrature (same rule, sub-triangles, area formula
  and density) -- an independent evaluation of the oracle's arithmetic, not
  of its definition, which tests/test_oracle_integrals.py pins.
"""
import math

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

import oracle
from paper_1709_06924_gb300 import inputs as I

mp.mp.dps = 40


def _v(x):
    return [mp.mpf(float(t)) for t in x]


def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def _cross(u, v):
    return [u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]]


def _sub(a, b):
    return [a[k] - b[k] for k in range(3)]


def _unit(a):
    r = mp.sqrt(_dot(a, a))
    return [t / r for t in a]


def _circumcentre(a, b, c):
    v = _unit(_cross(_sub(b, a), _sub(c, a)))
    return v if _dot(v, a) > 0 else [-t for t in v]


def _corners(z, i, nb):
    zi = _v(z[i])
    d = len(nb)
    return [_circumcentre(zi, _v(z[nb[t - 1]]), _v(z[nb[t]])) for t in range(d)]


def _girard_area(vs):
    """Area of a convex spherical polygon (corners counter-clockwise seen from
    outside): sum of the interior angles minus (d - 2) pi."""
    d = len(vs)
    tot = mp.mpf(0)
    for k in range(d):
        v, prev, nxt = vs[k], vs[k - 1], vs[(k + 1) % d]
        t1 = _sub(prev, [_dot(prev, v) * x for x in v])   # tangent toward the previous corner
        t2 = _sub(nxt, [_dot(nxt, v) * x for x in v])     # and toward the next one
        tot += mp.atan2(mp.sqrt(_dot(_cross(t1, t2), _cross(t1, t2))), _dot(t1, t2))
    return tot - (d - 2) * mp.pi


def _irregular_cells(z, deg, off, flat, count):
    """The cells whose neighbours' distances spread the most, and the smallest
    (the 12 wide cells of the icosahedron vertices left out)."""
    n = len(deg)
    spread = np.zeros(n)
    size = np.full(n, np.inf)
    for i in range(12, n):
        nb = flat[off[i]:off[i + 1]]
        d = np.linalg.norm(z[nb] - z[i], axis=1)
        spread[i] = d.max() / d.min()
        size[i] = d.max()
    a = np.argsort(-spread)[:count]
    b = np.argsort(size)[:count]
    return sorted(set(a.tolist()) | set(b.tolist()))


@pytest.fixture(scope="module")
def mesh():
    # the 12 icosahedron vertices and 4,000 points uniform in a cap of 0.02 rad
    # around a direction between them: cells ~1e-4 wide, as small as those of a
    # multi-million-generator mesh (tens of them far more irregular)
    rng = np.random.default_rng(424242)
    c = np.array([0.3, -0.5, 0.81])
    c /= np.linalg.norm(c)
    e1 = np.cross(c, [0.0, 0.0, 1.0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(c, e1)
    r = 0.02 * np.sqrt(rng.random(4000))
    t = 2 * np.pi * rng.random(4000)
    pts = c[None, :] + (r * np.cos(t))[:, None] * e1 + (r * np.sin(t))[:, None] * e2
    z = np.concatenate([I.platonic(12), pts / np.linalg.norm(pts, axis=1)[:, None]])
    deg, off, flat = oracle.voronoi_flat(z)
    return np.ascontiguousarray(z), deg, off, flat


def test_cell_areas_match_girard_on_irregular_cells(mesh):
    z, deg, off, flat = mesh
    o = oracle.energy_grad(z, I.density_uniform(), fan=True)
    worst = 0.0
    for i in _irregular_cells(z, deg, off, flat, 15):
        area = float(_girard_area(_corners(z, i, flat[off[i]:off[i + 1]])))
        worst = max(worst, abs(o["m"][i] - area) / area)
    assert worst <= 1e-14, worst


def _quadrature_40(z, i, nb, dens):
    s15 = mp.sqrt(15)
    a1, a2 = (6 - s15) / 21, (6 + s15) / 21
    w1, w2 = (155 - s15) / 1200, (155 + s15) / 1200
    rule = [((mp.mpf(1) / 3,) * 3, mp.mpf(9) / 40)]
    for a, wt in ((a1, w1), (a2, w2)):
        b = 1 - 2 * a
        rule += [((b, a, a), wt), ((a, b, a), wt), ((a, a, b), wt)]
    xc = _v(dens.xc)

    def rho(p):
        d = mp.atan2(mp.sqrt(_dot(_cross(p, xc), _cross(p, xc))), _dot(p, xc))
        return (1 - mp.mpf(dens.gamma)) / (1 + mp.exp(-2 * (mp.mpf(dens.beta) - d) / mp.mpf(dens.alpha))) \
            + mp.mpf(dens.gamma)

    zi = _v(z[i])
    vs = _corners(z, i, nb)
    m = F = mp.mpf(0)
    for t in range(len(nb)):
        mu = _unit([zi[k] + _v(z[nb[t]])[k] for k in range(3)])
        for a, b, c in ((zi, vs[t], mu), (zi, mu, vs[(t + 1) % len(nb)])):
            det = _dot(a, _cross(_sub(b, a), _sub(c, a)))
            den = 1 + _dot(a, b) + _dot(b, c) + _dot(c, a)
            area = 2 * mp.atan2(det, den)
            for (l0, l1, l2), wt in rule:
                p = _unit([l0 * a[k] + l1 * b[k] + l2 * c[k] for k in range(3)])
                r = rho(p) * wt * area
                dp = _sub(p, zi)
                m += r
                F += r * _dot(dp, dp)
    return float(m), float(F)


def test_cell_energies_match_a_40_digit_evaluation(mesh):
    z, deg, off, flat = mesh
    dens = I.Density(I.RHO_TANH_CAP, (1 / 8) ** 4, 0.10, math.pi / 9, tuple(z[77]))
    o = oracle.energy_grad(z, dens)
    worst = {"m": 0.0, "F": 0.0}
    for i in _irregular_cells(z, deg, off, flat, 5):
        m, F = _quadrature_40(z, i, flat[off[i]:off[i + 1]], dens)
        worst["m"] = max(worst["m"], abs(o["m"][i] - m) / m)
        worst["F"] = max(worst["F"], abs(o["Fi"][i] - F) / F)
    assert max(worst.values()) <= 1e-14, worst
