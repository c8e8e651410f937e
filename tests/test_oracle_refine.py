"""Bisection refinement and mesh quality (Sec. 4), oracle side.

Pins: bisecting the icosahedron gives the level-1 icosahedral grid (built
independently from its 20 faces); bisection adds E = 3N - 6 points; every
midpoint lies on its edge's bisector.  Quality: all cells of the icosahedral
and octahedral meshes are regular (cellQ = 1) and all their Delaunay
triangles equilateral (triQ = 1); triQ equals 2 r / R of the triangle of arc
lengths (inradius over circumradius from Heron's formula, a different
formula); triangle count 2N - 4."""
import math

import numpy as np

import oracle
from paper_1709_06924_gb300 import inputs as I


def _same_set(a, b, tol=1e-14):
    assert a.shape == b.shape
    d = np.linalg.norm(a[:, None, :] - b[None, :, :], axis=2)
    return d.min(axis=1).max() <= tol and d.min(axis=0).max() <= tol


def test_bisected_icosahedron_is_the_level1_grid():
    z = I.icosahedral_grid(0)
    zb = oracle.bisect(z)
    assert zb.shape == (42, 3)
    assert np.array_equal(zb[:12], z)
    assert _same_set(zb, I.icosahedral_grid(1))
    # and twice
    assert _same_set(oracle.bisect(zb), I.icosahedral_grid(2))


def test_bisection_count_and_midpoints_on_bisectors():
    z = I.uniform_sphere(1000, 4)
    zb = oracle.bisect(z)
    assert len(zb) == 4 * 1000 - 6
    deg, nbr, _ = oracle.voronoi(z)
    pairs = sorted((i, j) for i in range(1000) for j in nbr[i] if j > i)
    mids = zb[1000:]
    for (i, j), m in zip(pairs, mids):
        assert abs(np.linalg.norm(m) - 1) <= 1e-15
        assert abs(np.linalg.norm(m - z[i]) - np.linalg.norm(m - z[j])) <= 1e-15


def test_regular_meshes_have_quality_one():
    for z in (I.icosahedral_grid(0), I.platonic(6), I.platonic(4)):
        cq, tq = oracle.mesh_quality(z)
        assert len(tq) == 2 * len(z) - 4
        assert np.abs(cq - 1).max() <= 1e-13 and np.abs(tq - 1).max() <= 1e-13


def test_triq_is_twice_inradius_over_circumradius():
    z = I.uniform_sphere(300, 6)
    cq, tq = oracle.mesh_quality(z)
    assert np.all((cq > 0) & (cq <= 1)) and np.all((tq > 0) & (tq <= 1 + 1e-12))
    # rebuild the triangles from the Voronoi topology and compare with 2 r / R
    deg, nbr, _ = oracle.voronoi(z)
    tris = set()
    for i in range(300):
        c = nbr[i]
        for k in range(len(c)):
            tris.add(tuple(sorted((i, c[k], c[(k + 1) % len(c)]))))
    tris = sorted(tris)
    assert len(tris) == len(tq)

    def arc(p, q):
        return math.atan2(np.linalg.norm(np.cross(p, q)), p @ q)

    for (i, j, k), q in zip(tris, tq):
        a, b, c = arc(z[j], z[k]), arc(z[k], z[i]), arc(z[i], z[j])
        s = (a + b + c) / 2
        area = math.sqrt(s * (s - a) * (s - b) * (s - c))
        r, R = area / s, a * b * c / (4 * area)
        assert abs(q - 2 * r / R) <= 1e-10
