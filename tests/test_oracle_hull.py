"""Pins for the oracle's spherical Delaunay / Voronoi construction.

* Euler's formula on the sphere: V - E + F = 2 with 2N - 4 Voronoi vertices,
  3N - 6 edges and N cells (every cell closes, degrees sum to 6N - 12);
* empty circumcircle by brute force: every cell corner is equidistant from
  its cell's generator and the two neighbours of the adjacent edges, and no
  generator is closer (Sec. 2.1 definition of V_i^c);
* neighbour sets equal those of an independent library hull (scipy/Qhull);
* Platonic solids: closed-form degrees;
* invalid inputs (all generators in one hemisphere, duplicates) are refused.
"""
import numpy as np
import pytest

import oracle
from paper_1709_06924_gb300 import inputs as I


def in_closed_hemisphere(z):
    """Brute force: z lies in a closed hemisphere iff some great circle through
    two of the points (or a point's own tangent plane) leaves all on one side."""
    n = len(z)
    cands = [z[i] for i in range(n)]
    for i in range(n):
        for j in range(i + 1, n):
            c = np.cross(z[i], z[j])
            if np.linalg.norm(c) > 0:
                cands += [c, -c]
    return any((z @ u >= -1e-15).all() for u in cands)


def valid_small(n, seed):
    while True:
        z = I.uniform_sphere(n, seed)
        if not in_closed_hemisphere(z):
            return z
        seed += 1000


@pytest.mark.parametrize("n,seed", [(4, 0), (5, 1), (7, 2), (33, 3), (100, 4), (2562, 5), (40962, 6)])
def test_euler_and_cell_closure(n, seed):
    z = valid_small(n, seed) if n < 40 else I.uniform_sphere(n, seed)
    deg, nbr, vx = oracle.voronoi(z)
    assert deg.sum() == 6 * n - 12          # 2E
    assert (deg >= 3).all()
    # each Delaunay edge appears once from each side
    pairs = set()
    for i in range(n):
        assert len(set(nbr[i].tolist())) == len(nbr[i])
        for j in nbr[i]:
            pairs.add((i, int(j)))
    for (i, j) in pairs:
        assert (j, i) in pairs
    assert len(pairs) // 2 == 3 * n - 6
    # corners: distinct Voronoi vertices number 2N - 4
    allv = np.concatenate(vx)
    uniq = np.unique(np.round(allv, 9), axis=0)
    assert len(uniq) == 2 * n - 4


@pytest.mark.parametrize("n,seed", [(50, 10), (600, 11), (2000, 12)])
def test_empty_circumcircle_brute_force(n, seed):
    z = I.uniform_sphere(n, seed)
    deg, nbr, vx = oracle.voronoi(z)
    for i in range(n):
        d = deg[i]
        for t in range(d):
            v = vx[i][t]
            assert abs(np.linalg.norm(v) - 1) < 1e-14
            j_prev, j_next = nbr[i][(t - 1) % d], nbr[i][t]
            di = z[i] @ v
            # equidistant from the three generators of the corner
            assert abs(z[j_prev] @ v - di) < 1e-12
            assert abs(z[j_next] @ v - di) < 1e-12
            # nobody strictly closer (largest dot product = nearest)
            assert (z @ v).max() <= di + 1e-12


def test_neighbours_match_library_hull():
    spatial = pytest.importorskip("scipy.spatial")
    for n, seed in [(2562, 21), (10242, 22)]:
        z = I.uniform_sphere(n, seed)
        deg, nbr, _ = oracle.voronoi(z)
        hull = spatial.ConvexHull(z)
        ref = [set() for _ in range(n)]
        for a, b, c in hull.simplices:
            ref[a] |= {b, c}
            ref[b] |= {a, c}
            ref[c] |= {a, b}
        for i in range(n):
            assert set(nbr[i].tolist()) == ref[i]


@pytest.mark.parametrize("n,d", [(4, 3), (6, 4), (12, 5)])
def test_platonic_degrees(n, d):
    deg, nbr, vx = oracle.voronoi(I.platonic(n))
    assert (deg == d).all()


def test_cube_and_dodecahedron_cover_sphere():
    # degenerate Delaunay faces (squares / pentagons) are triangulated; the
    # cells still tile the sphere
    for n in (8, 20):
        deg, _, _ = oracle.voronoi(I.platonic(n))
        assert deg.sum() == 6 * n - 12


@pytest.mark.parametrize("n", [4, 5, 6, 8])
def test_small_sets_refused_iff_in_hemisphere(n):
    for seed in range(40):
        z = I.uniform_sphere(n, 500 + seed)
        if in_closed_hemisphere(z):
            with pytest.raises(oracle.OracleError):
                oracle.voronoi(z)
        else:
            deg, _, _ = oracle.voronoi(z)
            assert deg.sum() == 6 * n - 12


def test_hemisphere_and_duplicates_refused():
    z = I.uniform_sphere(200, 7)
    z[:, 2] = np.abs(z[:, 2]) + 1e-3
    z /= np.linalg.norm(z, axis=1)[:, None]
    with pytest.raises(oracle.OracleError) as e:
        oracle.voronoi(z)
    assert e.value.code == oracle.DEGENERATE
    z = I.uniform_sphere(50, 8)
    z[10] = z[3]
    with pytest.raises(oracle.OracleError):
        oracle.voronoi(z)


def test_cells_are_counter_clockwise():
    z = I.uniform_sphere(500, 9)
    deg, nbr, vx = oracle.voronoi(z)
    for i in range(500):
        c = vx[i]
        for t in range(deg[i]):
            a, b = c[t], c[(t + 1) % deg[i]]
            # (z_i, a, b) positively oriented seen from outside
            assert np.dot(z[i], np.cross(a, b)) > 0
