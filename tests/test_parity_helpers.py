"""The vectorised topology comparison used by the full-size parity tests,
checked on the CPU against the per-cell comparison (rotation invariance,
and that a swapped pair, a reversed cycle or a changed degree is caught)."""
import numpy as np
import pytest

import oracle
from paper_1709_06924_gb300 import inputs as I
from tests.parity import assert_topology_equal, assert_topology_equal_all, canon, canon_rows


def _flat(lists):
    deg = np.array([len(x) for x in lists], dtype=np.int32)
    off = np.zeros(len(lists) + 1, dtype=np.int64)
    off[1:] = np.cumsum(deg)
    flat = np.concatenate([np.asarray(x, dtype=np.int32) for x in lists])
    return deg, off, flat


def _padded(lists, rng, width=12):
    out = np.full((len(lists), width), 777, dtype=np.int32)  # junk past the degree
    for i, x in enumerate(lists):
        k = int(rng.integers(len(x)))
        out[i, :len(x)] = np.roll(np.asarray(x), -k)  # any rotation
    return out


def test_canon_rows_matches_canon():
    rng = np.random.default_rng(0)
    lists = [list(rng.permutation(50)[:int(rng.integers(3, 12))]) for _ in range(300)]
    deg = np.array([len(x) for x in lists])
    rows = canon_rows(deg, _padded(lists, rng))
    for i, x in enumerate(lists):
        assert list(rows[i, :deg[i]]) == canon(x)
        assert (rows[i, deg[i]:] == -1).all()


def test_all_cells_comparison_accepts_rotations_and_catches_changes():
    z = I.uniform_sphere(500, 3)
    _, lists, _ = oracle.voronoi(z)
    deg, off, flat = oracle.voronoi_flat(z)
    assert [list(flat[off[i]:off[i + 1]]) for i in range(len(z))] == [list(x) for x in lists]
    rng = np.random.default_rng(1)
    gpu = _padded(lists, rng)
    assert_topology_equal_all(deg, gpu, deg, off, flat)
    assert_topology_equal(deg, gpu, lists)
    swapped = gpu.copy()
    swapped[7, [0, 1]] = swapped[7, [1, 0]]
    with pytest.raises(AssertionError):
        assert_topology_equal_all(deg, swapped, deg, off, flat)
    rev = gpu.copy()
    rev[11, :deg[11]] = rev[11, :deg[11]][::-1]
    with pytest.raises(AssertionError):
        assert_topology_equal_all(deg, rev, deg, off, flat)
    d2 = deg.copy()
    d2[5] -= 1
    with pytest.raises(AssertionError):
        assert_topology_equal_all(d2, gpu, deg, off, flat)
