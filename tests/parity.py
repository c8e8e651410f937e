"""Comparison helpers for the CUDA-vs-oracle parity tests.

Tolerance (FP64 mode): 1e-12 relative.  Both sides evaluate the same
definitions in double precision with different formulas for the Voronoi
vertices (gnomonic line intersection vs. hull-facet normal) and different
summation orders; each vertex is then accurate to ~1e-16 absolute, which
moves a sub-triangle integral by ~1e-16/h relative (h = cell size, >= 1e-3
for N <= 2.6M), i.e. <= 1e-13.  The gradient g_i = 2(c.z)z - 2c cancels, so
it is compared relative to |c_i|, the scale of its terms.
"""
import numpy as np

RTOL = 1e-12


def canon(lst):
    """Rotate a cyclic neighbour list to start at its smallest id."""
    lst = [int(x) for x in lst]
    k = int(np.argmin(lst))
    return lst[k:] + lst[:k]


def assert_topology_equal(deg_gpu, nbr_gpu, nbr_orc):
    n = len(nbr_orc)
    assert len(deg_gpu) == n
    bad = [i for i in range(n) if canon(nbr_gpu[i, :deg_gpu[i]]) != canon(nbr_orc[i])]
    assert not bad, "cells with different neighbour cycles: %s (first: gpu %s oracle %s)" % (
        bad[:10], canon(nbr_gpu[bad[0], :deg_gpu[bad[0]]]), canon(nbr_orc[bad[0]]))


def canon_rows(deg, nbr):
    """Each row's first deg[i] entries rotated to start at their smallest id
    (vectorised canon); entries past deg[i] are -1."""
    deg = np.asarray(deg, dtype=np.int64)
    n = len(deg)
    w = int(deg.max()) if n else 0
    nbr = np.asarray(nbr)[:, :w].astype(np.int64)
    cols = np.arange(w)[None, :]
    valid = cols < deg[:, None]
    big = np.iinfo(np.int64).max
    k = np.where(valid, nbr, big).argmin(axis=1)
    src = (k[:, None] + cols) % np.maximum(deg, 1)[:, None]
    out = np.take_along_axis(nbr, src, axis=1)
    return np.where(valid, out, -1)


def pad_flat(deg, off, flat):
    """Flat neighbour lists (cell i at flat[off[i]:off[i+1]]) as a padded
    (n, max deg) array, -1 past each row's degree."""
    deg = np.asarray(deg, dtype=np.int64)
    n = len(deg)
    w = int(deg.max()) if n else 0
    out = np.full((n, w), -1, dtype=np.int64)
    rows = np.repeat(np.arange(n), deg)
    cols = np.arange(int(off[-1])) - np.repeat(np.asarray(off[:-1], dtype=np.int64), deg)
    out[rows, cols] = flat
    return out


def assert_topology_equal_all(deg_gpu, nbr_gpu, deg_orc, off_orc, flat_orc):
    """Every cell's neighbour cycle equal up to rotation (vectorised over
    millions of cells)."""
    deg_gpu = np.asarray(deg_gpu)
    bad_deg = np.nonzero(deg_gpu != np.asarray(deg_orc))[0]
    assert len(bad_deg) == 0, "cells with different degrees: %s" % bad_deg[:10]
    a = canon_rows(deg_gpu, nbr_gpu)
    b = canon_rows(deg_orc, pad_flat(deg_orc, off_orc, flat_orc))
    bad = np.nonzero((a != b).any(axis=1))[0]
    assert len(bad) == 0, "cells with different neighbour cycles: %s (first: gpu %s oracle %s)" % (
        bad[:10], a[bad[0]], b[bad[0]])


def rel_err(a, b, scale):
    return np.max(np.abs(a - b) / scale)


def assert_geometry_close(gpu, orc, rtol=RTOL, idx=None):
    sel = slice(None) if idx is None else idx
    m_o = orc["m"][sel]
    c_o = orc["c"][sel]
    cn = np.linalg.norm(c_o, axis=1)
    errs = {
        "m": rel_err(gpu["mass"][sel], m_o, m_o),
        "c": rel_err(gpu["moment"][sel], c_o, cn[:, None]),
        "F_i": rel_err(gpu["cell_energy"][sel], orc["Fi"][sel], orc["Fi"][sel]),
        "g": rel_err(gpu["grad"][sel], orc["g"][sel], cn[:, None]),
        "h": rel_err(gpu["precond"][sel], orc["h"][sel], orc["h"][sel]),
    }
    worst = max(errs.values())
    assert worst <= rtol, errs
    return errs


# Mixed form (precision = 1): per-quantity bounds against the FP64 oracle (the
# arithmetic behind them is stated in tests/test_gpu_mixed.py)
MIXED_BOUNDS = {"m": 1e-5, "c": 1e-5, "F_i": 2e-5, "g": 1e-6, "h": 1e-5, "F": 2e-6, "gnorm": 2e-6}


def mixed_errors(r, o):
    """Worst per-cell relative errors of a GPU evaluation r against the oracle
    o: m_i, c_i (per component, relative to |c_i|), F_i, g_i (relative to
    |c_i|), h_i, and the totals F, ||g||."""
    cn = np.linalg.norm(o["c"], axis=1)
    return {
        "m": float(np.max(np.abs(r["mass"] - o["m"]) / o["m"])),
        "c": float(np.max(np.abs(r["moment"] - o["c"]).max(axis=1) / cn)),
        "F_i": float(np.max(np.abs(r["cell_energy"] - o["Fi"]) / o["Fi"])),
        "g": float(np.max(np.abs(r["grad"] - o["g"]).max(axis=1) / cn)),
        "h": float(np.max(np.abs(r["precond"] - o["h"]) / o["h"])),
        "F": abs(r["energy"] - o["F"]) / o["F"],
        "gnorm": abs(r["grad_norm"] - o["gnorm"]) / o["gnorm"],
    }


def assert_mixed_within_bounds(r, o):
    err = mixed_errors(r, o)
    for k, v in err.items():
        assert v <= MIXED_BOUNDS[k], (k, v, err)
    return err

