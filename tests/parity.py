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
