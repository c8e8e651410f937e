"""Pins for the oracle's exact orientation predicate: the sign of
det[a-d; b-d; c-d] must equal the sign of the same determinant in exact
rational arithmetic (Python Fractions), including exactly degenerate and
one-ulp-perturbed configurations."""
from fractions import Fraction

import numpy as np
import pytest

import oracle


def exact_sign(a, b, c, d):
    A = [[Fraction(x) - Fraction(y) for x, y in zip(p, d)] for p in (a, b, c)]
    det = (A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
           - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
           + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]))
    return (det > 0) - (det < 0)


def test_random_quadruples():
    rng = np.random.default_rng(1)
    for _ in range(300):
        p = rng.standard_normal((4, 3))
        s = exact_sign(*p)
        assert oracle.orient3d(*p) == s
        assert oracle.orient3d(*p, exact_only=True) == s


def test_coplanar_and_ulp_perturbations():
    rng = np.random.default_rng(2)
    for _ in range(200):
        # four points on one circle of latitude (exactly in the plane
        # z = 0.25), then one z nudged by one ulp either way.  (The expansion
        # arithmetic is exact as long as no product underflows, the standing
        # assumption of Shewchuk's method; unit-sphere inputs are far from it.)
        ang = rng.uniform(0, 2 * np.pi, 4)
        p = np.stack([np.cos(ang), np.sin(ang), np.full(4, 0.25)], axis=1)
        assert exact_sign(*p) == 0
        assert oracle.orient3d(*p) == 0
        q = p.copy()
        k = rng.integers(0, 4)
        q[k, 2] = np.nextafter(0.25, 1.0) if rng.random() < 0.5 else np.nextafter(0.25, 0.0)
        assert exact_sign(*q) != 0
        assert oracle.orient3d(*q) == exact_sign(*q)
        # tilted plane: tiny relative perturbations of near-coplanar points
        r = rng.standard_normal((4, 3))
        n = rng.standard_normal(3)
        r -= np.outer(r @ n, n) / (n @ n)
        r[rng.integers(0, 4)] *= (1 + 2.0 ** -52)
        assert oracle.orient3d(*r) == exact_sign(*r)
        assert oracle.orient3d(*r, exact_only=True) == exact_sign(*r)


@pytest.mark.parametrize("scale", [1.0, 1e-8, 1e8])
def test_scaled_inputs(scale):
    rng = np.random.default_rng(3)
    for _ in range(50):
        p = rng.standard_normal((4, 3)) * scale
        assert oracle.orient3d(*p) == exact_sign(*p)
