"""Independent reference quantities used to pin the oracle (no oracle code).

* conical-product (Duffy) Gauss rules on a triangle from numpy's Gauss-Legendre
  nodes -- no stored quadrature tables;
* closed-form integrals over a spherical polygon for rho == 1: the area from the
  Van Oosterom-Strackee triangle formula and the first moment from Stokes'
  theorem, int_P y dsigma = 1/2 sum_edges theta_pq (p x q)/|p x q|;
* one-dimensional reductions of int_{S^2} sqrt(rho) for zonal densities
  (Archimedes: dsigma = dz dphi on the unit sphere).
"""
import math

import numpy as np


def conical_rule(n):
    """n*n-point rule on the triangle: barycentric points and weights summing to 1."""
    x, w = np.polynomial.legendre.leggauss(n)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    pts, wts = [], []
    for i in range(n):
        for j in range(n):
            u, v = x[i], x[j]
            l1 = u
            l2 = v * (1.0 - u)
            pts.append((1.0 - l1 - l2, l1, l2))
            wts.append(2.0 * w[i] * w[j] * (1.0 - u))
    return np.array(pts), np.array(wts)


def _tri_area(a, b, c):
    det = np.dot(a, np.cross(b - a, c - a))
    den = 1.0 + a @ b + b @ c + c @ a
    return 2.0 * math.atan2(det, den)


def polygon_area(zi, corners):
    d = len(corners)
    return sum(_tri_area(zi, corners[t], corners[(t + 1) % d]) for t in range(d))


def polygon_first_moment(corners):
    """int_P y dsigma for a CCW spherical polygon (rho == 1), Stokes' theorem."""
    d = len(corners)
    c = np.zeros(3)
    for t in range(d):
        p, q = corners[t], corners[(t + 1) % d]
        cr = np.cross(p, q)
        s = np.linalg.norm(cr)
        if s == 0.0:
            continue
        theta = math.atan2(s, p @ q)
        c += 0.5 * theta * cr / s
    return c


def zonal_integral(f_of_cos, n=4000):
    """int_{S^2} f(x . e) dsigma = 2 pi int_{-1}^{1} f(t) dt (Gauss-Legendre)."""
    t, w = np.polynomial.legendre.leggauss(n)
    return 2.0 * math.pi * float(np.sum(w * f_of_cos(t)))


HEX_G = 5.0 / (18.0 * math.sqrt(3.0))  # normalised second moment of the regular hexagon
