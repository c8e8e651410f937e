"""Seeded synthetic inputs for the spherical CVT workloads.

This module only *generates inputs*: generator sets on the unit sphere and the
parameters of the analytic point densities.  It holds none of the method's
arithmetic (no Voronoi construction, no quadrature, no density evaluation), so
that the CPU oracle and the CUDA path can both draw their inputs from it
without sharing any computation.

Input recipe (the paper's workloads are analytic densities on S^2, Sec. 4):

* generators: three independent standard normals per point from numpy's PCG64
  (``numpy.random.default_rng(seed)``), triples of norm < 1e-3 are redrawn,
  then each triple is scaled to unit length;
* densities: the X3 polar density (Sec. 4, X3 definition) and the tanh cap
  density of Sec. 4 (X64 definition, prefactor read as (1-gamma)/2), with the
  parameters of the workloads listed in ``WORKLOADS``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# density kinds (same numbering on both sides of the boundary)
RHO_UNIFORM = 0
RHO_POLAR_X3 = 1
RHO_TANH_CAP = 2
RHO_TANH_CAP_POW4 = 3


@dataclass(frozen=True)
class Density:
    kind: int = RHO_UNIFORM
    gamma: float = 1.0
    alpha: float = 1.0
    beta: float = 0.0
    xc: tuple = (0.0, 0.0, 1.0)


def latlon_to_xyz(lat_deg: float, lon_deg: float) -> tuple:
    """Unit vector at latitude/longitude (degrees); components below 1e-15 are
    snapped to exact zero so that e.g. 270 deg E gives x == 0 exactly."""
    la, lo = math.radians(lat_deg), math.radians(lon_deg)
    v = [math.cos(la) * math.cos(lo), math.cos(la) * math.sin(lo), math.sin(la)]
    v = [0.0 if abs(c) < 1e-15 else c for c in v]
    return tuple(v)


def mc_candidates(m: int, seed: int):
    """Inputs of the Monte Carlo initialisation: m candidate points uniform on
    S^2 and m acceptance variates uniform on [0, 1) (seeded)."""
    cand = uniform_sphere(m, seed)
    u = np.random.default_rng(seed + 7919).random(m)
    return cand, u


def uniform_sphere(n: int, seed: int) -> np.ndarray:
    """n points uniform on S^2 as a contiguous (n, 3) float64 array."""
    if n < 0:
        raise ValueError("n must be >= 0")
    rng = np.random.default_rng(seed)
    out = np.empty((n, 3), dtype=np.float64)
    filled = 0
    while filled < n:
        want = n - filled
        x = rng.standard_normal((want, 3))
        r = np.sqrt((x * x).sum(axis=1))
        ok = r >= 1e-3
        x = x[ok] / r[ok, None]
        out[filled:filled + len(x)] = x
        filled += len(x)
    return np.ascontiguousarray(out)


def uniform_sphere_device(n: int, seed: int, device):
    """n points uniform on S^2 drawn on a CUDA device (torch's Philox generator
    seeded with `seed`): three standard normals per point, scaled to unit
    length (the recipe of uniform_sphere, another generator).  For request
    streams of millions of generators per job, where drawing on the host
    would set the pace; nothing drawn here is compared with the oracle."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    x = torch.randn((n, 3), generator=gen, device=device, dtype=torch.float64)
    r = torch.linalg.vector_norm(x, dim=1, keepdim=True)
    bad = (r < 1e-3).squeeze(1)
    while bool(bad.any()):
        x[bad] = torch.randn((int(bad.sum()), 3), generator=gen, device=device, dtype=torch.float64)
        r = torch.linalg.vector_norm(x, dim=1, keepdim=True)
        bad = (r < 1e-3).squeeze(1)
    return (x / r).contiguous()


def _unit_rows(p) -> np.ndarray:
    p = np.asarray(p, dtype=np.float64)
    return np.ascontiguousarray(p / np.sqrt((p * p).sum(axis=1))[:, None])


def platonic(n: int) -> np.ndarray:
    """Vertices of the Platonic solid with n vertices (4, 6, 8, 12, 20) on S^2."""
    if n == 4:
        p = [(1, 1, 1), (1, -1, -1), (-1, 1, -1), (-1, -1, 1)]
    elif n == 6:
        p = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    elif n == 8:
        p = [(sx, sy, sz) for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)]
    elif n == 12:
        t = (1 + math.sqrt(5)) / 2
        p = []
        for a in (-1, 1):
            for b in (-t, t):
                p += [(0, a, b), (a, b, 0), (b, 0, a)]
    elif n == 20:
        t = (1 + math.sqrt(5)) / 2
        p = [(sx, sy, sz) for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)]
        for a in (-1 / t, 1 / t):
            for b in (-t, t):
                p += [(0, a, b), (a, b, 0), (b, 0, a)]
    else:
        raise ValueError("no Platonic solid with %d vertices" % n)
    return _unit_rows(p)


def icosahedral_grid(level: int) -> np.ndarray:
    """Recursively bisected icosahedron (10*4^level + 2 points): the
    bisection refinement used to build initial meshes (Sec. 4.3): every edge
    midpoint of the triangulation is added and scaled to the sphere.  Returned
    in a deterministic order."""
    t = (1 + math.sqrt(5)) / 2
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
             (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [tuple(np.array(v, float) / np.linalg.norm(v)) for v in verts]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9),
             (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2),
             (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10),
             (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        cache = {}
        nf = []

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = np.array(verts[a]) + np.array(verts[b])
                verts.append(tuple(m / np.linalg.norm(m)))
                cache[key] = len(verts) - 1
            return cache[key]

        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    return np.ascontiguousarray(np.array(verts, dtype=np.float64))


# --- densities ---------------------------------------------------------------

def density_uniform() -> Density:
    return Density(RHO_UNIFORM, 1.0, 1.0, 0.0, (0.0, 0.0, 1.0))


def density_x3() -> Density:
    """X3 polar density of Sec. 4: gamma = (1/3)^4."""
    return Density(RHO_POLAR_X3, (1.0 / 3.0) ** 4, 1.0, 0.0, (0.0, 0.0, 1.0))


def density_x64() -> Density:
    """X64 tanh cap of Sec. 4: z_c = (0, -cos 30deg, sin 30deg), beta = pi/6,
    alpha = 0.15, gamma = (1/64)^4."""
    return Density(RHO_TANH_CAP, (1.0 / 64.0) ** 4, 0.15, math.pi / 6,
                   latlon_to_xyz(30.0, 270.0))


def density_tanh(gamma: float, alpha: float, beta: float, xc) -> Density:
    xc = np.asarray(xc, dtype=np.float64)
    xc = xc / np.linalg.norm(xc)
    return Density(RHO_TANH_CAP, float(gamma), float(alpha), float(beta), tuple(float(v) for v in xc))


@dataclass(frozen=True)
class Workload:
    name: str
    n: int
    density: Density
    lbfgs_m: int
    grad_tol: float
    max_iter: int
    seeds: tuple = (0,)


WORKLOADS = {
    # 2,562 generators, rho == 1, m = 5, 200 iterations or ||g|| <= 1e-8
    "uniform-2562": Workload("uniform-2562", 2562, density_uniform(), 5, 1e-8, 200,
                             tuple(range(10))),
    # 163,842 generators, tanh cap at 30N 0E, alpha 0.15, beta pi/6, gamma (1/4)^4
    "tanh-163842": Workload("tanh-163842", 163842,
                            density_tanh((1 / 4) ** 4, 0.15, math.pi / 6, latlon_to_xyz(30, 0)),
                            7, 1e-7, 10**6, (0, 1, 2)),
    # 2,621,442 generators, tanh cap at 45N 270E, alpha 0.10, beta pi/9, gamma (1/8)^4
    "tanh-2621442": Workload("tanh-2621442", 2621442,
                             density_tanh((1 / 8) ** 4, 0.10, math.pi / 9, latlon_to_xyz(45, 270)),
                             7, 1e-6, 10**6, (0,)),
}


def sample_batched_instances(count: int, seed: int, n_lo: int = 10242, n_hi: int = 655362):
    """Sampler for many independent instances: N log-uniform in [n_lo, n_hi],
    tanh caps with x_c uniform on S^2, gamma^(1/4) ~ U[1/16, 1/2],
    alpha ~ U[0.05, 0.2], beta ~ U[pi/12, pi/4]."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        x = rng.standard_normal(3)
        x /= np.linalg.norm(x)
        g4 = rng.uniform(1 / 16, 1 / 2)
        d = density_tanh(g4 ** 4, rng.uniform(0.05, 0.2), rng.uniform(math.pi / 12, math.pi / 4), x)
        out.append((n, d, int(rng.integers(0, 2**31 - 1))))
    return out
