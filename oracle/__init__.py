"""FP64 CPU oracle for the spherical CVT path -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It wraps ``scvt_oracle.c`` (plain C, compiled
here with gcc) through ctypes; it shares no code with the CUDA library.

Functions and the passages of the paper they follow:

* ``voronoi``       spherical Voronoi cells (Sec. 2.1) as the dual of the 3D
                    convex hull with exact orientation signs;
* ``energy_grad``   m_i, c_i, F_i, F, g_i = 2(c_i.z_i)z_i - 2c_i,
                    h_i = 1/(2c_i.z_i) (Sec. 2.1, Sec. 3.1) with the signed
                    sub-triangle decomposition of Sec. 3.2.2;
* ``lloyd_step``    z_i <- c_i/|c_i| (Sec. 2.2.1 on S^2);
* ``two_loop``      LBFGS two-loop recursion (Sec. 2.2.2) with diag(h) as the
                    initial inverse Hessian (Sec. 3.1);
* ``line_search``   More-Thuente strong-Wolfe search (the search used by the
                    paper's LBFGS package, Sec. 4);
* ``lbfgs_solve``   Lloyd-preconditioned LBFGS (Sec. 3.1, serial core of the
                    algorithm of Sec. 3.3).

Every function here is pinned by ``tests/test_oracle_*.py`` against closed
forms, brute force and invariants; the solver's trajectory itself is "parity
unpinned" beyond single iterations (many local minima, Sec. 4.1).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "scvt_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, INVALID, DEGENERATE, NOMEM, LINESEARCH = 0, 1, 2, 3, 6


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP over cells)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Density(C.Structure):
    _fields_ = [("kind", C.c_int), ("gamma", C.c_double), ("alpha", C.c_double),
                ("beta", C.c_double), ("xc", C.c_double * 3)]


class _Opts(C.Structure):
    _fields_ = [("max_iter", C.c_int), ("grad_tol", C.c_double), ("rel_grad_tol", C.c_double),
                ("rel_df_tol", C.c_double), ("step_tol", C.c_double), ("ls_max_evals", C.c_int),
                ("c1", C.c_double), ("c2", C.c_double), ("lbfgs_m", C.c_int), ("nthreads", C.c_int),
                ("method", C.c_int)]

METHODS = {"plbfgs": 0, "lbfgs": 1, "lloyd": 2}


class _Report(C.Structure):
    _fields_ = [("iters", C.c_int), ("fevals", C.c_int), ("resets", C.c_int), ("skipped", C.c_int),
                ("energy", C.c_double), ("grad_norm", C.c_double), ("converged", C.c_int),
                ("status", C.c_int)]


PHI_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double))

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            L.orc_orient3d.argtypes = [_dp, _dp, _dp, _dp, C.c_int]
            L.orc_orient3d.restype = C.c_int
            L.orc_voronoi.argtypes = [C.c_int, _dp, _ip, _ip, _dp, C.c_int]
            L.orc_voronoi.restype = C.c_int
            L.orc_rho.argtypes = [C.POINTER(_Density), _dp]
            L.orc_rho.restype = C.c_double
            L.orc_energy_grad.argtypes = [C.c_int, _dp, C.POINTER(_Density), C.c_int, C.c_int, _dp, _dp,
                                          _dp, _dp, _dp, _dp, _dp, _dp, _dp, C.c_int]
            L.orc_energy_grad.restype = C.c_int
            L.orc_lloyd_step.argtypes = [C.c_int, _dp, C.POINTER(_Density), _dp, C.c_int]
            L.orc_lloyd_step.restype = C.c_int
            L.orc_two_loop.argtypes = [C.c_int, _dp, _dp, C.c_int, _dp, _dp, _dp]
            L.orc_two_loop.restype = C.c_int
            L.orc_two_loop_scalar.argtypes = [C.c_int, _dp, C.c_double, C.c_int, _dp, _dp, _dp]
            L.orc_two_loop_scalar.restype = C.c_int
            L.orc_line_search.argtypes = [PHI_FN, C.c_void_p, C.c_double, C.c_double, C.c_double,
                                          C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                          C.c_int, _dp, _dp, _dp, _ip]
            L.orc_line_search.restype = C.c_int
            L.orc_lbfgs_solve.argtypes = [C.c_int, _dp, C.POINTER(_Density), C.POINTER(_Opts),
                                          C.POINTER(_Report), _dp, _dp, _dp, _ip]
            L.orc_lbfgs_solve.restype = C.c_int
            L.orc_bisect.argtypes = [C.c_int, _dp, _dp, C.c_int, _ip]
            L.orc_bisect.restype = C.c_int
            L.orc_mesh_quality.argtypes = [C.c_int, _dp, _dp, _dp, C.c_int, _ip]
            L.orc_mesh_quality.restype = C.c_int
            L.orc_sample_density.argtypes = [C.POINTER(_Density), C.c_double, _dp, _dp, C.c_longlong, C.c_longlong,
                                             _dp]
            L.orc_sample_density.restype = C.c_longlong
            L.orc_max_threads.argtypes = []
            L.orc_max_threads.restype = C.c_int
            _lib = L
    return _lib


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s failed with oracle status %d" % (what, code))
        self.code = code


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _p(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _density(d) -> _Density:
    x = _Density()
    x.kind = int(d.kind)
    x.gamma, x.alpha, x.beta = float(d.gamma), float(d.alpha), float(d.beta)
    for k in range(3):
        x.xc[k] = float(d.xc[k])
    return x


def orient3d(a, b, c, d, exact_only=False) -> int:
    a, b, c, d = (_f64(v, (3,)) for v in (a, b, c, d))
    return lib().orc_orient3d(_p(a), _p(b), _p(c), _p(d), int(bool(exact_only)))


def rho(density, p) -> float:
    p = _f64(p, (3,))
    return lib().orc_rho(C.byref(_density(density)), _p(p))


def voronoi(z):
    """Cells as (deg[n], neighbour lists (CCW), corner coordinates (CCW))."""
    z = _f64(z)
    n = z.shape[0]
    cap = max(6 * n, 16)
    deg = np.zeros(n, dtype=np.int32)
    nbr = np.zeros(cap, dtype=np.int32)
    vx = np.zeros((cap, 3), dtype=np.float64)
    rc = lib().orc_voronoi(n, _p(z), deg.ctypes.data_as(_ip), nbr.ctypes.data_as(_ip), _p(vx), cap)
    if rc != OK:
        raise OracleError(rc, "voronoi")
    off = np.zeros(n + 1, dtype=np.int64)
    off[1:] = np.cumsum(deg)
    return deg, [nbr[off[i]:off[i + 1]].copy() for i in range(n)], [vx[off[i]:off[i + 1]].copy() for i in range(n)]


def voronoi_flat(z):
    """Cells as (deg[n], off[n+1], neighbour ids of all cells end to end, each
    cell's CCW cycle at off[i]:off[i+1]) -- the arrays of ``voronoi`` without
    the per-cell lists, for comparisons at millions of cells."""
    z = _f64(z)
    n = z.shape[0]
    cap = max(6 * n, 16)
    deg = np.zeros(n, dtype=np.int32)
    nbr = np.zeros(cap, dtype=np.int32)
    vx = np.zeros((cap, 3), dtype=np.float64)
    rc = lib().orc_voronoi(n, _p(z), deg.ctypes.data_as(_ip), nbr.ctypes.data_as(_ip), _p(vx), cap)
    if rc != OK:
        raise OracleError(rc, "voronoi")
    off = np.zeros(n + 1, dtype=np.int64)
    off[1:] = np.cumsum(deg)
    return deg, off, nbr[:off[-1]].copy()


def energy_grad(z, density, rule=None, exact_jacobian=False, nthreads=0, fan=False):
    """Evaluate the Sec. 3.1 quantities.  ``rule`` = (bary[nq,3], w[nq]) replaces
    the 7-point rule (weights summing to 1); ``exact_jacobian`` integrates with
    the exact Jacobian of the radial projection instead of area scaling;
    ``fan`` integrates one triangle (z_i, v_a, v_b) per Voronoi edge instead of
    the two sub-triangles through the Delaunay-edge midpoint."""
    z = _f64(z)
    n = z.shape[0]
    F = C.c_double(0.0)
    gn = C.c_double(0.0)
    g = np.zeros((n, 3))
    h = np.zeros(n)
    m = np.zeros(n)
    c = np.zeros((n, 3))
    Fi = np.zeros(n)
    if rule is None:
        mode, nq, qb, qw = 0, 0, None, None
    else:
        qb = _f64(rule[0], (-1, 3))
        qw = _f64(rule[1], (-1,))
        mode, nq = (2 if exact_jacobian else 1), qb.shape[0]
    if fan:
        mode |= 4
    rc = lib().orc_energy_grad(n, _p(z), C.byref(_density(density)), mode, nq, _p(qb), _p(qw),
                               C.byref(F), _p(g), _p(h), _p(m), _p(c), _p(Fi), C.byref(gn), int(nthreads))
    if rc != OK:
        raise OracleError(rc, "energy_grad")
    return {"F": F.value, "g": g, "h": h, "m": m, "c": c, "Fi": Fi, "gnorm": gn.value}


def lloyd_step(z, density, nthreads=0):
    z = _f64(z)
    out = np.zeros_like(z)
    rc = lib().orc_lloyd_step(z.shape[0], _p(z), C.byref(_density(density)), _p(out), int(nthreads))
    if rc != OK:
        raise OracleError(rc, "lloyd_step")
    return out


def two_loop(g, h, S, Y):
    """q = -H g with H0 = diag(h) per generator; S, Y: lists of (n,3) arrays, oldest first."""
    g = _f64(g)
    n = g.shape[0]
    h = _f64(h, (n,))
    mcount = len(S)
    Sa = _f64(np.stack(S) if mcount else np.zeros((1, n, 3)))
    Ya = _f64(np.stack(Y) if mcount else np.zeros((1, n, 3)))
    q = np.zeros_like(g)
    rc = lib().orc_two_loop(n, _p(g), _p(h), mcount, _p(Sa), _p(Ya), _p(q))
    if rc != OK:
        raise OracleError(rc, "two_loop")
    return q


def two_loop_scalar(g, gamma, S, Y):
    """q = -H g with H0 = gamma I (plain LBFGS); S, Y: lists of (n,3) arrays, oldest first."""
    g = _f64(g)
    n = g.shape[0]
    mcount = len(S)
    Sa = _f64(np.stack(S) if mcount else np.zeros((1, n, 3)))
    Ya = _f64(np.stack(Y) if mcount else np.zeros((1, n, 3)))
    q = np.zeros_like(g)
    rc = lib().orc_two_loop_scalar(n, _p(g), C.c_double(float(gamma)), mcount, _p(Sa), _p(Ya), _p(q))
    if rc != OK:
        raise OracleError(rc, "two_loop_scalar")
    return q


def line_search(phi, f0, g0, stp0=1.0, ftol=1e-4, gtol=0.9, xtol=1e-16, stpmin=1e-20, stpmax=1e20, maxfev=10):
    """More-Thuente search on a Python callable phi(a) -> (f, f'), or None
    when the trial point is not valid (the search then halves the step)."""
    calls = []

    def cb(_ctx, a, fp, gp):
        r = phi(a)
        if r is None:
            calls.append((a, None, None))
            return 2
        f, g = r
        calls.append((a, f, g))
        fp[0] = f
        gp[0] = g
        return 0

    cfn = PHI_FN(cb)
    stp, f, g, nfev = C.c_double(), C.c_double(), C.c_double(), C.c_int()
    info = lib().orc_line_search(cfn, None, f0, g0, stp0, ftol, gtol, xtol, stpmin, stpmax, maxfev,
                                 C.byref(stp), C.byref(f), C.byref(g), C.byref(nfev))
    return {"info": info, "stp": stp.value, "f": f.value, "g": g.value, "nfev": nfev.value, "calls": calls}


def lbfgs_solve(z, density, lbfgs_m=5, max_iter=200, grad_tol=1e-8, rel_grad_tol=0.0, rel_df_tol=0.0,
                step_tol=0.0, ls_max_evals=10, c1=1e-4, c2=0.9, nthreads=0, method="plbfgs"):
    """Solve from z with method "plbfgs" (Lloyd-preconditioned LBFGS), "lbfgs"
    (H0 = gamma_n I) or "lloyd"; returns (z_final, report, trace)."""
    z = _f64(z).copy()
    n = z.shape[0]
    o = _Opts(int(max_iter), float(grad_tol), float(rel_grad_tol), float(rel_df_tol), float(step_tol),
              int(ls_max_evals), float(c1), float(c2), int(lbfgs_m), int(nthreads), METHODS[method])
    rep = _Report()
    k = max(int(max_iter), 1)
    trF, trg, tra = np.zeros(k), np.zeros(k), np.zeros(k)
    trn = np.zeros(k, dtype=np.int32)
    rc = lib().orc_lbfgs_solve(n, _p(z), C.byref(_density(density)), C.byref(o), C.byref(rep),
                               _p(trF), _p(trg), _p(tra), trn.ctypes.data_as(_ip))
    report = {f: getattr(rep, f) for f, _ in _Report._fields_}
    it = rep.iters
    trace = {"F": trF[:it], "gnorm": trg[:it], "alpha": tra[:it], "nfev": trn[:it]}
    # a line search that cannot decrease F any more (rounding floor) ends the
    # solve with report["status"] == LINESEARCH and the last accepted iterate
    if rc not in (OK, LINESEARCH):
        raise OracleError(rc, "lbfgs_solve")
    return z, report, trace


def bisect(z):
    """Bisection refinement: z followed by the Delaunay-edge midpoints (i < j, lexicographic)."""
    z = _f64(z)
    n = z.shape[0]
    cap = 4 * n
    out = np.zeros((cap, 3))
    k = C.c_int()
    rc = lib().orc_bisect(n, _p(z), _p(out), cap, C.byref(k))
    if rc != OK:
        raise OracleError(rc, "bisect")
    return out[:k.value]


def mesh_quality(z):
    """(cellQ per generator, triQ per Delaunay triangle in sorted-triple order)."""
    z = _f64(z)
    n = z.shape[0]
    cq = np.zeros(n)
    tq = np.zeros(2 * n)
    k = C.c_int()
    rc = lib().orc_mesh_quality(n, _p(z), _p(cq), _p(tq), 2 * n, C.byref(k))
    if rc != OK:
        raise OracleError(rc, "mesh_quality")
    return cq, tq[:k.value]


def sample_density(density, cand, u, n_target, exponent=1.0):
    """Monte Carlo initialisation: the first n_target candidates with
    u_k rho_max^e <= rho(cand_k)^e, in order."""
    cand = _f64(cand)
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros((int(n_target), 3))
    k = lib().orc_sample_density(C.byref(_density(density)), float(exponent), _p(cand), _p(u), len(u),
                                 int(n_target), _p(out))
    return out[:k]


def max_threads() -> int:
    return lib().orc_max_threads()
