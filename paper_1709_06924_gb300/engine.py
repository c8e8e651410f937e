"""Convenience wrapper over the C ABI for PyTorch users.

Tensors supply device memory and the CUDA stream only; every step of the
computation runs in the CUDA library.  Arrays are float64, contiguous,
shaped (N, 3) for points and vectors and (N,) for per-point scalars.
Numpy arrays (host memory) are accepted too: the library stages them.
"""
from __future__ import annotations

import numpy as np
import torch

from . import capi
from .inputs import Density


METHODS = {"plbfgs": 0, "lbfgs": 1, "lloyd": 2}


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError("expected a torch.Tensor or numpy.ndarray")


def _density(d: Density) -> capi.scvt_density:
    r = capi.scvt_density()
    r.kind, r.gamma, r.alpha, r.beta = int(d.kind), float(d.gamma), float(d.alpha), float(d.beta)
    for k in range(3):
        r.xc[k] = float(d.xc[k])
    return r


class Engine:
    def __init__(self, n: int, density: Density, lbfgs_m: int = 7, knn_k0: int = 0,
                 device: int | torch.device = 0, stream: torch.cuda.Stream | None = None, precision: int = 0,
                 decomposition: int = 0):
        """precision: 0 = FP64 form (double-float corners and rule points relative to z_i,
        results within 1e-12 of FP64), 1 = mixed (FP32 corners and quadrature in local
        coordinates, FP64 predicates filter, sums and LBFGS), 2 = plain FP64 arithmetic.  decomposition: 0 = the
        paper's sub-triangles through the Delaunay-edge midpoints, 1 = the fan."""
        self.n = int(n)
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        cfg = capi.scvt_config()
        cfg.n = self.n
        cfg.rho = _density(density)
        cfg.quad_points = 7
        cfg.precision = int(precision)
        cfg.lbfgs_m = int(lbfgs_m)
        cfg.knn_k0 = int(knn_k0)
        cfg.knn_kmax = 0
        cfg.decomposition = int(decomposition)
        with torch.cuda.device(self.device):
            self._h = capi.scvt_create(cfg, self.stream.cuda_stream)

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            capi.scvt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _sync_inputs(self):
        # inputs written on torch's current stream must be visible on ours
        self.stream.wait_stream(torch.cuda.current_stream(self.device))

    def _tensor(self, *shape, dtype=torch.float64):
        return torch.empty(*shape, dtype=dtype, device=self.device)

    # -- entry points
    def energy_grad(self, z):
        g = self._tensor(self.n, 3)
        m = self._tensor(self.n)
        c = self._tensor(self.n, 3)
        self._sync_inputs()
        F = capi.scvt_energy_grad(self._h, _ptr(z), g.data_ptr(), m.data_ptr(), c.data_ptr())
        torch.cuda.current_stream(self.device).wait_stream(self.stream)
        return F, g, m, c

    def evaluate(self, z):
        """All per-cell outputs of one evaluation as tensors."""
        out = {k: self._tensor(self.n, 3) if k in ("grad", "moment") else self._tensor(self.n)
               for k in ("grad", "precond", "mass", "moment", "cell_energy")}
        self._sync_inputs()
        o = capi.scvt_eval_out()
        for k, t in out.items():
            setattr(o, k, t.data_ptr())
        capi.scvt_evaluate(self._h, _ptr(z), o)
        torch.cuda.current_stream(self.device).wait_stream(self.stream)
        out["energy"] = o.energy
        out["grad_norm"] = o.grad_norm
        return out

    def lloyd_step(self, z, out=None):
        if out is None:
            out = self._tensor(self.n, 3) if isinstance(z, torch.Tensor) else np.empty((self.n, 3))
        self._sync_inputs()
        capi.scvt_lloyd_step(self._h, _ptr(z), _ptr(out))
        torch.cuda.current_stream(self.device).wait_stream(self.stream)
        return out

    def lbfgs_solve(self, z, max_iter=200, grad_tol=1e-8, rel_grad_tol=0.0, rel_df_tol=0.0, step_tol=0.0,
                    ls_max_evals=10, c1=1e-4, c2=0.9, warm_start=False, method="plbfgs"):
        """In-place solve on z; returns the report as a dict.  method: "plbfgs"
        (Lloyd-preconditioned LBFGS), "lbfgs" (H0 = gamma_n I) or "lloyd"."""
        self._sync_inputs()
        o = capi.scvt_solve_opts(int(max_iter), float(grad_tol), float(rel_grad_tol), float(rel_df_tol),
                                 float(step_tol), int(ls_max_evals), float(c1), float(c2), int(warm_start),
                                 METHODS[method])
        rep = capi.scvt_lbfgs_solve(self._h, _ptr(z), o)
        torch.cuda.current_stream(self.device).wait_stream(self.stream)
        return {f: getattr(rep, f) for f, _ in capi.scvt_solve_report._fields_}

    def voronoi(self, z, max_deg=32):
        deg = self._tensor(self.n, dtype=torch.int32)
        nbr = torch.full((self.n, max_deg), -1, dtype=torch.int32, device=self.device)
        self._sync_inputs()
        capi.scvt_voronoi(self._h, _ptr(z), deg.data_ptr(), nbr.data_ptr(), max_deg)
        torch.cuda.current_stream(self.device).wait_stream(self.stream)
        return deg, nbr

    def lbfgs_direction(self, g, hdiag, S, Y):
        """q = -H g; S, Y: tensors (count, N, 3), oldest pair first."""
        q = self._tensor(self.n, 3)
        self._sync_inputs()
        count = 0 if S is None else int(S.shape[0])
        capi.scvt_lbfgs_direction(self._h, _ptr(g), _ptr(hdiag), count, _ptr(S) if count else None,
                                  _ptr(Y) if count else None, q.data_ptr())
        torch.cuda.current_stream(self.device).wait_stream(self.stream)
        return q

    def stats(self):
        s = capi.scvt_get_stats(self._h)
        return {f: getattr(s, f) for f, _ in capi.scvt_stats._fields_}

    def reset_stats(self):
        capi.scvt_reset_stats(self._h)

    def set_profiling(self, on=True):
        capi.scvt_set_profiling(self._h, on)

    def bisect(self, z):
        """Bisection refinement: z followed by its Delaunay-edge midpoints (i < j, lexicographic)."""
        out = self._tensor(4 * self.n, 3)
        self._sync_inputs()
        k = capi.scvt_bisect(self._h, _ptr(z), out.data_ptr(), 4 * self.n)
        torch.cuda.current_stream(self.device).wait_stream(self.stream)
        return out[:k]

    def mesh_quality(self, z):
        """(cellQ per generator, triQ per Delaunay triangle in lexicographic order)."""
        cq = self._tensor(self.n)
        tq = self._tensor(2 * self.n)
        self._sync_inputs()
        k = capi.scvt_mesh_quality(self._h, _ptr(z), cq.data_ptr(), tq.data_ptr(), 2 * self.n)
        torch.cuda.current_stream(self.device).wait_stream(self.stream)
        return cq, tq[:k]

    def set_tuning(self, **kw):
        """Launch shape / search parameters (results do not depend on them)."""
        t = capi.scvt_get_tuning(self._h)
        for k, v in kw.items():
            setattr(t, k, int(v))
        capi.scvt_set_tuning(self._h, t)

    def tuning(self):
        t = capi.scvt_get_tuning(self._h)
        return {f: getattr(t, f) for f, _ in capi.scvt_tuning._fields_}

    def tune(self, z):
        """Run the autotuner on evaluations at z; returns the chosen tuning."""
        self._sync_inputs()
        t = capi.scvt_tune(self._h, _ptr(z))
        return {f: getattr(t, f) for f, _ in capi.scvt_tuning._fields_}


def _config(n, density, lbfgs_m, precision, decomposition=0):
    cfg = capi.scvt_config()
    cfg.n = int(n)
    cfg.rho = _density(density)
    cfg.quad_points = 7
    cfg.precision = int(precision)
    cfg.lbfgs_m = int(lbfgs_m)
    cfg.knn_k0 = 0
    cfg.knn_kmax = 0
    cfg.decomposition = int(decomposition)
    return cfg


class Batch:
    """Independent problems (sizes ns, densities) solved together.

    Points of problem b are rows offsets[b]:offsets[b+1] of one (N_tot, 3)
    array; use split() / concat() to move between the two views."""

    def __init__(self, ns, densities, lbfgs_m: int = 7, precision: int = 0, device: int | torch.device = 0,
                 decomposition: int = 0):
        if len(ns) != len(densities):
            raise ValueError("one density per problem")
        self.ns = [int(n) for n in ns]
        self.count = len(self.ns)
        self.offsets = np.concatenate([[0], np.cumsum(self.ns)]).astype(np.int64)
        self.ntot = int(self.offsets[-1])
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        cfgs = [_config(n, d, lbfgs_m, precision, decomposition) for n, d in zip(self.ns, densities)]
        with torch.cuda.device(self.device):
            self._b = capi.scvt_batch_create(cfgs, torch.cuda.current_stream(self.device).cuda_stream)

    def close(self):
        if getattr(self, "_b", None):
            capi.scvt_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def concat(self, zs):
        if isinstance(zs[0], torch.Tensor):
            return torch.cat([z.to(self.device) for z in zs]).contiguous()
        return np.ascontiguousarray(np.concatenate(zs))

    def split(self, z):
        return [z[self.offsets[b]:self.offsets[b + 1]] for b in range(self.count)]

    def energy_grad(self, z):
        g = torch.empty((self.ntot, 3), dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            e = capi.scvt_batch_energy_grad(self._b, _ptr(z), self.count, g.data_ptr())
        return e, g

    def lbfgs_solve(self, z, max_iter=200, grad_tol=1e-8, rel_grad_tol=0.0, rel_df_tol=0.0, step_tol=0.0,
                    ls_max_evals=10, c1=1e-4, c2=0.9, warm_start=0, method="plbfgs"):
        o = capi.scvt_solve_opts(int(max_iter), float(grad_tol), float(rel_grad_tol), float(rel_df_tol),
                                 float(step_tol), int(ls_max_evals), float(c1), float(c2), int(warm_start),
                                 METHODS[method])
        with torch.cuda.device(self.device):
            reps = capi.scvt_batch_lbfgs_solve(self._b, _ptr(z), o, self.count)
        return [{f: getattr(r, f) for f, _ in capi.scvt_solve_report._fields_} for r in reps]

    def tune(self, z):
        with torch.cuda.device(self.device):
            t = capi.scvt_batch_tune(self._b, _ptr(z))
        return {f: getattr(t, f) for f, _ in capi.scvt_tuning._fields_}

    def set_tuning(self, **kw):
        t = capi.scvt_batch_get_tuning(self._b)
        for k, v in kw.items():
            setattr(t, k, int(v))
        capi.scvt_batch_set_tuning(self._b, t)

    def tuning(self):
        t = capi.scvt_batch_get_tuning(self._b)
        return {f: getattr(t, f) for f, _ in capi.scvt_tuning._fields_}

    def stats(self):
        s = capi.scvt_batch_get_stats(self._b)
        return {f: getattr(s, f) for f, _ in capi.scvt_stats._fields_}

    def reset_stats(self):
        capi.scvt_batch_reset_stats(self._b)


class Server:
    """Continuous-batching request loop: submit jobs, step, read and fetch results."""

    def __init__(self, max_generators: int, max_jobs: int, memory_budget: int = 0, precision: int = 0,
                 lbfgs_m: int = 7, device: int | torch.device = 0):
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        cfg = capi.scvt_server_config(int(memory_budget), int(max_generators), int(max_jobs), int(precision),
                                      int(lbfgs_m))
        with torch.cuda.device(self.device):
            self._s = capi.scvt_server_create(cfg, torch.cuda.current_stream(self.device).cuda_stream)
        self.sizes = {}

    def close(self):
        if getattr(self, "_s", None):
            capi.scvt_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, z0, density: Density, max_iter=200, grad_tol=1e-8, rel_grad_tol=0.0, rel_df_tol=0.0,
               step_tol=0.0, ls_max_evals=10, c1=1e-4, c2=0.9, method="plbfgs") -> int:
        o = capi.scvt_solve_opts(int(max_iter), float(grad_tol), float(rel_grad_tol), float(rel_df_tol),
                                 float(step_tol), int(ls_max_evals), float(c1), float(c2), 0, METHODS[method])
        n = int(z0.shape[0])
        with torch.cuda.device(self.device):
            jid = capi.scvt_server_submit(self._s, n, _density(density), _ptr(z0), o)
        self.sizes[jid] = n
        return jid

    def step(self):
        """One scheduling step; returns (running, queued)."""
        with torch.cuda.device(self.device):
            return capi.scvt_server_step(self._s)

    def job(self, jid: int) -> dict:
        i = capi.scvt_server_job(self._s, jid)
        d = {f: getattr(i, f) for f, _ in capi.scvt_job_info._fields_ if f != "report"}
        d["report"] = {f: getattr(i.report, f) for f, _ in capi.scvt_solve_report._fields_}
        return d

    def fetch(self, jid: int, out=None):
        """The finished job's generators: into `out` (a numpy array or a
        device tensor, n x 3) or a new numpy array."""
        z = np.empty((self.sizes[jid], 3)) if out is None else out
        capi.scvt_server_fetch(self._s, jid, _ptr(z))
        return z

    def clock(self) -> float:
        return capi.scvt_server_clock(self._s)

    def stats(self):
        s = capi.scvt_server_get_stats(self._s)
        return {f: getattr(s, f) for f, _ in capi.scvt_stats._fields_}


def sample_density(density: Density, cand, u, n_target: int, exponent: float = 1.0):
    """Monte Carlo initialisation by the density on the GPU: the first
    n_target candidates with u_k rho_max^e <= rho(cand_k)^e, in order (numpy
    in, numpy out)."""
    cand = np.ascontiguousarray(cand, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty((int(n_target), 3))
    k = capi.scvt_sample_density(_density(density), float(exponent), cand.ctypes.data, u.ctypes.data, len(u),
                                 int(n_target), out.ctypes.data)
    return out[:k]
