"""ctypes binding of ``include/scvt.h`` -- argument marshalling only.

Every function here forwards to the CUDA library ``libscvt.so`` under the
same name.  There is no CPU path: if the library cannot be loaded the import
of this module raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

from . import build as _build

OK = 0
ERR_INVALID = 1
ERR_DEGENERATE = 2
ERR_OOM = 3
ERR_CUDA = 4
ERR_KNN_EXHAUSTED = 5
ERR_LINESEARCH = 6
ERR_TIMEOUT = 7
ERR_UNIMPLEMENTED = 8


class scvt_density(C.Structure):
    _fields_ = [("kind", C.c_int), ("gamma", C.c_double), ("alpha", C.c_double), ("beta", C.c_double),
                ("xc", C.c_double * 3)]


class scvt_config(C.Structure):
    _fields_ = [("n", C.c_int64), ("rho", scvt_density), ("quad_points", C.c_int), ("precision", C.c_int),
                ("lbfgs_m", C.c_int), ("knn_k0", C.c_int), ("knn_kmax", C.c_int), ("decomposition", C.c_int)]


class scvt_solve_opts(C.Structure):
    _fields_ = [("max_iter", C.c_int), ("grad_tol", C.c_double), ("rel_grad_tol", C.c_double),
                ("rel_df_tol", C.c_double), ("step_tol", C.c_double), ("ls_max_evals", C.c_int),
                ("c1", C.c_double), ("c2", C.c_double), ("warm_start", C.c_int), ("method", C.c_int)]


class scvt_solve_report(C.Structure):
    _fields_ = [("iters", C.c_int), ("fevals", C.c_int), ("resets", C.c_int), ("skipped", C.c_int),
                ("knn_retries", C.c_int), ("energy", C.c_double), ("grad_norm", C.c_double),
                ("converged", C.c_int), ("status", C.c_int)]


class scvt_stats(C.Structure):
    _fields_ = [("evaluations", C.c_int64), ("cell_launches", C.c_int64), ("kernel_launches", C.c_int64),
                ("knn_retries", C.c_int64), ("ambiguous", C.c_int64), ("cell_kernel_ms", C.c_double),
                ("eval_ms", C.c_double), ("lbfgs_ms", C.c_double), ("cell_kernel_timed", C.c_int64),
                ("bytes_device", C.c_int64), ("series_edges", C.c_int64), ("series_terms", C.c_int64),
                ("topo_kernel_ms", C.c_double), ("topo_kernel_timed", C.c_int64)]


class scvt_eval_out(C.Structure):
    _fields_ = [("grad", C.c_void_p), ("precond", C.c_void_p), ("mass", C.c_void_p), ("moment", C.c_void_p),
                ("cell_energy", C.c_void_p), ("energy", C.c_double), ("grad_norm", C.c_double)]


class scvt_tuning(C.Structure):
    _fields_ = [("bin_load", C.c_int), ("knn_target", C.c_int), ("topo_warps", C.c_int),
                ("topo_blocks_per_sm", C.c_int), ("quad_block", C.c_int), ("topo_cell_lanes", C.c_int),
                ("chunks", C.c_int)]


class scvt_server_config(C.Structure):
    _fields_ = [("memory_budget", C.c_int64), ("max_generators", C.c_int64), ("max_jobs", C.c_int),
                ("precision", C.c_int), ("lbfgs_m", C.c_int)]


class scvt_job_info(C.Structure):
    _fields_ = [("state", C.c_int), ("n", C.c_int64), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double), ("bytes_resident", C.c_int64), ("report", scvt_solve_report)]


JOB_QUEUED, JOB_RUNNING, JOB_DONE, JOB_FAILED, JOB_FETCHED = range(5)

_H = C.c_void_p
_vp = C.c_void_p
_st = C.c_int

# name -> (restype, argtypes); mirrors include/scvt.h
SIGNATURES = {
    "scvt_create": (_st, [C.POINTER(scvt_config), _vp, C.POINTER(_H)]),
    "scvt_destroy": (None, [_H]),
    "scvt_energy_grad": (_st, [_H, _vp, C.POINTER(C.c_double), _vp, _vp, _vp]),
    "scvt_evaluate": (_st, [_H, _vp, C.POINTER(scvt_eval_out)]),
    "scvt_lloyd_step": (_st, [_H, _vp, _vp]),
    "scvt_lbfgs_solve": (_st, [_H, _vp, C.POINTER(scvt_solve_opts), C.POINTER(scvt_solve_report)]),
    "scvt_voronoi": (_st, [_H, _vp, _vp, _vp, C.c_int]),
    "scvt_lbfgs_direction": (_st, [_H, _vp, _vp, C.c_int, _vp, _vp, _vp]),
    "scvt_get_stats": (_st, [_H, C.POINTER(scvt_stats)]),
    "scvt_reset_stats": (_st, [_H]),
    "scvt_set_profiling": (_st, [_H, C.c_int]),
    "scvt_status_string": (C.c_char_p, [_st]),
    "scvt_last_error": (C.c_char_p, [_H]),
    "scvt_version": (C.c_char_p, []),
    "scvt_energy_grad_static": (_st, [C.c_int64, C.POINTER(scvt_density), _vp, _vp, C.POINTER(C.c_double),
                                      _vp, _vp, _vp]),
    "scvt_set_tuning": (_st, [_H, C.POINTER(scvt_tuning)]),
    "scvt_get_tuning": (_st, [_H, C.POINTER(scvt_tuning)]),
    "scvt_tune": (_st, [_H, _vp, C.POINTER(scvt_tuning)]),
    "scvt_batch_create": (_st, [C.POINTER(scvt_config), C.c_int, _vp, C.POINTER(_H)]),
    "scvt_batch_destroy": (None, [_H]),
    "scvt_batch_energy_grad": (_st, [_H, _vp, C.POINTER(C.c_double), _vp]),
    "scvt_batch_lbfgs_solve": (_st, [_H, _vp, C.POINTER(scvt_solve_opts), C.POINTER(scvt_solve_report)]),
    "scvt_batch_tune": (_st, [_H, _vp, C.POINTER(scvt_tuning)]),
    "scvt_batch_set_tuning": (_st, [_H, C.POINTER(scvt_tuning)]),
    "scvt_batch_get_tuning": (_st, [_H, C.POINTER(scvt_tuning)]),
    "scvt_batch_get_stats": (_st, [_H, C.POINTER(scvt_stats)]),
    "scvt_batch_reset_stats": (_st, [_H]),
    "scvt_batch_last_error": (C.c_char_p, [_H]),
    "scvt_server_create": (_st, [C.POINTER(scvt_server_config), _vp, C.POINTER(_H)]),
    "scvt_server_destroy": (None, [_H]),
    "scvt_server_submit": (_st, [_H, C.c_int64, C.POINTER(scvt_density), _vp, C.POINTER(scvt_solve_opts),
                                 C.POINTER(C.c_int64)]),
    "scvt_server_step": (_st, [_H, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "scvt_server_job": (_st, [_H, C.c_int64, C.POINTER(scvt_job_info)]),
    "scvt_server_fetch": (_st, [_H, C.c_int64, _vp]),
    "scvt_server_clock": (C.c_double, [_H]),
    "scvt_server_get_stats": (_st, [_H, C.POINTER(scvt_stats)]),
    "scvt_server_last_error": (C.c_char_p, [_H]),
    "scvt_bisect": (_st, [_H, _vp, _vp, C.c_int64, C.POINTER(C.c_int64)]),
    "scvt_mesh_quality": (_st, [_H, _vp, _vp, _vp, C.c_int64, C.POINTER(C.c_int64)]),
    "scvt_sample_density": (_st, [C.POINTER(scvt_density), C.c_double, _vp, _vp, C.c_int64, C.c_int64, _vp,
                                  C.POINTER(C.c_int64), _vp]),
}

STATIC_MAX_N = 16384  # SCVT_STATIC_MAX_N


def header_symbols():
    """Entry points declared in include/scvt.h."""
    path = os.path.join(_build.INCLUDE, "scvt.h")
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(scvt_[a-z_0-9]+)\s*\(", text)))


def load(path: str | None = None):
    """Load (building it first if it is missing or stale) the CUDA library."""
    path = path or _build.build()
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


class ScvtError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        s = lib().scvt_status_string(status).decode()
        super().__init__("%s: %s (status %d)%s" % (where, s, status, (": " + detail) if detail else ""))
        self.status = status


def check(status: int, where: str, handle=None, batch=None, server=None):
    if status != OK:
        if handle:
            detail = lib().scvt_last_error(handle).decode()
        elif batch:
            detail = lib().scvt_batch_last_error(batch).decode()
        elif server:
            detail = lib().scvt_server_last_error(server).decode()
        else:
            detail = ""
        raise ScvtError(status, where, detail)


# ---- same names as the C ABI -------------------------------------------------
def scvt_create(cfg: scvt_config, stream: int | None = None):
    h = _H()
    check(lib().scvt_create(C.byref(cfg), _vp(stream or 0), C.byref(h)), "scvt_create")
    return h


def scvt_destroy(h):
    lib().scvt_destroy(h)


def scvt_energy_grad(h, z_ptr: int, grad_ptr=None, mass_ptr=None, moment_ptr=None) -> float:
    e = C.c_double()
    check(lib().scvt_energy_grad(h, _vp(z_ptr), C.byref(e), _vp(grad_ptr), _vp(mass_ptr), _vp(moment_ptr)),
          "scvt_energy_grad", h)
    return e.value


def scvt_evaluate(h, z_ptr: int, out: scvt_eval_out) -> scvt_eval_out:
    check(lib().scvt_evaluate(h, _vp(z_ptr), C.byref(out)), "scvt_evaluate", h)
    return out


def scvt_lloyd_step(h, z_in_ptr: int, z_out_ptr: int):
    check(lib().scvt_lloyd_step(h, _vp(z_in_ptr), _vp(z_out_ptr)), "scvt_lloyd_step", h)


def scvt_lbfgs_solve(h, z_ptr: int, opts: scvt_solve_opts | None) -> scvt_solve_report:
    rep = scvt_solve_report()
    st = lib().scvt_lbfgs_solve(h, _vp(z_ptr), C.byref(opts) if opts is not None else None, C.byref(rep))
    if st not in (OK, ERR_LINESEARCH):
        check(st, "scvt_lbfgs_solve", h)
    return rep


def scvt_voronoi(h, z_ptr: int, deg_ptr: int, nbr_ptr: int, max_deg: int):
    check(lib().scvt_voronoi(h, _vp(z_ptr), _vp(deg_ptr), _vp(nbr_ptr), int(max_deg)), "scvt_voronoi", h)


def scvt_lbfgs_direction(h, g_ptr, h_ptr, count, S_ptr, Y_ptr, q_ptr):
    check(lib().scvt_lbfgs_direction(h, _vp(g_ptr), _vp(h_ptr), int(count), _vp(S_ptr), _vp(Y_ptr), _vp(q_ptr)),
          "scvt_lbfgs_direction", h)


def scvt_get_stats(h) -> scvt_stats:
    s = scvt_stats()
    check(lib().scvt_get_stats(h, C.byref(s)), "scvt_get_stats", h)
    return s


def scvt_reset_stats(h):
    check(lib().scvt_reset_stats(h), "scvt_reset_stats", h)


def scvt_set_profiling(h, on: bool):
    check(lib().scvt_set_profiling(h, int(bool(on))), "scvt_set_profiling", h)


def scvt_version() -> str:
    return lib().scvt_version().decode()


def scvt_set_tuning(h, t: scvt_tuning):
    check(lib().scvt_set_tuning(h, C.byref(t)), "scvt_set_tuning", h)


def scvt_get_tuning(h) -> scvt_tuning:
    t = scvt_tuning()
    check(lib().scvt_get_tuning(h, C.byref(t)), "scvt_get_tuning", h)
    return t


def scvt_tune(h, z_ptr: int) -> scvt_tuning:
    t = scvt_tuning()
    check(lib().scvt_tune(h, _vp(z_ptr), C.byref(t)), "scvt_tune", h)
    return t


def scvt_batch_create(cfgs, stream: int | None = None):
    arr = (scvt_config * len(cfgs))(*cfgs)
    b = _H()
    check(lib().scvt_batch_create(arr, len(cfgs), _vp(stream or 0), C.byref(b)), "scvt_batch_create")
    return b


def scvt_batch_destroy(b):
    lib().scvt_batch_destroy(b)


def scvt_batch_energy_grad(b, z_ptr: int, count: int, grad_ptr=None):
    e = (C.c_double * count)()
    check(lib().scvt_batch_energy_grad(b, _vp(z_ptr), e, _vp(grad_ptr)), "scvt_batch_energy_grad", batch=b)
    return list(e)


def scvt_batch_lbfgs_solve(b, z_ptr: int, opts: scvt_solve_opts | None, count: int):
    reps = (scvt_solve_report * count)()
    st = lib().scvt_batch_lbfgs_solve(b, _vp(z_ptr), C.byref(opts) if opts is not None else None, reps)
    # a problem's own failure is reported in its entry; anything else raises
    if st not in (OK, ERR_LINESEARCH) and not any(r.status == st for r in reps):
        check(st, "scvt_batch_lbfgs_solve", batch=b)
    return list(reps)


def scvt_batch_tune(b, z_ptr: int) -> scvt_tuning:
    t = scvt_tuning()
    check(lib().scvt_batch_tune(b, _vp(z_ptr), C.byref(t)), "scvt_batch_tune", batch=b)
    return t


def scvt_batch_set_tuning(b, t: scvt_tuning):
    check(lib().scvt_batch_set_tuning(b, C.byref(t)), "scvt_batch_set_tuning", batch=b)


def scvt_batch_get_tuning(b) -> scvt_tuning:
    t = scvt_tuning()
    check(lib().scvt_batch_get_tuning(b, C.byref(t)), "scvt_batch_get_tuning", batch=b)
    return t


def scvt_batch_get_stats(b) -> scvt_stats:
    s = scvt_stats()
    check(lib().scvt_batch_get_stats(b, C.byref(s)), "scvt_batch_get_stats", batch=b)
    return s


def scvt_batch_reset_stats(b):
    check(lib().scvt_batch_reset_stats(b), "scvt_batch_reset_stats", batch=b)


def scvt_server_create(cfg: scvt_server_config, stream: int | None = None):
    s = _H()
    check(lib().scvt_server_create(C.byref(cfg), _vp(stream or 0), C.byref(s)), "scvt_server_create")
    return s


def scvt_server_destroy(s):
    lib().scvt_server_destroy(s)


def scvt_server_submit(s, n: int, rho: scvt_density, z0_ptr: int, opts: scvt_solve_opts | None) -> int:
    jid = C.c_int64()
    check(lib().scvt_server_submit(s, int(n), C.byref(rho), _vp(z0_ptr),
                                   C.byref(opts) if opts is not None else None, C.byref(jid)),
          "scvt_server_submit", server=s)
    return jid.value


def scvt_server_step(s):
    r, q = C.c_int(), C.c_int()
    check(lib().scvt_server_step(s, C.byref(r), C.byref(q)), "scvt_server_step", server=s)
    return r.value, q.value


def scvt_server_job(s, jid: int) -> scvt_job_info:
    info = scvt_job_info()
    check(lib().scvt_server_job(s, int(jid), C.byref(info)), "scvt_server_job", server=s)
    return info


def scvt_server_fetch(s, jid: int, z_ptr: int):
    check(lib().scvt_server_fetch(s, int(jid), _vp(z_ptr)), "scvt_server_fetch", server=s)


def scvt_server_clock(s) -> float:
    return lib().scvt_server_clock(s)


def scvt_server_get_stats(s) -> scvt_stats:
    st = scvt_stats()
    check(lib().scvt_server_get_stats(s, C.byref(st)), "scvt_server_get_stats", server=s)
    return st


def scvt_sample_density(rho: scvt_density, exponent: float, cand_ptr: int, u_ptr: int, m: int, n_target: int,
                        out_ptr: int, stream: int | None = None) -> int:
    k = C.c_int64()
    check(lib().scvt_sample_density(C.byref(rho), float(exponent), _vp(cand_ptr), _vp(u_ptr), int(m), int(n_target),
                                    _vp(out_ptr), C.byref(k), _vp(stream or 0)), "scvt_sample_density")
    return k.value


def scvt_bisect(h, z_ptr: int, out_ptr: int, cap: int) -> int:
    k = C.c_int64()
    check(lib().scvt_bisect(h, _vp(z_ptr), _vp(out_ptr), int(cap), C.byref(k)), "scvt_bisect", h)
    return k.value


def scvt_mesh_quality(h, z_ptr: int, cellq_ptr, triq_ptr, tri_cap: int) -> int:
    k = C.c_int64()
    check(lib().scvt_mesh_quality(h, _vp(z_ptr), _vp(cellq_ptr), _vp(triq_ptr), int(tri_cap), C.byref(k)),
          "scvt_mesh_quality", h)
    return k.value
