"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point include/scvt.h declares, the ctypes structures have the C
layout (sizes and offsets printed by gcc from the header), and argument
validation that happens before any device work rejects bad configurations."""
import ctypes as C
import os
import subprocess

import pytest

from paper_1709_06924_gb300 import build as B
from paper_1709_06924_gb300 import capi


def test_library_exports_every_declared_symbol():
    lib = capi.lib()
    declared = capi.header_symbols()
    assert len(declared) >= 14
    for name in declared:
        assert hasattr(lib, name), name
        assert name in capi.SIGNATURES, name


def test_struct_layout_matches_header(tmp_path):
    structs = {
        "scvt_density": capi.scvt_density,
        "scvt_config": capi.scvt_config,
        "scvt_solve_opts": capi.scvt_solve_opts,
        "scvt_solve_report": capi.scvt_solve_report,
        "scvt_stats": capi.scvt_stats,
        "scvt_eval_out": capi.scvt_eval_out,
        "scvt_tuning": capi.scvt_tuning,
        "scvt_server_config": capi.scvt_server_config,
        "scvt_job_info": capi.scvt_job_info,
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "scvt.h"', "int main(void){"]
    for sname, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (sname, sname))
        for f, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (sname, f, sname, f))
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", B.INCLUDE, str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    for sname, cls in structs.items():
        assert int(out[sname]) == C.sizeof(cls), sname
        for f, _ in cls._fields_:
            assert int(out["%s.%s" % (sname, f)]) == getattr(cls, f).offset, (sname, f)


def test_status_strings_and_version():
    lib = capi.lib()
    for s in range(9):
        assert lib.scvt_status_string(s)
    assert b"sm_103a" in lib.scvt_version()


@pytest.mark.parametrize("field,value", [("n", 3), ("lbfgs_m", 33), ("quad_points", 4), ("knn_k0", 4), ("precision", 3)])
def test_create_rejects_bad_config_before_device_work(field, value):
    cfg = capi.scvt_config()
    cfg.n = 100
    cfg.rho.kind = 0
    cfg.quad_points = 7
    cfg.lbfgs_m = 5
    setattr(cfg, field, value)
    h = C.c_void_p()
    assert capi.lib().scvt_create(C.byref(cfg), None, C.byref(h)) == capi.ERR_INVALID
    assert not h.value


def test_null_handle_is_safe():
    lib = capi.lib()
    lib.scvt_destroy(None)
    assert lib.scvt_last_error(None) == b""
    assert lib.scvt_lloyd_step(None, None, None) == capi.ERR_INVALID
    lib.scvt_batch_destroy(None)
    assert lib.scvt_batch_last_error(None) == b""
    assert lib.scvt_batch_energy_grad(None, None, None, None) == capi.ERR_INVALID
    assert lib.scvt_set_tuning(None, None) == capi.ERR_INVALID


def _cfg(n, m=5, precision=0):
    cfg = capi.scvt_config()
    cfg.n = n
    cfg.rho.kind = 0
    cfg.quad_points = 7
    cfg.lbfgs_m = m
    cfg.precision = precision
    return cfg


@pytest.mark.parametrize("case", ["empty", "bad_n", "mixed_m", "mixed_precision"])
def test_batch_create_rejects_bad_configs_before_device_work(case):
    if case == "empty":
        cfgs = []
    elif case == "bad_n":
        cfgs = [_cfg(100), _cfg(3)]
    elif case == "mixed_m":
        cfgs = [_cfg(100, m=5), _cfg(100, m=7)]
    else:
        cfgs = [_cfg(100, precision=0), _cfg(100, precision=1)]
    arr = (capi.scvt_config * max(len(cfgs), 1))(*cfgs)
    b = C.c_void_p()
    assert capi.lib().scvt_batch_create(arr, len(cfgs), None, C.byref(b)) == capi.ERR_INVALID
    assert not b.value


def test_build_sources_target_sm103a():
    assert B.ARCH == "-gencode=arch=compute_103a,code=sm_103a"
    assert len(B.sources()) >= 3
    assert os.path.exists(capi.lib()._name)


@pytest.mark.parametrize("field,value", [("max_jobs", 0), ("max_generators", 3), ("precision", 3),
                                         ("lbfgs_m", 40), ("memory_budget", -1)])
def test_server_create_rejects_bad_config_before_device_work(field, value):
    cfg = capi.scvt_server_config(1 << 30, 100000, 8, 0, 7)
    setattr(cfg, field, value)
    s = C.c_void_p()
    assert capi.lib().scvt_server_create(C.byref(cfg), None, C.byref(s)) == capi.ERR_INVALID
    assert not s.value
    capi.lib().scvt_server_destroy(None)
    assert capi.lib().scvt_server_last_error(None) == b""
