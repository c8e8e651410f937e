"""The allocation-free entry point against the handle-based one (needs a GPU).

scvt_energy_grad_static serves callers that cannot allocate device memory
when they need an evaluation (a memory budget fixed up front, an allocator
that must not be re-entered, a host that forbids cudaMalloc after start-up):
its scratch is one fixed device array, sized for N <= SCVT_STATIC_MAX_N.
Two calls in a row, with different generators, must give the same energy,
gradient, masses and moments as scvt_energy_grad within the parity tolerance
(1e-12 relative) -- the second call shows that the array's leftover contents
from the first do not leak into the result.  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1709_06924_gb300 import capi
from paper_1709_06924_gb300 import inputs as I
from paper_1709_06924_gb300.engine import Engine, _density

RTOL = 1e-12


def static_eval(n, dens, z, stream):
    g = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    m = torch.empty(n, dtype=torch.float64, device="cuda")
    c = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    e = C.c_double()
    rho = _density(dens)
    torch.cuda.synchronize()
    st = capi.lib().scvt_energy_grad_static(n, C.byref(rho), C.c_void_p(z.data_ptr()),
                                            C.c_void_p(stream.cuda_stream), C.byref(e), C.c_void_p(g.data_ptr()),
                                            C.c_void_p(m.data_ptr()), C.c_void_p(c.data_ptr()))
    assert st == capi.OK, capi.lib().scvt_status_string(st)
    return e.value, g, m, c


def test_static_entry_matches_handle_entry_on_two_calls():
    dens = I.WORKLOADS["tanh-163842"].density
    stream = torch.cuda.Stream()
    for n, seed in ((12000, 21), (9001, 22)):
        z = torch.from_numpy(I.uniform_sphere(n, seed)).cuda()
        with Engine(n, dens) as e:
            F0, g0, m0, c0 = e.energy_grad(z)
        F1, g1, m1, c1 = static_eval(n, dens, z, stream)
        assert abs(F1 - F0) <= RTOL * abs(F0)
        m0n, m1n = m0.cpu().numpy(), m1.cpu().numpy()
        assert np.max(np.abs(m1n - m0n) / m0n) <= RTOL
        cn = np.linalg.norm(c0.cpu().numpy(), axis=1)[:, None]
        assert np.max(np.abs(c1.cpu().numpy() - c0.cpu().numpy()) / cn) <= RTOL
        assert np.max(np.abs(g1.cpu().numpy() - g0.cpu().numpy()) / cn) <= RTOL


def test_static_entry_rejects_sizes_beyond_the_maximum():
    rho = _density(I.density_uniform())
    e = C.c_double()
    z = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    st = capi.lib().scvt_energy_grad_static(capi.STATIC_MAX_N + 1, C.byref(rho), C.c_void_p(z.data_ptr()), None,
                                            C.byref(e), None, None, None)
    assert st == capi.ERR_INVALID
