"""The served form (needs a GPU): continuous batching of solve requests.

Jobs submitted over time are admitted as job slots, workspace rows and
device memory free up, run in lockstep with whatever else is on the device,
and retire on their own stopping test.  Each job's result must equal, bit
for bit, a single-problem solve of the same problem with the same options
from the same start -- alone and in the mix."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1709_06924_gb300 import capi
from paper_1709_06924_gb300 import inputs as I
from paper_1709_06924_gb300.engine import Engine, Server

JOBS = [
    # (n, density, max_iter, grad_tol): uneven sizes, densities and stopping rules
    (5003, I.density_x3(), 12, 0.0),
    (2562, I.density_uniform(), 40, 2e-4),
    (12001, I.WORKLOADS["tanh-163842"].density, 8, 0.0),
    (700, I.Density(I.RHO_TANH_CAP, (1 / 8) ** 4, 0.10, math.pi / 9, I.latlon_to_xyz(45, 270)), 20, 1e-6),
    (20001, I.WORKLOADS["tanh-2621442"].density, 5, 0.0),
    (3001, I.density_x64(), 15, 0.0),
]


def solo(z, dens, max_iter, grad_tol, precision=0):
    with Engine(len(z), dens, precision=precision) as e:
        zt = torch.from_numpy(z.copy()).cuda()
        r = e.lbfgs_solve(zt, max_iter=max_iter, grad_tol=grad_tol)
        return zt.cpu().numpy(), r


def drive(server, submit_plan):
    """submit_plan: list of (step_index, job) -- jobs arrive while others run."""
    ids, step, pending = {}, 0, list(submit_plan)
    max_running = 0
    while True:
        for k, (at, job) in enumerate(pending):
            if at == step:
                z, dens, mi, gt = job
                ids[k] = server.submit(z, dens, max_iter=mi, grad_tol=gt)
        running, queued = server.step()
        max_running = max(max_running, running)
        step += 1
        if running == 0 and queued == 0 and step > max(a for a, _ in pending):
            return ids, max_running
        assert step < 1000


@pytest.mark.parametrize("precision", [0, 1])
def test_each_job_equals_its_solo_solve(precision):
    zs = [I.uniform_sphere(n, 200 + k) for k, (n, *_ ) in enumerate(JOBS)]
    plan = [(2 * k, (zs[k], d, mi, gt)) for k, (n, d, mi, gt) in enumerate(JOBS)]
    with Server(max_generators=30000, max_jobs=3, precision=precision) as srv:
        ids, max_running = drive(srv, plan)
        infos = {k: srv.job(ids[k]) for k in ids}
        outs = {k: srv.fetch(ids[k]) for k in ids}
        st = srv.stats()
    assert max_running == 3  # jobs ran together, and the slot limit held
    keys = ("iters", "fevals", "resets", "skipped", "energy", "grad_norm", "converged", "status")
    for k, (n, d, mi, gt) in enumerate(JOBS):
        z_ref, r = solo(zs[k], d, mi, gt, precision)
        info = infos[k]
        assert info["state"] == capi.JOB_DONE
        assert 0 <= info["t_submit"] <= info["t_admit"] <= info["t_done"]
        for key in keys:
            assert info["report"][key] == r[key], (k, key, info["report"][key], r[key])
        assert np.array_equal(outs[k], z_ref), k
    assert st["evaluations"] > 0


def test_admission_follows_rows_and_memory_budget():
    # rows for two 20k jobs at most: the third waits in the queue until one retires
    n = 20001
    dens = I.WORKLOADS["tanh-163842"].density
    zs = [I.uniform_sphere(n, 300 + k) for k in range(3)]
    with Server(max_generators=2 * n + 10, max_jobs=8) as srv:
        ids = [srv.submit(z, dens, max_iter=4 + 2 * k, grad_tol=0.0) for k, z in enumerate(zs)]
        running, queued = srv.step()
        assert (running, queued) == (2, 1)
        assert srv.job(ids[2])["state"] == capi.JOB_QUEUED
        while running or queued:
            running, queued = srv.step()
        infos = [srv.job(i) for i in ids]
        z2 = srv.fetch(ids[2])
    assert infos[2]["t_admit"] >= infos[0]["t_done"]
    z_ref, r = solo(zs[2], dens, 8, 0.0)
    assert np.array_equal(z2, z_ref) and infos[2]["report"]["iters"] == r["iters"]


def test_a_failing_job_does_not_disturb_the_others():
    zs = [I.uniform_sphere(n, 400 + k) for k, (n, *_) in enumerate(JOBS[:3])]
    bad = zs[0].copy()
    bad[:, 2] = np.abs(bad[:, 2]) + 0.05  # all in one hemisphere: no bounded tessellation
    bad /= np.linalg.norm(bad, axis=1)[:, None]
    plan = [(0, (bad, JOBS[0][1], 5, 0.0))] + [(0, (zs[k], JOBS[k][1], JOBS[k][2], JOBS[k][3])) for k in (1, 2)]
    with Server(max_generators=40000, max_jobs=4) as srv:
        ids, _ = drive(srv, plan)
        infos = {k: srv.job(ids[k]) for k in ids}
        outs = {k: srv.fetch(ids[k]) for k in ids}
    assert infos[0]["state"] == capi.JOB_FAILED and infos[0]["report"]["status"] == capi.ERR_DEGENERATE
    for k in (1, 2):
        n, d, mi, gt = JOBS[k]
        z_ref, r = solo(zs[k], d, mi, gt)
        assert infos[k]["state"] == capi.JOB_DONE and np.array_equal(outs[k], z_ref)


def test_submit_rejects_jobs_that_can_never_run():
    with Server(max_generators=1000, max_jobs=2) as srv:
        z = I.uniform_sphere(2000, 1)
        with pytest.raises(capi.ScvtError):
            srv.submit(z, I.density_uniform())
        with pytest.raises(capi.ScvtError):  # no job 0
            capi.scvt_server_fetch(srv._s, 0, z.ctypes.data)


@pytest.mark.parametrize("iters", [1, 5])
def test_served_job_in_a_mix_matches_the_oracle(iters):
    # a 2,562-generator job served while larger jobs run beside it, against
    # the FP64 oracle's Lloyd-preconditioned LBFGS in lockstep: same accepted
    # iterations and evaluations, energy to 1e-12, iterate to 1e-11
    import oracle
    dens = I.density_x3()
    z = I.uniform_sphere(2562, 321)
    zo, rep_o, _ = oracle.lbfgs_solve(z, dens, lbfgs_m=7, max_iter=iters, grad_tol=0.0)
    others = [(I.uniform_sphere(20001, 322), I.WORKLOADS["tanh-163842"].density),
              (I.uniform_sphere(9001, 323), I.density_x64())]
    with Server(max_generators=40000, max_jobs=3, lbfgs_m=7) as srv:
        ids = [srv.submit(zz, d, max_iter=8, grad_tol=0.0) for zz, d in others[:1]]
        srv.step()
        jid = srv.submit(z, dens, max_iter=iters, grad_tol=0.0)
        ids.append(srv.submit(*others[1], max_iter=8, grad_tol=0.0))
        max_running = 0
        while True:
            running, queued = srv.step()
            max_running = max(max_running, running)
            if running == 0 and queued == 0:
                break
        info = srv.job(jid)
        zs = srv.fetch(jid)
    assert max_running == 3
    r = info["report"]
    assert r["iters"] == rep_o["iters"] == iters
    assert r["fevals"] == rep_o["fevals"]
    assert abs(r["energy"] - rep_o["energy"]) <= 1e-12 * rep_o["energy"]
    assert np.abs(zs - zo).max() <= 1e-11
