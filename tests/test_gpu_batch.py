"""Batches of independent problems (needs a GPU).

A batch evaluates every problem's cells in one launch sequence and steps
all problems' LBFGS in lockstep; each problem must reproduce a
single-problem handle bit for bit (same kernels on the same rows, per-cell
sums in edge order, per-problem reductions with the single-problem
chunking, the same line-search decisions).  The single-problem path is
itself checked against the oracle in test_gpu_parity.py; one batch is
checked against the oracle directly here too.  Tuning changes launch
shapes and search radii only, never a result."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
from paper_1709_06924_gb300 import inputs as I
from paper_1709_06924_gb300.engine import Batch, Engine
from tests.parity import RTOL

PROBLEMS = [
    # uneven sizes with ragged tails, four density kinds
    (2562, I.density_uniform()),
    (5003, I.density_x3()),
    (12001, I.WORKLOADS["tanh-163842"].density),
    (700, I.Density(I.RHO_TANH_CAP, (1 / 8) ** 4, 0.10, math.pi / 9, I.latlon_to_xyz(45, 270))),
    (40962, I.WORKLOADS["tanh-2621442"].density),
]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def inputs(problems, seed0=11):
    return [I.uniform_sphere(n, seed0 + k) for k, (n, _) in enumerate(problems)]


def solo_eval(z, dens, precision=0, **tune):
    with Engine(len(z), dens, precision=precision) as e:
        if tune:
            e.set_tuning(**tune)
        F, g, _, _ = e.energy_grad(dev(z))
        return F, g.cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_evaluation_equals_single_problems_bitwise(precision):
    zs = inputs(PROBLEMS)
    with Batch([n for n, _ in PROBLEMS], [d for _, d in PROBLEMS], precision=precision) as bt:
        e, g = bt.energy_grad(bt.concat([dev(z) for z in zs]))
        gs = bt.split(g.cpu().numpy())
    for k, (n, dens) in enumerate(PROBLEMS):
        F, gk = solo_eval(zs[k], dens, precision)
        assert e[k] == F, (k, e[k], F)
        assert np.array_equal(gs[k], gk), k


def test_batch_matches_the_oracle():
    zs = inputs(PROBLEMS[:4], seed0=31)
    with Batch([n for n, _ in PROBLEMS[:4]], [d for _, d in PROBLEMS[:4]]) as bt:
        e, g = bt.energy_grad(bt.concat([dev(z) for z in zs]))
        gs = bt.split(g.cpu().numpy())
    for k, (n, dens) in enumerate(PROBLEMS[:4]):
        o = oracle.energy_grad(zs[k], dens)
        assert abs(e[k] - o["F"]) <= RTOL * o["F"], k
        cn = np.linalg.norm(o["c"], axis=1)[:, None]
        assert np.max(np.abs(gs[k] - o["g"]) / cn) <= RTOL, k


@pytest.mark.parametrize("precision,method", [(0, "plbfgs"), (1, "plbfgs"), (0, "lbfgs"), (0, "lloyd")])
def test_batch_solve_equals_single_problem_solves_bitwise(precision, method):
    probs = PROBLEMS[:4]
    zs = inputs(probs, seed0=51)
    with Batch([n for n, _ in probs], [d for _, d in probs], precision=precision) as bt:
        zb = bt.concat([dev(z) for z in zs])
        reps = bt.lbfgs_solve(zb, max_iter=12, grad_tol=0.0, method=method)
        # and a continuation of the same solve
        reps2 = bt.lbfgs_solve(zb, max_iter=3, grad_tol=0.0, warm_start=1, method=method)
        zb_out = bt.split(zb.cpu().numpy())
    keys = ("iters", "fevals", "resets", "skipped", "energy", "grad_norm", "converged", "status")
    for k, (n, dens) in enumerate(probs):
        with Engine(n, dens, precision=precision) as e:
            z = dev(zs[k])
            r = e.lbfgs_solve(z, max_iter=12, grad_tol=0.0, method=method)
            r2 = e.lbfgs_solve(z, max_iter=3, grad_tol=0.0, warm_start=1, method=method)
            zk = z.cpu().numpy()
        for key in keys:
            assert reps[k][key] == r[key], (k, key, reps[k][key], r[key])
            assert reps2[k][key] == r2[key], (k, key, reps2[k][key], r2[key])
        assert np.array_equal(zb_out[k], zk), k


def test_batch_stopping_is_per_problem():
    # a loose tolerance stops the small uniform problem long before the others
    probs = PROBLEMS[:3]
    zs = inputs(probs, seed0=71)
    with Batch([n for n, _ in probs], [d for _, d in probs]) as bt:
        zb = bt.concat([dev(z) for z in zs])
        reps = bt.lbfgs_solve(zb, max_iter=30, grad_tol=2e-4)
        zb_out = bt.split(zb.cpu().numpy())
    for k, (n, dens) in enumerate(probs):
        with Engine(n, dens) as e:
            z = dev(zs[k])
            r = e.lbfgs_solve(z, max_iter=30, grad_tol=2e-4)
            assert reps[k]["iters"] == r["iters"] and reps[k]["converged"] == r["converged"]
            assert np.array_equal(zb_out[k], z.cpu().numpy())
    assert len({r["iters"] for r in reps}) > 1


def test_a_failing_problem_does_not_stop_the_others():
    probs = PROBLEMS[:3]
    zs = inputs(probs, seed0=81)
    bad = zs[1].copy()
    bad[:, 2] = np.abs(bad[:, 2]) + 0.05  # every generator in the upper hemisphere: no bounded tessellation
    bad /= np.linalg.norm(bad, axis=1)[:, None]
    zs[1] = bad
    with Batch([n for n, _ in probs], [d for _, d in probs]) as bt:
        zb = bt.concat([dev(z) for z in zs])
        reps = bt.lbfgs_solve(zb, max_iter=5, grad_tol=0.0)
        zb_out = bt.split(zb.cpu().numpy())
    assert reps[1]["status"] == 2  # DEGENERATE
    for k in (0, 2):
        n, dens = probs[k]
        with Engine(n, dens) as e:
            z = dev(zs[k])
            r = e.lbfgs_solve(z, max_iter=5, grad_tol=0.0)
            assert reps[k]["status"] == 0 and reps[k]["energy"] == r["energy"]
            assert np.array_equal(zb_out[k], z.cpu().numpy())


TUNINGS = [
    dict(bin_load=1), dict(bin_load=4), dict(bin_load=8), dict(topo_warps=2), dict(topo_warps=8),
    dict(topo_blocks_per_sm=4), dict(quad_block=128), dict(quad_block=512), dict(knn_target=12),
    dict(knn_target=48), dict(topo_cell_lanes=16), dict(topo_cell_lanes=16, topo_warps=8, bin_load=1),
    dict(topo_cell_lanes=16, knn_target=48), dict(chunks=1), dict(chunks=2), dict(chunks=4), dict(chunks=3, topo_cell_lanes=16),
]


@pytest.mark.parametrize("precision", [0, 1])
def test_tuning_never_changes_a_result(precision):
    n, dens = 20001, I.WORKLOADS["tanh-163842"].density
    z = I.uniform_sphere(n, 91)
    F0, g0 = solo_eval(z, dens, precision)
    for t in TUNINGS:
        F, g = solo_eval(z, dens, precision, **t)
        assert F == F0 and np.array_equal(g, g0), t


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_chunked_pipelines_keep_results(precision):
    """Cells split into concurrent chunks (edge lists chained on the device)
    give the batch's results bit for bit, graph replay included."""
    zs = inputs(PROBLEMS, seed0=77)
    with Batch([n for n, _ in PROBLEMS], [d for _, d in PROBLEMS], precision=precision) as bt:
        zb = bt.concat([dev(z) for z in zs])
        e0, g0 = bt.energy_grad(zb)
        for c in (2, 3, 4):
            bt.set_tuning(chunks=c)
            for _ in range(2):
                e1, g1 = bt.energy_grad(zb)
                assert e1 == e0 and torch.equal(g1, g0), c


def test_autotuner_picks_a_valid_tuning_and_keeps_results():
    zs = inputs(PROBLEMS, seed0=101)
    with Batch([n for n, _ in PROBLEMS], [d for _, d in PROBLEMS]) as bt:
        zb = bt.concat([dev(z) for z in zs])
        e0, g0 = bt.energy_grad(zb)
        t = bt.tune(zb)
        assert t == bt.tuning()
        assert t["bin_load"] in (1, 2, 4, 8) and t["topo_warps"] in (2, 4, 8)
        assert t["quad_block"] in (128, 256, 512) and t["knn_target"] in (16, 24, 32, 48)
        assert t["topo_cell_lanes"] in (16, 32) and t["chunks"] in (1, 2, 3, 4)
        e1, g1 = bt.energy_grad(zb)
        assert e1 == e0 and torch.equal(g1, g0)
        st = bt.stats()
        assert st["evaluations"] > 10 and st["kernel_launches"] > 0


def test_single_problem_autotuner_keeps_results():
    n, dens = 30001, I.WORKLOADS["tanh-2621442"].density
    z = dev(I.uniform_sphere(n, 121))
    with Engine(n, dens) as e:
        F0, g0, _, _ = e.energy_grad(z)
        t = e.tune(z)
        assert t == e.tuning()
        F1, g1, _, _ = e.energy_grad(z)
    assert F1 == F0 and torch.equal(g1, g0)


def test_fan_batch_equals_fan_single_problems():
    zs = inputs(PROBLEMS[:3], seed0=141)
    with Batch([n for n, _ in PROBLEMS[:3]], [d for _, d in PROBLEMS[:3]], decomposition=1) as bt:
        e, g = bt.energy_grad(bt.concat([dev(z) for z in zs]))
        gs = bt.split(g.cpu().numpy())
    for k, (n, dens) in enumerate(PROBLEMS[:3]):
        with Engine(n, dens, decomposition=1) as en:
            F, gk, _, _ = en.energy_grad(dev(zs[k]))
        assert e[k] == F and np.array_equal(gs[k], gk.cpu().numpy())
