"""The multi-GPU path of bench.py runs one replica per GPU and combines the
ranks with sum-of-units / max-of-time; that host logic is checked here with
two gloo processes on the CPU (no GPU)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units = 1000.0 * (rank + 1)        # replicas may process different amounts
    seconds = 2.0 if rank == 0 else 3.0
    u, t = bench.combine_ranks(units, seconds)
    out[rank] = (u, t)
    dist.barrier()
    dist.destroy_process_group()


def test_combine_ranks_two_gloo_processes():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        assert out[r] == (3000.0, 3.0)


def test_combine_ranks_single_process_is_identity():
    import bench
    assert bench.combine_ranks(5.0, 2.0) == (5.0, 2.0)


def test_roofline_figures_are_defined_for_every_density():
    import bench
    for kind in (0, 1, 2, 3):
        assert bench.fp64_flops_per_generator(kind) > 0
    # uniform < X3 < tanh cap: the density only adds work per rule point
    f = [bench.fp64_flops_per_generator(k) for k in (0, 1, 2)]
    assert f[0] < f[1] < f[2]
    assert abs(bench.fp64_peak_tflops() - 1.25856) < 1e-9
    assert bench.quad_traffic_bytes(163842) > 0


def test_roofline_of_both_forms():
    import bench
    from paper_1709_06924_gb300 import inputs as I
    w = I.WORKLOADS["tanh-2621442"]
    st = {"series_cells": w.n * 3, "series_terms": w.n * 3 * 5, "evaluations": 3}
    r0 = bench.roofline_of(0, w, 5.0, 4.0, st)
    r1 = bench.roofline_of(1, w, 1.0, 4.0, st, 16)
    for r, ms in ((r0, 5.0), (r1, 4.0)):
        assert r["bound"] == "alu" and r["unit"] == "Twarp-inst/s"
        assert abs(r["peak"] - 152 * 4 * 2.07e9 / 1e12) < 1e-12
        assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
        assert r["avg_launch_ms"] == ms
    assert r0["kernel"] == "k_quad" and r1["kernel"] == "k_topo_warp"
    assert r0["series_cell_fraction"] == 1.0 and r0["series_terms_avg"] == 5.0


def test_parse_tuning():
    import bench
    assert bench.parse_tuning("") == {}
    assert bench.parse_tuning("chunks=4, bin_load=8") == {"chunks": 4, "bin_load": 8}


def test_two_loop_roofline():
    import bench
    from paper_1709_06924_gb300 import inputs as I
    w = I.WORKLOADS["tanh-2621442"]
    r = bench.two_loop_roofline(w, 3, 5, 4.0)
    assert r["bound"] == "hbm" and r["pairs_per_iteration"] == [3, 4, 5, 6, 7]
    assert r["algorithmic_bytes"] == sum((4 * c + 2) * 24 for c in (3, 4, 5, 6, 7)) * w.n
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert bench.two_loop_roofline(w, 3, 0, 4.0) is None
