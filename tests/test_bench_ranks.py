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
    # a series term costs one double-float FMA per rule point: 6 edges x 14 points
    assert bench.df_inst_per_generator(6.0) - bench.df_inst_per_generator(5.0) == 6 * 14 * bench.DF_OPS["fma"]
    assert abs(bench.fp64_peak_flops(152, 2070.0) - 1.25856e12) < 1.0
    assert abs(bench.issue_peak(152, 2070.0) - 152 * 4 * 2.07e9) < 1.0


def test_roofline_of_the_three_forms():
    import bench
    from paper_1709_06924_gb300 import inputs as I
    w = I.WORKLOADS["tanh-2621442"]
    edges = (6 * w.n - 12) * 3
    st = {"series_edges": edges, "series_terms": edges * 5, "evaluations": 3}
    r0 = bench.roofline_of(0, w, 5.0, 4.0, st, 32, 152, 2070.0, "test")
    r1 = bench.roofline_of(1, w, 1.0, 4.0, st, 16, 152, 2070.0, "test")
    r2 = bench.roofline_of(2, w, 20.0, 4.0, st, 32, 152, 2070.0, "test")
    for r, ms in ((r0, 5.0), (r1, 4.0), (r2, 20.0)):
        assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
        assert r["avg_launch_ms"] == ms
    assert r0["bound"] == r1["bound"] == "alu" and r2["bound"] == "fp64"
    assert abs(r0["peak"] - 152 * 4 * 2.07e9 / 1e12) < 1e-12
    assert r0["kernel"] == "k_quad" and r1["kernel"] == "k_topo_warp"
    assert r0["series_edge_fraction"] == 1.0 and r0["series_terms_avg"] == 5.0
    # the method's arithmetic is a part of the executed instructions
    assert 0 < r0["algorithmic"]["frac"] < r0["frac"]
    # another SM count or clock scales the peak
    r0b = bench.roofline_of(0, w, 5.0, 4.0, st, 32, 76, 2070.0, "test")
    assert abs(r0b["frac"] - 2 * r0["frac"]) < 1e-12


def test_summary_collects_the_forms():
    import bench
    line = {"value": 2e8, "ms_per_step": 10.0, "roofline": {"frac": 0.7, "algorithmic": {"frac": 0.6}},
            "other_forms": [{"precision": "mixed", "value": 4e8}, {"precision": "plain", "value": 1e8}],
            "time_to_tol": {"mixed": {"paper_rules_without_movement": {"seconds": 3.0, "iters": 100}},
                            "served_mixed": {"paper_rules_without_movement": {"seconds": 4.0}}},
            "roofline_two_loop": {"frac": 0.5}, "serving": None, "cpu_baseline": None}
    s = bench.summary_of(line)
    assert s["fp64_form_M_per_s"] == 200.0 and s["mixed_M_per_s"] == 400.0 and s["plain_M_per_s"] == 100.0
    assert s["ttt_mixed_s"] == 3.0 and s["ttt_mixed_iters"] == 100 and s["ttt_served_mixed_s"] == 4.0
    assert s["two_loop_frac"] == 0.5


def test_parse_tuning():
    import bench
    assert bench.parse_tuning("") == {}
    assert bench.parse_tuning("chunks=4, bin_load=8") == {"chunks": 4, "bin_load": 8}


def test_two_loop_roofline():
    import bench
    from paper_1709_06924_gb300 import inputs as I
    w = I.WORKLOADS["tanh-2621442"]
    r = bench.two_loop_roofline(w, 3, 5, 4.0, 152, 2070.0)
    assert r["bound"] == "fp64" and r["pairs_per_iteration"] == [3, 4, 5, 6, 7]
    assert r["ms_total"] == 4.0
    # 4c + 2 FP64 operations per component, all multiply-adds but the initial matrix's multiply
    assert bench.two_loop_ops_per_component(7) == 30
    assert r["algorithmic_flops"] == sum(3 * (8 * c + 3) for c in (3, 4, 5, 6, 7)) * w.n
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert abs(r["peak"] - 1.25856) < 1e-9
    h = r["hbm"]
    assert h["algorithmic_bytes"] == sum((4 * c + 2) * 24 for c in (3, 4, 5, 6, 7)) * w.n
    assert abs(h["frac"] - h["achieved"] / h["peak"]) < 1e-12
    assert bench.two_loop_roofline(w, 3, 0, 4.0, 152, 2070.0) is None
