"""The N > 1 path of bench.py on CPU: world_size-2 gloo ranks, replicas only.

Each rank times its own reconstructions; the job time is the slowest rank's (all-reduce MAX) and
the whole-job figure is per reconstruction over all ranks.  The reference arm runs on rank 0 only.
"""
import os
import socket
import types

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (rank, world, rank)
        # rank r timed 5 reconstructions in 100 + 50 r ms, end to end 120 + 10 r ms per step
        res = bench.combine_ranks(100.0 + 50.0 * rank, 120.0 + 10.0 * rank, 5, world, "cpu")
        args = types.SimpleNamespace(workload="c1", cpu_iters=1, warmup=0, steps=1)
        ref = bench.run_reference(args, rank, world) if rank != 0 else "skipped"
        out.put((rank, res, ref))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(world):
        rank, res, ref = q.get(timeout=120)
        got[rank] = (res, ref)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in range(world):
        per_recon, e2e, total = got[rank][0]
        assert total == 150.0                       # slowest rank
        assert per_recon == 150.0 / (5 * world)     # whole-job throughput
        assert e2e == 130.0 / world
    assert got[1][1] is None                        # reference arm: rank 0 only, others do no work


def test_single_rank_needs_no_collective():
    per_recon, e2e, total = bench.combine_ranks(80.0, 90.0, 4, 1, "cpu")
    assert (per_recon, e2e, total) == (20.0, 90.0, 80.0)


@pytest.mark.parametrize("name,bmin_mb,bmodel_mb,half_unit", [("c1", 0.33, 0.98, 0.005), ("c2", 2.6, 7.9, 0.05),
                                                              ("c3", 23.6, 70.8, 0.05), ("c5", 94.4, 283.1, 0.05)])
def test_byte_models_per_iteration(name, bmin_mb, bmodel_mb, half_unit):
    # B_min = U + 2|G_S| and B_model = 11 U + 2|G_S| (U = Ni M 8 B, |G_S| = Nr M 8 B) for the
    # workload sizes with the unfolded data term; the fractions divide them by the loop time per
    # iteration and the copy peak
    import scenes
    w = scenes.workload(name)
    m = bench.hbm_model(w, loop_ms=w.iters * 1e-3, peaks={"hbm_gbs": 1000.0}, fold=0)   # 1 us per iteration
    assert abs(m["B_min_MB"] - bmin_mb) <= half_unit            # the figures as printed, rounded
    assert abs(m["B_model_MB"] - bmodel_mb) <= half_unit
    assert abs(m["t_iter_us"] - 1.0) < 1e-9
    assert abs(m["frac_min"] - m["B_min_MB"] * 1e6 / 1e-6 / 1e12) < 1e-9 * m["frac_min"]
    assert bench.hbm_model(w, None, {}) is None


def test_clock_sampler_parses_reasons(tmp_path, monkeypatch):
    # a stand-in nvidia-smi printing three samples (one with the power cap active) then idling
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "echo '0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "echo '0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active'\n"
                    "echo '0, 2040, 2070, 1200.5, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "exec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}:{os.environ['PATH']}")
    import time
    c = bench.Clocks(0)
    c.start()
    for _ in range(100):
        if len(c.lines) >= 3:
            break
        time.sleep(0.05)
    out = c.stop()
    assert out["samples"] == 3 and out["sm_mhz"] == 2040.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_nvidia_smi(monkeypatch, tmp_path):
    monkeypatch.setenv("PATH", str(tmp_path))
    c = bench.Clocks(0)
    c.start()
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_byte_models_count_the_folded_operator():
    # with the folded data term the operator read twice per iteration is G_S Phi, Nr K^2 8 B
    # (c2: 32 x 225 x 8 = 57.6 kB) instead of G_S (32 x 4096 x 8 = 1.05 MB); U = 16 x 4096 x 8
    import scenes
    w = scenes.workload("c2")
    m = bench.hbm_model(w, loop_ms=w.iters * 1e-3, peaks={"hbm_gbs": 1000.0}, fold=1)
    U, G = 16 * 4096 * 8, 32 * 225 * 8
    assert m["B_min_MB"] == pytest.approx((U + 2 * G) / 1e6)
    assert m["B_model_MB"] == pytest.approx((11 * U + 2 * G) / 1e6)


def test_cluster_flops_c2_both_forms():
    # c2 by hand: 64 x 64 grid, padding 128, K = 15, Nr = 32, Ni = 16.  Per incidence:
    #   synthesis 8 (64 15 15 + 64 64 15) = 606 720, analysis the same;
    #   G_D: 2 x 64 row + 2 x 128 column 128-point FFTs at 5 x 128 x 7 = 4 480 flops, plus
    #        6 x 128 x 128 spectrum products = 1 818 624, G_D^H the same;
    #   data term: folded 8 x 32 x 225 = 57 600 each way, unfolded 8 x 32 x 4096 = 1 048 576.
    import scenes
    w = scenes.workload("c2")
    per_inc = 2 * 606720 + 2 * 1818624
    assert bench.cluster_flops(w, fold=1) == 16 * (per_inc + 2 * 57600) == 79454208
    assert bench.cluster_flops(w, fold=0) == 16 * (per_inc + 2 * 1048576) == 111165440
    # the network (H = 64, D = 450) per incidence: forward 28 800 + 4 096 + 28 800 MACs, chain rule
    # 28 800 + 4 096, weight gradients 28 800 + 4 096 + 28 800: 156 288 MACs, 312 576 flops
    assert bench.cluster_flops(w, fold=1, hidden=64) == 79454208 + 16 * 312576 == 84455424
