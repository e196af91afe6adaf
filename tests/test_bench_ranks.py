"""Multi-rank bench logic on CPU: two gloo ranks, no GPU.

The benchmark runs one independent replica per GPU (the method does not
shard). Its whole-job figure is the entries of every rank over the slowest
rank's time; these tests run that aggregation on two CPU processes.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 + 50.0 * rank  # rank 1 is the slowest
        slowest = bench.rank_max(dist, world, local_ms, "cpu")
        value = bench.job_throughput(16384.0 * 16384.0, 5, world, slowest)
        results[rank] = (slowest, value)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_slowest_time_and_job_value():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        results = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, results)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        got = dict(results)
    assert got[0] == got[1]
    slowest, value = got[0]
    assert slowest == 150.0
    # 2 ranks x 5 steps x N^2 entries over 150 ms
    assert value == pytest.approx(2 * 5 * 16384.0 ** 2 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.rank_max(None, 1, 42.0, "cpu") == 42.0
    assert bench.job_throughput(100.0, 2, 1, 1000.0) == pytest.approx(200.0)


def test_clock_records_rejected():
    """Throttled or clock-locked timed regions are measured again; a power
    cap alone is kept."""
    import bench
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}
    assert not bench.clocks_rejected(ok)
    assert not bench.clocks_rejected({**ok, "reasons": ["sw_power_cap"], "sm_mhz": 1500.0})
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.clocks_rejected({**ok, "reasons": [r]})
    assert bench.clocks_rejected({**ok, "sm_mhz": 1200.0})  # locked well below the maximum
    assert not bench.clocks_rejected({"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]})


def test_roofline_arithmetic():
    """The roofline entries from a fill's counts and per-kernel times: the
    fill's algorithmic bytes (8 per new pair) over the fill and mirror-pass
    time, the step's 4 N^2 bytes over the step time, the propagation's
    relaxations over its launches, and the dominant kernel picked by time."""
    import bench

    class W:  # a 4 x 4 grey image, 8-connected
        N, conn, kind, mask = 16, 8, "grey", None

    st = {"new_pairs": 120, "propagations": 3, "prepass_propagations": 2}
    peaks = {"hbm_gbs": 1000.0, "sm_max_mhz": 2000.0}
    prof = {"_fills": 2, "fill": (4.0, 8), "mirror": (1.0, 2), "propagate": (1.0, 6), "lookahead": (0.0, 0),
            "tree": (0.5, 8)}
    r = bench.roofline(W, st, dict(prof), ms_per_step=10.0, peaks=peaks,
                       dram={"kernel": "k_fill", "bytes": 1e4, "launch": "round 0"})
    fill = r["kernels"]["fill"]
    # 8 B x 120 pairs x 2 fills over (4 + 1) ms of fill and mirror
    assert fill["achieved"] == pytest.approx(8 * 120 * 2 / 5e-3 / 1e9)
    assert fill["frac"] == pytest.approx(fill["achieved"] / 1000.0)
    assert fill["mirror_ms_per_fill"] == pytest.approx(0.5)
    assert fill["traffic"] == 1e4 and fill["traffic_launch"] == "round 0"
    assert r["step_hbm"]["achieved"] == pytest.approx(4 * 16 * 16 / 10e-3 / 1e9)
    prop = r["kernels"]["propagate"]
    # 2 conn relaxations per free pixel for each of the P + 2 propagations, both fills
    assert prop["achieved"] == pytest.approx(2 * 8 * 16 * 5 * 2 / 1e-3 / 1e12)
    assert r["kernel"] == "k_fill"  # 5 ms of fill against 1 ms of propagation
    assert r["kernel_ms_per_fill"]["mirror"] == pytest.approx(0.5)
