"""Replica aggregation of bench.py under torch.distributed, on CPU with the
gloo backend and world_size 2: every rank times its own replica, the job's
time is the max over ranks (after a barrier), and units add up."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    r, w, dist = bench.dist_setup()
    assert (r, w) == (rank, world) and dist is not None
    bench.barrier(dist)
    t = bench.reduce_max(10.0 * (rank + 1), dist)   # rank-dependent "time"
    out[rank] = t
    dist.destroy_process_group()


def test_two_rank_max_time_over_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert dict(out) == {0: 20.0, 1: 20.0}


def test_single_process_has_no_group():
    import bench
    os.environ.pop("WORLD_SIZE", None)
    assert bench.dist_setup() == (0, 1, None)
    assert bench.reduce_max(3.5, None) == 3.5


def test_clock_regime_picks_the_peak_and_scales_fp8():
    import bench
    pk = {"hbm_gbs": 6800.0, "bf16": 2000.0, "bf16_sustained": 1600.0, "source": "measured"}
    obj = {"plane": {"roofline": {"bound": "tensor", "unit": "TFLOP/s", "achieved": 1000.0}},
           "extras": {"b": {"roofline": {"bound": "tensor", "unit": "TFLOP/s",
                                         "achieved": 400.0, "peak_scale": 2.0}}},
           "redq": {"roofline": {"bound": "hbm", "unit": "GB/s", "achieved": 6000.0,
                                 "peak": 6800.0}}}
    bench.apply_clock_regime(obj, {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}, pk)
    assert obj["plane"]["roofline"]["peak"] == 2000.0
    assert obj["plane"]["roofline"]["frac"] == 0.5
    assert obj["extras"]["b"]["roofline"]["peak"] == 4000.0
    assert obj["extras"]["b"]["roofline"]["frac"] == 0.1
    assert obj["redq"]["roofline"]["peak"] == 6800.0 and "frac_of_burst" not in obj["redq"]["roofline"]
    # power-capped (or below the maximum clock): the sustained figure
    bench.apply_clock_regime(obj, {"sm_mhz": 1800.0, "sm_max_mhz": 2070.0,
                                   "reasons": ["sw_power_cap"]}, pk)
    assert obj["plane"]["roofline"]["peak"] == 1600.0
    assert obj["extras"]["b"]["roofline"]["frac_of_sustained"] == 400.0 / 3200.0
