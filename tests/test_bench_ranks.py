"""Host logic of the benchmark's multi-GPU mode (replicas only): every rank
inpaints its own clip of the same size (weak scaling) and rank 0 reports the
maximum time and the summed work over ranks. Exercised here with two gloo
ranks on CPU; no GPU and no collective on the data path."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (10 + r) ms and did (100 * (r + 1)) evaluations
        mx, sm = bench.combine_ranks([10.0 + rank, 100.0 * (rank + 1)], dist, "cpu")
        out[rank] = (mx, sm)
    finally:
        dist.destroy_process_group()


def test_combine_ranks_gloo_two_ranks():
    world = 2
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        mx, sm = out[rank]
        assert mx[0] == 11.0                      # slowest rank's time
        assert sm[1] == 300.0                     # work of all ranks
    # one rank: the values themselves
    assert bench.combine_ranks([1.0, 2.0]) == ([1.0, 2.0], [1.0, 2.0])


def test_replicas_are_independent_clips_of_the_same_size():
    a = bench.make_clip(0)
    b = bench.make_clip(1)
    assert a.rgb.shape == b.rgb.shape and a.levels == b.levels
    assert not np.array_equal(a.rgb, b.rgb)
    assert abs(a.mask.mean() - b.mask.mean()) < 0.01


def test_clock_summary_from_nvidia_smi_samples():
    # the clocks object of the JSON line: median SM clock, the maximum, and
    # every throttle reason active in any sample ("Not Active" is not)
    text = "\n".join([
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ])
    c = bench.summarise_clocks(text)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    hot = text + "\n0, 1500, 2070, 1400.0, 0x48, Active, Not Active, Active, Not Active"
    assert bench.summarise_clocks(hot)["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert bench.summarise_clocks("") is None
