"""Multi-rank bookkeeping of bench.py on CPU with two gloo ranks: disjoint
slots per rank, max-over-ranks timing and the whole-job aggregate.  The NRX
path shards by slot with no data-path collective, so only this host logic is
distributed."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import bench
    from paper_2409_02912_b300 import synth
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    batch = 3
    start = bench.rank_slot_start(rank, batch)
    starts = [None] * world
    dist.all_gather_object(starts, start)
    local_ms = 10.0 + 5.0 * rank
    mx = bench.reduce_max_ms(local_ms, world, "cpu")
    w = synth.WORKLOADS["su_2rx_4prb"]
    value = bench.aggregate_value(world, 4, batch * bench.res_per_slot(w), mx)
    # ranks' first slots are different draws of the generator
    y0 = synth.workload_slots(w, 1, start=start)[0].y
    ys = [None] * world
    dist.all_gather_object(ys, y0.tobytes())
    out[rank] = (starts, mx, value, len(set(ys)))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        starts, mx, value, n_distinct = out[rank]
        assert starts == [0, 3]
        assert mx == 15.0
        assert n_distinct == world
        assert abs(value - world * 4 * 3 * 14 * 48 / 15e-3) < 1e-6
