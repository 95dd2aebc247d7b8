"""The multi-rank path of bench.py on CPU: two gloo ranks on 127.0.0.1 run
independent jobs; the reported throughput is the units of all ranks over
the slowest rank's time (weak scaling), with no data-path collective."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units = 1000.0 * (rank + 1)   # rank 0: 1000 voxel updates, rank 1: 2000
    ms = 10.0 * (rank + 1)        # rank 0: 10 ms, rank 1: 20 ms
    out[rank] = (bench.weak_scaling_value(torch, units, ms, device="cpu"),
                 bench.allreduce_max(torch, ms, device="cpu"), bench.allreduce_sum(torch, units, device="cpu"))
    bench.barrier(torch)
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    for r in range(world):
        value, ms_max, units = res[r]
        assert ms_max == 20.0 and units == 3000.0
        assert abs(value - 3000.0 / 20e-3) < 1e-6


def test_single_process_needs_no_process_group():
    import bench
    assert not dist.is_initialized()
    assert bench.weak_scaling_value(torch, 500.0, 5.0, device="cpu") == 500.0 / 5e-3
