"""Volumes of one map partitioned across ranks (mv_pack_hits, all-reduce MIN,
mv_merge_hits, all-reduce SUM): the merged maps equal those of one mapper
holding every volume.  Ranks are emulated on the one GPU of the test box:
in one process (the MIN and SUM taken in the test), and as two processes
whose collectives go through gloo -- host-side, so no kernel of one process
waits on the other's."""
import os
import socket

import numpy as np
import pytest

from paper_1511_07106_b300 import Mapper, synth
from paper_1511_07106_b300.partition import PartitionedMapper, assign
from parity_utils import dev, gpu_maps

pytestmark = pytest.mark.gpu

KEYS = ("depth", "normal", "rgba", "vertex", "vol_id")


def workload():
    return synth.uneven_volumes(n_volumes=12, frames=4, edges=(16, 24, 40), pitch_mm=(15.0, 40.0),
                                half_extent=1.6, height_m=2.2, width=160, height=120)


def specs_of(wl):
    return [(v.h, v.r, v.s) for v in wl.volumes]


def single_mapper_maps(wl):
    m = Mapper()
    for v in wl.volumes:
        m.add_volume(v.h, v.r, v.s)
    out = []
    for i in range(wl.n_frames):
        d, c = wl.frame(i)
        out.append(gpu_maps(m.frame(dev(d), dev(c), wl.cam, wl.poses[i])))
    m.close()
    return out


@pytest.mark.parametrize("world", [2, 3])
def test_partitioned_frames_equal_one_mapper_in_one_process(world):
    import torch
    wl = workload()
    ref = single_mapper_maps(wl)
    ranks = [PartitionedMapper(specs_of(wl), r, world) for r in range(world)]
    assert sorted(g for pm in ranks for g in pm.global_of.values()) == list(range(len(wl.volumes)))
    for i in range(wl.n_frames):
        d, c = wl.frame(i)
        local = [pm.local_frame(dev(d), dev(c), wl.cam, wl.poses[i]) for pm in ranks]
        best = local[0][1].clone()
        for _, k in local[1:]:
            best = torch.minimum(best, k)  # the all-reduce MIN
        for pm, (maps, k) in zip(ranks, local):
            pm.apply_merge(maps, k, best)
        merged = {key: sum(maps[key].double() if key != "rgba" else maps[key].int() for maps, _ in local)
                  for key in ("normal", "vertex", "rgba")}  # the all-reduce SUM
        for maps, _ in local:
            np.testing.assert_array_equal(maps["depth"].cpu().numpy(), ref[i]["depth"])
            np.testing.assert_array_equal(maps["vol_id"].cpu().numpy(), ref[i]["vol_id"])
        np.testing.assert_array_equal(merged["normal"].cpu().numpy(), ref[i]["normal"])
        np.testing.assert_array_equal(merged["vertex"].cpu().numpy(), ref[i]["vertex"])
        np.testing.assert_array_equal(merged["rgba"].cpu().numpy(), ref[i]["rgba"])
        # exactly one rank holds each hit
        holders = sum((maps["rgba"][..., 3] != 0).int() for maps, _ in local).cpu().numpy()
        assert np.all(holders == (ref[i]["depth"] > 0))
    assert (ref[-1]["depth"] > 0).mean() > 0.05
    for pm in ranks:
        pm.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = workload()
    pm = PartitionedMapper(specs_of(wl), rank, world)
    res = []
    for i in range(wl.n_frames):
        d, c = wl.frame(i)
        if rank == 0:
            dd, dc = dev(d), dev(c)
        else:  # the frame arrives by broadcast from rank 0
            dd = torch.zeros(d.shape, dtype=torch.float32, device="cuda")
            dc = torch.zeros(c.shape, dtype=torch.uint8, device="cuda")
        maps = pm.frame(dd, dc, wl.cam, wl.poses[i])
        torch.cuda.synchronize()
        res.append({k: maps[k].cpu().numpy() for k in KEYS})
    out[rank] = (res, sorted(pm.global_of.values()))
    pm.close()
    dist.barrier()
    dist.destroy_process_group()


def test_partitioned_frames_over_two_gloo_processes():
    import torch.multiprocessing as mp
    wl = workload()
    ref = single_mapper_maps(wl)
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    owned = [res[r][1] for r in range(world)]
    assert sorted(owned[0] + owned[1]) == list(range(len(wl.volumes))) and owned[0] and owned[1]
    assert owned == [[g for g, o in enumerate(assign([int(np.prod(v.r)) for v in wl.volumes], world)) if o == r]
                     for r in range(world)]
    for r in range(world):
        for i in range(wl.n_frames):
            for k in KEYS:
                np.testing.assert_array_equal(res[r][0][i][k], ref[i][k], err_msg=f"rank {r} frame {i} {k}")
