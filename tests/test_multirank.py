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


# ---------------------------------------------------------------------------
# volumes partitioned across ranks: the merge of per-rank raycast maps
# ---------------------------------------------------------------------------

def _hit_key(depth, gid):
    """Key of one hit in the layout mv_pack_hits documents: the float bits of
    the ray distance above the global volume id (test stand-in for the
    library kernel, which needs a GPU)."""
    import numpy as np
    return (int(np.float32(depth).view(np.uint32)) << 32) | int(gid)


def _rank_maps(rank, world, H=6, W=7, n_vol=5):
    """Deterministic per-rank maps: each global volume belongs to one rank and
    hits some pixels at a random distance (some distances tie across
    volumes); a pixel keeps the rank's nearest hit, ties to the lower id."""
    import numpy as np
    from paper_1511_07106_b300.partition import NO_HIT, assign
    rng = np.random.default_rng(3)
    owner = assign([100, 80, 80, 60, 10], world)
    depth_v = rng.choice([0.5, 0.75, 1.0, 1.25], size=(n_vol, H, W)).astype(np.float32)
    hit_v = rng.uniform(size=(n_vol, H, W)) < 0.5
    keys = np.full((H, W), NO_HIT, np.int64)
    normal = np.zeros((H, W, 3), np.float32)
    rgba = np.zeros((H, W, 4), np.uint8)
    for g in range(n_vol):
        if owner[g] != rank:
            continue
        k = np.where(hit_v[g], [[_hit_key(depth_v[g, y, x], g) for x in range(W)] for y in range(H)], NO_HIT)
        better = k < keys
        keys = np.where(better, k, keys)
        normal[better] = (g + 1) * np.array([0.1, -0.2, 0.3], np.float32)
        rgba[better] = np.array([g * 40 + 1, 255 - g, 7 * g, 255], np.uint8)
    return keys, normal, rgba


def _merge_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np
    from paper_1511_07106_b300.partition import NO_HIT, merge_collectives
    keys, normal, rgba = _rank_maps(rank, world)
    maps = {"normal": torch.from_numpy(normal.copy()), "rgba": torch.from_numpy(rgba.copy()),
            "depth": torch.zeros(keys.shape), "vol_id": torch.zeros(keys.shape, dtype=torch.int32)}
    own = torch.from_numpy(keys.copy())

    def merge(best):  # stand-in for mv_merge_hits (the per-pixel rule it documents)
        b = best.numpy()
        hit = b != NO_HIT
        maps["depth"][:] = torch.from_numpy(np.where(hit, (b >> 32).astype(np.uint32).view(np.float32), 0.0))
        maps["vol_id"][:] = torch.from_numpy(np.where(hit, (b & 0xFFFFFFFF), -1).astype(np.int32))
        lost = torch.from_numpy(~hit | (own.numpy() != b))
        maps["normal"][lost] = 0.0
        maps["rgba"][lost] = 0

    best = merge_collectives(own, maps, merge)
    out[rank] = (best.numpy(), maps["depth"].numpy(), maps["vol_id"].numpy(), maps["normal"].numpy(),
                 maps["rgba"].numpy())
    dist.destroy_process_group()


def test_partitioned_merge_equals_single_rank_on_two_gloo_ranks():
    """Two gloo ranks each hold some of five volumes; after the all-reduce
    MIN of the packed keys and the SUM of the cleared maps, both ranks hold
    the maps of one rank owning all five volumes: nearest hit, equal
    distances to the lower global id, the winner's normal and colour."""
    import numpy as np
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_merge_rank, args=(world, _free_port(), out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    keys1, normal1, rgba1 = _rank_maps(0, 1)
    for r in range(world):
        best, depth, vol_id, normal, rgba = res[r]
        np.testing.assert_array_equal(best, keys1)
        hit = keys1 != np.iinfo(np.int64).max
        assert hit.mean() > 0.5
        np.testing.assert_array_equal(vol_id, np.where(hit, keys1 & 0xFFFFFFFF, -1))
        np.testing.assert_array_equal(depth[hit] > 0, True)
        np.testing.assert_array_equal(normal, normal1)
        np.testing.assert_array_equal(rgba, rgba1)
    # ties across ranks exist in this fixture, and the lower id won them
    k0, _, _ = _rank_maps(0, world)
    k1, _, _ = _rank_maps(1, world)
    tie = (k0 >> 32 == k1 >> 32) & (k0 != np.iinfo(np.int64).max) & (k1 != np.iinfo(np.int64).max)
    assert tie.any()
    assert np.all((keys1 & 0xFFFFFFFF)[tie] == np.minimum(k0 & 0xFFFFFFFF, k1 & 0xFFFFFFFF)[tie])


def test_partition_assignment_is_balanced_and_deterministic():
    from paper_1511_07106_b300.partition import assign
    vox = [768 ** 3, 128 ** 3, 512 ** 3, 512 ** 3, 256 ** 3, 384 ** 3, 192 ** 3, 128 ** 3]
    for world in (1, 2, 3, 4):
        a = assign(vox, world)
        assert a == assign(vox, world)
        assert sorted(set(a)) == list(range(min(world, len(vox))))
        load = [sum(v for v, r in zip(vox, a) if r == k) for k in range(world)]
        # greedy largest-first: no rank exceeds the lightest by more than the largest volume
        assert max(load) - min(load) <= max(vox)
    assert assign(vox, 1) == [0] * len(vox)
