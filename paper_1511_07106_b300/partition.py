"""Volumes of one map partitioned across GPUs, one process per GPU.

Integration of different volumes is independent (Sec. Comparison to
KinectFusion) and every volume writes into one map where the shortest ray
distance wins (Sec. Raycasting, last paragraph), so the set H of a map can be
split across GPUs: each rank holds, integrates and raycasts its own volumes,
the frame reaches every rank by one broadcast, and the maps are merged by

  1. ``mv_pack_hits``: per pixel the key (bits of tau << 32 | global id);
  2. all-reduce MIN of the keys (the per-pixel winner on every rank);
  3. ``mv_merge_hits``: depth and volume id from the winning key, and the
     pixels this rank did not win cleared in its normal / colour / vertex maps;
  4. all-reduce SUM of those maps (exactly one rank holds each hit).

The merged maps equal those of one GPU holding every volume.  The collectives
are torch.distributed calls (NCCL on GPUs); every per-pixel step runs in the
library's kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _abi
from .mapper import Mapper, _stream

NO_HIT = np.iinfo(np.int64).max


def assign(voxels, world: int) -> list:
    """Owner rank of each volume: largest first, each to the rank holding the
    fewest voxels so far (ties to the lower rank).  Deterministic, so every
    rank computes the same partition."""
    load = [0] * world
    owner = [0] * len(voxels)
    for g in sorted(range(len(voxels)), key=lambda i: (-int(voxels[i]), i)):
        r = min(range(world), key=lambda k: (load[k], k))
        owner[g] = r
        load[r] += int(voxels[g])
    return owner


def merge_collectives(keys, maps, merge, group=None):
    """Steps 2-4 on this rank: all-reduce MIN of the packed keys, `merge`
    (best_keys) clears the pixels this rank did not win and writes depth and
    volume id from the winning keys, then all-reduce SUM of the cleared normal,
    colour and vertex maps.  `maps` holds tensors on the collective's device;
    colour is summed as one int32 word per pixel (only one rank's word is
    non-zero, so no byte carries into another)."""
    import torch
    import torch.distributed as dist
    best = keys.clone()
    dist.all_reduce(best, op=dist.ReduceOp.MIN, group=group)
    merge(best)
    for k in ("normal", "vertex"):
        if maps.get(k) is not None:
            dist.all_reduce(maps[k], op=dist.ReduceOp.SUM, group=group)
    if maps.get("rgba") is not None:
        dist.all_reduce(maps["rgba"].view(-1).view(dtype=torch.int32), op=dist.ReduceOp.SUM,
                        group=group)
    return best


class PartitionedMapper:
    """This rank's share of a multi-volume map (volumes given as
    (h_t, h_r, voxel_size) specs with global ids 0..n-1)."""

    def __init__(self, specs, rank: int, world: int, fmt="f32", config=None, device: int = 0, group=None):
        import torch
        self.rank, self.world, self.group = rank, world, group
        self.owner = assign([int(np.prod(s[1])) for s in specs], world)
        self.mapper = Mapper(config, device)
        self.global_of = {}
        for g, (h, r, s) in enumerate(specs):  # ascending global id: local ids keep that order
            if self.owner[g] == rank:
                self.global_of[self.mapper.add_volume(h, r, s, fmt)] = g
        n = max(self.global_of, default=-1) + 1
        table = np.full(max(n, 1), -1, np.int32)
        for lid, g in self.global_of.items():
            table[lid] = g
        self.dev = torch.device("cuda", device)
        self.id_map = torch.from_numpy(table).to(self.dev)
        self._lib = _abi.lib()
        self._keys = None

    def close(self):
        self.mapper.close()

    def local_frame(self, depth, rgb, cam, T, out=None, stream=None):
        """Step 1 on this rank: integrate and raycast its own volumes
        (mv_frame) and pack the per-pixel keys (mv_pack_hits).  Returns
        (maps, keys); `keys` is reused by the next call."""
        import torch
        maps = self.mapper.frame(depth, rgb, cam, T, out=out, stream=stream)
        n = cam.width * cam.height
        if self._keys is None or self._keys.numel() != n:
            self._keys = torch.empty(n, dtype=torch.int64, device=self.dev)
        st = self._lib.mv_pack_hits(C.c_void_p(maps["depth"].data_ptr()), C.c_void_p(maps["vol_id"].data_ptr()),
                                    C.c_void_p(self.id_map.data_ptr()), int(self.id_map.numel()), n,
                                    C.c_void_p(self._keys.data_ptr()), _stream(stream))
        if st != _abi.MV_OK:
            raise _abi.MVError(st, "mv_pack_hits")
        return maps, self._keys

    def apply_merge(self, maps, keys, best, stream=None):
        """Step 3 on this rank (mv_merge_hits): depth and volume id from the
        winning keys `best`, the pixels this rank did not win cleared."""
        ptr = (lambda k: C.c_void_p(maps[k].data_ptr()) if maps.get(k) is not None else None)
        st = self._lib.mv_merge_hits(C.c_void_p(best.data_ptr()), C.c_void_p(keys.data_ptr()), keys.numel(),
                                     ptr("depth"), ptr("vol_id"), ptr("normal"), ptr("rgba"), ptr("vertex"),
                                     _stream(stream))
        if st != _abi.MV_OK:
            raise _abi.MVError(st, "mv_merge_hits")

    def frame(self, depth, rgb, cam, T, out=None, src: int = 0, broadcast: bool = True, stream=None):
        """Integrate and raycast one frame on every rank: the frame of rank
        `src` is broadcast (broadcast=False: every rank passes the same frame),
        each rank runs its volumes, and the maps are merged (steps 1-4).
        Returns the merged maps, identical on every rank."""
        import torch.distributed as dist
        if self.world > 1 and broadcast:
            dist.broadcast(depth, src, group=self.group)
            if rgb is not None:
                dist.broadcast(rgb, src, group=self.group)
        maps, keys = self.local_frame(depth, rgb, cam, T, out=out, stream=stream)
        if self.world > 1:
            merge_collectives(keys, maps, lambda best: self.apply_merge(maps, keys, best, stream), self.group)
        else:
            self.apply_merge(maps, keys, keys, stream)
        return maps
