"""The worked-example fixture of tests/golden (written by make_golden.py from
the FP64 oracle; the paper prints no worked example of its own): the oracle
must keep reproducing it (CPU), and the CUDA path must match it within the
parity tolerances (GPU): |dF| <= 1e-4 of the truncation distance with equal
weights and colours on voxels away from a decision threshold, raycast depth
within 0.1 voxel on pixels away from one (Sec. Volumetric Integration,
Sec. Raycasting)."""
import json
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
FIXTURE = os.path.join(HERE, "golden", "tilted_plane_8.json")


class _Cam:
    def __init__(self, d):
        self.fx, self.fy, self.cx, self.cy = d["fx"], d["fy"], d["cx"], d["cy"]
        self.width, self.height = d["width"], d["height"]


def _load():
    with open(FIXTURE) as f:
        g = json.load(f)
    cam = _Cam(g["intrinsics"])
    frames = [(np.array(fr["depth"], np.float32), np.array(fr["rgb"], np.uint8), np.array(fr["pose"]))
              for fr in g["frames"]]
    return g, cam, frames


def test_oracle_reproduces_worked_example(oracle_lib):
    g, cam, frames = _load()
    v = g["volume"]
    cfg = oracle.Config(trunc_vox=g["config"]["trunc_voxels"], w_max=g["config"]["w_max"],
                        color_w_max=g["config"]["color_w_max"], step_vox=g["config"]["ray_step"])
    vol = oracle.Volume(tuple(v["h"]), tuple(v["r"]), v["s"])
    for D, rgb, T in frames:
        oracle.integrate(vol, D, rgb, cam, T, cfg)
    assert np.array_equal(vol.W, np.array(g["W"]))
    assert np.array_equal(vol.rgba, np.array(g["rgba"], np.uint8))
    assert np.abs(vol.F - np.array(g["F"])).max() <= 1e-12
    out = oracle.raycast([vol], cam, np.array(g["raycast_pose"]), cfg, ids=[0])
    assert np.abs(out["depth"] - np.array(g["raycast_depth"])).max() <= 1e-12
    # the example exercises the method: observed voxels, a running average
    # over two frames, colour, and a surface the raycast finds
    W = np.array(g["W"])
    assert (W == 2).sum() > 100 and (np.array(g["raycast_depth"]) > 0).sum() > 20


@pytest.mark.gpu
def test_cuda_path_matches_worked_example():
    import torch
    from paper_1511_07106_b300 import Config, Mapper
    g, cam, frames = _load()
    v = g["volume"]
    cfg = Config()
    cfg.trunc_voxels, cfg.w_max = g["config"]["trunc_voxels"], g["config"]["w_max"]
    cfg.color_w_max, cfg.ray_step = g["config"]["color_w_max"], g["config"]["ray_step"]
    with Mapper(cfg) as m:
        vid = m.add_volume(v["h"], v["r"], v["s"], "f32")
        for D, rgb, T in frames:
            m.integrate(torch.from_numpy(D).cuda(), torch.from_numpy(rgb).cuda(), cam, T)
        F, W, rgba = m.read_decoded(vid)
        # the raycast of the stored example volume itself (the oracle raycast
        # its own FP64 state; off-threshold voxels may differ after integration)
        m.write_decoded(vid, np.array(g["F"], np.float32), np.array(g["W"], np.float32),
                        np.array(g["rgba"], np.uint8))
        out = m.raycast(cam, np.array(g["raycast_pose"]))
        depth = out["depth"].cpu().numpy()
    ok = np.array(g["decided"], bool)
    assert np.abs(F - np.array(g["F"]))[ok].max() <= 1e-4
    assert np.array_equal(W[ok], np.array(g["W"])[ok])
    assert np.array_equal(rgba[ok], np.array(g["rgba"], np.uint8)[ok])
    rd = np.array(g["raycast_depth"])
    rok = np.array(g["raycast_decided"], bool)
    assert np.array_equal((depth > 0)[rok], (rd > 0)[rok])
    both = rok & (depth > 0) & (rd > 0)
    assert both.sum() > 20
    # depth error in voxels along the ray: |d tau| |d| / s, |d| = |K^-1 [x, y, 1]|
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    dn = np.sqrt(((xs - cam.cx) / cam.fx) ** 2 + ((ys - cam.cy) / cam.fy) ** 2 + 1.0)
    assert (np.abs(depth - rd) * dn / v["s"])[both].max() <= 0.1
