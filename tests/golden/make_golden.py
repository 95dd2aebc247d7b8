"""Write the small worked-example fixtures of this directory from the FP64
oracle (the only code this script runs besides numpy).

The paper prints no worked example, so the fixtures are the oracle's values on
a tiny, hand-checkable scene: two 8x6 depth + RGB frames of a tilted plane
integrated into one 8^3 volume (Sec. Volumetric Integration; Algorithm 1,
integration loop), then one raycast of the result (Sec. Raycasting;
Algorithm 1, raycast loop).  Every value in them can also be derived by hand
from the formulas the tests restate; tests/test_golden.py checks the oracle
against them (and against those closed forms) on the CPU, and the CUDA path
against them on the GPU.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


class Cam:
    fx, fy, cx, cy, width, height = 24.0, 24.0, 3.5, 2.5, 8, 6


def plane_depth(cam, T, n, d):
    """z-depth of the plane n.p = d seen from pose T (camera to world)."""
    R, t = T[:3, :3], T[:3, 3]
    D = np.zeros((cam.height, cam.width), np.float32)
    for y in range(cam.height):
        for x in range(cam.width):
            ray = R @ np.array([(x - cam.cx) / cam.fx, (y - cam.cy) / cam.fy, 1.0])
            tau = (d - n @ t) / (n @ ray)
            D[y, x] = tau if tau > 0 else 0.0
    return D


def pose(yaw_deg, t):
    a = np.radians(yaw_deg)
    T = np.eye(4)
    T[:3, :3] = [[np.cos(a), 0, np.sin(a)], [0, 1, 0], [-np.sin(a), 0, np.cos(a)]]
    T[:3, 3] = t
    return T


def main():
    cam = Cam()
    h, r, s = (-4, -3, 16), (8, 8, 8), 0.05      # voxel i at (h + i) s: x in [-0.2, 0.15], z in [0.8, 1.15]
    n = np.array([0.2, 0.0, 1.0]); n /= np.linalg.norm(n)
    d = n @ np.array([0.0, 0.0, 0.97])
    poses = [pose(0.0, (0.0, 0.0, 0.0)), pose(3.0, (0.02, 0.01, 0.0))]
    cfg = oracle.Config()
    vol = oracle.Volume(h, r, s)
    frames = []
    decided = np.ones((8, 8, 8), bool)
    for i, T in enumerate(poses):
        D = plane_depth(cam, T, n, d)
        rgb = np.zeros((cam.height, cam.width, 3), np.uint8)
        rgb[..., 0], rgb[..., 1], rgb[..., 2] = 40 + 20 * i, 120, 200 - 10 * i
        _, flags = oracle.integrate(vol, D, rgb, cam, T, cfg, want_flags=True)
        decided &= flags == 0
        frames.append({"pose": T.tolist(), "depth": D.tolist(), "rgb": rgb.tolist()})
    T_ray = pose(1.5, (0.01, 0.0, 0.0))
    out = oracle.raycast([vol], cam, T_ray, cfg, ids=[0])
    ray_ok = (out["flags"] & (oracle.RF_SIGN | oracle.RF_CELL | oracle.RF_RANGE)) == 0
    fixture = {
        "about": "Two frames of a tilted plane integrated into one 8^3 volume, then raycast once; "
                 "values from the FP64 oracle (oracle/), written by tests/golden/make_golden.py. "
                 "The paper prints no worked example: Sec. Volumetric Integration and Algorithm 1 "
                 "(integration loop) define F and W, Sec. Raycasting and Algorithm 1 (raycast loop) "
                 "the depth map.",
        "intrinsics": {"fx": cam.fx, "fy": cam.fy, "cx": cam.cx, "cy": cam.cy, "width": cam.width,
                       "height": cam.height},
        "config": {"trunc_voxels": cfg.trunc_vox, "w_max": cfg.w_max, "color_w_max": cfg.color_w_max,
                   "ray_step": cfg.step_vox},
        "plane": {"n": n.tolist(), "d": float(d)},
        "volume": {"h": list(h), "r": list(r), "s": s},
        "frames": frames,
        "F": vol.F.tolist(), "W": vol.W.tolist(), "rgba": vol.rgba.tolist(),
        "decided": decided.astype(int).tolist(),
        "raycast_pose": T_ray.tolist(),
        "raycast_depth": out["depth"].tolist(),
        "raycast_decided": ray_ok.astype(int).tolist(),
    }
    path = os.path.join(HERE, "tilted_plane_8.json")
    with open(path, "w") as f:
        json.dump(fixture, f, indent=None, separators=(",", ":"))
    print(path, int(decided.sum()), "decided voxels,", int((vol.W > 0).sum()), "observed,",
          int((out["depth"] > 0).sum()), "raycast hits")


if __name__ == "__main__":
    main()
